"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a library routine applied to the definition, a brute-force enumeration
on a tiny graph, an invariant, or a worked case of the paper. Section numbers
refer to Konolige & Brown, "A Parallel Solver for Graph Laplacians".
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, laplacian

SEED = 0x5EED
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_adj(g):
    A = np.zeros((g.n, g.n))
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            A[i, g.col[p]] = g.w[p]
    return A


def dense_lap(g):
    A = dense_adj(g)
    return np.diag(A.sum(1)) - A


def sp_adj(g):
    return sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))


# --------------------------------------------------------------------------
# Random streams
# --------------------------------------------------------------------------
def test_splitmix64_published_outputs(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    for ctr, val in rows:
        assert oracle.splitmix64(1234567, int(ctr)) == int(val)


def test_uniform_stream_range_and_independence(oracle):
    u = np.array([oracle.uniform(SEED, 1, 0, i) for i in range(4000)])
    v = np.array([oracle.uniform(SEED, 2, 0, i) for i in range(4000)])
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.05 and abs(u.var() - 1.0 / 3.0) < 0.03
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.05
    # 53 random bits: 2u - 1 with u a multiple of 2^-53
    assert np.all(((u + 1.0) * 2.0 ** 52) == np.floor((u + 1.0) * 2.0 ** 52))


# --------------------------------------------------------------------------
# Laplacian (Section 2.1)
# --------------------------------------------------------------------------
def test_laplacian_matches_scipy_and_properties(oracle, inputs):
    g = inputs.random_graph(300, 7, seed=3)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(g.n), rng.standard_normal(g.n)
    Ls = laplacian(sp_adj(g))
    np.testing.assert_allclose(oracle.apply_L(g, x), Ls @ x, rtol=1e-12, atol=1e-12)
    # zero row sums, symmetry, quadratic form 1/2 sum w (x_i - x_j)^2 >= 0
    assert np.abs(oracle.apply_L(g, np.ones(g.n))).max() < 1e-12
    assert abs(x @ oracle.apply_L(g, y) - y @ oracle.apply_L(g, x)) < 1e-10
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    q = 0.5 * np.sum(g.w * (x[rows] - x[g.col]) ** 2)
    assert abs(x @ oracle.apply_L(g, x) - q) < 1e-9 * q
    np.testing.assert_allclose(oracle.diag(g), np.asarray(sp_adj(g).sum(1)).ravel(), rtol=1e-14)


def test_components_match_scipy(oracle, inputs):
    g = inputs.random_graph(200, 3, seed=5)
    # two copies side by side: exactly two components
    n2 = 2 * g.n
    rp = np.concatenate([g.rowptr, g.rowptr[1:] + g.rowptr[-1]])
    cl = np.concatenate([g.col, g.col + g.n]).astype(np.int32)
    w = np.concatenate([g.w, g.w])
    two = inputs.Graph(n2, rp, cl, w)
    nc, lab = oracle.components(two)
    ref_nc, ref_lab = connected_components(sp_adj(two), directed=False)
    assert nc == ref_nc == 2
    assert len(set(zip(lab, ref_lab))) == 2
    assert oracle.check_graph(two) == oracle.DISCONNECTED
    assert oracle.check_graph(g) == oracle.OK


def test_check_graph_rejects_bad_input(oracle, inputs):
    g = inputs.path(5)
    bad_w = inputs.Graph(g.n, g.rowptr, g.col, g.w.copy())
    bad_w.w[0] = -1.0
    bad_w.w[2] = -1.0  # keep the pair equal, still negative
    assert oracle.check_graph(bad_w) == oracle.INVALID
    asym = inputs.Graph(g.n, g.rowptr, g.col, g.w.copy())
    asym.w[0] = 2.0
    assert oracle.check_graph(asym) == oracle.INVALID
    selfloop = inputs.Graph(2, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.ones(2))
    assert oracle.check_graph(selfloop) == oracle.INVALID
    unsorted = inputs.complete(3)
    c = unsorted.col.copy()
    c[0], c[1] = c[1], c[0]
    assert oracle.check_graph(inputs.Graph(3, unsorted.rowptr, c, unsorted.w)) == oracle.INVALID
    single = inputs.Graph(1, np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.check_graph(single) == oracle.OK


# --------------------------------------------------------------------------
# Low-degree elimination (Section 3.4)
# --------------------------------------------------------------------------
def brute_force_elim(g, seed):
    deg = np.diff(g.rowptr)
    h = [int(v) for v in oracle_hashes(g.n, seed)]
    out = np.zeros(g.n, np.uint8)
    for i in range(g.n):
        if deg[i] > 4:
            continue
        nbrs = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        if all(h[i] < h[j] for j in nbrs if deg[j] <= 4):
            out[i] = 1
    return out


def oracle_hashes(n, seed):
    import oracle as O

    return O.vertex_hash(seed, range(n))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_elim_select_brute_force(oracle, inputs, seed):
    g = inputs.random_graph(400, 3.5, seed=seed)
    f = oracle.elim_select(g, 4, SEED)
    np.testing.assert_array_equal(f, brute_force_elim(g, SEED))
    deg = np.diff(g.rowptr)
    assert np.all(deg[f == 1] <= 4)  # F within the candidates
    for i in np.nonzero(f)[0]:  # F is an independent set
        assert not np.any(f[g.col[g.rowptr[i]:g.rowptr[i + 1]]])


def test_elim_star_and_path(oracle, inputs):
    s = inputs.star(9)
    f = oracle.elim_select(s, 4, SEED)
    assert f[0] == 0 and np.all(f[1:] == 1)  # hub has degree 9, every leaf goes
    coarse, cmap = oracle.schur(s, f)
    assert coarse.n == 1 and coarse.nnz_off == 0  # the 1x1 zero Laplacian
    assert cmap[0] == 0 and np.all(cmap[1:] == -1)
    p = inputs.path(50)
    f = oracle.elim_select(p, 4, SEED)
    h = oracle_hashes(50, SEED)
    for i in range(50):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < 50]
        assert f[i] == all(h[i] < h[j] for j in nb)


def test_elim_grids(oracle, inputs):
    g2 = inputs.grid2d(40, 40)
    frac2 = oracle.elim_select(g2, 4, SEED).mean()
    assert 0.15 < frac2 < 0.25  # every vertex is a candidate: about 1/5 win their neighbourhood
    g3 = inputs.grid3d(10, 10, 10)
    f3 = oracle.elim_select(g3, 4, SEED)
    deg = np.diff(g3.rowptr)
    assert np.all(deg[f3 == 1] <= 4) and f3.mean() < 0.05  # only cube edges/corners, below the gate


@pytest.mark.parametrize("seed", [4, 5])
def test_schur_complement_dense(oracle, inputs, seed):
    g = inputs.random_graph(120, 3.0, seed=seed)
    f = oracle.elim_select(g, 4, SEED).astype(bool)
    assert f.sum() > 0
    coarse, cmap = oracle.schur(g, f)
    L = dense_lap(g)
    C = ~f
    S = L[np.ix_(C, C)] - L[np.ix_(C, f)] @ np.linalg.inv(L[np.ix_(f, f)]) @ L[np.ix_(f, C)]
    np.testing.assert_allclose(dense_lap(coarse), S, rtol=1e-12, atol=1e-12)
    assert np.array_equal(cmap[C], np.arange(C.sum())) and np.all(cmap[f] == -1)


def test_two_level_elimination_identity(oracle, inputs):
    """L^+ b = P L_c^+ P^T b + Fsmooth(b) up to constants (Section 3.4)."""
    g = inputs.random_graph(90, 3.0, seed=8, weights="uniform")
    f = oracle.elim_select(g, 4, SEED).astype(bool)
    coarse, cmap = oracle.schur(g, f)
    L = dense_lap(g)
    Fi, Ci = np.nonzero(f)[0], np.nonzero(~f)[0]
    P = np.zeros((g.n, Ci.size))
    P[Ci, np.arange(Ci.size)] = 1.0
    P[np.ix_(Fi, np.arange(Ci.size))] = -np.linalg.inv(L[np.ix_(Fi, Fi)]) @ L[np.ix_(Fi, Ci)]
    b = inputs.rhs(g.n, seed=3)
    fs = np.zeros(g.n)
    fs[Fi] = b[Fi] / np.diag(L)[Fi]
    x2 = P @ np.linalg.pinv(dense_lap(coarse)) @ P.T @ b + fs
    x1 = np.linalg.pinv(L) @ b
    np.testing.assert_allclose(x2 - x2.mean(), x1 - x1.mean(), atol=1e-9)
    # the V-cycle over [elimination, exact coarsest] is the exact solve
    h = oracle.Hierarchy(g, oracle.default_opts(coarse_nnz=float(coarse.nnz_off + coarse.n)))
    assert [h.level(l).kind for l in range(h.nlevels)] == [oracle.ELIM, oracle.COARSEST]
    xc = h.vcycle(b)
    np.testing.assert_allclose(xc - xc.mean(), x1 - x1.mean(), atol=1e-9)


# --------------------------------------------------------------------------
# Strength of connection (Section 3.5)
# --------------------------------------------------------------------------
def test_jacobi_on_eigenvectors(oracle, inputs):
    n = 24
    g = inputs.cycle(n)
    i = np.arange(n)
    omega = 2.0 / 3.0
    for k in (1, 3, 6, 12):
        v = np.cos(2 * np.pi * k * i / n)
        mu = 1.0 - np.cos(2 * np.pi * k / n)  # eigenvalue of D^-1 L on the cycle
        x = oracle.jacobi(g, v[:, None], sweeps=3, omega=omega)[:, 0]
        np.testing.assert_allclose(x, (1 - omega * mu) ** 3 * v, atol=1e-13)


def test_affinity_closed_forms(oracle, inputs):
    p = inputs.path(3)  # edges 0-1, 1-2
    x = np.array([[1.0, 0.0], [2.0, 0.0], [1.0, 1.0]])
    S = oracle.affinity(p, x)
    # C_01 = (x0.x1)^2/(|x0|^2 |x1|^2) = 4/(1*4) = 1; C_12 = (2)^2/(4*2) = 0.5
    C01, C12 = 1.0, 0.5
    rowmax = [C01, max(C01, C12), C12]
    expect = {(0, 1): C01 / max(rowmax[0], rowmax[1]), (1, 0): C01 / max(rowmax[1], rowmax[0]),
              (1, 2): C12 / max(rowmax[1], rowmax[2]), (2, 1): C12 / max(rowmax[2], rowmax[1])}
    for i in range(3):
        for q in range(p.rowptr[i], p.rowptr[i + 1]):
            assert S[q] == pytest.approx(expect[(i, int(p.col[q]))], abs=1e-15)
    # orthogonal rows give 0
    x = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    assert np.all(oracle.affinity(p, x) == 0.0)


def test_strength_invariants(oracle, inputs):
    g = inputs.random_graph(500, 6, seed=11)
    S = oracle.strength(g, SEED, 0)
    assert S.min() >= 0.0 and S.max() == 1.0
    Ssp = sp.csr_matrix((S, g.col, g.rowptr), shape=(g.n, g.n))
    assert abs(Ssp - Ssp.T).max() == 0.0  # bitwise symmetric
    y = oracle.strength_vectors(SEED, 0, g.n, 4)
    x = oracle.jacobi(g, y, 3, 2.0 / 3.0)
    C = oracle.affinity(g, x)
    assert np.all(C <= 1.0 + 1e-15) and np.all(C >= 0.0)  # Cauchy-Schwarz
    # row i's strongest edge is 1 whenever i is its partner's strongest too
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    assert np.all(S <= 1.0)
    assert np.any(S[rows == rows[np.argmax(S)]] == 1.0)


# --------------------------------------------------------------------------
# Aggregation (Section 3.5, Algorithm 3)
# --------------------------------------------------------------------------
def check_partition(oracle, g, S, nc, agg, st, votes, threshold=8, iters=10):
    assert agg.min() == 0 and agg.max() == nc - 1 and np.unique(agg).size == nc
    roots = {}
    for i in range(g.n):
        if st[i] in (oracle.SEED, oracle.UNDECIDED):
            assert agg[i] not in roots
            roots[agg[i]] = i
    assert len(roots) == nc
    assert np.all(votes[st == oracle.SEED] >= threshold)
    fmin = 0.5 ** iters
    for i in range(g.n):
        if st[i] == oracle.DECIDED:
            r = roots[agg[i]]
            assert st[r] == oracle.SEED
            cols = g.col[g.rowptr[i]:g.rowptr[i + 1]]
            q = g.rowptr[i] + np.searchsorted(cols, r)
            assert cols[q - g.rowptr[i]] == r and S[q] >= fmin  # an S-neighbour of its seed
    # roots are numbered in ascending vertex order
    assert [agg[roots[c]] for c in sorted(roots, key=lambda c: roots[c])] == list(range(nc))


@pytest.mark.parametrize("seed", [1, 2])
def test_aggregation_partition(oracle, inputs, seed):
    g = inputs.random_graph(2000, 8, seed=seed)
    S = oracle.strength(g, SEED, 0)
    nc, agg, st, votes = oracle.aggregate(g, S)
    check_partition(oracle, g, S, nc, agg, st, votes)
    assert nc < g.n // 2


def test_aggregation_star_worked_cases(oracle, inputs):
    # 8 leaves: all vote for the hub in step 1 (8 votes, a seed), join it in step 2
    s = inputs.star(8)
    nc, agg, st, votes = oracle.aggregate(s, np.ones(s.nnz_off))
    assert nc == 1 and st[0] == oracle.SEED and np.all(st[1:] == oracle.DECIDED)
    assert votes[0] == 8 and votes[1] == 1 and np.all(votes[2:] == 0)  # the hub picks leaf 1 on the tie
    # 5 leaves: 5 votes after step 1, 10 after step 2, the leaves join in step 3
    s = inputs.star(5)
    nc, agg, st, votes = oracle.aggregate(s, np.ones(s.nnz_off))
    assert nc == 1 and votes[0] == 10 and votes[1] == 2
    nc2, *_ = oracle.aggregate(s, np.ones(s.nnz_off), iters=2)
    assert nc2 == 6  # after two steps the hub is a seed but nobody has joined yet


def test_aggregation_pair_and_filter(oracle, inputs):
    k2 = inputs.path(2)
    nc, agg, st, votes = oracle.aggregate(k2, np.ones(2))
    # each votes for the other once per step; both reach 8 in step 8 and become seeds
    # together, after which neither is Undecided and the voting stops
    assert nc == 2 and np.all(st == oracle.SEED) and np.all(votes == 8)
    nc, _, st, votes = oracle.aggregate(k2, np.ones(2), iters=7)
    assert nc == 2 and np.all(st == oracle.UNDECIDED) and np.all(votes == 7)
    g = inputs.random_graph(100, 4, seed=1)
    nc, agg, *_ = oracle.aggregate(g, np.full(g.nnz_off, 0.5 ** 11))  # all filtered out
    assert nc == g.n and np.array_equal(agg, np.arange(g.n))


# --------------------------------------------------------------------------
# Galerkin product (Section 3.5)
# --------------------------------------------------------------------------
def test_galerkin_dense_and_energy(oracle, inputs):
    g = inputs.random_graph(400, 6, seed=12)
    S = oracle.strength(g, SEED, 0)
    nc, agg, _, _ = oracle.aggregate(g, S)
    c = oracle.galerkin(g, agg, nc)
    R = np.zeros((nc, g.n))
    R[agg, np.arange(g.n)] = 1.0
    np.testing.assert_allclose(dense_lap(c), R @ dense_lap(g) @ R.T, rtol=1e-12, atol=1e-12)
    u = np.random.default_rng(1).standard_normal(nc)
    Lc_u = oracle.apply_L(c, u)
    Pu = R.T @ u
    assert u @ Lc_u == pytest.approx(Pu @ oracle.apply_L(g, Pu), rel=1e-12)


def test_post_smoothing_residual_through_w(oracle, inputs):
    """The identity behind the W = L P pass that starts post-smoothing (the
    CUDA cycle's reading of Section 3.6): after the coarse correction
    x = x_pre + P x_c, r_0 = f - L x equals r_pre - (L P) x_c, and
    (L P x_c)_i = sum_a W_ia (x_c[agg_i] - x_c[a]) with W_ia the weight from i
    into aggregate a != agg_i (the rows of L sum to zero, so the own aggregate
    drops out). Checked with numpy against dense products on the oracle's
    aggregates."""
    g = inputs.random_graph(500, 6, seed=13)
    S = oracle.strength(g, SEED, 0)
    nc, agg, _, _ = oracle.aggregate(g, S)
    L = dense_lap(g)
    P = np.zeros((g.n, nc))
    P[np.arange(g.n), agg] = 1.0
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    off = agg[g.col] != agg[rows]
    W = sp.csr_matrix((g.w[off], (rows[off], agg[g.col][off])), shape=(g.n, nc))  # equal keys summed
    assert W.nnz == len(set(zip(rows[off].tolist(), agg[g.col][off].tolist())))
    rng = np.random.default_rng(4)
    xc, xpre, f = rng.standard_normal(nc), rng.standard_normal(g.n), rng.standard_normal(g.n)
    lp_xc = np.asarray(W.sum(axis=1)).ravel() * xc[agg] - W @ xc
    np.testing.assert_allclose(lp_xc, L @ P @ xc, rtol=1e-12, atol=1e-12)
    r_pre = f - L @ xpre
    np.testing.assert_allclose(r_pre - lp_xc, f - L @ (xpre + P @ xc), rtol=1e-11, atol=1e-11)


# --------------------------------------------------------------------------
# Eigenvalue estimate and Chebyshev smoothing (Section 3.6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 5, 8, 11])
def test_lanczos_complete_graph(oracle, inputs, n):
    assert oracle.lanczos(inputs.complete(n)) == pytest.approx(n / (n - 1), rel=1e-12)


@pytest.mark.parametrize("g_name", ["path6", "cycle8", "grid3"])
def test_lanczos_bipartite_small(oracle, inputs, g_name):
    g = {"path6": inputs.path(6), "cycle8": inputs.cycle(8), "grid3": inputs.grid2d(3, 3)}[g_name]
    assert oracle.lanczos(g) == pytest.approx(2.0, rel=1e-10)


def test_lanczos_bounds(oracle, inputs):
    g = inputs.random_graph(300, 6, seed=2, weights="uniform")
    L = dense_lap(g)
    d = np.diag(L)
    lam_max = np.linalg.eigvalsh(L / np.sqrt(np.outer(d, d))).max()
    lam = oracle.lanczos(g)
    assert lam <= lam_max * (1 + 1e-12) and lam > 0.9 * lam_max
    rng = np.random.default_rng(3)
    for m in (1, 2, 5, 10):
        a, b = rng.standard_normal(m), rng.standard_normal(m - 1)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        assert oracle.tridiag_max(a, b) == pytest.approx(np.linalg.eigvalsh(T).max(), abs=1e-13)


def cheb_poly(mu, lam, lo, hi, k):
    a, b = lo * lam, hi * lam
    theta, delta = (a + b) / 2, (b - a) / 2
    Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
    return Tk((theta - mu) / delta) / Tk(theta / delta)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_chebyshev_error_polynomial(oracle, inputs, degree):
    n = 32
    g = inputs.cycle(n)
    i = np.arange(n)
    lam = 2.0  # lambda_max of D^-1 L on an even cycle
    for k in (2, 5, 9, 16):
        v = np.cos(2 * np.pi * k * i / n)
        mu = 1.0 - np.cos(2 * np.pi * k / n)
        f = oracle.apply_L(g, v)
        p = cheb_poly(mu, lam, 0.3, 1.1, degree)
        x, r = oracle.cheb_pre(g, lam, f, degree=degree)
        np.testing.assert_allclose(x, (1 - p) * v, atol=1e-12)  # error v - x = p(mu) v
        np.testing.assert_allclose(r, p * f, atol=1e-12)
        x2 = oracle.cheb_post(g, lam, f, 0.25 * v, degree=degree)
        np.testing.assert_allclose(v - x2, p * 0.75 * v, atol=1e-12)


# --------------------------------------------------------------------------
# Coarsest level, cycle, PCG
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 6])
def test_pinv_complete_graph(oracle, inputs, n):
    if n == 1:
        g = inputs.Graph(1, np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0))
    else:
        g = inputs.complete(n)
    np.testing.assert_allclose(oracle.pinv(g), (np.eye(n) - 1.0 / n) / n, atol=1e-14)


def test_pinv_random(oracle, inputs):
    g = inputs.random_graph(60, 4, seed=9, weights="uniform")
    np.testing.assert_allclose(oracle.pinv(g), np.linalg.pinv(dense_lap(g)), atol=1e-10)


def test_vcycle_symmetric_positive(oracle, inputs):
    g = inputs.random_graph(3000, 6, seed=4, weights="uniform")
    h = oracle.Hierarchy(g)
    assert h.nlevels >= 3
    rng = np.random.default_rng(5)
    u = rng.standard_normal(g.n); u -= u.mean()
    v = rng.standard_normal(g.n); v -= v.mean()
    Mu, Mv = h.vcycle(u), h.vcycle(v)
    assert abs(u @ Mv - v @ Mu) < 1e-10 * np.linalg.norm(Mu) * np.linalg.norm(v)
    assert u @ Mu > 0 and v @ Mv > 0


def test_hierarchy_structure(oracle, inputs):
    g = inputs.grid2d(64, 64)
    h = oracle.Hierarchy(g)
    kinds = [h.level(l).kind for l in range(h.nlevels)]
    assert kinds[0] == oracle.ELIM and kinds[-1] == oracle.COARSEST
    for a, b in zip(kinds, kinds[1:]):
        assert not (a == oracle.ELIM and b == oracle.ELIM)  # stages alternate
    last = h.level(h.nlevels - 1)
    assert last.a.nnz_off + last.a.n <= 1000
    for l in range(h.nlevels - 1):
        L = h.level(l)
        assert L.a.nnz_off + L.a.n > 1000 and h.level(l + 1).a.n == L.nc
        if L.kind == oracle.AGG:
            assert 1.0 < L.lam <= 2.0 + 1e-12  # lambda_max(D^-1 L) <= 2
    g3 = inputs.grid3d(12, 12, 12)
    assert oracle.Hierarchy(g3).level(0).kind == oracle.AGG  # elimination below the 5% gate


def test_pcg_grid_matches_dense(oracle, inputs):
    g = inputs.grid2d(64, 64)
    b = inputs.rhs(g.n, seed=2)
    h = oracle.Hierarchy(g)
    x, st, it, rel = h.pcg(b, tol=1e-8)
    assert st == oracle.OK and rel <= 1e-8 and it < 60
    Ls = laplacian(sp_adj(g))
    assert np.linalg.norm(b - Ls @ x) <= 1e-8 * np.linalg.norm(b)
    L = dense_lap(g)
    xs = np.linalg.solve(L + 1.0 / g.n, b)
    xs -= xs.mean()
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    xd = oracle.dense_solve(g, b)
    np.testing.assert_allclose(xd, xs, atol=1e-9 * np.abs(xs).max())


def test_pcg_power_law(oracle, inputs):
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    b = inputs.rhs(g.n, seed=2)
    h = oracle.Hierarchy(g)
    x, st, it, rel = h.pcg(b, tol=1e-8)
    assert st == oracle.OK and it < 40
    assert np.linalg.norm(b - laplacian(sp_adj(g)) @ x) <= 1e-8 * np.linalg.norm(b)


def test_setup_errors(oracle, inputs):
    with pytest.raises(RuntimeError, match="status 2"):
        g = inputs.random_graph(50, 2, seed=1)
        rp = np.concatenate([g.rowptr, [g.rowptr[-1]]])  # extra isolated vertex
        oracle.Hierarchy(inputs.Graph(g.n + 1, rp, g.col, g.w))
    with pytest.raises(RuntimeError, match="status 3"):
        oracle.Hierarchy(inputs.grid2d(30, 30), oracle.default_opts(max_levels=1, max_coarse_n=100))


# ---------------------------------------------------------------------------
# K-cycle (Section 3.7): two FCG iterations from x = 0 with a fixed linear
# preconditioner B give the L-orthogonal projection of the solution onto
# span{B f, B L B f}, x = V (V^T L V)^-1 V^T f. On a hierarchy whose second
# aggregation level sits right above the coarsest (exact) solve, that level's
# cycle body is linear, so the K-solve there is pinned by this closed form.
# ---------------------------------------------------------------------------
def _lap_dense(a):
    n = a.n
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(a.rowptr[i], a.rowptr[i + 1]):
            A[i, a.col[k]] -= a.w[k]
            A[i, i] += a.w[k]
    return A


@pytest.mark.parametrize("name", ["grid24", "rand800"])
def test_kcycle_two_fcg_steps_are_an_energy_projection(oracle, inputs, name):
    g = inputs.grid2d(24, 24) if name == "grid24" else inputs.random_graph(800, 6, seed=3)
    h = oracle.Hierarchy(g, oracle.default_opts(elim_enable=0, coarse_nnz=600, kcycle=1))
    kinds = [h.level(l).kind for l in range(h.nlevels)]
    assert kinds == [oracle.AGG, oracle.AGG, oracle.COARSEST]
    lv = h.level(1)
    n1 = lv.a.n
    A = _lap_dense(lv.a)
    B = np.column_stack([h.level_cycle(1, np.eye(n1)[j], body_only=True) for j in range(n1)])
    f = np.random.default_rng(5).standard_normal(n1)
    f -= f.mean()
    V = np.column_stack([B @ f, B @ (A @ (B @ f))])
    ref = V @ np.linalg.solve(V.T @ A @ V, V.T @ f)
    x = h.level_cycle(1, f)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # the first aggregation level is left to the outer Krylov method
    f0 = np.random.default_rng(6).standard_normal(g.n)
    f0 -= f0.mean()
    np.testing.assert_array_equal(h.level_cycle(0, f0), h.level_cycle(0, f0, body_only=True))
    # with the V-cycle every level is its body
    hv = oracle.Hierarchy(g, oracle.default_opts(elim_enable=0, coarse_nnz=600, kcycle=0))
    np.testing.assert_array_equal(hv.level_cycle(1, f), hv.level_cycle(1, f, body_only=True))


def test_kcycle_pcg_matches_dense(oracle, inputs):
    g = inputs.grid2d(64, 64)
    b = inputs.rhs(g.n, seed=2)
    h = oracle.Hierarchy(g, oracle.default_opts(kcycle=1))
    x, st, it, rel = h.pcg(b, tol=1e-8)
    assert st == oracle.OK and rel <= 1e-8
    ref = oracle.dense_solve(g, b)
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)
    _, _, it_v, _ = oracle.Hierarchy(g).pcg(b, tol=1e-8)
    assert it <= it_v  # the K-cycle is the stronger preconditioner here


# ---------------------------------------------------------------------------
# Repeated elimination rounds (Section 3.4). Elimination is exact (a Schur
# complement), so a hierarchy made only of elimination levels above the
# coarsest dense solve is a direct solver: one cycle gives L^+ f.
# ---------------------------------------------------------------------------
def test_elim_rounds_path_is_exact(oracle, inputs):
    g = inputs.path(2000)
    h = oracle.Hierarchy(g, oracle.default_opts(elim_rounds=20))
    kinds = [h.level(l).kind for l in range(h.nlevels)]
    assert kinds[-1] == oracle.COARSEST and all(k == oracle.ELIM for k in kinds[:-1])
    f = inputs.rhs(g.n, seed=3)
    ref = oracle.dense_solve(g, f)
    x = h.vcycle(f)
    # exact up to rounding: the path Laplacian's condition number is ~n^2 = 4e6, so both this and the
    # dense reference carry errors of order 4e6 * 1e-16; an inexact cycle would be off by ~1e-1
    assert np.linalg.norm(x - x.mean() - ref) <= 1e-8 * np.linalg.norm(ref)
    _, st, it, rel = h.pcg(f, tol=1e-8)
    assert st == oracle.OK and it == 1


@pytest.mark.parametrize("name", ["grid64", "chunglu"])
def test_elim_rounds_stop_at_the_gate(oracle, inputs, name):
    g = inputs.grid2d(64, 64) if name == "grid64" else inputs.chung_lu(20000, m_target=100000, seed=3)
    h = oracle.Hierarchy(g, oracle.default_opts(elim_rounds=20))
    kinds = [h.level(l).kind for l in range(h.nlevels)]
    for l, k in enumerate(kinds[:-1]):
        lv = h.level(l)
        G = inputs.Graph(lv.a.n, lv.a.rowptr, lv.a.col, lv.a.w)
        nf = int(oracle.elim_select(G, 4, 0x5EED).sum())
        if k == oracle.ELIM:
            assert nf > 0.05 * lv.a.n and lv.nc == lv.a.n - nf
        else:  # an aggregation level: the gate failed on it
            assert nf <= 0.05 * lv.a.n
    # one round is the default hierarchy
    h1 = oracle.Hierarchy(g, oracle.default_opts(elim_rounds=1))
    hd = oracle.Hierarchy(g)
    assert [h1.level(l).a.n for l in range(h1.nlevels)] == [hd.level(l).a.n for l in range(hd.nlevels)]


def test_setup_is_a_function_of_the_graph_and_the_seed(oracle, inputs):
    """Two setups of one graph with one seed give the same hierarchy, bit for
    bit (every random choice comes from the counter-based streams); another
    seed changes the random choices (elimination hashes, test vectors)."""
    g = inputs.chung_lu(3000, m_target=15000, seed=11)

    def levels(seed):
        o = oracle.default_opts()
        o.seed = seed
        H = oracle.Hierarchy(g, o)
        out = []
        for l in range(H.nlevels):
            L = H.level(l)
            out.append((L.kind, L.a.rowptr.copy(), L.a.col.copy(), L.a.w.copy(),
                        None if L.map is None else L.map.copy(), L.lam))
        return out

    a, b, c = levels(0x5EED), levels(0x5EED), levels(12345)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x[0] == y[0] and x[5] == y[5]
        for p, q in zip(x[1:5], y[1:5]):
            assert (p is None and q is None) or np.array_equal(p, q)
    differs = len(a) != len(c) or any(
        x[4] is not None and y[4] is not None and not np.array_equal(x[4], y[4]) for x, y in zip(a, c))
    assert differs


# ---------------------------------------------------------------------------
# The composition of the cycle (Algorithm 1 with Sections 3.4-3.6), pinned
# against a dense two-grid operator assembled here in numpy from its parts:
# the degree-2 Chebyshev smoother as a matrix polynomial (numpy's Chebyshev
# basis), R = P^T from the aggregates, the dense Galerkin product P^T L P and
# numpy's pseudo-inverse of it. Only the aggregates and the eigenvalue
# estimate come from the oracle (both pinned on their own above).
# ---------------------------------------------------------------------------
def _cheb_smoother(L, lam, lo=0.3, hi=1.1, degree=2):
    """S with x = S f the Chebyshev smoother from x = 0 on D^-1 L over
    [lo lam, hi lam]: the error after `degree` steps is r(D^-1 L) e with
    r(t) = T_k((theta - t) / delta) / T_k(theta / delta), so the iterate is
    s(D^-1 L) D^-1 f with s(t) = (1 - r(t)) / t, a polynomial since r(0) = 1."""
    from numpy.polynomial import Chebyshev, Polynomial

    a, b = lo * lam, hi * lam
    theta, delta = (b + a) / 2, (b - a) / 2
    Tk = Chebyshev.basis(degree).convert(kind=Polynomial)
    u = Polynomial([theta / delta, -1.0 / delta])          # t -> (theta - t) / delta
    r = Tk(u) / Tk(theta / delta)
    s, rem = divmod(Polynomial([1.0]) - r, Polynomial([0.0, 1.0]))
    assert np.allclose(rem.coef, 0.0, atol=1e-12 * np.abs(r.coef).max())
    Dinv = np.diag(1.0 / np.diag(L))
    A = Dinv @ L
    S = np.zeros_like(L)
    Ak = np.eye(L.shape[0])
    for c in s.coef:
        S += c * Ak
        Ak = Ak @ A
    return S @ Dinv


def _agg_two_grid(L, agg, nc, lam, coarse):
    """x = M f for one aggregation level over a coarse solve `coarse`:
    pre-smooth, restrict the residual by R = P^T, coarse solve, prolong,
    post-smooth from the current x."""
    n = L.shape[0]
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = 1.0
    S = _cheb_smoother(L, lam)

    def M(f):
        x = S @ f
        xc = coarse(P.T @ (f - L @ x))
        x = x + P @ xc
        return x + S @ (f - L @ x)

    return M, P


def _pinv_solve(Lc):
    # the Laplacian of a connected graph has one zero eigenvalue; rounding
    # leaves it at ~1e-16 of the largest, so the cut-off drops it explicitly
    Lp = np.linalg.pinv(Lc, rcond=1e-10, hermitian=True)
    return lambda fc: Lp @ fc


@pytest.mark.parametrize("name", ["grid2d_16", "random_150_weighted"])
def test_vcycle_equals_dense_two_grid(oracle, inputs, name):
    g = inputs.grid2d(16, 16) if name == "grid2d_16" else inputs.random_graph(150, 6, seed=21, weights="uniform")
    h = oracle.Hierarchy(g, oracle.default_opts(elim_enable=0))
    assert [h.level(l).kind for l in range(h.nlevels)] == [oracle.AGG, oracle.COARSEST]
    lv = h.level(0)
    L = dense_lap(g)
    P = np.zeros((g.n, lv.nc))
    P[np.arange(g.n), lv.map] = 1.0
    M, _ = _agg_two_grid(L, lv.map, lv.nc, lv.lam, _pinv_solve(P.T @ L @ P))
    rng = np.random.default_rng(7)
    for _ in range(3):
        f = rng.standard_normal(g.n)
        f -= f.mean()
        want = M(f)
        got = h.vcycle(f)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_vcycle_equals_dense_three_level(oracle, inputs):
    """An elimination level over an aggregation level over the coarsest: the
    elimination level's additive form x = Fsmooth(f) + P_e M_agg(P_e^T f)
    (Section 3.4) with P_e = [L_FF^-1 A_FC ; I] built densely from the
    eliminated set, the coarse operator as the dense Schur complement."""
    g = inputs.grid2d(24, 24)  # every vertex a candidate: level 0 eliminates ~1/5
    h = oracle.Hierarchy(g)
    kinds = [h.level(l).kind for l in range(h.nlevels)]
    assert kinds == [oracle.ELIM, oracle.AGG, oracle.COARSEST]
    L = dense_lap(g)
    e = h.level(0)
    F = np.flatnonzero(e.map < 0)
    C = np.flatnonzero(e.map >= 0)
    assert np.array_equal(e.map[C], np.arange(len(C)))  # kept vertices numbered in order
    Pe = np.zeros((g.n, len(C)))
    Pe[C, e.map[C]] = 1.0
    dF = np.diag(L)[F]
    Pe[F] = -L[np.ix_(F, C)] / dF[:, None]
    Lc = Pe.T @ L @ Pe                                  # = the Schur complement (F independent)
    a = h.level(1)
    Pa = np.zeros((len(C), a.nc))
    Pa[np.arange(len(C)), a.map] = 1.0
    Magg, _ = _agg_two_grid(Lc, a.map, a.nc, a.lam, _pinv_solve(Pa.T @ Lc @ Pa))

    def M(f):
        x = Pe @ Magg(Pe.T @ f)
        x[F] += f[F] / dF
        return x

    rng = np.random.default_rng(8)
    for _ in range(3):
        f = rng.standard_normal(g.n)
        f -= f.mean()
        want = M(f)
        got = h.vcycle(f)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
