"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer work (degrees, elimination sets, aggregates given the same strength
values) must match bit for bit. Floating-point results are compared with
tolerances derived from the arithmetic:
  * one SpMV / strength pass in FP64: |diff| <= 1e-12 relative to the row scale
    (a few ulps of a reordered sum of O(degree) terms);
  * coarse operators: 1e-12 relative (sums of at most a few thousand terms);
  * Lanczos estimate: 1e-9 relative (10 steps amplify rounding mildly);
  * solves: true relative residual <= 1e-8 (recomputed here with scipy), and
    the mean-removed solution within 1e-6 relative of the oracle's reference
    solution (dense direct solve, or oracle PCG at tol 1e-12).
"""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian

pytestmark = pytest.mark.gpu

SEED = 0x5EED


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relres(g, b, x):
    A = sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))
    bm = b - b.mean()
    return np.linalg.norm(bm - laplacian(A) @ x) / np.linalg.norm(bm)


GRAPHS = {
    "grid2d_20": lambda I: I.grid2d(20, 20),
    "grid3d_8": lambda I: I.grid3d(8, 8, 8),
    "random_3k": lambda I: I.random_graph(3000, 5, seed=3),
    "chunglu_20k": lambda I: I.chung_lu(20000, m_target=100000, seed=3),
    "rmat_12": lambda I: I.rmat(12, seed=2),
    "star_5000": lambda I: I.star(5000),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_laplacian_apply(torch_cuda, lgmod, oracle, inputs, name):
    torch = torch_cuda
    g = GRAPHS[name](inputs)
    x = np.random.default_rng(1).standard_normal(g.n)
    y = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    lgmod.lg_laplacian_apply(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.w), dev(torch, x), y)
    ref = oracle.apply_L(g, x)
    scale = np.abs(g.w).max() * (np.abs(x).max()) * np.diff(g.rowptr).clip(1)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * scale)


SEG_GRAPHS = {  # every row above 2048 entries and a short vector: the long rows go column-segmented
    "complete_3000w": lambda I: I.complete(3000, weights="uniform", seed=5),
}


@pytest.mark.parametrize("name", ["chunglu_20k", "star_5000", "rmat_12", "complete_3000w"])
def test_level_apply_matches_oracle(torch_cuda, lgmod, oracle, inputs, name):
    """lg_level_apply on every non-coarsest level (the cycle's tuned plans,
    chunked long rows included) against the oracle's L x on that level's CSR:
    FP64 within a few ulps of the row scale, FP32 within its own rounding
    (2^-24 per term, O(degree) terms, the difference form's x_i - x_j)."""
    torch = torch_cuda
    g = {**GRAPHS, **SEG_GRAPHS}[name](inputs)
    H = lgmod.Hierarchy(g)
    if name in SEG_GRAPHS:
        assert lgmod.lg_level_plan(H.h, 0)["seg_tiles"] > 0
    rng = np.random.default_rng(4)
    for l in range(H.nlevels - 1):
        rp, cl, w, _ = H.level(l)
        G = inputs.Graph(len(rp) - 1, rp, cl, w)
        x = rng.standard_normal(G.n)
        ref = oracle.apply_L(G, x)
        scale = np.abs(w).max(initial=0.0) * np.abs(x).max() * np.diff(rp).clip(1)
        y = torch.zeros(G.n, dtype=torch.float64, device="cuda")
        lgmod.lg_level_apply(H.h, l, lgmod.FP64, dev(torch, x), y)
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * scale), l
        x32 = x.astype(np.float32)
        ref32 = oracle.apply_L(G, x32.astype(np.float64))
        y32 = torch.zeros(G.n, dtype=torch.float32, device="cuda")
        lgmod.lg_level_apply(H.h, l, lgmod.FP32_HIER, dev(torch, x32), y32)
        assert np.all(np.abs(y32.cpu().numpy() - ref32) <= 2e-6 * scale), l
    with pytest.raises(lgmod.LGError):
        lgmod.lg_level_apply(H.h, H.nlevels - 1, lgmod.FP64, y, y)  # the coarsest has no row pass
    H.close()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_elim_select_bit_exact(torch_cuda, lgmod, oracle, inputs, name):
    torch = torch_cuda
    g = GRAPHS[name](inputs)
    is_f = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
    nf = lgmod.lg_elim_select(g.n, dev(torch, g.rowptr), dev(torch, g.col), 4, SEED, is_f)
    ref = oracle.elim_select(g, 4, SEED)
    np.testing.assert_array_equal(is_f.cpu().numpy(), ref)
    assert nf == int(ref.sum())


@pytest.mark.parametrize("name", list(GRAPHS))
def test_strength_and_aggregation(torch_cuda, lgmod, oracle, inputs, name):
    torch = torch_cuda
    g = GRAPHS[name](inputs)
    rp, cl, w = dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.w)
    S = torch.zeros(max(g.nnz_off, 1), dtype=torch.float64, device="cuda")
    lgmod.lg_strength(g.n, rp, cl, w, SEED, 3, 4, 3, 2.0 / 3.0, S)
    S_gpu = S.cpu().numpy()[: g.nnz_off]
    S_ref = oracle.strength(g, SEED, 3)
    np.testing.assert_allclose(S_gpu, S_ref, rtol=0, atol=1e-12)
    # aggregation on identical strength values: bit-exact
    agg = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    st = torch.zeros(g.n, dtype=torch.int8, device="cuda")
    votes = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    nc = lgmod.lg_aggregate(g.n, rp, cl, S, 10, 8, agg, st, votes)
    nc_ref, agg_ref, st_ref, votes_ref = oracle.aggregate(g, S_gpu)
    assert nc == nc_ref
    np.testing.assert_array_equal(agg.cpu().numpy(), agg_ref)
    np.testing.assert_array_equal(st.cpu().numpy(), st_ref)
    np.testing.assert_array_equal(votes.cpu().numpy(), votes_ref)


def renumbered(g, perm):
    """The graph with vertex i of the result being vertex perm[i] of g."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(g.n, dtype=perm.dtype)
    rows = inv[np.repeat(np.arange(g.n), np.diff(g.rowptr))].astype(np.int64)
    cols = inv[g.col].astype(np.int64)
    order = np.lexsort((cols, rows))
    rp = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=g.n), out=rp[1:])
    return rp, cols[order].astype(np.int32), g.w[order]


def same_csr(a_rp, a_cl, a_w, b, rtol=1e-12):
    np.testing.assert_array_equal(a_rp, b.rowptr)
    np.testing.assert_array_equal(a_cl, b.col)
    np.testing.assert_allclose(a_w, b.w, rtol=rtol, atol=0)


@pytest.mark.parametrize("name", ["grid2d_20", "grid3d_8", "random_3k", "chunglu_20k", "rmat_12"])
def test_hierarchy_per_level_reinjection(torch_cuda, lgmod, oracle, inputs, name):
    """Each GPU level, fed to the oracle's stage, reproduces the GPU's next level."""
    torch = torch_cuda
    g = GRAPHS[name](inputs)
    H = lgmod.Hierarchy(g)
    nl = H.nlevels
    assert nl >= 2
    for l in range(nl):
        info = H.level_info(l)
        rp, cl, w, mp = H.level(l)
        G = inputs.Graph(info["n"], rp, cl, w)
        if l == 0:
            prp, pcl, pw = renumbered(g, H.permutation())
            np.testing.assert_array_equal(rp, prp)
            np.testing.assert_array_equal(cl, pcl)
            np.testing.assert_array_equal(w, pw)
        if info["kind"] == lgmod.LEVEL_ELIM:
            is_f = oracle.elim_select(G, 4, SEED)
            np.testing.assert_array_equal((mp < 0).astype(np.uint8), is_f)
            coarse, cmap = oracle.schur(G, is_f)
            np.testing.assert_array_equal(mp, cmap)
            nrp, ncl, nw, _ = H.level(l + 1)
            same_csr(nrp, ncl, nw, coarse)
        elif info["kind"] == lgmod.LEVEL_AGG:
            S = torch.zeros(max(G.nnz_off, 1), dtype=torch.float64, device="cuda")
            lgmod.lg_strength(G.n, dev(torch, rp), dev(torch, cl), dev(torch, w), SEED, l, 4, 3, 2.0 / 3.0, S)
            S_gpu = S.cpu().numpy()[: G.nnz_off]
            np.testing.assert_allclose(S_gpu, oracle.strength(G, SEED, l), rtol=0, atol=1e-12)
            nc_ref, agg_ref, _, _ = oracle.aggregate(G, S_gpu)
            assert info["nc"] == nc_ref
            np.testing.assert_array_equal(mp, agg_ref)
            nrp, ncl, nw, _ = H.level(l + 1)
            same_csr(nrp, ncl, nw, oracle.galerkin(G, agg_ref, nc_ref))
            lam_ref = oracle.lanczos(G, SEED, l)
            assert info["lambda"] == pytest.approx(lam_ref, rel=1e-9)
        else:
            assert l == nl - 1
            assert info["nnz"] + info["n"] <= 1000 or nl == 64
            P = lgmod.lg_coarsest_pinv(H.h, info["n"])
            np.testing.assert_allclose(P, oracle.pinv(G), rtol=0, atol=1e-9 * max(1.0, np.abs(P).max()))
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_grid64_matches_dense(lgmod, oracle, inputs, prec):
    g = inputs.grid2d(64, 64)
    b = inputs.rhs(g.n, seed=2)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g, precision=p)
    x, info = H.solve(b, tol=1e-8)
    assert info.status == lgmod.OK
    assert relres(g, b, x) <= 1e-8
    assert abs(info.relres - relres(g, b, x)) <= 1e-10
    ref = oracle.dense_solve(g, b)
    assert np.linalg.norm(x - x.mean() - ref) <= 1e-6 * np.linalg.norm(ref)
    assert abs(x.mean()) < 1e-12
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["chunglu_20k", "rmat_12", "grid3d_8", "star_5000"])
def test_solve_matches_oracle_pcg(lgmod, oracle, inputs, name, prec):
    g = GRAPHS[name](inputs)
    b = inputs.rhs(g.n, seed=5)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g, precision=p)
    x, info = H.solve(b, tol=1e-8)
    assert info.status == lgmod.OK and relres(g, b, x) <= 1e-8
    ref, st, it, rel = oracle.Hierarchy(g).pcg(b, tol=1e-12, maxit=1000)
    assert st == oracle.OK
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)
    H.close()


def test_vcycle_fp64_matches_oracle_cycle(lgmod, oracle, inputs):
    """Where the oracle builds the identical hierarchy, one V-cycle agrees to rounding."""
    g = inputs.random_graph(3000, 6, seed=4, weights="uniform")
    H = lgmod.Hierarchy(g, reorder=0)  # the oracle works in the caller's numbering
    R = oracle.Hierarchy(g)
    assert H.nlevels == R.nlevels
    for l in range(H.nlevels):
        rp, cl, w, mp = H.level(l)
        Lr = R.level(l)
        np.testing.assert_array_equal(rp, Lr.a.rowptr)
        np.testing.assert_array_equal(cl, Lr.a.col)
        if mp is not None:
            np.testing.assert_array_equal(mp, Lr.map)
    f = inputs.rhs(g.n, seed=9)
    xg = H.vcycle(f, lgmod.FP64)
    xr = R.vcycle(f)
    assert np.linalg.norm(xg - xr) <= 1e-11 * np.linalg.norm(xr)
    x32 = H.vcycle(f, lgmod.FP32_HIER)
    assert np.linalg.norm(x32 - xr) <= 1e-4 * np.linalg.norm(xr)
    H.close()


def test_vcycle_with_w_pass_matches_oracle_cycle(lgmod, oracle, inputs):
    """As above on a graph large enough for the W = L P post-smoothing pass
    (the oracle computes r_0 = f - L x directly)."""
    g = inputs.random_graph(9000, 6, seed=6, weights="uniform")
    H = lgmod.Hierarchy(g, reorder=0)
    R = oracle.Hierarchy(g)
    assert H.nlevels == R.nlevels
    for l in range(H.nlevels):
        rp, cl, w, mp = H.level(l)
        Lr = R.level(l)
        np.testing.assert_array_equal(rp, Lr.a.rowptr)
        np.testing.assert_array_equal(cl, Lr.a.col)
        if mp is not None:
            np.testing.assert_array_equal(mp, Lr.map)
    assert sum(H.level_lp_nnz(l) for l in range(H.nlevels)) > 0
    f = inputs.rhs(g.n, seed=9)
    xg = H.vcycle(f, lgmod.FP64)
    xr = R.vcycle(f)
    assert np.linalg.norm(xg - xr) <= 1e-11 * np.linalg.norm(xr)
    x32 = H.vcycle(f, lgmod.FP32_HIER)
    assert np.linalg.norm(x32 - xr) <= 1e-4 * np.linalg.norm(xr)
    H.close()


def test_edge_cases(lgmod, inputs):
    one = inputs.Graph(1, np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0))
    H = lgmod.Hierarchy(one)
    x, info = H.solve(np.array([3.0]))
    assert info.status == lgmod.OK and x[0] == 0.0
    H.close()
    p2 = inputs.path(2)
    H = lgmod.Hierarchy(p2)
    x, info = H.solve(np.array([1.0, -1.0]))
    assert info.status == lgmod.OK and np.allclose(x, [0.5, -0.5])
    H.close()
    g = inputs.grid2d(10, 10)
    H = lgmod.Hierarchy(g)
    x, info = H.solve(np.ones(g.n))  # b is constant: zero after projection
    assert info.status == lgmod.OK and info.iterations == 0 and np.all(x == 0)
    H.close()
    # disconnected and malformed graphs
    rp = np.concatenate([g.rowptr, [g.rowptr[-1]]])
    with pytest.raises(lgmod.LGError) as e:
        lgmod.Hierarchy(inputs.Graph(g.n + 1, rp, g.col, g.w))
    assert e.value.status == lgmod.ERR_DISCONNECTED
    bad = g.w.copy()
    bad[0] = 2.0
    with pytest.raises(lgmod.LGError) as e:
        lgmod.Hierarchy(inputs.Graph(g.n, g.rowptr, g.col, bad))
    assert e.value.status == lgmod.ERR_INVALID
    badc = g.col.copy()
    badc[3] = g.n + 5
    with pytest.raises(lgmod.LGError) as e:
        lgmod.Hierarchy(inputs.Graph(g.n, g.rowptr, badc, g.w))
    assert e.value.status == lgmod.ERR_INVALID
    # a self-loop, a repeated column, a negative weight
    for mutate in ("self", "dup", "neg"):
        c2, w2 = g.col.copy(), g.w.copy()
        r = 55  # an interior vertex with four neighbours
        k0 = g.rowptr[r]
        if mutate == "self":
            c2[k0] = r
        elif mutate == "dup":
            c2[k0 + 1] = c2[k0]
        else:
            w2[k0] = -w2[k0]
        with pytest.raises(lgmod.LGError) as e:
            lgmod.Hierarchy(inputs.Graph(g.n, g.rowptr, c2, w2))
        assert e.value.status == lgmod.ERR_INVALID, mutate


def test_deterministic(lgmod, inputs):
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    b = inputs.rhs(g.n, seed=1)
    xs = []
    for _ in range(2):
        H = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER)
        xs.append(H.solve(b)[0])
        H.close()
    np.testing.assert_array_equal(xs[0], xs[1])


def test_device_pointers(torch_cuda, lgmod, inputs):
    torch = torch_cuda
    g = inputs.grid2d(30, 30)
    H = lgmod.Hierarchy(n=g.n, rowptr=dev(torch, g.rowptr), col=dev(torch, g.col), w=dev(torch, g.w))
    b = inputs.rhs(g.n, seed=3)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    info = lgmod.lg_solve(H.h, dev(torch, b), x, 1e-8)
    xh, _ = H.solve(b)
    np.testing.assert_array_equal(x.cpu().numpy(), xh)
    assert info.status == lgmod.OK
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_loop_matches_host_loop(lgmod, inputs, prec):
    """The PCG loop replayed as one CUDA graph (device-side WHILE node) gives
    bitwise the same iterate and iteration count as the host-driven loop."""
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    b = inputs.rhs(g.n, seed=4)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    out = []
    for use_graphs in (1, 0):
        H = lgmod.Hierarchy(g, precision=p, use_graphs=use_graphs)
        x, info = H.solve(b)
        x2, info2 = H.solve(b)  # the second solve replays the cached graph
        np.testing.assert_array_equal(x, x2)
        out.append((x, info.iterations, info.relres))
        H.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


def test_max_iter_and_tolerance(lgmod, inputs):
    g = inputs.grid2d(40, 40)
    b = inputs.rhs(g.n, seed=6)
    H = lgmod.Hierarchy(g, max_iter=3)
    x, info = H.solve(b, check=False)
    assert info.status == lgmod.ERR_NOT_CONVERGED and info.iterations == 3 and info.relres > 1e-8
    H.close()
    H = lgmod.Hierarchy(g)
    x1, i1 = H.solve(b, tol=1e-4)
    x2, i2 = H.solve(b, tol=1e-10)
    assert i1.relres <= 1e-4 and i2.relres <= 1e-10 and i2.iterations > i1.iterations
    H.close()


@pytest.mark.parametrize("name", ["chunglu_20k", "grid3d_8", "star_5000"])
def test_degree_renumbering(lgmod, oracle, inputs, name):
    """The renumbering is a permutation by non-increasing degree (ties by id),
    and solves with and without it agree within the solve tolerance."""
    g = GRAPHS[name](inputs)
    H = lgmod.Hierarchy(g)
    perm = H.permutation()
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    deg = np.diff(g.rowptr)[perm]
    assert np.all(deg[:-1] >= deg[1:])
    same = deg[:-1] == deg[1:]
    assert np.all(perm[:-1][same] < perm[1:][same])
    b = inputs.rhs(g.n, seed=8)
    x1, i1 = H.solve(b)
    H.close()
    H0 = lgmod.Hierarchy(g, reorder=0)
    assert np.array_equal(H0.permutation(), np.arange(g.n))
    x0, i0 = H0.solve(b)
    H0.close()
    assert relres(g, b, x1) <= 1e-8 and relres(g, b, x0) <= 1e-8
    assert np.linalg.norm(x1 - x0) <= 1e-6 * np.linalg.norm(x0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [2, 5, 32])
@pytest.mark.parametrize("name", ["chunglu_20k", "grid3d_8", "star_5000"])
def test_solve_batch_matches_single(lgmod, oracle, inputs, name, k, prec):
    """Multi-RHS solve (SpMM cycles, per-column CG scalars): every column meets
    the tolerance and agrees with the single-RHS solve of that column."""
    g = GRAPHS[name](inputs)
    B = inputs.rhs(g.n, k, seed=11)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g, precision=p)
    X, infos = H.solve_batch(B)
    ref_pcg = oracle.Hierarchy(g)
    for c in range(k):
        assert infos[c].status == lgmod.OK and infos[c].relres <= 1e-8
        assert relres(g, B[:, c], X[:, c]) <= 1e-8
        xs, inf = H.solve(np.ascontiguousarray(B[:, c]))
        assert abs(infos[c].iterations - inf.iterations) <= 1
        assert np.linalg.norm(X[:, c] - xs) <= 1e-6 * np.linalg.norm(xs)
        if c < 2:
            xr, st, _, _ = ref_pcg.pcg(np.ascontiguousarray(B[:, c]), tol=1e-12, maxit=1000)
            assert np.linalg.norm(X[:, c] - xr) <= 1e-6 * np.linalg.norm(xr)
    H.close()


def test_batch_plan_reports_schedule(lgmod, inputs):
    """lg_batch_plan: refused before the first multi-column solve builds the
    plans; afterwards the operator plan of every aggregation level (and of
    the finest) has a stretch length from the tuner's set and virtual rows at
    least its rows, and a level with W = L P has a W plan too."""
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    H = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER)
    with pytest.raises(lgmod.LGError):
        lgmod.lg_batch_plan(H.h, 0)
    H.solve_batch(inputs.rhs(g.n, 4, seed=2))
    for l in range(H.nlevels):
        info, plan = H.level_info(l), lgmod.lg_batch_plan(H.h, l)
        if info["kind"] == lgmod.LEVEL_AGG or l == 0:
            assert plan["op_ch"] in (64, 256, 1024) and plan["op_vrows"] >= info["n"]
        else:
            assert plan["op_ch"] == 0 and plan["op_vrows"] == 0
        assert plan["w_ch"] in (0, 64, 256, 1024)
    assert any(lgmod.lg_batch_plan(H.h, l)["w_vrows"] > 0 for l in range(H.nlevels))
    H.close()


def test_batch_columns_independent(lgmod, inputs):
    g = inputs.grid2d(48, 48)
    B = inputs.rhs(g.n, 4, seed=12)
    B[:, 1] = 0.0      # zero right-hand side: done at once
    B[:, 2] = 3.0      # constant: zero after the projection
    B[:, 3] *= 1e-6    # tiny but nonzero: same relative tolerance
    H = lgmod.Hierarchy(g)
    X, infos = H.solve_batch(B)
    assert [i.status for i in infos] == [lgmod.OK] * 4
    assert infos[1].iterations == 0 and infos[2].iterations == 0
    assert np.all(X[:, 1] == 0) and np.all(X[:, 2] == 0)
    assert infos[0].iterations > 0 and abs(infos[3].iterations - infos[0].iterations) <= 1
    assert relres(g, np.ascontiguousarray(B[:, 3]), X[:, 3]) <= 1e-8
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["chunglu_20k", "grid3d_8"])
def test_vcycle_batch_matches_single(lgmod, inputs, name, prec):
    """The multi-column cycle applies the same preconditioner to every column."""
    g = GRAPHS[name](inputs)
    F = inputs.rhs(g.n, 3, seed=13)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g)
    X = H.vcycle_batch(F, p)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for c in range(3):
        xs = H.vcycle(np.ascontiguousarray(F[:, c]), p)
        assert np.linalg.norm(X[:, c] - xs) <= tol * np.linalg.norm(xs), c
    H.close()


# ---------------------------------------------------------------------------
# K-cycle (Section 3.7): every aggregation level below the first solved by two
# FCG iterations preconditioned by its own cycle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,n", [(4, 3000), (5, 6000)])
def test_kcycle_matches_oracle(lgmod, oracle, inputs, seed, n):
    """Where the oracle builds the identical hierarchy, one application of the
    K-cycle preconditioner agrees to rounding (FP64)."""
    g = inputs.random_graph(n, 6, seed=seed, weights="uniform")
    H = lgmod.Hierarchy(g, reorder=0, kcycle=1)
    R = oracle.Hierarchy(g, oracle.default_opts(kcycle=1))
    assert H.nlevels == R.nlevels
    kinds = [R.level(l).kind for l in range(R.nlevels)]
    assert kinds.count(oracle.AGG) >= 2  # the K-cycle acts below the first aggregation level
    for l in range(H.nlevels):
        rp, cl, w, mp = H.level(l)
        Lr = R.level(l)
        np.testing.assert_array_equal(rp, Lr.a.rowptr)
        np.testing.assert_array_equal(cl, Lr.a.col)
        if mp is not None:
            np.testing.assert_array_equal(mp, Lr.map)
    f = inputs.rhs(g.n, seed=9)
    xr = R.vcycle(f)
    assert np.linalg.norm(xr - oracle.Hierarchy(g).vcycle(f)) > 1e-6 * np.linalg.norm(xr)  # differs from V
    xg = H.vcycle(f, lgmod.FP64)
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
    x32 = H.vcycle(f, lgmod.FP32_HIER)
    assert np.linalg.norm(x32 - xr) <= 1e-3 * np.linalg.norm(xr)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["grid2d_64", "grid3d_16", "chunglu_20k"])
def test_kcycle_solve(lgmod, oracle, inputs, name, prec):
    g = {"grid2d_64": lambda: inputs.grid2d(64, 64), "grid3d_16": lambda: inputs.grid3d(16, 16, 16),
         "chunglu_20k": lambda: inputs.chung_lu(20000, m_target=100000, seed=3)}[name]()
    b = inputs.rhs(g.n, seed=2)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g, precision=p, kcycle=1)
    x, info = H.solve(b, tol=1e-8)
    assert info.status == lgmod.OK
    assert relres(g, b, x) <= 1e-8
    R = oracle.Hierarchy(g, oracle.default_opts(kcycle=1))
    xr, st, it, _ = R.pcg(b, tol=1e-12)
    xr -= xr.mean()
    assert np.linalg.norm(x - x.mean() - xr) <= 1e-6 * np.linalg.norm(xr)
    _, _, it8, _ = R.pcg(b, tol=1e-8)
    assert abs(info.iterations - it8) <= (1 if prec == "fp64" else 3)
    H.close()


def test_kcycle_batch_runs_columns(lgmod, inputs):
    g = inputs.grid3d(12, 12, 12)
    B = inputs.rhs(g.n, 3, seed=4)
    H = lgmod.Hierarchy(g, kcycle=1)
    X, infos = H.solve_batch(B)
    for c in range(3):
        assert infos[c].status == lgmod.OK
        xs, _ = H.solve(np.ascontiguousarray(B[:, c]))
        np.testing.assert_array_equal(X[:, c], xs)
    H.close()


# ---------------------------------------------------------------------------
# Repeated elimination rounds (Section 3.4).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["path_3000", "grid2d_20", "chunglu_20k"])
def test_elim_rounds_hierarchy(torch_cuda, lgmod, oracle, inputs, name):
    """With several rounds, each elimination level matches the oracle's Schur
    complement of the GPU's previous level (reinjection), and the kinds of the
    levels match the oracle's hierarchy."""
    g = {"path_3000": lambda: inputs.path(3000), "grid2d_20": lambda: inputs.grid2d(20, 20),
         "chunglu_20k": lambda: inputs.chung_lu(20000, m_target=100000, seed=3)}[name]()
    H = lgmod.Hierarchy(g, elim_rounds=8, reorder=0)  # the oracle hashes the caller's vertex ids
    R = oracle.Hierarchy(g, oracle.default_opts(elim_rounds=8))
    kinds = [H.level_info(l)["kind"] for l in range(H.nlevels)]
    assert kinds == [R.level(l).kind for l in range(R.nlevels)]
    assert kinds.count(lgmod.LEVEL_ELIM) > (1 if name != "grid2d_20" else 0)
    for l in range(H.nlevels - 1):
        if kinds[l] != lgmod.LEVEL_ELIM:
            continue
        rp, cl, w, mp = H.level(l)
        G = inputs.Graph(len(rp) - 1, rp, cl, w)
        is_f = oracle.elim_select(G, 4, SEED)
        np.testing.assert_array_equal((mp < 0).astype(np.uint8), is_f)
        coarse, cmap = oracle.schur(G, is_f)
        nrp, ncl, nw, _ = H.level(l + 1)
        same_csr(nrp, ncl, nw, coarse)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_elim_rounds_path_solve_is_direct(lgmod, oracle, inputs, prec):
    """Only elimination levels over the dense coarsest solve: one cycle is the
    exact solve, so PCG converges in one iteration."""
    g = inputs.path(2000)
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    H = lgmod.Hierarchy(g, elim_rounds=20, precision=p)
    kinds = [H.level_info(l)["kind"] for l in range(H.nlevels)]
    assert kinds[-1] == lgmod.LEVEL_COARSEST and all(k == lgmod.LEVEL_ELIM for k in kinds[:-1])
    b = inputs.rhs(g.n, seed=3)
    x, info = H.solve(b, tol=1e-8)
    assert info.status == lgmod.OK and relres(g, b, x) <= 1e-8
    if prec == "fp64":
        assert info.iterations == 1
    ref = oracle.dense_solve(g, b)
    assert np.linalg.norm(x - x.mean() - ref) <= 1e-6 * np.linalg.norm(ref)
    H.close()


# ---------------------------------------------------------------------------
# Work units (Section 2.3.1, WDA): recomputed here from the level structure.
# ---------------------------------------------------------------------------
def _iteration_work(lgmod, H, kcycle, deg=2):
    """A level with W = L P starts post-smoothing with a pass over W, whose
    cost is nnz(W) + n in place of one Laplacian pass."""
    lv = [H.level_info(l) for l in range(H.nlevels)]
    first_agg = next((l for l, d in enumerate(lv) if d["kind"] == lgmod.LEVEL_AGG), -1)

    def solve(l):
        d = lv[l]
        A = d["nnz"] + d["n"]
        if d["kind"] == lgmod.LEVEL_COARSEST:
            return d["n"] ** 2
        if d["kind"] == lgmod.LEVEL_ELIM:
            rp, _, _, mp = H.level(l)
            nnz_f = int(np.diff(rp)[mp < 0].sum())
            return 2 * nnz_f + d["nc"] + d["n"] + solve(l + 1)
        body = 2 * deg * A + 2 * d["n"] + solve(l + 1)
        w = H.level_lp_nnz(l)
        if w > 0:
            body += w + d["n"] - A
        return 2 * body + 2 * A if (kcycle and l != first_agg) else body

    A0 = lv[0]["nnz"] + lv[0]["n"]
    return (A0 + solve(0)) / A0


@pytest.mark.parametrize("kcycle", [0, 1])
def test_work_units(lgmod, inputs, kcycle):
    g = inputs.grid3d(16, 16, 16)
    H = lgmod.Hierarchy(g, kcycle=kcycle)
    b = inputs.rhs(g.n, seed=2)
    _, info = H.solve(b)
    w = _iteration_work(lgmod, H, kcycle)
    assert info.work_units == pytest.approx(info.iterations * w, rel=1e-12)
    wda = info.work_units / -np.log10(info.relres)
    assert 1.0 < wda < 1000.0
    X, infos = H.solve_batch(inputs.rhs(g.n, 2, seed=5))
    for inf in infos:
        assert inf.work_units == pytest.approx(inf.iterations * w, rel=1e-12)
    H.close()


@pytest.mark.parametrize("name", ["chunglu_20k", "grid3d_8", "rmat_12"])
def test_random_ordering(lgmod, oracle, inputs, name):
    """reorder = 2 (Section 3.3's random ordering): the permutation sorts the
    vertices by the counter-based hash of the seed and id (recomputed here with
    the published SplitMix64), level 0 is the graph in that numbering, and the
    solve agrees with the oracle's solution."""
    g = GRAPHS[name](inputs)
    H = lgmod.Hierarchy(g, reorder=2)
    perm = H.permutation()
    ids = np.arange(g.n, dtype=np.uint64)
    counter = (np.uint64(9) << np.uint64(56)) | ids
    keys = np.array([oracle.splitmix64(SEED, int(c)) >> 32 for c in counter], dtype=np.uint64)
    expect = np.lexsort((ids, keys))  # by key, then by id
    np.testing.assert_array_equal(perm, expect)
    prp, pcl, pw = renumbered(g, perm)
    rp, cl, w, _ = H.level(0)
    np.testing.assert_array_equal(rp, prp)
    np.testing.assert_array_equal(cl, pcl)
    np.testing.assert_array_equal(w, pw)
    b = inputs.rhs(g.n, seed=8)
    x, info = H.solve(b)
    assert info.status == lgmod.OK and relres(g, b, x) <= 1e-8
    xr, _, _, _ = oracle.Hierarchy(g).pcg(b, tol=1e-12)
    xr -= xr.mean()
    assert np.linalg.norm(x - x.mean() - xr) <= 1e-6 * np.linalg.norm(xr)
    H.close()


LP_GRAPHS = {
    "chunglu_20k": GRAPHS["chunglu_20k"],
    "grid3d_16": lambda I: I.grid3d(16, 16, 16),
    "random_8k": lambda I: I.random_graph(8000, 5, seed=5),
}


@pytest.mark.parametrize("name", list(LP_GRAPHS))
def test_lp_residual(lgmod, inputs, name):
    """Post-smoothing from r_0 = r_pre - (L P) x_c (lp_residual = 1) against
    r_0 = f - L x (lp_residual = 0): W = L P has one entry per (row, other
    aggregate among the row's neighbours) (counted here with numpy), the FP64
    cycles agree to rounding, and both solves converge in the same number of
    iterations. (test_vcycle_fp64_matches_oracle_cycle checks the default,
    W-based, cycle against the oracle's.)"""
    g = LP_GRAPHS[name](inputs)
    H1 = lgmod.Hierarchy(g, lp_residual=1)
    H0 = lgmod.Hierarchy(g, lp_residual=0)
    assert H1.nlevels == H0.nlevels
    built = 0
    for l in range(H1.nlevels):
        d = H1.level_info(l)
        assert H0.level_lp_nnz(l) == 0
        if d["kind"] != lgmod.LEVEL_AGG or d["n"] < 4096:  # W only on aggregation levels of >= 4096 vertices
            assert H1.level_lp_nnz(l) == 0
            continue
        rp, cl, _, agg = H1.level(l)
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        off = agg[cl] != agg[rows]
        pairs = np.unique(rows[off].astype(np.int64) * (int(agg.max()) + 1) + agg[cl][off])
        assert H1.level_lp_nnz(l) == pairs.size
        built += pairs.size > 0
    assert built > 0
    f = inputs.rhs(g.n, seed=12)
    x1 = H1.vcycle(f, lgmod.FP64)
    x0 = H0.vcycle(f, lgmod.FP64)
    assert np.linalg.norm(x1 - x0) <= 1e-11 * np.linalg.norm(x0)
    for prec in (lgmod.FP64, lgmod.FP32_HIER):
        _, i1 = H1.solve(f, precision=prec)
        _, i0 = H0.solve(f, precision=prec)
        assert i1.status == lgmod.OK and i0.status == lgmod.OK
        assert abs(i1.iterations - i0.iterations) <= 1
    H1.close()
    H0.close()


def test_segmented_long_rows_solve(torch_cuda, lgmod, oracle, inputs):
    """Solves through a hierarchy whose finest operator serves its long rows
    column-segmented (every pass of level 0: the Chebyshev steps, the
    residuals, the PCG's q = L p, the true residual) reach the tolerance and
    the oracle's solution, in both precisions, and repeat bit for bit."""
    g = SEG_GRAPHS["complete_3000w"](inputs)
    H = lgmod.Hierarchy(g)
    assert lgmod.lg_level_plan(H.h, 0)["seg_tiles"] > 0
    b = inputs.rhs(g.n, seed=6)
    ref = oracle.dense_solve(g, b)
    for prec in (lgmod.FP64, lgmod.FP32_HIER):
        x, info = H.solve(b, precision=prec)
        assert info.status == lgmod.OK and relres(g, b, x) <= 1e-8
        xm = x - x.mean()
        assert np.linalg.norm(xm - ref) <= 1e-6 * np.linalg.norm(ref)
        x2, info2 = H.solve(b, precision=prec)
        np.testing.assert_array_equal(x2, x)
    H.close()
