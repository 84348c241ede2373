"""Degenerate and extreme inputs through the C ABI, against the oracle.

Each case is a shape the method meets at its edges: a graph small enough to
be its own coarsest level, dense rows, a row spanning dozens of chunks,
a long chain between dense blocks, weights over six orders of magnitude
(solved) and over twelve (beyond the method, as for the oracle: reported
as not converged), the widest batch, and iteration limits of zero and one.
"""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian

pytestmark = pytest.mark.gpu


def relres(g, b, x):
    A = sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))
    bm = b - b.mean()
    return np.linalg.norm(bm - laplacian(A) @ x) / np.linalg.norm(bm)


def check_solve(lgmod, oracle, g, b, tol=1e-8, compare_x=True, **kw):
    H = lgmod.Hierarchy(g, **kw)
    x, info = H.solve(b, tol=tol)
    assert info.status == lgmod.OK
    assert relres(g, b, x) <= tol * 1.0001
    ref = oracle.dense_solve(g, b) if (compare_x and g.n <= 4096) else None
    if ref is not None:
        assert np.linalg.norm(x - x.mean() - ref) <= 1e-6 * max(np.linalg.norm(ref), 1e-300)
    H.close()
    return info


def test_small_graph_is_its_own_coarsest(lgmod, oracle, inputs):
    g = inputs.random_graph(60, 4, seed=2)  # nnz + n well below the coarsest threshold
    H = lgmod.Hierarchy(g)
    assert H.nlevels == 1 and H.level_info(0)["kind"] == lgmod.LEVEL_COARSEST
    b = inputs.rhs(g.n, seed=1)
    x, info = H.solve(b)
    assert info.status == lgmod.OK and info.iterations == 1
    ref = oracle.dense_solve(g, b)
    assert np.linalg.norm(x - x.mean() - ref) <= 1e-10 * np.linalg.norm(ref)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_complete_graph(lgmod, oracle, inputs, prec):
    g = inputs.complete(300)  # dense rows of 299 entries
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    check_solve(lgmod, oracle, g, inputs.rhs(g.n, seed=3), precision=p)


def test_star_with_a_row_of_many_chunks(lgmod, inputs):
    g = inputs.star(100000)  # hub row: 100,000 entries, ~49 chunks of 2048
    b = inputs.rhs(g.n, seed=4)
    H = lgmod.Hierarchy(g)
    x, info = H.solve(b)
    assert info.status == lgmod.OK and relres(g, b, x) <= 1e-8
    # the exact solution of a unit star: x_leaf = b_leaf - ... has a closed form
    # (L x = b with the hub at index 0 after renumbering); check against scipy
    A = laplacian(sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))).tocsc()
    bm = b - b.mean()
    Ar = A[1:, 1:]
    xr = np.zeros(g.n)
    xr[1:] = sp.linalg.spsolve(Ar, bm[1:])
    xr -= xr.mean()
    assert np.linalg.norm(x - x.mean() - xr) <= 1e-6 * np.linalg.norm(xr)
    H.close()


def test_barbell(lgmod, oracle, inputs):
    """Two 40-cliques joined by a 400-vertex path: dense blocks, a long chain,
    a bottleneck edge."""
    k, L = 40, 400
    u, v = [], []
    for off in (0, k + L):
        for i in range(k):
            for j in range(i + 1, k):
                u.append(off + i)
                v.append(off + j)
    chain = [k - 1] + list(range(k, k + L)) + [k + L]
    u += chain[:-1]
    v += chain[1:]
    g = inputs.from_edges(2 * k + L, np.array(u), np.array(v), weights="uniform", seed=5)
    for kw in ({}, {"elim_rounds": 8}, {"kcycle": 1}):
        check_solve(lgmod, oracle, g, inputs.rhs(g.n, seed=6), **kw)


def _spread_weights(inputs, decades, seed=7):
    """The 40x40 grid with one weight per undirected edge, log-uniform over
    10^-decades .. 10^decades."""
    g = inputs.grid2d(40, 40)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    lo, hi = np.minimum(rows, g.col), np.maximum(rows, g.col)
    _, inv = np.unique(lo * g.n + hi, return_inverse=True)
    wk = 10.0 ** rng.uniform(-decades, decades, size=inv.max() + 1)
    return inputs.Graph(g.n, g.rowptr, g.col, wk[inv])


def test_weights_over_six_orders(lgmod, oracle, inputs):
    g = _spread_weights(inputs, 3)
    b = inputs.rhs(g.n, seed=8)
    # the condition number is far beyond 1e6 here, so a dense solve is no reference for x;
    # the residual (recomputed with scipy) is the check, and the oracle's iteration count
    info = check_solve(lgmod, oracle, g, b, tol=1e-8, compare_x=False)
    _, st, it, _ = oracle.Hierarchy(g).pcg(b, tol=1e-8, maxit=500)
    assert st == oracle.OK
    assert abs(info.iterations - it) <= 0.1 * it


def test_weights_over_twelve_orders_do_not_converge(lgmod, oracle, inputs):
    """Beyond the method's reach (the oracle does not converge either): the
    library stops at max_iter with LG_ERR_NOT_CONVERGED, a finite iterate and
    the true residual of that iterate."""
    g = _spread_weights(inputs, 6)
    b = inputs.rhs(g.n, seed=8)
    _, st, _, rel_o = oracle.Hierarchy(g).pcg(b, tol=1e-8, maxit=100)
    assert st == oracle.NOT_CONVERGED and rel_o > 1e-8
    H = lgmod.Hierarchy(g, max_iter=100)
    x, info = H.solve(b, check=False)
    assert info.status == lgmod.ERR_NOT_CONVERGED and info.iterations == 100
    assert np.all(np.isfinite(x))
    assert info.relres == pytest.approx(relres(g, b, x), rel=1e-6)
    H.close()


def test_widest_batch(lgmod, inputs):
    g = inputs.chung_lu(5000, m_target=25000, seed=9)
    B = inputs.rhs(g.n, 32, seed=10)
    H = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER)
    X, infos = H.solve_batch(B)
    for c in range(32):
        assert infos[c].status == lgmod.OK
        assert relres(g, B[:, c], X[:, c]) <= 1e-8 * 1.0001
    with pytest.raises(lgmod.LGError):
        H.solve_batch(inputs.rhs(g.n, 33, seed=10))  # beyond the widest column block
    H.close()


def test_iteration_limits(lgmod, inputs):
    g = inputs.grid2d(30, 30)
    b = inputs.rhs(g.n, seed=11)
    H = lgmod.Hierarchy(g, max_iter=0)
    x, info = H.solve(b, check=False)
    assert info.status == lgmod.ERR_NOT_CONVERGED and info.iterations == 0
    assert info.relres == pytest.approx(1.0, rel=1e-12)  # x = 0
    H.close()
    H = lgmod.Hierarchy(g, max_iter=1)
    x, info = H.solve(b, check=False)
    assert info.status == lgmod.ERR_NOT_CONVERGED and info.iterations == 1
    assert info.relres == pytest.approx(relres(g, b, x), rel=1e-9)
    H.close()
