"""Many small solves in one launch (lg_solve_many): each graph's result
against the oracle's dense solve and against lg_solve on the same hierarchy,
over a mix of graph types, both cycle precisions, the K-cycle, repeated
elimination, device vectors, more graphs than the GPU holds blocks at once,
and the degenerate cases (zero right-hand side, iteration limits, rejected
arguments)."""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian

pytestmark = pytest.mark.gpu


def relres(g, b, x):
    A = sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))
    bm = b - b.mean()
    return np.linalg.norm(bm - laplacian(A) @ x) / np.linalg.norm(bm)


def mix(inputs):
    gs = inputs.serving_mix(20, 200, 6000, seed=21)
    gs += [inputs.complete(60), inputs.star(3000), inputs.random_graph(60, 4, seed=2),
           inputs.road_like(40, 40, seed=3), inputs.grid2d(30, 30)]
    return gs


def check_against_single(lgmod, oracle, g, H, b, x, info, tol=1e-8):
    assert info.status == lgmod.OK
    rr = relres(g, b, x)
    assert rr <= tol * 1.0001
    assert info.relres == pytest.approx(rr, rel=1e-6, abs=1e-14)
    assert abs(x.mean()) <= 1e-12 * max(np.abs(x).max(), 1.0)
    x1, i1 = H.solve(b, tol=tol)
    # the same arithmetic up to the order of additions: the same iteration
    # count unless a residual lands within rounding of the tolerance (then
    # one more iteration's correction separates the two results)
    assert abs(info.iterations - i1.iterations) <= 1
    same = info.iterations == i1.iterations
    assert np.linalg.norm(x - x1) <= (1e-9 if same else 1e-5) * np.linalg.norm(x1)
    if g.n <= 2000:
        ref = oracle.dense_solve(g, b)
        assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_many_match_oracle_and_single_solves(lgmod, oracle, inputs, prec):
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    gs = mix(inputs)
    Hs = [lgmod.Hierarchy(g, precision=p) for g in gs]
    bs = [inputs.rhs(g.n, seed=30 + i) for i, g in enumerate(gs)]
    xs, infos = lgmod.solve_many(Hs, bs)
    assert len({H.nlevels for H in Hs}) > 1  # hierarchies of different depths in one launch
    for g, H, b, x, info in zip(gs, Hs, bs, xs, infos):
        check_against_single(lgmod, oracle, g, H, b, x, info)
        H.close()


def test_many_mixed_options_in_one_launch(lgmod, oracle, inputs):
    """FP64 and FP32 cycles, the K-cycle, several elimination rounds, a
    graph that is its own coarsest level and a degree-3 smoother together."""
    gs = [inputs.grid2d(40, 40), inputs.chung_lu(3000, m_target=15000, seed=3), inputs.road_like(50, 50, seed=4),
          inputs.random_graph(60, 4, seed=2), inputs.grid3d(12, 12, 12), inputs.chung_lu(5000, m_target=25000, seed=5)]
    kws = [dict(precision=lgmod.FP32_HIER), dict(kcycle=1), dict(elim_rounds=4, precision=lgmod.FP32_HIER),
           dict(), dict(cheb_degree=3), dict(kcycle=1, precision=lgmod.FP32_HIER)]
    Hs = [lgmod.Hierarchy(g, **kw) for g, kw in zip(gs, kws)]
    assert Hs[3].nlevels == 1
    bs = [inputs.rhs(g.n, seed=50 + i) for i, g in enumerate(gs)]
    xs, infos = lgmod.solve_many(Hs, bs)
    for g, H, b, x, info in zip(gs, Hs, bs, xs, infos):
        check_against_single(lgmod, oracle, g, H, b, x, info)
        H.close()


def fuzz_graphs(inputs, count=60, seed=77):
    """Small graphs of six shapes, sizes and weights drawn from one seed."""
    rng = np.random.default_rng(seed)
    gs = []
    for q in range(count):
        n = int(rng.integers(8, 2500))
        kind = q % 6
        if kind == 0:
            g = inputs.random_graph(n, float(rng.uniform(2.5, 12.0)), seed=q + 1)
        elif kind == 1:
            g = inputs.chung_lu(max(n, 60), m_target=5 * max(n, 60), seed=q + 1)
        elif kind == 2:
            side = max(2, int(np.sqrt(n)))
            g = inputs.grid2d(side, side + int(rng.integers(0, 5)), weights="uniform", seed=q + 1)
        elif kind == 3:
            g = inputs.path(n, weights="uniform", seed=q + 1)
        elif kind == 4:
            g = inputs.star(max(n // 4, 3), weights="uniform", seed=q + 1)
        else:
            g = inputs.cycle(n, weights="uniform", seed=q + 1)
        gs.append(g)
    return gs


def test_fuzz_small_graphs_against_the_oracle(lgmod, oracle, inputs):
    """Sixty seeded small graphs (random, power-law, grids, paths, stars,
    cycles; unit and spread weights), both cycle precisions, solved in one
    packed launch: each solution against the oracle's dense solve. Solved to
    1e-10 so that the error bound kappa * relres stays below 1e-6 on the
    grids (kappa about 2.4e3 at 50 x 54)."""
    gs = fuzz_graphs(inputs)
    Hs = [lgmod.Hierarchy(g, precision=lgmod.FP32_HIER if q % 2 else lgmod.FP64) for q, g in enumerate(gs)]
    bs = [inputs.rhs(g.n, seed=500 + q) for q, g in enumerate(gs)]
    xs, infos = lgmod.solve_many(Hs, bs, tol=1e-10)
    for q, (g, b, x, info) in enumerate(zip(gs, bs, xs, infos)):
        assert info.status == lgmod.OK, (q, g.name)
        assert relres(g, b, x) <= 1e-10 * 1.0001, (q, g.name)
        ref = oracle.dense_solve(g, b)
        assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref), (q, g.name)
    for H in Hs:
        H.close()


def test_many_device_vectors(lgmod, inputs, torch_cuda):
    torch = torch_cuda
    gs = inputs.serving_mix(6, 300, 3000, seed=8)
    Hs = [lgmod.Hierarchy(g) for g in gs]
    bs = [inputs.rhs(g.n, seed=60 + i) for i, g in enumerate(gs)]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xd = [torch.zeros(g.n, dtype=torch.float64, device="cuda") for g in gs]
    infos = lgmod.lg_solve_many([H.h for H in Hs], bd, xd)
    for g, b, x, info in zip(gs, bs, xd, infos):
        assert info.status == lgmod.OK
        assert relres(g, b, x.cpu().numpy()) <= 1e-8 * 1.0001
    for H in Hs:
        H.close()


def test_more_graphs_than_resident_blocks(lgmod, inputs):
    """700 graphs: more blocks than the GPU runs at once, so blocks start as
    earlier ones finish."""
    gs = [inputs.grid2d(8 + i % 9, 8 + i % 7) if i % 2 else inputs.chung_lu(300 + 7 * (i % 40), m_target=1500,
                                                                           seed=100 + i) for i in range(700)]
    Hs = [lgmod.Hierarchy(g, precision=lgmod.FP32_HIER if i % 3 else lgmod.FP64) for i, g in enumerate(gs)]
    bs = [inputs.rhs(g.n, seed=i) for i, g in enumerate(gs)]
    xs, infos = lgmod.solve_many(Hs, bs)
    for g, b, x, info in zip(gs, bs, xs, infos):
        assert info.status == lgmod.OK
        assert relres(g, b, x) <= 1e-8 * 1.0001
    for H in Hs:
        H.close()


def test_many_degenerate_cases(lgmod, inputs):
    g = inputs.grid2d(30, 30)
    H0 = lgmod.Hierarchy(g)
    H1 = lgmod.Hierarchy(g, max_iter=1)
    H2 = lgmod.Hierarchy(g, max_iter=0)
    H3 = lgmod.Hierarchy(g)
    b = inputs.rhs(g.n, seed=11)
    bs = [np.full(g.n, 3.0), b, b, b]  # a constant b projects to zero
    xs, infos = lgmod.solve_many([H0, H1, H2, H3], bs, check=False)
    assert infos[0].status == lgmod.OK and infos[0].iterations == 0 and np.all(xs[0] == 0.0)
    assert infos[1].status == lgmod.ERR_NOT_CONVERGED and infos[1].iterations == 1
    assert infos[1].relres == pytest.approx(relres(g, b, xs[1]), rel=1e-9)
    assert infos[2].status == lgmod.ERR_NOT_CONVERGED and infos[2].iterations == 0
    assert infos[2].relres == pytest.approx(1.0, rel=1e-12) and np.all(xs[2] == 0.0)
    assert infos[3].status == lgmod.OK
    # the first failing status in argument order
    st = lgmod.lib().lg_solve_many(4, (lgmod.C.c_void_p * 4)(H0.h.value, H1.h.value, H2.h.value, H3.h.value),
                                   (lgmod.C.c_void_p * 4)(*[b.ctypes.data] * 4),
                                   (lgmod.C.c_void_p * 4)(*[x.ctypes.data for x in xs]), 1e-8, None)
    assert st == lgmod.ERR_NOT_CONVERGED
    with pytest.raises(lgmod.LGError) as e:
        lgmod.solve_many([H0, H3, H0], [b, b, b])  # a repeated handle
    assert e.value.status == lgmod.ERR_INVALID
    with pytest.raises(lgmod.LGError) as e:
        lgmod.solve_many([H0], [b], tol=0.0)
    assert e.value.status == lgmod.ERR_INVALID
    for H in (H0, H1, H2, H3):
        H.close()


def test_graph_over_the_size_limit_rejected(lgmod, inputs):
    g = inputs.grid2d(1100, 1100)  # nnz(L_0) = 5.8M > 2^22
    H = lgmod.Hierarchy(g)
    with pytest.raises(lgmod.LGError) as e:
        lgmod.solve_many([H], [inputs.rhs(g.n)])
    assert e.value.status == lgmod.ERR_INVALID
    H.close()
