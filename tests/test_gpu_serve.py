"""The continuous-batching server (lg_serve_*).

Requests on graphs of different sizes arrive while others are running; each
must be admitted as slots and budget free up, join other requests in one
multi-column batch (same hierarchy) or one packed launch (single columns on
small graphs), overlap on the device with the others, and give the same
result as when it runs alone. A column is computed the same way whatever it
is grouped with and every reduction is in a fixed order, so "the same" is
bitwise here; each result is also checked for a true relative residual
<= 1e-8 recomputed with scipy, and against the oracle's solution.
"""

import time

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian

pytestmark = pytest.mark.gpu

TOL = 1e-8

GRAPHS = {
    "grid2d_40": lambda I: I.grid2d(40, 40),
    "grid3d_12": lambda I: I.grid3d(12, 12, 12),
    "chunglu_30k": lambda I: I.chung_lu(30000, m_target=150000, seed=5),
    "rmat_13": lambda I: I.rmat(13, seed=4),
}


def rhs2(inputs, n, k, seed):
    return inputs.rhs(n, k, seed=seed).reshape(n, k)


def relres_cols(g, B, X):
    A = laplacian(sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n)))
    Bm = B - B.mean(axis=0)
    return np.linalg.norm(Bm - A @ X, axis=0) / np.linalg.norm(Bm, axis=0)


@pytest.fixture(scope="module")
def graphs(lgmod, inputs):
    out = {}
    for name, make in GRAPHS.items():
        g = make(inputs)
        out[name] = (g, lgmod.Hierarchy(g))
    yield out
    for _, H in out.values():
        H.close()


def request_mix(graphs, inputs, count, seed):
    rng = np.random.default_rng(seed)
    names = list(graphs)
    reqs = []
    for q in range(count):
        name = names[q % len(names)]
        k = int(rng.integers(1, 5))
        reqs.append((name, rhs2(inputs, graphs[name][0].n, k, 100 + q)))
    order = rng.permutation(count)
    return [reqs[i] for i in order]


@pytest.fixture(scope="module")
def oracle_x(oracle, graphs):
    """The oracle's solution of a column (PCG to 1e-12), per graph."""
    hs = {name: oracle.Hierarchy(g) for name, (g, _) in graphs.items()}

    def solve(name, b):
        x, st, it, rel = hs[name].pcg(b, tol=1e-12, maxit=1000)
        assert st == oracle.OK
        return x - x.mean()

    return solve


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_serve_same_alone_and_in_mix(lgmod, inputs, graphs, oracle_x, prec):
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    reqs = request_mix(graphs, inputs, 16, seed=7)

    alone = []
    sv = lgmod.Server(slots=1, precision=p)
    for _, H in graphs.values():
        sv.register(H)
    for name, B in reqs:  # one at a time: nothing else on the device
        t = sv.submit(graphs[name][1], B, TOL)
        X, info = sv.wait(t)
        assert info.status == lgmod.OK
        alone.append(X)
    sv.close()

    sv = lgmod.Server(slots=4, precision=p)
    for _, H in graphs.values():
        sv.register(H)
    tickets = [sv.submit(graphs[name][1], B, TOL) for name, B in reqs]  # all in flight together
    mixed = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()

    assert st.completed == len(reqs) and st.failed == 0
    for (name, B), Xa, (Xm, info) in zip(reqs, alone, mixed):
        assert info.status == lgmod.OK
        assert np.array_equal(Xa, Xm), name
        assert relres_cols(graphs[name][0], B, Xm).max() <= TOL * 1.0001
        assert np.abs(Xm.mean(axis=0)).max() <= 1e-12 * np.abs(Xm).max()
        for c in range(B.shape[1]):
            ref = oracle_x(name, B[:, c])
            assert np.linalg.norm(Xm[:, c] - ref) <= 1e-6 * np.linalg.norm(ref), name


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_serve_merges_and_packs(lgmod, inputs, graphs, prec):
    """Requests queued behind a running one are taken together: the ones on
    one hierarchy as one multi-column batch, the single columns on small
    graphs as one packed launch; results equal those of each request alone."""
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    g_big, H_big = graphs["chunglu_30k"]
    smalls = ["grid2d_40", "grid3d_12", "rmat_13"]
    reqs = [("chunglu_30k", rhs2(inputs, g_big.n, 2, 200 + q)) for q in range(4)]  # 8 columns: one batch
    reqs += [(name, rhs2(inputs, graphs[name][0].n, 1, 300 + q)) for q, name in enumerate(smalls)]
    sv = lgmod.Server(slots=1, precision=p)
    for _, H in graphs.values():
        sv.register(H)
    alone = []
    for name, B in reqs:
        X, info = sv.wait(sv.submit(graphs[name][1], B, TOL))
        assert info.status == lgmod.OK
        alone.append(X)
    sv.close()
    sv = lgmod.Server(slots=1, precision=p)
    for _, H in graphs.values():
        sv.register(H)
    blocker = sv.submit(H_big, rhs2(inputs, g_big.n, 8, 99), TOL)  # holds the one slot while the rest queue up
    tickets = [sv.submit(graphs[name][1], B, TOL) for name, B in reqs]
    sv.wait(blocker)
    mixed = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()
    assert st.completed == len(reqs) + 1
    assert st.packed_groups >= 1
    assert st.groups <= 3  # the blocker, one batch of the four requests on one graph, one packed launch
    for (name, B), Xa, (Xm, info) in zip(reqs, alone, mixed):
        assert info.status == lgmod.OK
        assert np.array_equal(Xa, Xm), name


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_columns_independent_of_width(lgmod, inputs, prec):
    """lg_solve_batch's columns do not depend on the batch: 5 columns solved
    together equal the same columns solved as batches of 2 and 3."""
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    H = lgmod.Hierarchy(g)
    B = inputs.rhs(g.n, 5, seed=8).reshape(g.n, 5)
    X5, i5 = H.solve_batch(B, precision=p)
    X2, i2 = H.solve_batch(np.ascontiguousarray(B[:, :2]), precision=p)
    X3, i3 = H.solve_batch(np.ascontiguousarray(B[:, 2:]), precision=p)
    np.testing.assert_array_equal(X5, np.concatenate([X2, X3], axis=1))
    assert [i.iterations for i in i5] == [i.iterations for i in i2 + i3]
    H.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_serve_least_work_policy(lgmod, inputs, graphs, oracle_x, prec):
    """Policy least work first: with the one slot held, three long requests
    (8 columns each, so none merge) and then a short one queue up. Under
    arrival order the short request is served last; under least work it
    leads the next group and finishes before every queued long one. Each
    result is bitwise the same under both policies (a column does not depend
    on its group) and matches the oracle."""
    p = lgmod.FP64 if prec == "fp64" else lgmod.FP32_HIER
    g_big, H_big = graphs["chunglu_30k"]
    g_s, H_s = graphs["grid2d_40"]
    longs = [rhs2(inputs, g_big.n, 8, 400 + q) for q in range(3)]
    Bs = rhs2(inputs, g_s.n, 2, 500)
    runs = {}
    for pol in (lgmod.SERVE_ARRIVAL, lgmod.SERVE_LEAST_WORK):
        sv = lgmod.Server(slots=1, precision=p, policy=pol)
        for _, H in graphs.values():
            sv.register(H)
        blocker = sv.submit(H_big, rhs2(inputs, g_big.n, 8, 99), TOL)
        tl = [sv.submit(H_big, B, TOL) for B in longs]
        ts = sv.submit(H_s, Bs, TOL)
        outs = [sv.wait(t) for t in tl]
        short = sv.wait(ts)
        sv.wait(blocker)
        sv.close()
        assert all(i.status == lgmod.OK for _, i in outs) and short[1].status == lgmod.OK
        runs[pol] = (outs, short)
    arr_long, arr_short = runs[lgmod.SERVE_ARRIVAL]
    lw_long, lw_short = runs[lgmod.SERVE_LEAST_WORK]
    assert arr_short[1].solve_ms > max(i.solve_ms for _, i in arr_long)
    assert lw_short[1].solve_ms < min(i.solve_ms for _, i in lw_long)
    for (Xa, _), (Xl, _) in zip(arr_long, lw_long):
        assert np.array_equal(Xa, Xl)
    assert np.array_equal(arr_short[0], lw_short[0])
    for c in range(Bs.shape[1]):
        ref = oracle_x("grid2d_40", Bs[:, c])
        assert np.linalg.norm(lw_short[0][:, c] - ref) <= 1e-6 * np.linalg.norm(ref)


def test_serve_least_work_ages_passed_requests(lgmod, inputs, graphs):
    """Under least work first a long request is passed by every short one,
    but only 16 times: with the one slot held, a long request and then 90
    single-column requests on the small graphs (packed, at most one per graph
    and group) queue up; the long request leads once 16 groups have started
    ahead of it, so it finishes before the last of the short ones, after at
    most 16 groups of them."""
    g_big, H_big = graphs["chunglu_30k"]
    smalls = ["grid2d_40", "grid3d_12", "rmat_13"]
    sv = lgmod.Server(slots=1, precision=lgmod.FP32_HIER, policy=lgmod.SERVE_LEAST_WORK)
    for _, H in graphs.values():
        sv.register(H)
    blocker = sv.submit(H_big, rhs2(inputs, g_big.n, 8, 98), TOL)
    t_long = time.perf_counter()
    tl = sv.submit(H_big, rhs2(inputs, g_big.n, 8, 97), TOL)
    shorts = []
    for q in range(90):
        name = smalls[q % 3]
        shorts.append((time.perf_counter(), sv.submit(graphs[name][1], rhs2(inputs, graphs[name][0].n, 1, 600 + q),
                                                       TOL)))
    _, info_l = sv.wait(tl)
    done_long = t_long + info_l.solve_ms * 1e-3
    done_short = []
    for t0, t in shorts:
        _, inf = sv.wait(t)
        assert inf.status == lgmod.OK
        done_short.append(t0 + inf.solve_ms * 1e-3)
    sv.wait(blocker)
    st = sv.stats()
    sv.close()
    assert info_l.status == lgmod.OK
    before = sum(d < done_long for d in done_short)
    assert before < len(done_short)  # not starved: some short requests finish after it
    assert before <= 16 * 3  # at most 16 groups of at most one request per small graph went first
    assert st.packed_groups >= 16


def test_serve_short_request_overtakes_long(lgmod, inputs):
    """A short request submitted right after a long one finishes first: it is
    admitted into a free slot while the long one is still on the device."""
    big = inputs.chung_lu(300000, m_target=2000000, seed=9)
    small = inputs.grid2d(32, 32)
    Hb, Hs = lgmod.Hierarchy(big), lgmod.Hierarchy(small)
    sv = lgmod.Server(slots=2, precision=lgmod.FP64)
    sv.register(Hb)
    sv.register(Hs)
    Bb = rhs2(inputs, big.n, 8, 1)
    Bs = rhs2(inputs, small.n, 1, 2)
    tb = sv.submit(Hb, Bb, TOL)
    ts = sv.submit(Hs, Bs, TOL)
    Xs, infs = sv.wait(ts)
    Xb, infb = sv.wait(tb)
    sv.close()
    assert infs.status == lgmod.OK and infb.status == lgmod.OK
    assert infs.solve_ms < infb.solve_ms  # latency from submission
    assert relres_cols(small, Bs, Xs).max() <= TOL * 1.0001
    assert relres_cols(big, Bb, Xb).max() <= TOL * 1.0001
    Hb.close()
    Hs.close()


def test_serve_admission_budget(lgmod, inputs, graphs):
    """With a budget that holds the hierarchies and one request's workspace,
    requests run one at a time (never two in flight) and all complete."""
    g, H = graphs["chunglu_30k"]
    hb, _ = lgmod.lg_hier_bytes(H.h)
    req = lgmod.lg_serve_request_bytes(H.h, 2)
    assert req > 0
    sv = lgmod.Server(slots=4, precision=lgmod.FP32_HIER, hbm_budget_bytes=float(hb + 1.5 * req))
    sv.register(H)
    assert sv.stats().resident_bytes == hb
    Bs = [rhs2(inputs, g.n, 2, 30 + q) for q in range(6)]
    tickets = [sv.submit(H, B, TOL) for B in Bs]
    max_running = 0
    results = {}
    t0 = time.monotonic()
    while len(results) < len(tickets) and time.monotonic() - t0 < 120:
        max_running = max(max_running, sv.stats().running)
        for t in tickets:
            if t not in results:
                X, info = sv.poll(t)
                if X is not None:
                    results[t] = (X, info)
    st = sv.stats()
    # a request that could never fit the budget is refused at submission
    with pytest.raises(lgmod.LGError) as e:
        sv.submit(H, inputs.rhs(g.n, 32, seed=1), TOL)
    assert e.value.status == lgmod.ERR_NOMEM
    sv.close()
    assert len(results) == len(tickets)
    assert max_running <= 1
    assert st.completed == len(tickets) and st.failed == 0
    assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
    for t, B in zip(tickets, Bs):
        X, info = results[t]
        assert info.status == lgmod.OK
        assert relres_cols(g, B, X).max() <= TOL * 1.0001


def test_serve_errors(lgmod, inputs, graphs):
    g, H = graphs["grid2d_40"]
    sv = lgmod.Server(slots=1)
    with pytest.raises(lgmod.LGError) as e:  # not registered
        sv.submit(H, inputs.rhs(g.n, 1, seed=1), TOL)
    assert e.value.status == lgmod.ERR_INVALID
    with pytest.raises(lgmod.LGError):
        lgmod.lg_serve_poll(sv.s, 12345)  # unknown ticket
    sv.register(H)
    t = sv.submit(H, inputs.rhs(g.n, 1, seed=1), TOL)
    sv.wait(t)
    with pytest.raises(lgmod.LGError):
        lgmod.lg_serve_poll(sv.s, t)  # a ticket is polled done once
    sv.close()
    # the budget refuses a hierarchy that does not fit
    sv = lgmod.Server(slots=1, hbm_budget_bytes=1000.0)
    with pytest.raises(lgmod.LGError) as e:
        sv.register(H)
    assert e.value.status == lgmod.ERR_NOMEM
    sv.close()
