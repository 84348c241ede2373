"""Constant-weight finest operators (option const_weights): a graph whose
weights are all one value keeps only the pattern of L_0 and applies the value
as a constant. The solves must equal, bit for bit, those of the same
hierarchy with the weights stored, in both precisions, batched, packed with
other graphs and after a save and load; lg_level_copy must give the value
back; and the device bytes must drop by the weight arrays."""

import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _scaled(g, v):
    return dataclasses.replace(g, w=np.full_like(g.w, v))


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_HIER"])
@pytest.mark.parametrize("value", [1.0, 2.5])
def test_const_weights_same_bits(lgmod, inputs, prec_name, value, tmp_path):
    prec = getattr(lgmod, prec_name)
    g = _scaled(inputs.chung_lu(30000, m_target=150000, seed=4), value)
    stored = lgmod.Hierarchy(g, precision=prec, const_weights=0)
    pattern = lgmod.Hierarchy(g, precision=prec)
    assert pattern.nlevels == stored.nlevels
    assert lgmod.lg_level_plan(pattern.h, 0)["const_weights"] == 1
    assert lgmod.lg_level_plan(stored.h, 0)["const_weights"] == 0
    assert all(lgmod.lg_level_plan(pattern.h, l)["const_weights"] == 0 for l in range(1, pattern.nlevels))
    hb_stored, _ = lgmod.lg_hier_bytes(stored.h)
    hb_pattern, _ = lgmod.lg_hier_bytes(pattern.h)
    assert hb_stored - hb_pattern >= 12 * g.nnz_off  # the FP64 and FP32 weights of L_0
    b = inputs.rhs(g.n, seed=7)
    x1, i1 = stored.solve(b)
    x2, i2 = pattern.solve(b)
    assert i1.status == lgmod.OK and i2.iterations == i1.iterations and i2.relres == i1.relres
    np.testing.assert_array_equal(x2, x1)
    B = inputs.rhs(g.n, 3, seed=9)
    X1, _ = stored.solve_batch(B)
    X2, _ = pattern.solve_batch(B)
    np.testing.assert_array_equal(X2, X1)
    other = inputs.grid2d(40, 30, weights="uniform", seed=2)
    ho = lgmod.Hierarchy(other, precision=prec)
    bo = inputs.rhs(other.n, seed=3)
    xs1, _ = lgmod.solve_many([stored, ho], [b, bo])
    xs2, inf = lgmod.solve_many([pattern, ho], [b, bo])
    assert all(i.status == lgmod.OK for i in inf)
    np.testing.assert_array_equal(xs2[0], xs1[0])
    np.testing.assert_array_equal(xs2[1], xs1[1])
    rp, cl, w, _ = lgmod.lg_level_copy(pattern.h, 0)
    for a, c in zip((rp, cl, w), stored.level(0)[:3]):
        np.testing.assert_array_equal(a, c)
    assert np.all(w == value)
    path = str(tmp_path / "h.lgh")
    pattern.save(path)
    back = lgmod.Hierarchy.load(path)
    assert lgmod.lg_level_plan(back.h, 0)["const_weights"] == 1
    x3, _ = back.solve(b)
    np.testing.assert_array_equal(x3, x1)
    for h in (stored, pattern, ho, back):
        h.close()


def test_const_weights_level_apply_and_fp32_only(torch_cuda, lgmod, inputs):
    torch = torch_cuda
    g = inputs.chung_lu(20000, m_target=100000, seed=3, weights="unit")
    stored = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER, const_weights=0)
    lean = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER, fp32_only=1)
    x = torch.from_numpy(inputs.rhs(g.n, seed=11)).cuda()
    for prec, dt in ((lgmod.FP64, torch.float64), (lgmod.FP32_HIER, torch.float32)):
        xs = x.to(dt)
        ys = [torch.zeros(g.n, dtype=dt, device="cuda") for _ in range(2)]
        lgmod.lg_level_apply(stored.h, 0, prec, xs, ys[0])
        lgmod.lg_level_apply(lean.h, 0, prec, xs, ys[1])
        assert torch.equal(ys[0], ys[1])
    b = inputs.rhs(g.n, seed=5)
    x1, _ = stored.solve(b)
    x2, info = lean.solve(b)
    assert info.status == lgmod.OK
    np.testing.assert_array_equal(x2, x1)
    stored.close()
    lean.close()
