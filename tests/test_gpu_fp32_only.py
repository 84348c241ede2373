"""FP32-only hierarchies (option fp32_only): once built, the handle releases
the FP64 copies an FP32-hierarchy solve never reads, and the kept vertices'
rows of the elimination levels below the finest. Its solves must equal, bit
for bit, those of the same hierarchy with everything kept (the FP32 arrays and
the order of every sum are the same), on fewer device bytes; calls that need
the released arrays are refused."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [{}, {"kcycle": 1}, {"elim_rounds": 3}])
def test_fp32_only_same_bits_fewer_bytes(lgmod, inputs, kw):
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    full = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER, **kw)
    lean = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER, fp32_only=1, **kw)
    kinds = [full.level_info(l)["kind"] for l in range(full.nlevels)]
    assert lgmod.LEVEL_ELIM in kinds[1:]  # an elimination level below the finest is compacted
    assert lean.nlevels == full.nlevels
    for l in range(full.nlevels):
        assert lean.level_info(l) == full.level_info(l)  # logical sizes unchanged
    hb_full, _ = lgmod.lg_hier_bytes(full.h)
    hb_lean, _ = lgmod.lg_hier_bytes(lean.h)
    assert hb_lean < 0.8 * hb_full
    b = inputs.rhs(g.n, seed=3)
    x1, i1 = full.solve(b)
    x2, i2 = lean.solve(b)
    assert i1.status == lgmod.OK and i2.iterations == i1.iterations and i2.relres == i1.relres
    np.testing.assert_array_equal(x2, x1)
    B = inputs.rhs(g.n, 4, seed=5)
    X1, _ = full.solve_batch(B)
    X2, _ = lean.solve_batch(B)
    np.testing.assert_array_equal(X2, X1)
    xs1, _ = lgmod.solve_many([full], [b])
    xs2, inf = lgmod.solve_many([lean], [b])
    assert inf[0].status == lgmod.OK
    np.testing.assert_array_equal(xs2[0], xs1[0])
    full.close()
    lean.close()


def test_fp32_only_refuses_fp64_use(lgmod, inputs, tmp_path):
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    with pytest.raises(lgmod.LGError) as e:  # fp32_only needs the FP32 hierarchy
        lgmod.Hierarchy(g, precision=lgmod.FP64, fp32_only=1)
    assert e.value.status == lgmod.ERR_INVALID
    lean = lgmod.Hierarchy(g, precision=lgmod.FP32_HIER, fp32_only=1)
    for call in (lambda: lgmod.lg_set_precision(lean.h, lgmod.FP64),
                 lambda: lean.save(str(tmp_path / "h.lgh")),
                 lambda: lgmod.lg_level_copy(lean.h, 1),
                 lambda: lgmod.lg_vcycle(lean.h, np.ones(g.n), np.zeros(g.n), lgmod.FP64)):
        with pytest.raises(lgmod.LGError) as e:
            call()
        assert e.value.status == lgmod.ERR_INVALID
    rp, cl, w, _ = lgmod.lg_level_copy(lean.h, 0)  # the finest operator is kept in FP64
    full = lgmod.Hierarchy(g)
    for a, b in zip((rp, cl, w), full.level(0)[:3]):
        np.testing.assert_array_equal(a, b)
    full.close()
    sv = lgmod.lg_serve_create(lgmod.serve_options(precision=lgmod.FP64))
    with pytest.raises(lgmod.LGError) as e:
        lgmod.lg_serve_register(sv, lean.h)
    assert e.value.status == lgmod.ERR_INVALID
    lgmod.lg_serve_destroy(sv)
    x, info = lean.solve(inputs.rhs(g.n, seed=1))
    assert info.status == lgmod.OK
    lean.close()
