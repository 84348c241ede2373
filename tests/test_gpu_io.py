"""Save and load of a hierarchy (lg_save / lg_load): the loaded handle has
the same levels, plans, vertex order and coarsest pseudo-inverse, and its
solves (FP64 and FP32 hierarchy, single, multi-column and packed) return the
same bits; damaged files are refused."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = {
    "chunglu_20k": (lambda I: I.chung_lu(20000, m_target=100000, seed=3), {}),
    "grid3d_16_kcycle": (lambda I: I.grid3d(16, 16, 16), {"kcycle": 1}),
    "road_elim4": (lambda I: I.road_like(60, 60, seed=4), {"elim_rounds": 4}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_save_load_round_trip(lgmod, inputs, tmp_path, name):
    make, kw = CASES[name]
    g = make(inputs)
    H = lgmod.Hierarchy(g, **kw)
    path = str(tmp_path / "h.lgh")
    H.save(path)
    H2 = lgmod.Hierarchy.load(path)
    assert H2.nlevels == H.nlevels and H2.n == H.n
    for l in range(H.nlevels):
        assert H2.level_info(l) == H.level_info(l)
        assert H2.level_lp_nnz(l) == H.level_lp_nnz(l)
        assert lgmod.lg_level_plan(H2.h, l) == lgmod.lg_level_plan(H.h, l)
        for a, b in zip(H.level(l), H2.level(l)):
            if a is None:
                assert b is None
            else:
                np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(H2.permutation(), H.permutation())
    nc = H.level_info(H.nlevels - 1)["n"]
    np.testing.assert_array_equal(lgmod.lg_coarsest_pinv(H2.h, nc), lgmod.lg_coarsest_pinv(H.h, nc))
    assert H2.info().setup_ms == H.info().setup_ms
    b = inputs.rhs(g.n, seed=3)
    for prec in (lgmod.FP64, lgmod.FP32_HIER):
        x1, i1 = H.solve(b, precision=prec)
        x2, i2 = H2.solve(b, precision=prec)
        assert i1.status == lgmod.OK and i2.iterations == i1.iterations and i2.relres == i1.relres
        np.testing.assert_array_equal(x2, x1)
    B = inputs.rhs(g.n, 4, seed=5)
    X1, _ = H.solve_batch(B)
    X2, _ = H2.solve_batch(B)
    np.testing.assert_array_equal(X2, X1)
    xs, infos = lgmod.solve_many([H2], [b])
    assert infos[0].status == lgmod.OK
    H.close()
    H2.close()


def test_damaged_files_refused(lgmod, inputs, tmp_path):
    g = inputs.grid2d(40, 40)
    H = lgmod.Hierarchy(g)
    path = tmp_path / "h.lgh"
    H.save(str(path))
    data = path.read_bytes()
    for cut in (len(data) // 2, len(data) - 1):
        bad = tmp_path / f"cut{cut}.lgh"
        bad.write_bytes(data[:cut])
        with pytest.raises(lgmod.LGError) as e:
            lgmod.Hierarchy.load(str(bad))
        assert e.value.status == lgmod.ERR_INVALID
    longer = tmp_path / "longer.lgh"
    longer.write_bytes(data + b"\0")
    with pytest.raises(lgmod.LGError) as e:
        lgmod.Hierarchy.load(str(longer))
    assert e.value.status == lgmod.ERR_INVALID
    x1, _ = H.solve(inputs.rhs(g.n, seed=1))  # the saved handle is untouched
    H.close()


def test_solve_log(lgmod, inputs, tmp_path, monkeypatch):
    """With LG_LOG set, every setup and every solved right-hand side appends
    one JSON line with the figures the call returned."""
    import json

    log = tmp_path / "solves.jsonl"
    monkeypatch.setenv("LG_LOG", str(log))
    g = inputs.grid2d(30, 30)
    H = lgmod.Hierarchy(g)
    b = inputs.rhs(g.n, seed=1)
    _, info = H.solve(b)
    _, binfos = H.solve_batch(inputs.rhs(g.n, 2, seed=2))
    H2 = lgmod.Hierarchy(inputs.grid2d(20, 20))
    _, minfos = lgmod.solve_many([H, H2], [b, inputs.rhs(400, seed=3)])
    monkeypatch.delenv("LG_LOG")
    H.solve(b)  # not logged
    lines = [json.loads(s) for s in log.read_text().splitlines()]
    assert [x["call"] for x in lines] == ["lg_setup", "lg_solve", "lg_solve_batch", "lg_solve_batch", "lg_setup",
                                          "lg_solve_many", "lg_solve_many"]
    assert lines[0]["n"] == g.n and lines[0]["levels"] == H.nlevels
    for line, inf in zip(lines[1:4] + lines[5:], [info] + binfos + minfos):
        assert line["status"] == inf.status == lgmod.OK
        assert line["iterations"] == inf.iterations and line["relres"] == inf.relres
        assert line["wda"] == pytest.approx(inf.work_units / -np.log10(inf.relres), rel=1e-6)
    assert [x["index"] for x in lines[5:]] == [0, 1]
    H.close()
    H2.close()


def _level0_offsets(lgmod, data, n0):
    """Byte offsets of level 0's col values and, on an aggregation level, its
    agg values in a hierarchy file (the layout lg_save writes: header, vertex
    order, then the level's sizes and arrays, each array a uint64 count
    followed by its values). Each count is checked on the way, so a layout
    misread fails here rather than corrupting the wrong bytes."""
    import ctypes

    def u64(at):
        return int(np.frombuffer(data, dtype=np.uint64, count=1, offset=at)[0])

    at = 8 + 4 + 4 + ctypes.sizeof(lgmod.Options) + 4 + 8 + 8 + 8 + 4
    assert u64(at) == n0
    at += 8 + 4 * n0                       # vertex order
    kind = int(np.frombuffer(data, dtype=np.int32, count=1, offset=at)[0])
    n, nnz, nc = (int(v) for v in np.frombuffer(data, dtype=np.int64, count=3, offset=at + 4))
    at += 4 + 5 * 8 + 4                    # kind, n, nnz, nc, nf, lambda, binning
    wconst = int(np.frombuffer(data, dtype=np.int32, count=1, offset=at)[0])
    assert wconst in (0, 1)
    at += 4 + 8                            # constant-weight flag and value
    nw = 0 if wconst else nnz              # a constant-weight level stores no weight arrays
    assert n == n0 and u64(at) == n + 1
    at += 8 + 8 * (n + 1)                  # rowptr
    rowptr_at = at - 8 * (n + 1)
    assert u64(at) == nnz
    col_at = at + 8
    at += 8 + 4 * nnz
    for count, size in ((nw, 8), (n, 8), (n, 8), (nw, 4), (n, 4)):  # w, d, dinv, w32, dinv32
        assert u64(at) == count
        at += 8 + size * count
    agg_at = None
    if kind == lgmod.LEVEL_AGG:
        assert u64(at) == n
        agg_at = at + 8
    return rowptr_at, col_at, agg_at, n, nc


def test_out_of_range_indices_refused(lgmod, inputs, tmp_path):
    """A file whose sizes agree but whose index values point outside their
    arrays (a flipped byte in a column, an aggregate id, a row pointer) is
    refused with LG_ERR_INVALID before any solve could index with it. The
    checks only compare values, so the damaged arrays are never used to
    address memory."""
    g = inputs.grid3d(20, 20, 20)  # level 0 is an aggregation level (elimination gated out)
    H = lgmod.Hierarchy(g)
    assert H.level_info(0)["kind"] == lgmod.LEVEL_AGG
    path = tmp_path / "h.lgh"
    H.save(str(path))
    data = path.read_bytes()
    rowptr_at, col_at, agg_at, n, nc = _level0_offsets(lgmod, data, g.n)
    assert agg_at is not None
    damages = {
        "col": (col_at + 4 * 5, np.int32(n + 7)),
        "col_negative": (col_at + 4 * 11, np.int32(-3)),
        "agg": (agg_at + 4 * 3, np.int32(nc + 1)),
        "rowptr_decreasing": (rowptr_at + 8 * 2, np.int64(0)),
    }
    good = lgmod.Hierarchy.load(str(path))  # the undamaged file still loads
    good.close()
    for name, (at, val) in damages.items():
        buf = bytearray(data)
        raw = val.tobytes()
        buf[at:at + len(raw)] = raw
        bad = tmp_path / f"{name}.lgh"
        bad.write_bytes(bytes(buf))
        with pytest.raises(lgmod.LGError) as e:
            lgmod.Hierarchy.load(str(bad))
        assert e.value.status == lgmod.ERR_INVALID, name
        assert "out of range" in str(e.value), name
    x, info = H.solve(inputs.rhs(g.n, seed=1))
    assert info.status == lgmod.OK
    H.close()
