"""The C ABI library loads and exports every entry point include/lg.h declares
(no compute calls: these run without a GPU)."""

import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lg_[a-z0-9_]+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["lg_setup", "lg_solve", "lg_solve_batch", "lg_serve_submit", "lg_serve_poll",
                     "lg_serve_create", "lg_serve_register", "lg_serve_stats", "lg_destroy", "lg_error_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lgmod):
    lib = lgmod.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", lgmod.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lg_[a-z0-9_]+)\b", out))
    missing = declared_symbols() - exported
    assert not missing, missing
    for name in declared_symbols():
        assert hasattr(lib, name)


def test_options_defaults_match_paper(lgmod):
    o = lgmod.options()
    assert o.coarse_nnz == 1000.0 and o.elim_max_degree == 4 and abs(o.elim_min_frac - 0.05) < 1e-15
    assert o.agg_iters == 10 and o.vote_threshold == 8 and o.strength_vecs == 4 and o.strength_sweeps == 3
    assert o.cheb_degree == 2 and o.cheb_lo == 0.3 and o.cheb_hi == 1.1 and o.eig_iters == 10
    assert o.kcycle == 0 and o.elim_rounds == 1  # V-cycle, one elimination round (Sections 3.4, 4)
    assert o.lp_residual == 1
    assert o.const_weights == 1 and o.row_sorts == 1 and o.fp32_only == 0
    assert lgmod.serve_options().policy == lgmod.SERVE_ARRIVAL
    assert lgmod.lib().lg_error_string(0) == b"ok"


def test_serve_options_checked_without_gpu_work(lgmod):
    import ctypes as C

    lib = lgmod.lib()
    s = C.c_void_p()
    for bad in ({"policy": 2}, {"policy": -1}, {"slots": 0}, {"hbm_budget_bytes": 0.0}):
        o = lgmod.serve_options(**bad)
        assert lib.lg_serve_create(C.byref(o), C.byref(s)) == lgmod.ERR_INVALID
    assert lib.lg_serve_set_policy(None, 1) == lgmod.ERR_INVALID


def test_bad_arguments_rejected_without_gpu_work(lgmod):
    import ctypes as C

    lib = lgmod.lib()
    h = C.c_void_p()
    assert lib.lg_setup(0, None, None, None, None, C.byref(h)) == lgmod.ERR_INVALID
    assert lib.lg_solve(None, None, None, 1e-8, None) == lgmod.ERR_INVALID
    assert lib.lg_solve_many(0, None, None, None, 1e-8, None) == lgmod.ERR_INVALID
    one = (C.c_void_p * 1)(None)
    assert lib.lg_solve_many(1, one, one, one, 1e-8, None) == lgmod.ERR_INVALID  # a NULL handle
    assert lib.lg_save(None, b"/nonexistent/x") == lgmod.ERR_INVALID
    assert lib.lg_load(None, None, C.byref(h)) == lgmod.ERR_INVALID


def test_load_refuses_other_files_before_device_work(lgmod, tmp_path):
    import ctypes as C

    lib = lgmod.lib()
    h = C.c_void_p()
    assert lib.lg_load(str(tmp_path / "missing.lgh").encode(), None, C.byref(h)) == lgmod.ERR_INVALID
    junk = tmp_path / "junk.lgh"
    junk.write_bytes(b"not a hierarchy file at all" * 10)
    assert lib.lg_load(str(junk).encode(), None, C.byref(h)) == lgmod.ERR_INVALID
    assert not h.value
    # the right magic with a wrong version, options layout or level count
    import struct

    magic = b"LGHIERF1"
    opts_size = C.sizeof(lgmod.Options)
    good_opts = bytes(opts_size)
    cases = [
        magic + struct.pack("<II", 2, opts_size),                                   # version
        magic + struct.pack("<II", 1, opts_size + 8),                               # options layout
        magic + struct.pack("<II", 1, opts_size) + good_opts + struct.pack("<iqqdi", 0, 10, 50, 1.0, -1),  # no levels
        magic + struct.pack("<II", 1, opts_size) + good_opts + struct.pack("<iqqdi", 3, 0, 50, 1.0, -1),   # n = 0
        magic + struct.pack("<II", 1, opts_size) + good_opts,                       # truncated header
    ]
    for q, data in enumerate(cases):
        bad = tmp_path / f"bad{q}.lgh"
        bad.write_bytes(data)
        assert lib.lg_load(str(bad).encode(), None, C.byref(h)) == lgmod.ERR_INVALID, q
        assert not h.value


def test_oracle_and_cuda_path_share_no_code():
    """The oracle never imports the package and the package never touches the oracle."""
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "paper_1705_06266_gb300" not in src and "lg.h" not in src.replace("lgref.h", "")
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_1705_06266_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower().replace("the oracle", "") or f == "inputs.py", f
                assert "lgref" not in src, f
