"""Python binding of the C ABI in ``include/lg.h`` (ctypes, marshalling only).

Every computation runs in ``liblg.so``; this module converts arguments. Arrays
may be numpy arrays (host memory) or torch CUDA tensors (device memory, passed
by ``data_ptr()``). The library is loaded from this package's directory;
importing works without it, but the first call raises if it is missing, so a
missing CUDA build never goes unnoticed.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblg.so")

OK, ERR_INVALID, ERR_DISCONNECTED, ERR_SETUP, ERR_NOMEM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, \
    ERR_TIMEOUT, ERR_CUDA, ERR_BUSY = range(10)
FP64, FP32_HIER = 0, 1
AUTO, HOST, DEVICE = -1, 0, 1
LEVEL_AGG, LEVEL_ELIM, LEVEL_COARSEST = 1, 2, 3
SERVE_ARRIVAL, SERVE_LEAST_WORK = 0, 1
DECIDED, UNDECIDED, SEED = 0, 1, 2


class Options(C.Structure):
    _fields_ = [
        ("coarse_nnz", C.c_double), ("elim_min_frac", C.c_double), ("jacobi_omega", C.c_double),
        ("cheb_lo", C.c_double), ("cheb_hi", C.c_double), ("stagnation_frac", C.c_double),
        ("seed", C.c_uint64), ("stream", C.c_void_p),
        ("precision", C.c_int32), ("max_levels", C.c_int32), ("max_iter", C.c_int32),
        ("elim_enable", C.c_int32), ("elim_max_degree", C.c_int32), ("agg_iters", C.c_int32),
        ("vote_threshold", C.c_int32), ("strength_vecs", C.c_int32), ("strength_sweeps", C.c_int32),
        ("cheb_degree", C.c_int32), ("eig_iters", C.c_int32), ("max_coarse_n", C.c_int32),
        ("residual_replace", C.c_int32), ("memory_space", C.c_int32), ("use_graphs", C.c_int32),
        ("autotune", C.c_int32), ("reorder", C.c_int32), ("kcycle", C.c_int32),
        ("elim_rounds", C.c_int32), ("lp_residual", C.c_int32), ("fp32_only", C.c_int32),
        ("const_weights", C.c_int32), ("row_sorts", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("relres", C.c_double), ("op_complexity", C.c_double), ("setup_ms", C.c_double),
        ("solve_ms", C.c_double), ("work_units", C.c_double), ("nnz", C.c_int64),
        ("status", C.c_int32), ("iterations", C.c_int32), ("levels", C.c_int32), ("reserved", C.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class KernelProfile(C.Structure):
    _fields_ = [("total_ms", C.c_double), ("bytes", C.c_double), ("launches", C.c_int64), ("reserved", C.c_int64)]


class ServeOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("slots", C.c_int32), ("max_queue", C.c_int32),
                ("precision", C.c_int32), ("policy", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double), ("solves_per_s", C.c_double), ("resident_bytes", C.c_double),
                ("completed", C.c_int64), ("failed", C.c_int64), ("pending", C.c_int64),
                ("running", C.c_int64), ("groups", C.c_int64), ("packed_groups", C.c_int64),
                ("workspaces_made", C.c_int64), ("workspace_ms", C.c_double), ("copy_ms", C.c_double),
                ("solve_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P, _I64, _I32, _U64, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
_SIGS = {
    "lg_options_default": (C.c_int, [_P]),
    "lg_error_string": (C.c_char_p, [C.c_int]),
    "lg_last_error_detail": (C.c_char_p, []),
    "lg_setup": (C.c_int, [_I64, _P, _P, _P, _P, _P]),
    "lg_destroy": (None, [_P]),
    "lg_solve": (C.c_int, [_P, _P, _P, _D, _P]),
    "lg_solve_batch": (C.c_int, [_P, _I32, _P, _I64, _P, _I64, _D, _P]),
    "lg_set_precision": (C.c_int, [_P, _I32]),
    "lg_hier_info": (C.c_int, [_P, _P]),
    "lg_hier_bytes": (C.c_int, [_P, _P, _P]),
    "lg_level_info": (C.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    "lg_level_copy": (C.c_int, [_P, _I32, _P, _P, _P, _P]),
    "lg_coarsest_pinv": (C.c_int, [_P, _P]),
    "lg_permutation": (C.c_int, [_P, _P]),
    "lg_vcycle": (C.c_int, [_P, _P, _P, _I32]),
    "lg_vcycle_batch": (C.c_int, [_P, _I32, _P, _I64, _P, _I64, _I32]),
    "lg_laplacian_apply": (C.c_int, [_I64, _P, _P, _P, _P, _P, _P]),
    "lg_elim_select": (C.c_int, [_I64, _P, _P, _I32, _U64, _P, _P, _P]),
    "lg_elim_select_noalloc": (C.c_int, [_I64, _P, _P, _I32, _U64, _P, _P, _P]),
    "lg_strength": (C.c_int, [_I64, _P, _P, _P, _U64, _I32, _I32, _I32, _D, _P, _P]),
    "lg_aggregate": (C.c_int, [_I64, _P, _P, _P, _I32, _I32, _P, _P, _P, _P, _P]),
    "lg_level_apply": (C.c_int, [_P, _I32, _I32, _P, _P]),
    "lg_kernel_launches": (C.c_uint64, []),
    "lg_profile": (C.c_int, [_P, _I32]),
    "lg_profile_read": (C.c_int, [_P, _I32, _P]),
    "lg_level_plan": (C.c_int, [_P, _I32, _P]),
    "lg_batch_plan": (C.c_int, [_P, _I32, _P]),
    "lg_solve_many": (C.c_int, [_I32, _P, _P, _P, _D, _P]),
    "lg_level_lp_nnz": (C.c_int, [_P, _I32, _P]),
    "lg_save": (C.c_int, [_P, C.c_char_p]),
    "lg_load": (C.c_int, [C.c_char_p, _P, _P]),
    "lg_serve_options_default": (C.c_int, [_P]),
    "lg_serve_create": (C.c_int, [_P, _P]),
    "lg_serve_register": (C.c_int, [_P, _P]),
    "lg_serve_submit": (C.c_int, [_P, _P, _I32, _P, _P, _D, _P]),
    "lg_serve_poll": (C.c_int, [_P, _U64, _P, _P]),
    "lg_serve_stats": (C.c_int, [_P, _P]),
    "lg_serve_reset_stats": (C.c_int, [_P]),
    "lg_serve_set_policy": (C.c_int, [_P, _I32]),
    "lg_serve_request_bytes": (C.c_int, [_P, _I32, _P]),
    "lg_serve_destroy": (None, [_P]),
}

_lib = None


class LGError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _load()
        msg = lib.lg_error_string(status).decode()
        detail = lib.lg_last_error_detail().decode()
        super().__init__(f"{where}: status {status} ({msg}){': ' + detail if detail else ''}")
        self.status = status


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def lib():
    return _load()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _check(st: int, where: str):
    if st != OK:
        raise LGError(st, where)


def options(**kw) -> Options:
    o = Options()
    _check(_load().lg_options_default(C.byref(o)), "lg_options_default")
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lg_setup(n, rowptr, col, w, opts: Options | None = None):
    """Returns an opaque handle (c_void_p); release with lg_destroy."""
    h = C.c_void_p()
    _check(_load().lg_setup(int(n), _ptr(rowptr), _ptr(col), _ptr(w),
                            C.byref(opts) if opts is not None else None, C.byref(h)), "lg_setup")
    return h


def lg_destroy(h):
    _load().lg_destroy(h)


def lg_solve(h, b, x, tol: float = 1e-8, check: bool = True) -> Info:
    info = Info()
    st = _load().lg_solve(h, _ptr(b), _ptr(x), float(tol), C.byref(info))
    if check and st not in (OK,):
        raise LGError(st, "lg_solve")
    return info


def lg_solve_batch(h, k, B, ldb, X, ldx, tol: float = 1e-8, check: bool = True):
    infos = (Info * k)()
    st = _load().lg_solve_batch(h, int(k), _ptr(B), int(ldb), _ptr(X), int(ldx), float(tol), infos)
    if check and st != OK:
        raise LGError(st, "lg_solve_batch")
    return list(infos)


def lg_solve_many(hs, bs, xs, tol: float = 1e-8, check: bool = True):
    """hs: handles; bs / xs: one vector per handle (numpy or torch CUDA)."""
    count = len(hs)

    def addr(p):
        return p.value if isinstance(p, C.c_void_p) else p

    H = (C.c_void_p * count)(*[addr(h) for h in hs])
    B = (C.c_void_p * count)(*[addr(_ptr(b)) for b in bs])
    X = (C.c_void_p * count)(*[addr(_ptr(x)) for x in xs])
    infos = (Info * count)()
    st = _load().lg_solve_many(int(count), H, B, X, float(tol), infos)
    if check and st != OK:
        raise LGError(st, "lg_solve_many")
    return list(infos)


def solve_many(hierarchies, bs, tol: float = 1e-8, check: bool = True):
    """Solve one right-hand side on each of several hierarchies in one launch
    (lg_solve_many). Returns (xs, infos)."""
    bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    xs = [np.zeros(H.n) for H in hierarchies]
    infos = lg_solve_many([H.h for H in hierarchies], bs, xs, tol, check=check)
    return xs, infos


def lg_set_precision(h, precision: int):
    _check(_load().lg_set_precision(h, int(precision)), "lg_set_precision")


def lg_hier_info(h) -> Info:
    info = Info()
    _check(_load().lg_hier_info(h, C.byref(info)), "lg_hier_info")
    return info


def lg_hier_bytes(h):
    a, b = C.c_int64(), C.c_int64()
    _check(_load().lg_hier_bytes(h, C.byref(a), C.byref(b)), "lg_hier_bytes")
    return a.value, b.value


def lg_level_info(h, l: int):
    kind, n, nnz, nc, lam = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
    _check(_load().lg_level_info(h, l, C.byref(kind), C.byref(n), C.byref(nnz), C.byref(nc), C.byref(lam)),
           "lg_level_info")
    return {"kind": kind.value, "n": n.value, "nnz": nnz.value, "nc": nc.value, "lambda": lam.value}


def lg_level_copy(h, l: int):
    """Returns (rowptr, col, w, map) as numpy arrays (map None for the coarsest)."""
    d = lg_level_info(h, l)
    rp = np.zeros(d["n"] + 1, np.int64)
    cl = np.zeros(max(d["nnz"], 1), np.int32)
    w = np.zeros(max(d["nnz"], 1), np.float64)
    mp = np.zeros(d["n"], np.int32) if d["kind"] != LEVEL_COARSEST else None
    _check(_load().lg_level_copy(h, l, _ptr(rp), _ptr(cl), _ptr(w), _ptr(mp)), "lg_level_copy")
    return rp, cl[: d["nnz"]], w[: d["nnz"]], mp


def lg_permutation(h, n: int) -> np.ndarray:
    perm = np.zeros(n, np.int32)
    _check(_load().lg_permutation(h, _ptr(perm)), "lg_permutation")
    return perm


def lg_coarsest_pinv(h, nc: int) -> np.ndarray:
    out = np.zeros((nc, nc))
    _check(_load().lg_coarsest_pinv(h, _ptr(out)), "lg_coarsest_pinv")
    return out


def lg_vcycle(h, f, x, precision: int = FP64):
    _check(_load().lg_vcycle(h, _ptr(f), _ptr(x), int(precision)), "lg_vcycle")


def lg_vcycle_batch(h, k: int, F, ldf: int, X, ldx: int, precision: int = FP64):
    """X = M F on k column-major columns (leading dimensions ldf, ldx), host or device."""
    _check(_load().lg_vcycle_batch(h, int(k), _ptr(F), int(ldf), _ptr(X), int(ldx), int(precision)),
           "lg_vcycle_batch")


def lg_kernel_launches() -> int:
    return int(_load().lg_kernel_launches())


def lg_level_apply(h, level: int, precision: int, x, y):
    """y = L_level x on the device (float64 tensors for FP64, float32 for FP32_HIER)."""
    _check(_load().lg_level_apply(h, int(level), int(precision), _ptr(x), _ptr(y)), "lg_level_apply")


def lg_profile(h, enable: bool):
    _check(_load().lg_profile(h, 1 if enable else 0), "lg_profile")


def lg_profile_read(h, level: int = -1) -> KernelProfile:
    p = KernelProfile()
    _check(_load().lg_profile_read(h, int(level), C.byref(p)), "lg_profile_read")
    return p


def lg_batch_plan(h, l: int) -> dict:
    out = (C.c_int64 * 4)()
    _check(_load().lg_batch_plan(h, int(l), out), "lg_batch_plan")
    return {"op_ch": out[0], "op_vrows": out[1], "w_ch": out[2], "w_vrows": out[3]}


def lg_level_plan(h, l: int) -> dict:
    out = (C.c_int64 * 8)()
    _check(_load().lg_level_plan(h, int(l), out), "lg_level_plan")
    return {"E": out[0], "group_rows": out[1], "warp_rows": out[2], "long_rows": out[3], "chunks": out[4],
            "blocks": out[5], "seg_tiles": out[6], "const_weights": out[7]}


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def lg_laplacian_apply(n, rowptr, col, w, x, y, stream=None):
    _check(_load().lg_laplacian_apply(int(n), _ptr(rowptr), _ptr(col), _ptr(w), _ptr(x), _ptr(y),
                                      _stream(stream)), "lg_laplacian_apply")


def lg_elim_select(n, rowptr, col, max_degree, seed, is_f, stream=None) -> int:
    nf = C.c_int64()
    _check(_load().lg_elim_select(int(n), _ptr(rowptr), _ptr(col), int(max_degree), int(seed), _ptr(is_f),
                                  C.byref(nf), _stream(stream)), "lg_elim_select")
    return nf.value


def lg_elim_select_noalloc(n, rowptr, col, max_degree, seed, is_f, stream=None) -> int:
    """lg_elim_select with its scratch in a fixed device array (no allocation)."""
    nf = C.c_int64()
    _check(_load().lg_elim_select_noalloc(int(n), _ptr(rowptr), _ptr(col), int(max_degree), int(seed), _ptr(is_f),
                                          C.byref(nf), _stream(stream)), "lg_elim_select_noalloc")
    return nf.value


def lg_strength(n, rowptr, col, w, seed, level, m, sweeps, omega, S, stream=None):
    _check(_load().lg_strength(int(n), _ptr(rowptr), _ptr(col), _ptr(w), int(seed), int(level), int(m),
                               int(sweeps), float(omega), _ptr(S), _stream(stream)), "lg_strength")


def lg_aggregate(n, rowptr, col, S, iters, threshold, agg, state=None, votes=None, stream=None) -> int:
    nc = C.c_int64()
    _check(_load().lg_aggregate(int(n), _ptr(rowptr), _ptr(col), _ptr(S), int(iters), int(threshold),
                                _ptr(agg), C.byref(nc), _ptr(state), _ptr(votes), _stream(stream)),
           "lg_aggregate")
    return nc.value


def serve_options(**kw) -> ServeOptions:
    o = ServeOptions()
    _check(_load().lg_serve_options_default(C.byref(o)), "lg_serve_options_default")
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lg_serve_create(opts: ServeOptions | None = None):
    s = C.c_void_p()
    _check(_load().lg_serve_create(C.byref(opts) if opts is not None else None, C.byref(s)), "lg_serve_create")
    return s


def lg_serve_register(s, h):
    _check(_load().lg_serve_register(s, h), "lg_serve_register")


def lg_serve_submit(s, h, k, B, X, tol: float = 1e-8) -> int:
    t = C.c_uint64()
    _check(_load().lg_serve_submit(s, h, int(k), _ptr(B), _ptr(X), float(tol), C.byref(t)), "lg_serve_submit")
    return t.value


def lg_serve_poll(s, ticket: int):
    done, info = C.c_int32(), Info()
    _check(_load().lg_serve_poll(s, C.c_uint64(ticket), C.byref(done), C.byref(info)), "lg_serve_poll")
    return bool(done.value), info


def lg_serve_stats(s) -> ServeStats:
    st = ServeStats()
    _check(_load().lg_serve_stats(s, C.byref(st)), "lg_serve_stats")
    return st


def lg_serve_reset_stats(s):
    _check(_load().lg_serve_reset_stats(s), "lg_serve_reset_stats")


def lg_serve_set_policy(s, policy: int):
    _check(_load().lg_serve_set_policy(s, int(policy)), "lg_serve_set_policy")


def lg_serve_destroy(s):
    _load().lg_serve_destroy(s)


def lg_serve_request_bytes(h, k: int) -> float:
    b = C.c_double()
    _check(_load().lg_serve_request_bytes(h, int(k), C.byref(b)), "lg_serve_request_bytes")
    return b.value


class Server:
    """A continuous-batching solve server (lg_serve_*). Right-hand sides are
    [n][k] numpy arrays; the column-major copies handed to the server are kept
    alive here until the request is polled done."""

    def __init__(self, **kw):
        self.s = lg_serve_create(serve_options(**kw))
        self._live = {}

    def register(self, H):
        lg_serve_register(self.s, H.h)

    def submit(self, H, B, tol=1e-8) -> int:
        B = np.asarray(B, dtype=np.float64)
        if B.ndim == 1:
            B = B[:, None]
        Bc = np.ascontiguousarray(B.T)
        Xc = np.zeros_like(Bc)
        t = lg_serve_submit(self.s, H.h, B.shape[1], Bc, Xc, tol)
        self._live[t] = (Bc, Xc)
        return t

    def poll(self, ticket):
        """(X [n][k], info) once done, else (None, None)."""
        done, info = lg_serve_poll(self.s, ticket)
        if not done:
            return None, None
        _, Xc = self._live.pop(ticket)
        return np.ascontiguousarray(Xc.T), info

    def wait(self, ticket, timeout=120.0):
        import time
        t0 = time.monotonic()
        while True:
            X, info = self.poll(ticket)
            if X is not None:
                return X, info
            if time.monotonic() - t0 > timeout:
                raise TimeoutError(f"request {ticket} not done after {timeout} s")
            time.sleep(2e-4)

    def stats(self) -> ServeStats:
        return lg_serve_stats(self.s)

    def close(self):
        if getattr(self, "s", None):
            lg_serve_destroy(self.s)
            self.s = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Owning wrapper of an lg handle built from a CSR graph (numpy or torch arrays)."""

    def __init__(self, g=None, *, n=None, rowptr=None, col=None, w=None, opts: Options | None = None, **kw):
        if g is not None:
            n, rowptr, col, w = g.n, g.rowptr, g.col, g.w
        self.opts = opts if opts is not None else options(**kw)
        self.n = int(n)
        self.h = lg_setup(n, rowptr, col, w, self.opts)

    def close(self):
        if getattr(self, "h", None):
            lg_destroy(self.h)
            self.h = None

    def save(self, path: str):
        """Write the hierarchy to a file (lg_save)."""
        _check(_load().lg_save(self.h, os.fsencode(path)), "lg_save")

    @classmethod
    def load(cls, path: str, opts: Options | None = None, **kw):
        """A hierarchy read back from a file written by save (lg_load); opts
        or keyword options give only the stream and memory space."""
        self = cls.__new__(cls)
        self.opts = opts if opts is not None else options(**kw)
        h = C.c_void_p()
        _check(_load().lg_load(os.fsencode(path), C.byref(self.opts), C.byref(h)), "lg_load")
        self.h = h
        self.n = int(lg_level_info(h, 0)["n"])
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> Info:
        return lg_hier_info(self.h)

    @property
    def nlevels(self) -> int:
        return self.info().levels

    def level_info(self, l):
        return lg_level_info(self.h, l)

    def level_lp_nnz(self, l) -> int:
        v = C.c_int64()
        _check(_load().lg_level_lp_nnz(self.h, int(l), C.byref(v)), "lg_level_lp_nnz")
        return v.value

    def level(self, l):
        return lg_level_copy(self.h, l)

    def permutation(self):
        return lg_permutation(self.h, self.n)

    def solve(self, b, x=None, tol=1e-8, precision=None, check=True):
        if precision is not None:
            lg_set_precision(self.h, precision)
        if x is None:
            x = np.zeros(self.n)
        info = lg_solve(self.h, b, x, tol, check=check)
        return x, info

    def solve_batch(self, B, tol=1e-8, precision=None, check=True):
        """B: [n][k] (one right-hand side per column). Returns (X [n][k], infos)."""
        if precision is not None:
            lg_set_precision(self.h, precision)
        B = np.asarray(B, dtype=np.float64)
        k = B.shape[1]
        Bc = np.ascontiguousarray(B.T)  # column-major n x k, leading dimension n
        Xc = np.zeros_like(Bc)
        infos = lg_solve_batch(self.h, k, Bc, self.n, Xc, self.n, tol, check=check)
        return np.ascontiguousarray(Xc.T), infos

    def vcycle_batch(self, F, precision=FP64):
        """F: [n][k]. One multi-column V-cycle; returns X [n][k]."""
        F = np.asarray(F, dtype=np.float64)
        k = F.shape[1]
        Fc = np.ascontiguousarray(F.T)
        Xc = np.zeros_like(Fc)
        _check(_load().lg_vcycle_batch(self.h, int(k), _ptr(Fc), self.n, _ptr(Xc), self.n, int(precision)),
               "lg_vcycle_batch")
        return np.ascontiguousarray(Xc.T)

    def vcycle(self, f, precision=FP64):
        x = np.zeros(self.n)
        lg_vcycle(self.h, np.ascontiguousarray(f, dtype=np.float64), x, precision)
        return x
