"""ctypes binding of the FP64 oracle (``oracle/lgref.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the CUDA library and its Python
binding never import it. Arrays are numpy; every function copies its outputs
into fresh numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgref.c")
_HDR = os.path.join(_HERE, "lgref.h")
_LIB = os.path.join(_HERE, "liblgref.so")

OK, INVALID, DISCONNECTED, SETUP, NOT_CONVERGED, BREAKDOWN = range(6)
AGG, ELIM, COARSEST = 1, 2, 3
DECIDED, UNDECIDED, SEED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no CUDA)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [
        ("coarse_nnz", C.c_double), ("elim_min_frac", C.c_double), ("jacobi_omega", C.c_double),
        ("cheb_lo", C.c_double), ("cheb_hi", C.c_double), ("stagnation_frac", C.c_double),
        ("seed", C.c_uint64),
        ("max_levels", C.c_int32), ("elim_max_degree", C.c_int32), ("agg_iters", C.c_int32),
        ("vote_threshold", C.c_int32), ("strength_vecs", C.c_int32), ("strength_sweeps", C.c_int32),
        ("cheb_degree", C.c_int32), ("eig_iters", C.c_int32), ("max_coarse_n", C.c_int32),
        ("elim_enable", C.c_int32),
        ("kcycle", C.c_int32), ("elim_rounds", C.c_int32),
    ]


_lib = None

_P = C.c_void_p
_I64, _I32, _U64, _D = C.c_int64, C.c_int32, C.c_uint64, C.c_double


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    sig = {
        "lgref_opts_default": (None, [_P]),
        "lgref_splitmix64": (_U64, [_U64, _U64]),
        "lgref_vertex_hash": (_U64, [_U64, _I64]),
        "lgref_uniform": (_D, [_U64, _I32, _I32, _I64]),
        "lgref_check_graph": (C.c_int, [_I64, _P, _P, _P]),
        "lgref_components": (_I64, [_I64, _P, _P, _P]),
        "lgref_diag": (None, [_I64, _P, _P, _P]),
        "lgref_apply_L": (None, [_I64, _P, _P, _P, _P, _P]),
        "lgref_elim_select": (_I64, [_I64, _P, _P, _I32, _U64, _P]),
        "lgref_schur": (_P, [_I64, _P, _P, _P, _P, _P]),
        "lgref_strength_vectors": (None, [_U64, _I32, _I64, _I32, _P]),
        "lgref_jacobi": (None, [_I64, _P, _P, _P, _I32, _I32, _D, _P]),
        "lgref_affinity": (None, [_I64, _P, _P, _I32, _P, _P]),
        "lgref_strength": (None, [_I64, _P, _P, _P, _U64, _I32, _I32, _I32, _D, _P]),
        "lgref_aggregate": (_I64, [_I64, _P, _P, _P, _I32, _I32, _P, _P, _P]),
        "lgref_galerkin": (_P, [_I64, _P, _P, _P, _P, _I64]),
        "lgref_tridiag_max": (_D, [_I32, _P, _P]),
        "lgref_lanczos": (_D, [_I64, _P, _P, _P, _U64, _I32, _I32]),
        "lgref_cheb_pre": (None, [_I64, _P, _P, _P, _D, _D, _D, _I32, _P, _P, _P]),
        "lgref_cheb_post": (None, [_I64, _P, _P, _P, _D, _D, _D, _I32, _P, _P]),
        "lgref_pinv": (C.c_int, [_I64, _P, _P, _P, _P]),
        "lgref_dense_solve": (C.c_int, [_I64, _P, _P, _P, _P, _P]),
        "lgref_setup": (_P, [_I64, _P, _P, _P, _P, _P]),
        "lgref_hier_free": (None, [_P]),
        "lgref_hier_nlevels": (_I32, [_P]),
        "lgref_hier_level_info": (None, [_P, _I32, _P, _P, _P, _P, _P]),
        "lgref_hier_level_csr": (None, [_P, _I32, _P, _P, _P]),
        "lgref_hier_level_map": (None, [_P, _I32, _P]),
        "lgref_hier_coarsest_pinv": (None, [_P, _P]),
        "lgref_vcycle": (None, [_P, _P, _P]),
        "lgref_level_cycle": (None, [_P, C.c_int32, _P, _P, C.c_int32]),
        "lgref_pcg": (C.c_int, [_P, _P, _P, _D, _I32, _P, _P]),
        "lgref_csr_n": (_I64, [_P]),
        "lgref_csr_nnz": (_I64, [_P]),
        "lgref_csr_copy": (None, [_P, _P, _P, _P]),
        "lgref_csr_free": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr_args(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    return rp, cl, w


class CSR:
    """A plain CSR graph (same fields as inputs.Graph)."""

    def __init__(self, n, rowptr, col, w):
        self.n, self.rowptr, self.col, self.w = int(n), rowptr, col, w

    @property
    def nnz_off(self):
        return int(self.rowptr[-1])


def _take_csr(handle) -> CSR:
    lib = _load()
    n = lib.lgref_csr_n(handle)
    nnz = lib.lgref_csr_nnz(handle)
    rp = np.zeros(n + 1, np.int64)
    cl = np.zeros(max(nnz, 1), np.int32)
    w = np.zeros(max(nnz, 1), np.float64)
    lib.lgref_csr_copy(handle, _ptr(rp), _ptr(cl), _ptr(w))
    lib.lgref_csr_free(handle)
    return CSR(n, rp, cl[:nnz], w[:nnz])


def default_opts(**kw) -> Opts:
    o = Opts()
    _load().lgref_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def splitmix64(seed: int, counter: int) -> int:
    return int(_load().lgref_splitmix64(seed, counter))


def vertex_hash(seed: int, ids) -> np.ndarray:
    lib = _load()
    return np.array([lib.lgref_vertex_hash(seed, int(i)) for i in ids], dtype=np.uint64)


def uniform(seed: int, stream: int, level: int, idx: int) -> float:
    return float(_load().lgref_uniform(seed, stream, level, idx))


def check_graph(g) -> int:
    rp, cl, w = _csr_args(g)
    return int(_load().lgref_check_graph(g.n, _ptr(rp), _ptr(cl), _ptr(w)))


def components(g):
    rp, cl, _ = _csr_args(g)
    lab = np.zeros(g.n, np.int32)
    nc = _load().lgref_components(g.n, _ptr(rp), _ptr(cl), _ptr(lab))
    return int(nc), lab


def diag(g) -> np.ndarray:
    rp, _, w = _csr_args(g)
    d = np.zeros(g.n)
    _load().lgref_diag(g.n, _ptr(rp), _ptr(w), _ptr(d))
    return d


def apply_L(g, x) -> np.ndarray:
    rp, cl, w = _csr_args(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(g.n)
    _load().lgref_apply_L(g.n, _ptr(rp), _ptr(cl), _ptr(w), _ptr(x), _ptr(y))
    return y


def elim_select(g, max_degree: int = 4, seed: int = 0x5EED) -> np.ndarray:
    rp, cl, _ = _csr_args(g)
    f = np.zeros(g.n, np.uint8)
    _load().lgref_elim_select(g.n, _ptr(rp), _ptr(cl), max_degree, seed, _ptr(f))
    return f


def schur(g, is_f):
    rp, cl, w = _csr_args(g)
    is_f = np.ascontiguousarray(is_f, dtype=np.uint8)
    cmap = np.zeros(g.n, np.int32)
    h = _load().lgref_schur(g.n, _ptr(rp), _ptr(cl), _ptr(w), _ptr(is_f), _ptr(cmap))
    return _take_csr(h), cmap


def strength_vectors(seed: int, level: int, n: int, m: int = 4) -> np.ndarray:
    y = np.zeros((n, m))
    _load().lgref_strength_vectors(seed, level, n, m, _ptr(y))
    return y


def jacobi(g, x, sweeps: int = 3, omega: float = 2.0 / 3.0) -> np.ndarray:
    rp, cl, w = _csr_args(g)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    m = 1 if x.ndim == 1 else x.shape[1]
    _load().lgref_jacobi(g.n, _ptr(rp), _ptr(cl), _ptr(w), m, sweeps, omega, _ptr(x))
    return x


def affinity(g, x) -> np.ndarray:
    rp, cl, _ = _csr_args(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = 1 if x.ndim == 1 else x.shape[1]
    S = np.zeros(g.nnz_off)
    _load().lgref_affinity(g.n, _ptr(rp), _ptr(cl), m, _ptr(x), _ptr(S))
    return S


def strength(g, seed: int = 0x5EED, level: int = 0, m: int = 4, sweeps: int = 3,
             omega: float = 2.0 / 3.0) -> np.ndarray:
    rp, cl, w = _csr_args(g)
    S = np.zeros(max(g.nnz_off, 1))
    _load().lgref_strength(g.n, _ptr(rp), _ptr(cl), _ptr(w), seed, level, m, sweeps, omega, _ptr(S))
    return S[: g.nnz_off]


def aggregate(g, S, iters: int = 10, threshold: int = 8):
    """Returns (nc, agg, state, votes)."""
    rp, cl, _ = _csr_args(g)
    S = np.ascontiguousarray(S, dtype=np.float64)
    agg = np.zeros(g.n, np.int32)
    st = np.zeros(g.n, np.int8)
    votes = np.zeros(g.n, np.int32)
    nc = _load().lgref_aggregate(g.n, _ptr(rp), _ptr(cl), _ptr(S), iters, threshold,
                                 _ptr(agg), _ptr(st), _ptr(votes))
    return int(nc), agg, st, votes


def galerkin(g, agg, nc: int) -> CSR:
    rp, cl, w = _csr_args(g)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    h = _load().lgref_galerkin(g.n, _ptr(rp), _ptr(cl), _ptr(w), _ptr(agg), nc)
    return _take_csr(h)


def tridiag_max(alpha, beta) -> float:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(np.append(beta, 0.0), dtype=np.float64)
    return float(_load().lgref_tridiag_max(len(a), _ptr(a), _ptr(b)))


def lanczos(g, seed: int = 0x5EED, level: int = 0, iters: int = 10) -> float:
    rp, cl, w = _csr_args(g)
    return float(_load().lgref_lanczos(g.n, _ptr(rp), _ptr(cl), _ptr(w), seed, level, iters))


def cheb_pre(g, lam, f, lo=0.3, hi=1.1, degree=2):
    rp, cl, w = _csr_args(g)
    f = np.ascontiguousarray(f, dtype=np.float64)
    x = np.zeros(g.n)
    r = np.zeros(g.n)
    _load().lgref_cheb_pre(g.n, _ptr(rp), _ptr(cl), _ptr(w), lam, lo, hi, degree, _ptr(f), _ptr(x), _ptr(r))
    return x, r


def cheb_post(g, lam, f, x0, lo=0.3, hi=1.1, degree=2):
    rp, cl, w = _csr_args(g)
    f = np.ascontiguousarray(f, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    _load().lgref_cheb_post(g.n, _ptr(rp), _ptr(cl), _ptr(w), lam, lo, hi, degree, _ptr(f), _ptr(x))
    return x


def pinv(g) -> np.ndarray:
    rp, cl, w = _csr_args(g)
    out = np.zeros((g.n, g.n))
    st = _load().lgref_pinv(g.n, _ptr(rp), _ptr(cl), _ptr(w), _ptr(out))
    if st != OK:
        raise RuntimeError(f"lgref_pinv status {st}")
    return out


def dense_solve(g, b) -> np.ndarray:
    rp, cl, w = _csr_args(g)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(g.n)
    st = _load().lgref_dense_solve(g.n, _ptr(rp), _ptr(cl), _ptr(w), _ptr(b), _ptr(x))
    if st != OK:
        raise RuntimeError(f"lgref_dense_solve status {st}")
    return x


class Level:
    def __init__(self, kind, a: CSR, nc, lam, mapping):
        self.kind, self.a, self.nc, self.lam, self.map = kind, a, nc, lam, mapping


class Hierarchy:
    """An oracle hierarchy; the C object is freed with the Python object."""

    def __init__(self, g, opts: Opts | None = None):
        lib = _load()
        self.opts = opts or default_opts()
        rp, cl, w = _csr_args(g)
        st = C.c_int(0)
        self._h = lib.lgref_setup(g.n, _ptr(rp), _ptr(cl), _ptr(w), C.byref(self.opts), C.byref(st))
        self.status = st.value
        if not self._h:
            raise RuntimeError(f"lgref_setup status {self.status}")
        self.n = g.n

    def __del__(self):
        if getattr(self, "_h", None):
            _load().lgref_hier_free(self._h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return int(_load().lgref_hier_nlevels(self._h))

    def level(self, l: int) -> Level:
        lib = _load()
        kind, n, nnz, nc = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
        lam = C.c_double()
        lib.lgref_hier_level_info(self._h, l, C.byref(kind), C.byref(n), C.byref(nnz), C.byref(nc), C.byref(lam))
        rp = np.zeros(n.value + 1, np.int64)
        cl = np.zeros(max(nnz.value, 1), np.int32)
        w = np.zeros(max(nnz.value, 1), np.float64)
        lib.lgref_hier_level_csr(self._h, l, _ptr(rp), _ptr(cl), _ptr(w))
        mp = None
        if kind.value in (AGG, ELIM):
            mp = np.zeros(n.value, np.int32)
            lib.lgref_hier_level_map(self._h, l, _ptr(mp))
        return Level(kind.value, CSR(n.value, rp, cl[: nnz.value], w[: nnz.value]), nc.value, lam.value, mp)

    def coarsest_pinv(self) -> np.ndarray:
        last = self.level(self.nlevels - 1)
        out = np.zeros((last.a.n, last.a.n))
        _load().lgref_hier_coarsest_pinv(self._h, _ptr(out))
        return out

    def vcycle(self, f) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(self.n)
        _load().lgref_vcycle(self._h, _ptr(f), _ptr(x))
        return x

    def level_cycle(self, l: int, f, body_only: bool = False) -> np.ndarray:
        """The cycle at level l from x = 0 (body_only: without that level's own
        K-cycle acceleration)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(len(f))
        _load().lgref_level_cycle(self._h, int(l), _ptr(f), _ptr(x), 1 if body_only else 0)
        return x

    def pcg(self, b, tol: float = 1e-8, maxit: int = 500):
        """Returns (x, status, iterations, relres)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        it, rel = C.c_int32(), C.c_double()
        st = _load().lgref_pcg(self._h, _ptr(b), _ptr(x), tol, maxit, C.byref(it), C.byref(rel))
        return x, int(st), int(it.value), float(rel.value)
