"""ctypes binding of the C ABI in include/amg.h (argument marshalling only).

Every function here forwards to the symbol of the same name in
libamg_gb300.so; all computation happens in that library's CUDA kernels.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
pointers are taken from them without copies.  There is no fallback: if the
library cannot be built or loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

AMG_OK = 0
AMG_ERR_INVALID_ARG = 1
AMG_ERR_NOT_SYMMETRIC = 2
AMG_ERR_SELF_LOOP = 3
AMG_ERR_BAD_WEIGHT = 4
AMG_ERR_DISCONNECTED = 5
AMG_ERR_OOM = 6
AMG_ERR_CUDA = 7
AMG_ERR_NOT_CONVERGED = 8
AMG_ERR_BREAKDOWN = 9
AMG_ERR_TIMEOUT = 10
AMG_ERR_SETUP_STALL = 11
AMG_MEM_HOST = 0
AMG_MEM_DEVICE = 1
AMG_PREC_FP64 = 0
AMG_PREC_FP32 = 1
AMG_CYCLE_K = 0
AMG_CYCLE_AMLI = 1
AMG_AGG_MATCHING = 0
AMG_AGG_MIS = 1

# every symbol declared in include/amg.h
SYMBOLS = [
    "amg_default_options", "amg_degree_for", "amg_setup", "amg_solve", "amg_free", "amg_last_error",
    "amg_num_levels", "amg_level_n", "amg_level_nnz", "amg_level_csr", "amg_level_agg",
    "amg_level_smoother", "amg_apply_spmv", "amg_apply_smoother", "amg_apply_restrict",
    "amg_apply_prolong_add", "amg_apply_coarse_solve", "amg_apply_kcycle", "amg_match", "amg_match_noalloc",
    "amg_kernel_timing", "amg_kernel_timing_read", "amg_kernel_timing_read_kind", "amg_launch_count",
    "amg_server_create", "amg_server_add_graph", "amg_server_submit", "amg_server_poll", "amg_server_wait",
    "amg_server_stats", "amg_server_destroy",
]


class amg_options(C.Structure):
    _fields_ = [("degree", C.c_int), ("passes", C.c_int), ("coarse_max", C.c_int),
                ("max_levels", C.c_int), ("inner_iters", C.c_int), ("restart", C.c_int),
                ("max_iters", C.c_int), ("precision", C.c_int), ("lambda0_ratio", C.c_double),
                ("hash_salt", C.c_uint64), ("cycle", C.c_int), ("amli_alpha", C.c_double),
                ("rho", C.c_double), ("aggregation", C.c_int), ("mis_k", C.c_int)]


class amg_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("n_levels", C.c_int),
                ("grid_complexity", C.c_double), ("op_complexity", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("history", C.POINTER(C.c_double)), ("history_cap", C.c_int), ("history_len", C.c_int)]


class amg_server_config(C.Structure):
    _fields_ = [("mem_cap_bytes", C.c_size_t), ("max_active", C.c_int), ("batch_max", C.c_int),
                ("opt", amg_options)]


class amg_server_stats_t(C.Structure):
    _fields_ = [("resident_bytes", C.c_size_t), ("peak_resident_bytes", C.c_size_t), ("active", C.c_int),
                ("peak_active", C.c_int), ("queued", C.c_int64), ("completed", C.c_int64),
                ("setups", C.c_int64), ("evictions", C.c_int64), ("solves", C.c_int64),
                ("setup_retries", C.c_int64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libamg_gb300.so (building it with nvcc if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path}")
            L = C.CDLL(path)
            P, I64, I = C.c_void_p, C.c_int64, C.c_int
            L.amg_default_options.argtypes = [C.POINTER(amg_options)]
            L.amg_default_options.restype = None
            L.amg_degree_for.argtypes = [C.c_double, C.c_double]
            L.amg_degree_for.restype = C.c_int
            L.amg_setup.argtypes = [I64, P, P, P, P, C.POINTER(amg_options), I, P, C.POINTER(C.c_void_p)]
            L.amg_solve.argtypes = [P, P, P, I, I64, C.c_double, C.POINTER(amg_info)]
            L.amg_free.argtypes = [P]
            L.amg_free.restype = None
            L.amg_last_error.argtypes = [P]
            L.amg_last_error.restype = C.c_char_p
            L.amg_num_levels.argtypes = [P]
            L.amg_level_n.argtypes = [P, I]
            L.amg_level_n.restype = I64
            L.amg_level_nnz.argtypes = [P, I]
            L.amg_level_nnz.restype = I64
            L.amg_level_csr.argtypes = [P, I, P, P, P, P, P]
            L.amg_level_agg.argtypes = [P, I, P]
            L.amg_level_smoother.argtypes = [P, I, C.POINTER(C.c_double), C.POINTER(C.c_double), P]
            for name in ("amg_apply_spmv", "amg_apply_smoother", "amg_apply_restrict",
                         "amg_apply_prolong_add", "amg_apply_kcycle"):
                getattr(L, name).argtypes = [P, I, P, P]
            L.amg_apply_coarse_solve.argtypes = [P, P, P]
            L.amg_match.argtypes = [I64, P, P, P, C.c_uint64, P, P, C.POINTER(I64), C.POINTER(I), P]
            L.amg_match_noalloc.argtypes = [I64, P, P, P, C.c_uint64, P, P, C.POINTER(I64), C.POINTER(I), P]
            L.amg_kernel_timing.argtypes = [P, I]
            L.amg_kernel_timing_read.argtypes = [P, C.POINTER(I64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.amg_kernel_timing_read_kind.argtypes = [P, I, C.POINTER(I64), C.POINTER(C.c_double),
                                                      C.POINTER(C.c_double)]
            L.amg_launch_count.argtypes = [P]
            L.amg_launch_count.restype = I64
            L.amg_server_create.argtypes = [C.POINTER(amg_server_config), C.POINTER(C.c_void_p)]
            L.amg_server_add_graph.argtypes = [P, I64, P, P, P, P, C.POINTER(I64)]
            L.amg_server_submit.argtypes = [P, I64, P, C.c_double, C.POINTER(I64)]
            L.amg_server_poll.argtypes = [P, I64, P, C.POINTER(amg_info), C.POINTER(I), C.POINTER(C.c_double)]
            L.amg_server_wait.argtypes = [P, I64, P, C.POINTER(amg_info), C.POINTER(C.c_double)]
            L.amg_server_stats.argtypes = [P, C.POINTER(amg_server_stats_t)]
            L.amg_server_destroy.argtypes = [P]
            L.amg_server_destroy.restype = None
            _lib = L
    return _lib


def ptr(a) -> int | None:
    """Raw address of a numpy array / torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


class AmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"amg status {status}: {msg}")
        self.status = status


# ---- thin wrappers with the C names ----------------------------------------
def amg_degree_for(rho: float, lambda0_ratio: float = 0.1) -> int:
    """Smoother degree of Eq. (bound-on-m) for damping rho (-1: none <= 16)."""
    return lib().amg_degree_for(rho, lambda0_ratio)


def amg_default_options(**overrides) -> amg_options:
    o = amg_options()
    lib().amg_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def amg_setup(n, row_ptr, col_idx, w, d=None, opt=None, mem_space=AMG_MEM_HOST, stream=None):
    """Returns (status, handle)."""
    h = C.c_void_p()
    st = lib().amg_setup(n, ptr(row_ptr), ptr(col_idx), ptr(w), ptr(d),
                         C.byref(opt) if opt is not None else None, mem_space, stream, C.byref(h))
    return st, h


def amg_solve(h, rhs, x, nrhs, ld, tol, info=None):
    return lib().amg_solve(h, ptr(rhs), ptr(x), nrhs, ld, tol, C.byref(info) if info is not None else None)


def amg_free(h):
    lib().amg_free(h)


def amg_last_error(h=None) -> str:
    m = lib().amg_last_error(h)
    return m.decode() if m else ""


def amg_match(n, row_ptr, col_idx, s, salt, mate, agg, stream=None):
    nH = C.c_int64(0)
    rounds = C.c_int(0)
    st = lib().amg_match(n, ptr(row_ptr), ptr(col_idx), ptr(s), C.c_uint64(salt), ptr(mate), ptr(agg),
                         C.byref(nH), C.byref(rounds), stream)
    return st, nH.value, rounds.value


def amg_match_noalloc(n, row_ptr, col_idx, s, salt, mate, agg, stream=None):
    """amg_match without device allocation (fixed in-library scratch, n <= 2^20)."""
    nH = C.c_int64(0)
    rounds = C.c_int(0)
    st = lib().amg_match_noalloc(n, ptr(row_ptr), ptr(col_idx), ptr(s), C.c_uint64(salt), ptr(mate),
                                 ptr(agg), C.byref(nH), C.byref(rounds), stream)
    return st, nH.value, rounds.value


class Hierarchy:
    """Owns one amg_handle (the C handle); methods forward to the C ABI."""

    def __init__(self, n, row_ptr, col_idx, w, d=None, mem_space=AMG_MEM_HOST, stream=None, **opts):
        self.opt = amg_default_options(**opts)
        self._keep = (row_ptr, col_idx, w, d)
        self.status, self.h = amg_setup(n, row_ptr, col_idx, w, d, self.opt, mem_space, stream)
        self.error = amg_last_error(None) if self.status else ""
        self.n = n
        if self.status != AMG_OK:
            self.h = None
        elif self.opt.rho > 0:  # the degree the handle derived from rho
            self.opt.degree = amg_degree_for(self.opt.rho, self.opt.lambda0_ratio)

    @classmethod
    def from_graph(cls, g, mem_space=AMG_MEM_HOST, stream=None, device="cuda", **opts):
        if mem_space == AMG_MEM_DEVICE:
            import torch

            t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
            args = (t(g.rowptr, torch.int64), t(g.col, torch.int32), t(g.w, torch.float64),
                    None if g.d is None else t(g.d, torch.float64))
        else:
            args = (np.ascontiguousarray(g.rowptr, np.int64), np.ascontiguousarray(g.col, np.int32),
                    np.ascontiguousarray(g.w, np.float64),
                    None if g.d is None else np.ascontiguousarray(g.d, np.float64))
        return cls(g.n, *args, mem_space=mem_space, stream=stream, **opts)

    def close(self):
        if getattr(self, "h", None):
            amg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st not in (AMG_OK,):
            raise AmgError(st, amg_last_error(self.h))

    @property
    def n_levels(self) -> int:
        return lib().amg_num_levels(self.h)

    def level_n(self, k: int) -> int:
        return lib().amg_level_n(self.h, k)

    def level_csr(self, k: int):
        n = self.level_n(k)
        nnz = lib().amg_level_nnz(self.h, k)
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1))
        diag = np.zeros(n)
        dlow = np.zeros(n)
        self._check(lib().amg_level_csr(self.h, k, ptr(rp), ptr(col), ptr(val), ptr(diag), ptr(dlow)))
        return rp, col[:nnz], val[:nnz], diag, dlow

    def level_agg(self, k: int) -> np.ndarray:
        agg = np.zeros(self.level_n(k), np.int32)
        self._check(lib().amg_level_agg(self.h, k, ptr(agg)))
        return agg

    def level_smoother(self, k: int):
        l0, l1 = C.c_double(), C.c_double()
        coef = np.zeros(self.opt.degree + 1)
        self._check(lib().amg_level_smoother(self.h, k, C.byref(l0), C.byref(l1), ptr(coef)))
        return l0.value, l1.value, coef

    def apply(self, name: str, k: int, a, b):
        fn = getattr(lib(), "amg_apply_" + name)
        self._check(fn(self.h, k, ptr(a), ptr(b)))

    def coarse_solve(self, b, x):
        self._check(lib().amg_apply_coarse_solve(self.h, ptr(b), ptr(x)))

    def solve(self, rhs, x, tol=1e-8, nrhs=1, ld=None, history_cap=4096):
        info = amg_info()
        hist = np.zeros(history_cap)
        info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
        info.history_cap = history_cap
        st = amg_solve(self.h, rhs, x, nrhs, self.n if ld is None else ld, tol, info)
        return st, info, hist[: info.history_len].copy()

    def kernel_timing(self, enable: bool):
        self._check(lib().amg_kernel_timing(self.h, 1 if enable else 0))

    def kernel_timing_read(self):
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        self._check(lib().amg_kernel_timing_read(self.h, C.byref(n), C.byref(ms), C.byref(b)))
        return n.value, ms.value, b.value

    def launch_count(self) -> int:
        return lib().amg_launch_count(self.h)


class Server:
    """Continuous-batching solve server (amg_server_* of the C ABI)."""

    def __init__(self, mem_cap_bytes: int, max_active: int, batch_max: int = 8, **opts):
        cfg = amg_server_config()
        cfg.mem_cap_bytes = int(mem_cap_bytes)
        cfg.max_active = int(max_active)
        cfg.batch_max = int(batch_max)
        cfg.opt = amg_default_options(**opts)
        h = C.c_void_p()
        self.status = lib().amg_server_create(C.byref(cfg), C.byref(h))
        if self.status != AMG_OK:
            raise AmgError(self.status, amg_last_error(None))
        self.h = h
        self._n = {}

    def add_graph(self, g) -> int:
        rp = np.ascontiguousarray(g.rowptr, np.int64)
        col = np.ascontiguousarray(g.col, np.int32)
        w = np.ascontiguousarray(g.w, np.float64)
        d = None if g.d is None else np.ascontiguousarray(g.d, np.float64)
        gid = C.c_int64()
        st = lib().amg_server_add_graph(self.h, g.n, ptr(rp), ptr(col), ptr(w), ptr(d), C.byref(gid))
        if st != AMG_OK:
            raise AmgError(st, amg_last_error(None))
        self._n[gid.value] = g.n
        return gid.value

    def submit(self, graph_id: int, rhs: np.ndarray, tol: float = 1e-8) -> int:
        rhs = np.ascontiguousarray(rhs, np.float64)
        t = C.c_int64()
        st = lib().amg_server_submit(self.h, graph_id, ptr(rhs), tol, C.byref(t))
        if st != AMG_OK:
            raise AmgError(st, amg_last_error(None))
        self._n[("t", t.value)] = self._n[graph_id]
        return t.value

    def wait(self, ticket: int):
        """(status, x, info, latency_ms)"""
        x = np.zeros(self._n.pop(("t", ticket)))
        info = amg_info()
        lat = C.c_double()
        st = lib().amg_server_wait(self.h, ticket, ptr(x), C.byref(info), C.byref(lat))
        return st, x, info, lat.value

    def stats(self) -> amg_server_stats_t:
        s = amg_server_stats_t()
        lib().amg_server_stats(self.h, C.byref(s))
        return s

    def close(self):
        if getattr(self, "h", None):
            lib().amg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
