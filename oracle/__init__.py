"""Python loader for the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg and ``--impl reference`` arm may import this package.  It compiles ``amg_oracle.c`` with gcc on first
use (or via :func:`build`) and wraps it with ctypes; nothing here shares code
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_HDR = os.path.join(_HERE, "amg_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_NOT_SYMMETRIC, ERR_SELF_LOOP, ERR_BAD_WEIGHT = 0, 1, 2, 3, 4
ERR_DISCONNECTED, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_SETUP_STALL = 5, 6, 8, 9, 11
PREC_KCYCLE, PREC_IDENTITY, PREC_EXACT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (plain C99, -O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_OUT)
    if force or stale:
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class Options(C.Structure):
    _fields_ = [("degree", C.c_int), ("passes", C.c_int), ("coarse_max", C.c_int),
                ("max_levels", C.c_int), ("inner_iters", C.c_int), ("restart", C.c_int),
                ("max_iters", C.c_int), ("precond", C.c_int), ("lambda0_ratio", C.c_double),
                ("hash_salt", C.c_uint64), ("cycle", C.c_int), ("amli_alpha", C.c_double),
                ("rho", C.c_double), ("aggregation", C.c_int), ("mis_k", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("n_levels", C.c_int),
                ("grid_complexity", C.c_double), ("op_complexity", C.c_double),
                ("history", C.POINTER(C.c_double)), ("history_cap", C.c_int), ("history_len", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_default_options.argtypes = [C.POINTER(Options)]
            L.orc_match.argtypes = [C.c_int, P, P, P, C.c_uint64, P, P, C.POINTER(C.c_int)]
            L.orc_match.restype = C.c_int
            L.orc_remez_inverse.argtypes = [C.c_int, C.c_double, C.c_double, P, C.POINTER(C.c_double), P]
            L.orc_jacobi_eigen.argtypes = [C.c_int, P, P, P]
            L.orc_setup.argtypes = [C.c_int64, P, P, P, P, C.POINTER(Options), C.POINTER(C.c_void_p)]
            L.orc_solve.argtypes = [C.c_void_p, P, P, C.c_double, C.POINTER(Info)]
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_num_levels.argtypes = [C.c_void_p]
            for name in ("orc_level_n", "orc_level_nnz"):
                getattr(L, name).argtypes = [C.c_void_p, C.c_int]
                getattr(L, name).restype = C.c_int64
            L.orc_level_csr.argtypes = [C.c_void_p, C.c_int, P, P, P, P, P]
            L.orc_level_agg.argtypes = [C.c_void_p, C.c_int, P]
            L.orc_level_pass_count.argtypes = [C.c_void_p, C.c_int]
            L.orc_level_pass_n.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_level_pass_n.restype = C.c_int64
            L.orc_level_pass_agg.argtypes = [C.c_void_p, C.c_int, C.c_int, P]
            L.orc_level_lambda.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_level_cheb.argtypes = [C.c_void_p, C.c_int, P]
            L.orc_amli_coef.argtypes = [C.c_void_p, P]
            L.orc_mis_aggregate.argtypes = [C.c_int, P, P, C.c_int, C.c_uint64, P, P]
            L.orc_mis_aggregate.restype = C.c_int
            L.orc_degree_for.argtypes = [C.c_double, C.c_double]
            L.orc_degree_for.restype = C.c_int
            for name in ("orc_spmv", "orc_smooth", "orc_restrict", "orc_prolong_add", "orc_kcycle",
                         "orc_inner_fcg", "orc_amli_cycle"):
                getattr(L, name).argtypes = [C.c_void_p, C.c_int, P, P]
            L.orc_coarse_solve.argtypes = [C.c_void_p, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_options(**kw) -> Options:
    o = Options()
    lib().orc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def match(rowptr, col, w, salt: int = 0):
    """One handshake matching pass: returns (mate, agg, n_coarse, rounds)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = rowptr.size - 1
    mate = np.empty(n, np.int32)
    agg = np.empty(n, np.int32)
    rounds = C.c_int(0)
    nH = lib().orc_match(n, _p(rowptr), _p(col), _p(w), C.c_uint64(salt), _p(mate), _p(agg), C.byref(rounds))
    return mate, agg, nH, rounds.value


def mis_aggregate(rowptr, col, k: int = 4, salt: int = 0):
    """Sec. 2 aggregation: (agg, is_root, n_aggregates) from the MIS of the graph of A^k."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = rowptr.size - 1
    agg = np.empty(n, np.int32)
    root = np.empty(n, np.int32)
    nH = lib().orc_mis_aggregate(n, _p(rowptr), _p(col), k, C.c_uint64(salt), _p(agg), _p(root))
    return agg, root.astype(bool), nH


def degree_for(rho: float, lambda0_ratio: float = 0.1) -> int:
    """Smoother degree from Eq. (bound-on-m): smallest m with E_m <= rho and E_m < 1 (-1: none)."""
    return lib().orc_degree_for(rho, lambda0_ratio)


def remez_inverse(m: int, l0: float, l1: float):
    """(coefficients, max error on [l0,l1], alternation points) of q_m, Eq. (1x-1-min)."""
    c = np.zeros(m + 1)
    alt = np.zeros(m + 2)
    err = C.c_double(0)
    rc = lib().orc_remez_inverse(m, l0, l1, _p(c), C.byref(err), _p(alt))
    if rc:
        raise RuntimeError(f"remez failed: {rc}")
    return c, err.value, alt


def jacobi_eigen(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    ev = np.zeros(n)
    V = np.zeros((n, n))
    lib().orc_jacobi_eigen(n, _p(A), _p(ev), _p(V))
    return ev, V


@dataclass
class SolveResult:
    status: int
    x: np.ndarray
    iterations: int
    converged: bool
    rel_residual: float
    true_rel_residual: float
    n_levels: int
    grid_complexity: float
    op_complexity: float
    history: np.ndarray = field(repr=False)


class Hierarchy:
    """Oracle hierarchy built by orc_setup; owns the C handle."""

    def __init__(self, g, **opts):
        self._keep = (np.ascontiguousarray(g.rowptr, np.int64), np.ascontiguousarray(g.col, np.int32),
                      np.ascontiguousarray(g.w, np.float64),
                      None if g.d is None else np.ascontiguousarray(g.d, np.float64))
        rp, col, w, d = self._keep
        self.opts = default_options(**opts)
        h = C.c_void_p()
        self.status = lib().orc_setup(g.n, _p(rp), _p(col), _p(w), None if d is None else _p(d),
                                      C.byref(self.opts), C.byref(h))
        self.h = h if self.status == 0 else None
        self.n = g.n
        if self.status == 0 and self.opts.rho > 0:  # the degree the hierarchy uses
            self.opts.degree = degree_for(self.opts.rho, self.opts.lambda0_ratio)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    @property
    def n_levels(self) -> int:
        return lib().orc_num_levels(self.h)

    def level_n(self, k: int) -> int:
        return lib().orc_level_n(self.h, k)

    def level_csr(self, k: int):
        """(rowptr, col, val, diag, dlow) of level k; val = off-diagonal a_ij."""
        n = self.level_n(k)
        nnz = lib().orc_level_nnz(self.h, k)
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1))
        diag = np.zeros(n)
        dlow = np.zeros(n)
        lib().orc_level_csr(self.h, k, _p(rp), _p(col), _p(val), _p(diag), _p(dlow))
        return rp, col[:nnz], val[:nnz], diag, dlow

    def level_dense(self, k: int) -> np.ndarray:
        rp, col, val, diag, _ = self.level_csr(k)
        n = rp.size - 1
        A = np.diag(diag)
        rows = np.repeat(np.arange(n), np.diff(rp))
        A[rows, col] = val
        return A

    def level_agg(self, k: int) -> np.ndarray:
        agg = np.zeros(self.level_n(k), np.int32)
        rc = lib().orc_level_agg(self.h, k, _p(agg))
        if rc:
            raise IndexError(k)
        return agg

    def level_pass_aggs(self, k: int):
        out = []
        for p in range(lib().orc_level_pass_count(self.h, k)):
            a = np.zeros(lib().orc_level_pass_n(self.h, k, p), np.int32)
            lib().orc_level_pass_agg(self.h, k, p, _p(a))
            out.append(a)
        return out

    def level_lambda(self, k: int):
        l0, l1 = C.c_double(), C.c_double()
        lib().orc_level_lambda(self.h, k, C.byref(l0), C.byref(l1))
        return l0.value, l1.value

    def level_cheb(self, k: int) -> np.ndarray:
        c = np.zeros(self.opts.degree + 1)
        lib().orc_level_cheb(self.h, k, _p(c))
        return c

    def _op(self, name: str, k: int, v: np.ndarray, n_out: int) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(n_out)
        if name == "orc_prolong_add":
            out = v[1].copy()
            v = np.ascontiguousarray(v[0])
        rc = getattr(lib(), name)(self.h, k, _p(v), _p(out))
        if rc:
            raise RuntimeError(f"{name} failed: {rc}")
        return out

    def spmv(self, k, x):
        return self._op("orc_spmv", k, x, self.level_n(k))

    def smooth(self, k, r):
        return self._op("orc_smooth", k, r, self.level_n(k))

    def restrict(self, k, s):
        return self._op("orc_restrict", k, s, self.level_n(k + 1))

    def prolong_add(self, k, eH, x):
        eH = np.ascontiguousarray(eH, np.float64)
        out = np.ascontiguousarray(x, np.float64).copy()
        rc = lib().orc_prolong_add(self.h, k, _p(eH), _p(out))
        if rc:
            raise RuntimeError(rc)
        return out

    def kcycle(self, k, r):
        return self._op("orc_kcycle", k, r, self.level_n(k))

    def amli_cycle(self, k, r):
        """x = B_k r, the stationary AMLI W-cycle (cycle=1 hierarchies)."""
        return self._op("orc_amli_cycle", k, r, self.level_n(k))

    def amli_coef(self) -> np.ndarray:
        c = np.zeros(self.opts.inner_iters)
        if lib().orc_amli_coef(self.h, _p(c)):
            raise RuntimeError("not an AMLI-cycle hierarchy")
        return c

    def inner_fcg(self, k, b):
        return self._op("orc_inner_fcg", k, b, self.level_n(k))

    def coarse_solve(self, b):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        lib().orc_coarse_solve(self.h, _p(b), _p(x))
        return x

    def solve(self, b: np.ndarray, tol: float = 1e-8, history_cap: int = 4096) -> SolveResult:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        hist = np.zeros(history_cap)
        info = Info()
        info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
        info.history_cap = history_cap
        st = lib().orc_solve(self.h, _p(b), _p(x), tol, C.byref(info))
        return SolveResult(st, x, info.iterations, bool(info.converged), info.rel_residual,
                           info.true_rel_residual, info.n_levels, info.grid_complexity,
                           info.op_complexity, hist[: info.history_len].copy())
