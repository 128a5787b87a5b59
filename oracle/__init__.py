"""CPU oracle for block principal pivoting NNLS -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it: the two meet only on the seeded inputs of the
``workloads`` package.

Contents
  * ``tsnnls_oracle.c`` (built here into ``_build/liboracle.so``): plain FP64
    BPP following the algorithm box of Section 2, the column-dot Gram of
    Section 3, a textbook Cholesky, Householder QR and LSQR final steps.
  * ``lcp_enumerate``: the plain definition of the solution of Eq. 3 by
    enumerating every complementary split (F, G), for n <= 12.
  * ``kkt``: the optimality certificate of Eq. 3 for any x.

Parity status: every function here is pinned by a CPU test (brute-force
enumeration, scipy's Lawson-Hanson NNLS, numpy's lstsq/cholesky, closed
forms, constructed solutions); the exchange rule of the algorithm box,
including the index the single-variable fallback moves, by a hand-worked
example and by a numpy replay of every trace row.  The only unpinned
quantity is the pivot *count* of the paper's own problems: the paper prints
no worked iteration, so iteration counts have no external reference (parity
unpinned for iteration counts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsnnls_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

OK, EMAXITER, ENOTPD, EINVAL, ENOMEM = 0, 1, 2, 3, 4
INNER_CHOLESKY, INNER_LSQR = 0, 1
FINAL_NONE, FINAL_QR, FINAL_LSQR = 0, 1, 2


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O3 -ffp-contract=off)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
                    "-shared", "-Wall", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Opts(ctypes.Structure):
    _fields_ = [("zero_tol", ctypes.c_double), ("p_max", ctypes.c_int64),
                ("max_iter", ctypes.c_int64), ("inner", ctypes.c_int32),
                ("final_step", ctypes.c_int32), ("lsqr_atol", ctypes.c_double),
                ("lsqr_max_it", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("final_k", ctypes.c_int64),
                ("lsqr_steps", ctypes.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        _lib.oracle_gram.argtypes = [i64, i64, p, p, p, p]
        _lib.oracle_atb.argtypes = [i64, i64, p, p, p, p, p]
        _lib.oracle_cholesky.argtypes = [i64, p]
        _lib.oracle_cholesky_solve.argtypes = [i64, p, p, p]
        _lib.oracle_qr_lstsq.argtypes = [i64, i64, p, p, p]
        _lib.oracle_bpp_solve.argtypes = [i64, i64, p, p, p, p, ctypes.POINTER(_Opts), p, p, p,
                                          ctypes.POINTER(_Info), p, i64]
        for f in ("oracle_gram", "oracle_atb", "oracle_cholesky", "oracle_qr_lstsq",
                  "oracle_bpp_solve"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(prob):
    rp = np.ascontiguousarray(prob.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(prob.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(prob.val, dtype=np.float64)
    return rp, ci, va


def gram(prob) -> np.ndarray:
    """A^T A by column dot products (Section 3), dense n x n."""
    rp, ci, va = _csr(prob)
    g = np.empty((prob.n, prob.n))
    st = _load().oracle_gram(prob.m, prob.n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(g))
    if st:
        raise OracleError(st, "gram")
    return g


def atb(prob) -> np.ndarray:
    """A^T b (Eq. 2's linear term)."""
    rp, ci, va = _csr(prob)
    b = np.ascontiguousarray(prob.b, dtype=np.float64)
    c = np.empty(prob.n)
    st = _load().oracle_atb(prob.m, prob.n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b), _ptr(c))
    if st:
        raise OracleError(st, "atb")
    return c


def cholesky(s: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of a symmetric positive definite matrix."""
    a = np.array(s, dtype=np.float64, order="C", copy=True)
    st = _load().oracle_cholesky(a.shape[0], _ptr(a))
    if st:
        raise OracleError(st, "cholesky")
    return np.tril(a)


def cholesky_solve(L: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    r = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.empty_like(r)
    _load().oracle_cholesky_solve(L.shape[0], _ptr(L), _ptr(r), _ptr(x))
    return x


def qr_lstsq(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """min ||M z - rhs|| by Householder QR."""
    m, k = M.shape
    a = np.asfortranarray(np.array(M, dtype=np.float64, copy=True))
    r = np.array(rhs, dtype=np.float64, copy=True)
    z = np.empty(k)
    st = _load().oracle_qr_lstsq(m, k, _ptr(a), _ptr(r), _ptr(z))
    if st:
        raise OracleError(st, "qr_lstsq")
    return z


class Result:
    def __init__(self, x, y, inF, iters, final_k, lsqr_steps, trace):
        self.x, self.y, self.inF = x, y, inF
        self.iters, self.final_k, self.lsqr_steps = iters, final_k, lsqr_steps
        self.trace = trace


def bpp_solve(prob, *, zero_tol=1e-12, p_max=3, max_iter=None, inner=INNER_CHOLESKY,
              final_step=FINAL_QR, lsqr_atol=1e-15, lsqr_max_it=None,
              trace_cap=1000) -> Result:
    """Block principal pivoting (Section 2, algorithm box) in FP64."""
    rp, ci, va = _csr(prob)
    b = np.ascontiguousarray(prob.b, dtype=np.float64)
    n, m = prob.n, prob.m
    opts = _Opts(zero_tol, p_max, max_iter if max_iter is not None else 10 * n + 100, inner,
                 final_step, lsqr_atol, lsqr_max_it if lsqr_max_it is not None else 4 * n + 100)
    info = _Info()
    x = np.empty(n)
    y = np.empty(n)
    inF = np.empty(n, dtype=np.uint8)
    trace = np.zeros((trace_cap, 6), dtype=np.int64)
    st = _load().oracle_bpp_solve(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b),
                                  ctypes.byref(opts), _ptr(x), _ptr(y), _ptr(inF),
                                  ctypes.byref(info), _ptr(trace), trace_cap)
    if st:
        raise OracleError(st, "bpp_solve")
    return Result(x, y, inF.astype(bool), info.iters, info.final_k, info.lsqr_steps,
                  trace[: min(info.iters, trace_cap)])
