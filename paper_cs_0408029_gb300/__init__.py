"""Python binding of libtsnnls (include/tsnnls.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels.  There is no CPU
path: if the library is missing or no GPU is usable, the calls raise.

Host inputs are numpy arrays; device inputs are torch CUDA tensors (PyTorch
provides device memory and streams here, nothing else).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

(OK, EINVAL, ENOMEM, EADMIT, ENOTPD, EMAXITER, ENOCONV, ETIMEOUT, PENDING, ECUDA, ENODEV, ENOTFOUND,
 EBOUNDS) = range(13)
MIXED, FP64 = 0, 1
PATH_AUTO, PATH_FACTOR, PATH_LSQR, PATH_SPARSE = 0, 1, 2, 3
WAIT_PROBE_MAX_POLLS = 1 << 22  # TSNNLS_WAIT_PROBE_MAX_POLLS

# every entry point declared in include/tsnnls.h
EXPORTS = (
    "tsnnls_opts_default", "tsnnls_strerror", "tsnnls_ctx_create", "tsnnls_ctx_destroy",
    "tsnnls_solve", "tsnnls_solve_ex", "tsnnls_submit", "tsnnls_poll", "tsnnls_wait",
    "tsnnls_solve_batch_dense", "tsnnls_gram", "tsnnls_gather", "tsnnls_cholesky",
    "tsnnls_chol_solve", "tsnnls_spmv", "tsnnls_profile_enable", "tsnnls_profile_read",
    "tsnnls_chol_solve_noalloc", "tsnnls_batch_autotune", "tsnnls_batch_set_panel",
    "tsnnls_queue_stats_read", "tsnnls_wait_probe", "tsnnls_submit_batch",
    "tsnnls_batch_member_info", "tsnnls_sparse_analyze", "tsnnls_solve_batch_dense_ex",
    "tsnnls_batch_autotune_cached", "tsnnls_batch_tune_key", "tsnnls_tune_cache_get",
    "tsnnls_tune_cache_put", "tsnnls_check_build", "tsnnls_check_report", "tsnnls_sparse_supernodes",
)

PHASES = ("setup", "gram", "exchange", "gather", "factor", "trsv", "spmv", "vector", "lsqr",
          "factor_diag", "factor_panel", "factor_update", "reuse")


class TsnnlsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} (status {status})")


class CSR(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("zero_tol", ctypes.c_double),
                ("p_max", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("path", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("full_refine", ctypes.c_int32),
                ("no_fallback", ctypes.c_int32), ("cond_est", ctypes.c_int32),
                ("no_reuse", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("nF", ctypes.c_int32),
                ("path_used", ctypes.c_int32), ("precision_used", ctypes.c_int32),
                ("last_rel_step", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("cond_est", ctypes.c_double),
                ("fallback_used", ctypes.c_int32), ("factor_reuses", ctypes.c_int32),
                ("kkt_viol", ctypes.c_double), ("rel_resid_change", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SparseStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_gram", ctypes.c_int64), ("nnz_l", ctypes.c_int64),
                ("supernodes", ctypes.c_int64), ("max_height", ctypes.c_int64),
                ("factor_flops", ctypes.c_double), ("analysis_ms", ctypes.c_double),
                ("nnz_l_stored", ctypes.c_int64), ("update_entries", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build_mod.LIB


def load(build_if_missing: bool = True):
    """Load libtsnnls.so (building it first if needed); with TSNNLS_CHECK=1
    in the environment, the bounds-checked libtsnnls_check.so instead."""
    global _lib
    if _lib is not None:
        return _lib
    variant = "check" if os.environ.get("TSNNLS_CHECK", "") not in ("", "0") else "normal"
    path = _build_mod.VARIANTS[variant][0]
    if build_if_missing and not _build_mod.up_to_date(variant):
        _build_mod.build(variants=(variant,))
    if not os.path.exists(path):
        raise RuntimeError(f"libtsnnls is not built ({path}); run paper_cs_0408029_gb300.build")
    lib = ctypes.CDLL(path)
    p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sigs = {
        "tsnnls_opts_default": ([ctypes.POINTER(Opts)], None),
        "tsnnls_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "tsnnls_ctx_create": ([ctypes.POINTER(p), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "tsnnls_ctx_destroy": ([p], None),
        "tsnnls_solve": ([p, ctypes.POINTER(CSR), p, p, ctypes.POINTER(Opts), ctypes.POINTER(Info)],
                         ctypes.c_int),
        "tsnnls_solve_ex": ([p, ctypes.POINTER(CSR), p, p, p, p, p, i64, ctypes.POINTER(Opts),
                             ctypes.POINTER(Info)], ctypes.c_int),
        "tsnnls_submit": ([p, ctypes.POINTER(CSR), p, p, ctypes.POINTER(Opts),
                           ctypes.POINTER(i64)], ctypes.c_int),
        "tsnnls_poll": ([p, i64, ctypes.POINTER(Info)], ctypes.c_int),
        "tsnnls_wait": ([p, i64, i64, ctypes.POINTER(Info)], ctypes.c_int),
        "tsnnls_solve_batch_dense": ([p, i32, p, p, p, p, p, ctypes.POINTER(Opts), p,
                                      ctypes.POINTER(Info)], ctypes.c_int),
        "tsnnls_solve_batch_dense_ex": ([p, i32, p, p, p, p, p, ctypes.POINTER(Opts), p,
                                         ctypes.POINTER(Info), p, i64], ctypes.c_int),
        "tsnnls_gram": ([p, ctypes.POINTER(CSR), p, i32, p, i64, p], ctypes.c_int),
        "tsnnls_gather": ([p, i32, p, i64, p, i64, p, i64], ctypes.c_int),
        "tsnnls_cholesky": ([p, i32, p, i64, i64, ctypes.POINTER(i32)], ctypes.c_int),
        "tsnnls_chol_solve": ([p, i32, p, i64, i64, p], ctypes.c_int),
        "tsnnls_spmv": ([p, ctypes.POINTER(CSR), i32, d, p, d, p, p], ctypes.c_int),
        "tsnnls_profile_enable": ([p, i32], ctypes.c_int),
        "tsnnls_profile_read": ([p, p, i32], ctypes.c_int),
        "tsnnls_chol_solve_noalloc": ([i32, p, i64, i64, p, p], ctypes.c_int),
        "tsnnls_wait_probe": ([i64], ctypes.c_int),
        "tsnnls_batch_autotune": ([p, i32, i32, p], ctypes.c_int),
        "tsnnls_batch_set_panel": ([i32, p], ctypes.c_int),
        "tsnnls_batch_autotune_cached": ([p, i32, i32, ctypes.c_char_p, p, ctypes.POINTER(i32)], ctypes.c_int),
        "tsnnls_batch_tune_key": ([p, i32, i32, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "tsnnls_check_build": ([], ctypes.c_int),
        "tsnnls_check_report": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "tsnnls_tune_cache_get": ([ctypes.c_char_p, ctypes.c_char_p, p], ctypes.c_int),
        "tsnnls_tune_cache_put": ([ctypes.c_char_p, ctypes.c_char_p, p], ctypes.c_int),
        "tsnnls_queue_stats_read": ([p, p], ctypes.c_int),
        "tsnnls_submit_batch": ([p, i32, p, p, p, ctypes.POINTER(Opts), ctypes.POINTER(i64)],
                                ctypes.c_int),
        "tsnnls_batch_member_info": ([p, i64, i32, ctypes.POINTER(Info)], ctypes.c_int),
        "tsnnls_sparse_analyze": ([i64, i64, p, p, i32, p, p, ctypes.POINTER(SparseStats)], ctypes.c_int),
        "tsnnls_sparse_supernodes": ([i64, i64, p, p, i32, p, p, p, p, p], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def check_build():
    """True if the loaded library is the bounds-checked build."""
    return bool(load().tsnnls_check_build())


def check_report():
    """(failing accesses since the last call, first one's description)."""
    buf = ctypes.create_string_buffer(512)
    hits = load().tsnnls_check_report(buf, len(buf))
    return hits, buf.value.decode()


def tune_cache_get(path, key):
    """The 5 cached widths for key, or None if the file or the key is absent."""
    nb = np.zeros(5, dtype=np.int32)
    st = load().tsnnls_tune_cache_get(os.fsencode(path), key.encode(), _np_ptr(nb))
    if st == ENOTFOUND:
        return None
    _check(st, "tune_cache_get")
    return nb


def tune_cache_put(path, key, nb):
    arr = np.ascontiguousarray(nb, dtype=np.int32)
    if arr.shape != (5,):
        raise ValueError("five widths expected")
    _check(load().tsnnls_tune_cache_put(os.fsencode(path), key.encode(), _np_ptr(arr)), "tune_cache_put")


def strerror(status: int) -> str:
    try:
        return load(build_if_missing=False).tsnnls_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return f"status {status}"


def _check(st, what):
    if st != OK:
        raise TsnnlsError(st, what)


def default_opts(**kw) -> Opts:
    o = Opts()
    load().tsnnls_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"mixed": MIXED, "fp64": FP64}[v]
        if k == "path" and isinstance(v, str):
            v = {"auto": PATH_AUTO, "factor": PATH_FACTOR, "lsqr": PATH_LSQR, "sparse": PATH_SPARSE}[v]
        setattr(o, k, v)
    return o


def sparse_analyze(m, n, row_ptr, col_idx, max_width=64):
    """Host-only symbolic analysis of the sparse path: (perm, parent, stats dict)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    perm = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    st = SparseStats()
    _check(load().tsnnls_sparse_analyze(int(m), int(n), _np_ptr(rp), _np_ptr(ci), int(max_width), _np_ptr(perm),
                                        _np_ptr(parent), ctypes.byref(st)), "sparse_analyze")
    return perm, parent, {f: getattr(st, f) for f, _ in st._fields_}


def sparse_supernodes(m, n, row_ptr, col_idx, max_width=64):
    """Host-only supernodal tree of the sparse analysis: (sn_first, sparent,
    order_up, order_down) as int32 arrays."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    ns = ctypes.c_int64(0)
    f = load().tsnnls_sparse_supernodes
    _check(f(int(m), int(n), _np_ptr(rp), _np_ptr(ci), int(max_width), ctypes.byref(ns), None, None, None, None),
           "sparse_supernodes")
    k = int(ns.value)
    first = np.empty(k + 1, dtype=np.int32)
    sparent, up, down = (np.empty(k, dtype=np.int32) for _ in range(3))
    _check(f(int(m), int(n), _np_ptr(rp), _np_ptr(ci), int(max_width), ctypes.byref(ns), _np_ptr(first),
             _np_ptr(sparent), _np_ptr(up), _np_ptr(down)), "sparse_supernodes")
    return first, sparent, up, down


def wait_probe(polls: int) -> int:
    """Status of one bounded device wait on a flag nothing sets (ETIMEOUT expected)."""
    return load().tsnnls_wait_probe(int(polls))


def chol_solve_noalloc(L, k, lds, rhs, precision=MIXED, stream=None):
    """Context-free, allocation-free factor solve on device tensors (in place
    on rhs) using the library's static scratch; returns the status code."""
    sp = ctypes.c_void_p(stream) if stream else ctypes.c_void_p(0)
    return load().tsnnls_chol_solve_noalloc(precision, _dev_ptr(L), int(k), int(lds), _dev_ptr(rhs), sp)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class HostCSR:
    """CSR arrays in host memory (keeps contiguous copies alive)."""

    def __init__(self, m, n, row_ptr, col_idx, val):
        self.m, self.n = int(m), int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @classmethod
    def from_problem(cls, p):
        return cls(p.m, p.n, p.row_ptr, p.col_idx, p.val)

    def struct(self):
        return CSR(self.m, self.n, int(self.row_ptr[-1]), _np_ptr(self.row_ptr),
                   _np_ptr(self.col_idx), _np_ptr(self.val), 0)


class DeviceCSR:
    """CSR arrays resident in device memory (torch CUDA tensors)."""

    def __init__(self, m, n, row_ptr, col_idx, val):
        self.m, self.n = int(m), int(n)
        self.row_ptr, self.col_idx, self.val = row_ptr, col_idx, val
        self.nnz = int(val.numel())

    @classmethod
    def from_problem(cls, p, device="cuda"):
        import torch

        return cls(p.m, p.n, torch.as_tensor(p.row_ptr, dtype=torch.int64, device=device),
                   torch.as_tensor(p.col_idx, dtype=torch.int32, device=device),
                   torch.as_tensor(p.val, dtype=torch.float64, device=device))

    def struct(self):
        return CSR(self.m, self.n, self.nnz, _dev_ptr(self.row_ptr), _dev_ptr(self.col_idx),
                   _dev_ptr(self.val), 1)


class QueueStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("max_in_use_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("lanes", ctypes.c_int32), ("max_active", ctypes.c_int32)]


class PhaseStat(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_int64), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


class Context:
    """A tsnnls context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self._inflight = {}  # ticket -> buffers that must outlive the asynchronous solve
        _check(self._lib.tsnnls_ctx_create(ctypes.byref(self._h), device, hbm_budget), "ctx_create")

    def close(self):
        if self._h:
            self._lib.tsnnls_ctx_destroy(self._h)  # waits for every outstanding ticket
            self._h = ctypes.c_void_p()
            self._inflight.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # -- solves -------------------------------------------------------------

    def solve(self, A, b, x_out=None, opts=None, raise_on_error=True, **kw):
        """Solve Eq. 1.  A is HostCSR (b numpy) or DeviceCSR (b a CUDA tensor).
        Returns (x, Info)."""
        o = opts if opts is not None else default_opts(**kw)
        info = Info()
        s = A.struct()
        if isinstance(A, HostCSR):
            b = np.ascontiguousarray(b, dtype=np.float64)
            x = np.empty(A.n) if x_out is None else x_out
            st = self._lib.tsnnls_solve(self._h, ctypes.byref(s), _np_ptr(b), _np_ptr(x),
                                        ctypes.byref(o), ctypes.byref(info))
        else:
            import torch

            x = torch.empty(A.n, dtype=torch.float64, device=b.device) if x_out is None else x_out
            st = self._lib.tsnnls_solve(self._h, ctypes.byref(s), _dev_ptr(b), _dev_ptr(x),
                                        ctypes.byref(o), ctypes.byref(info))
        if raise_on_error:
            _check(st, "solve")
        return x, info

    def solve_ex(self, A: HostCSR, b, trace_cap=1000, opts=None, **kw):
        """Host solve returning (x, y, inF(bool), trace[iters, 6], Info)."""
        o = opts if opts is not None else default_opts(**kw)
        info = Info()
        s = A.struct()
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(A.n)
        y = np.empty(A.n)
        f = np.empty(A.n, dtype=np.uint8)
        tr = np.zeros((trace_cap, 6), dtype=np.int64)
        st = self._lib.tsnnls_solve_ex(self._h, ctypes.byref(s), _np_ptr(b), _np_ptr(x), _np_ptr(y),
                                       _np_ptr(f), _np_ptr(tr), trace_cap, ctypes.byref(o),
                                       ctypes.byref(info))
        _check(st, "solve_ex")
        return x, y, f.astype(bool), tr[: min(info.iters, trace_cap)], info

    def submit(self, A, b, x_out, opts=None, **kw):
        o = opts if opts is not None else default_opts(**kw)
        s = A.struct()
        t = ctypes.c_int64()
        bp = _np_ptr(b) if isinstance(b, np.ndarray) else _dev_ptr(b)
        xp = _np_ptr(x_out) if isinstance(x_out, np.ndarray) else _dev_ptr(x_out)
        _check(self._lib.tsnnls_submit(self._h, ctypes.byref(s), bp, xp, ctypes.byref(o),
                                       ctypes.byref(t)), "submit")
        self._inflight[t.value] = (A, b, x_out)
        return t.value

    def submit_batch(self, As, bs, xs, opts=None, **kw):
        """One ticket for len(As) independent solves (HostCSR with numpy b / x,
        or DeviceCSR with CUDA tensors, per member)."""
        o = opts if opts is not None else default_opts(**kw)
        cnt = len(As)
        arr = (CSR * cnt)(*[a.struct() for a in As])
        bp = np.array([b.ctypes.data if isinstance(b, np.ndarray) else b.data_ptr() for b in bs],
                      dtype=np.uint64)
        xp = np.array([x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr() for x in xs],
                      dtype=np.uint64)
        t = ctypes.c_int64()
        _check(self._lib.tsnnls_submit_batch(self._h, cnt, ctypes.cast(arr, ctypes.c_void_p), _np_ptr(bp),
                                             _np_ptr(xp), ctypes.byref(o), ctypes.byref(t)), "submit_batch")
        self._inflight[t.value] = (As, bs, xs, arr)
        return t.value

    def batch_member_info(self, ticket, i):
        info = Info()
        st = self._lib.tsnnls_batch_member_info(self._h, ticket, int(i), ctypes.byref(info))
        return st, info

    def poll(self, ticket):
        info = Info()
        st = self._lib.tsnnls_poll(self._h, ticket, ctypes.byref(info))
        if st != PENDING:
            self._inflight.pop(ticket, None)
        return st, info

    def wait(self, ticket, timeout_us=-1):
        info = Info()
        st = self._lib.tsnnls_wait(self._h, ticket, timeout_us, ctypes.byref(info))
        if st != PENDING:
            self._inflight.pop(ticket, None)
        return st, info

    def queue_stats(self):
        q = QueueStats()
        _check(self._lib.tsnnls_queue_stats_read(self._h, ctypes.byref(q)), "queue_stats")
        return {f: getattr(q, f) for f, _ in q._fields_}

    def solve_batch_dense(self, a_list, b_list, x_list, opts=None, trace_cap=0, **kw):
        """Dense batched solve; a_list: CUDA float32 [m_i, n_i] row-major, b_list,
        x_list: CUDA float64.  Returns (status, status array, Info), plus the
        list of per-problem pivot traces [iters_i, 6] when trace_cap > 0."""
        o = opts if opts is not None else default_opts(**kw)
        cnt = len(a_list)
        ms = np.array([a.shape[0] for a in a_list], dtype=np.int32)
        ns = np.array([a.shape[1] for a in a_list], dtype=np.int32)
        ap = np.array([t.data_ptr() for t in a_list], dtype=np.uint64)
        bp = np.array([t.data_ptr() for t in b_list], dtype=np.uint64)
        xp = np.array([t.data_ptr() for t in x_list], dtype=np.uint64)
        stat = np.zeros(cnt, dtype=np.int32)
        info = Info()
        if trace_cap <= 0:
            st = self._lib.tsnnls_solve_batch_dense(self._h, cnt, _np_ptr(ms), _np_ptr(ns), _np_ptr(ap),
                                                    _np_ptr(bp), _np_ptr(xp), ctypes.byref(o),
                                                    _np_ptr(stat), ctypes.byref(info))
            return st, stat, info
        trs = [np.full((trace_cap, 6), -7, dtype=np.int64) for _ in range(cnt)]
        tp = np.array([t.ctypes.data for t in trs], dtype=np.uint64)
        st = self._lib.tsnnls_solve_batch_dense_ex(self._h, cnt, _np_ptr(ms), _np_ptr(ns), _np_ptr(ap),
                                                   _np_ptr(bp), _np_ptr(xp), ctypes.byref(o),
                                                   _np_ptr(stat), ctypes.byref(info), _np_ptr(tp), trace_cap)
        return st, stat, info, [t[t[:, 0] > 0] for t in trs]

    def batch_autotune(self, precision=MIXED, per_bucket=64):
        nb = np.zeros(5, dtype=np.int32)
        _check(self._lib.tsnnls_batch_autotune(self._h, precision, per_bucket, _np_ptr(nb)),
               "batch_autotune")
        return nb

    def batch_autotune_cached(self, cache_path, precision=MIXED, per_bucket=64):
        """Autotune through the JSON cache at cache_path: (widths, hit)."""
        nb = np.zeros(5, dtype=np.int32)
        hit = ctypes.c_int32(-1)
        _check(self._lib.tsnnls_batch_autotune_cached(self._h, precision, per_bucket, os.fsencode(cache_path),
                                                      _np_ptr(nb), ctypes.byref(hit)), "batch_autotune_cached")
        return nb, bool(hit.value)

    def batch_tune_key(self, precision=MIXED, per_bucket=64):
        buf = ctypes.create_string_buffer(1024)
        _check(self._lib.tsnnls_batch_tune_key(self._h, precision, per_bucket, buf, len(buf)), "batch_tune_key")
        return buf.value.decode()

    @staticmethod
    def batch_set_panel(nb, precision=MIXED):
        arr = np.ascontiguousarray(nb, dtype=np.int32)
        _check(load().tsnnls_batch_set_panel(precision, _np_ptr(arr)), "batch_set_panel")

    # -- per-phase device time ---------------------------------------------

    def profile(self, enable=True, kernels=False):
        """Per-phase device time; kernels=True times the factorisation's
        kernels one by one (diag / panel / update)."""
        mode = (2 if kernels else 1) if enable else 0
        _check(self._lib.tsnnls_profile_enable(self._h, mode), "profile_enable")

    def profile_read(self):
        arr = (PhaseStat * len(PHASES))()
        _check(self._lib.tsnnls_profile_read(self._h, ctypes.cast(arr, ctypes.c_void_p), len(PHASES)),
               "profile_read")
        return {name: {"ms": s.ms, "launches": s.launches, "bytes": s.bytes, "flops": s.flops}
                for name, s in zip(PHASES, arr)}

    # -- step-level entry points (device tensors) ----------------------------

    def gram(self, A: DeviceCSR, b, precision=MIXED):
        import torch

        ldg = ((A.n + 31) // 32) * 32
        dt = torch.float32 if precision == MIXED else torch.float64
        G = torch.zeros((A.n, ldg), dtype=dt, device=b.device)  # column j = row j of this tensor
        c = torch.empty(A.n, dtype=torch.float64, device=b.device)
        s = A.struct()
        _check(self._lib.tsnnls_gram(self._h, ctypes.byref(s), _dev_ptr(b), precision, _dev_ptr(G),
                                     ldg, _dev_ptr(c)), "gram")
        return G, ldg, c

    def gather(self, G, ldg, F, precision=MIXED):
        import torch

        k = int(F.numel())
        lds = max(k, 1)
        S = torch.zeros((max(k, 1), lds), dtype=G.dtype, device=G.device)
        _check(self._lib.tsnnls_gather(self._h, precision, _dev_ptr(G), ldg, _dev_ptr(F), k,
                                       _dev_ptr(S), lds), "gather")
        return S

    def cholesky(self, S, k, lds, precision=MIXED):
        """In place; S holds column j at S.view(-1)[j*lds : j*lds + k]."""
        info = ctypes.c_int32()
        st = self._lib.tsnnls_cholesky(self._h, precision, _dev_ptr(S), k, lds, ctypes.byref(info))
        return st, info.value

    def chol_solve(self, L, k, lds, rhs, precision=MIXED):
        _check(self._lib.tsnnls_chol_solve(self._h, precision, _dev_ptr(L), k, lds, _dev_ptr(rhs)),
               "chol_solve")
        return rhs

    def spmv(self, A: DeviceCSR, trans, alpha, x, beta=0.0, z=None):
        import torch

        rows = A.n if trans else A.m
        out = torch.empty(rows, dtype=torch.float64, device=x.device)
        zp = _dev_ptr(z) if z is not None else ctypes.c_void_p(0)
        s = A.struct()
        _check(self._lib.tsnnls_spmv(self._h, ctypes.byref(s), int(trans), float(alpha), _dev_ptr(x),
                                     float(beta), zp, _dev_ptr(out)), "spmv")
        return out
