"""Python binding of libmcinv (include/mcinv.h): argument marshalling only.

Every function keeps the C name and forwards to the CUDA library through
ctypes; all computation happens in the library's kernels.  There is no CPU
fallback: if ``_build/libmcinv.so`` is missing, :func:`lib` raises.

PyTorch supplies the CUDA stream (``torch.cuda.current_stream()``) when it
is importable and a GPU is present; otherwise the legacy default stream is used.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmcinv.so")

MCINV_OK = 0
STATUS_NAMES = {0: "MCINV_OK", 1: "MCINV_E_ARG", 2: "MCINV_E_SINGULAR_DIAG", 3: "MCINV_E_DIVERGED",
                4: "MCINV_E_NOMEM", 5: "MCINV_E_CUDA", 6: "MCINV_E_TIMEOUT", 7: "MCINV_E_STATE",
                8: "MCINV_E_UNSUPPORTED"}
globals().update({name: code for code, name in STATUS_NAMES.items()})
MCINV_REAL64, MCINV_COMPLEX128 = 0, 1
MCINV_ACC_FP32_SIMT, MCINV_ACC_BF16_TC = 0, 1
MCINV_EST_BLOCK, MCINV_EST_DIAG, MCINV_EST_TRACE = 0, 1, 2
MCINV_F_NO_DIAG = 1
MCINV_F_AUTOTUNE = 2
MCINV_F_COLOR_ORDER = 4
MCINV_F_STAGED = 8
MCINV_F_GRID = 16
MCINV_F_GRID_BULK = 32
MCINV_F_GRID_NOPAIR = 64
MCINV_F_GRID_PAIR = 128
MCINV_F_GRID_TILE = 256
MCINV_F_GRID_WAVE = 512
MCINV_F_TEST_EXPIRE_WAIT = 1024

# every symbol include/mcinv.h declares
EXPORTS = ("mcinv_default_options", "mcinv_create", "mcinv_create_partitioned", "mcinv_burnin", "mcinv_burnin_coupled", "mcinv_sample",
           "mcinv_estimate", "mcinv_set_trace_weights", "mcinv_trace_mc_error", "mcinv_trace_series",
           "mcinv_sample_until", "mcinv_sync", "mcinv_get_state", "mcinv_set_state",
           "mcinv_reset_estimates", "mcinv_info", "mcinv_profile", "mcinv_profile_read",
           "mcinv_selftest_tc_gemm", "mcinv_block_accumulate_noalloc", "mcinv_destroy",
           "mcinv_last_error", "mcinv_color_order",
           "mcinv_pool_default_options", "mcinv_pool_create", "mcinv_pool_footprint", "mcinv_pool_submit",
           "mcinv_pool_step", "mcinv_pool_poll", "mcinv_pool_estimate", "mcinv_pool_get_state",
           "mcinv_pool_release", "mcinv_pool_info", "mcinv_pool_sync", "mcinv_pool_destroy",
           "mcinv_pool_last_error",
           "mcinv_server_create", "mcinv_server_submit", "mcinv_server_wait", "mcinv_server_stats",
           "mcinv_server_reset_stats", "mcinv_server_last_error", "mcinv_server_destroy")
MCINV_KERNEL_NOISE, MCINV_KERNEL_SWEEP, MCINV_KERNEL_BLOCK, MCINV_KERNEL_FOLD, MCINV_KERNEL_ESTIMATE = range(5)
KERNEL_NAMES = ("noise", "sweep", "block", "fold", "estimate")


class McinvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mcinv_options(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("seed", ctypes.c_uint64), ("chain_base", ctypes.c_int64),
                ("matrix_id", ctypes.c_uint32), ("groups", ctypes.c_int32),
                ("batch_cycles", ctypes.c_int32), ("acc", ctypes.c_int32),
                ("chains_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("block_rows", ctypes.POINTER(ctypes.c_int64)), ("n_block_rows", ctypes.c_int64),
                ("block_cols", ctypes.POINTER(ctypes.c_int64)), ("n_block_cols", ctypes.c_int64),
                ("ctas_per_slice", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mcinv_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("K", ctypes.c_int64),
                ("is_complex", ctypes.c_int32), ("chains_per_cta", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("ctas_per_slice", ctypes.c_int32), ("chains_per_lane", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("batch_cycles", ctypes.c_int32), ("acc", ctypes.c_int32),
                ("cycle", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("block_batches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("sweep_kernel", ctypes.c_int32), ("grid_ctas", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mcinv_pool_options(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("seed", ctypes.c_uint64), ("chain_base", ctypes.c_int64),
                ("mem_budget", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("batch_cycles", ctypes.c_int32), ("groups", ctypes.c_int32), ("fold_steps", ctypes.c_int32),
                ("chains_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class mcinv_pool_info_t(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("steps", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("arena_bytes", ctypes.c_int64), ("arena_used", ctypes.c_int64),
                ("chains_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("batch_cycles", ctypes.c_int32), ("active", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("fold_steps", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mcinv_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("elapsed_s", ctypes.c_double), ("busy_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libmcinv.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.mcinv_default_options.argtypes = [ctypes.POINTER(mcinv_options)]
        L.mcinv_default_options.restype = None
        L.mcinv_create.argtypes = [ctypes.POINTER(vp), i64, vp, vp, vp, ctypes.c_int,
                                   ctypes.POINTER(mcinv_options)]
        for name in ("mcinv_burnin", "mcinv_sample"):
            getattr(L, name).argtypes = [vp, i64]
        L.mcinv_burnin_coupled.argtypes = [vp, ctypes.c_double, i64, ctypes.POINTER(i64)]
        L.mcinv_burnin_coupled.restype = ctypes.c_int
        L.mcinv_create_partitioned.argtypes = [ctypes.POINTER(vp), i64, vp, vp, vp, ctypes.c_int,
                                               ctypes.POINTER(mcinv_options), i64, vp]
        L.mcinv_create_partitioned.restype = ctypes.c_int
        L.mcinv_color_order.argtypes = [i64, vp, vp, vp, ctypes.POINTER(i32)]
        L.mcinv_color_order.restype = ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        L.mcinv_set_trace_weights.argtypes = [vp, vp]
        L.mcinv_trace_mc_error.argtypes = [vp, dp, dp, dp, dp]
        L.mcinv_trace_series.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.mcinv_sample_until.argtypes = [vp, ctypes.c_double, i64, i64, ctypes.POINTER(i64)]
        for name in ("mcinv_set_trace_weights", "mcinv_trace_mc_error", "mcinv_trace_series", "mcinv_sample_until"):
            getattr(L, name).restype = ctypes.c_int
        L.mcinv_estimate.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.mcinv_sync.argtypes = [vp]
        L.mcinv_get_state.argtypes = [vp, i64, i64, vp, vp, ctypes.POINTER(i64)]
        L.mcinv_set_state.argtypes = [vp, vp, vp, i64]
        L.mcinv_reset_estimates.argtypes = [vp]
        L.mcinv_info.argtypes = [vp, ctypes.POINTER(mcinv_info_t)]
        L.mcinv_profile.argtypes = [vp, ctypes.c_int]
        L.mcinv_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64),
                                         ctypes.POINTER(ctypes.c_double)]
        L.mcinv_selftest_tc_gemm.argtypes = [i64, i64, i64, vp, vp, vp]
        L.mcinv_selftest_tc_gemm.restype = ctypes.c_int
        L.mcinv_block_accumulate_noalloc.argtypes = [i64, i64, i64, vp, i64, vp, i64, ctypes.c_double,
                                                     vp, vp, vp, ctypes.POINTER(ctypes.c_char_p)]
        L.mcinv_block_accumulate_noalloc.restype = ctypes.c_int
        L.mcinv_destroy.argtypes = [vp]
        L.mcinv_destroy.restype = None
        L.mcinv_pool_default_options.argtypes = [ctypes.POINTER(mcinv_pool_options)]
        L.mcinv_pool_default_options.restype = None
        L.mcinv_pool_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mcinv_pool_options)]
        L.mcinv_pool_footprint.argtypes = [vp, i64, i64, i32, ctypes.POINTER(i64)]
        L.mcinv_pool_submit.argtypes = [vp, i64, vp, vp, vp, ctypes.c_uint32, i64, i64, i32, ctypes.POINTER(i64)]
        L.mcinv_pool_step.argtypes = [vp]
        L.mcinv_pool_poll.argtypes = [vp, i64, ctypes.POINTER(i32)]
        L.mcinv_pool_estimate.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp]
        L.mcinv_pool_get_state.argtypes = [vp, i64, i64, i64, vp, vp, ctypes.POINTER(i64)]
        L.mcinv_pool_release.argtypes = [vp, i64]
        L.mcinv_pool_info.argtypes = [vp, ctypes.POINTER(mcinv_pool_info_t)]
        L.mcinv_pool_sync.argtypes = [vp]
        L.mcinv_pool_destroy.argtypes = [vp]
        L.mcinv_pool_destroy.restype = None
        L.mcinv_pool_last_error.argtypes = [vp]
        L.mcinv_pool_last_error.restype = ctypes.c_char_p
        L.mcinv_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mcinv_pool_options)]
        L.mcinv_server_submit.argtypes = [vp, i64, vp, vp, vp, ctypes.c_uint32, i64, i64, ctypes.c_int, vp,
                                          ctypes.POINTER(i64)]
        L.mcinv_server_wait.argtypes = [vp, i64, ctypes.c_double, vp, vp, ctypes.POINTER(ctypes.c_double)]
        L.mcinv_server_stats.argtypes = [vp, ctypes.POINTER(mcinv_server_stats_t)]
        L.mcinv_server_reset_stats.argtypes = [vp]
        L.mcinv_server_last_error.argtypes = [vp]
        L.mcinv_server_last_error.restype = ctypes.c_char_p
        L.mcinv_server_destroy.argtypes = [vp]
        L.mcinv_server_destroy.restype = None
        for name in ("mcinv_server_create", "mcinv_server_submit", "mcinv_server_wait", "mcinv_server_stats",
                     "mcinv_server_reset_stats"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("mcinv_pool_create", "mcinv_pool_footprint", "mcinv_pool_submit", "mcinv_pool_step",
                     "mcinv_pool_poll", "mcinv_pool_estimate", "mcinv_pool_get_state", "mcinv_pool_release",
                     "mcinv_pool_info", "mcinv_pool_sync"):
            getattr(L, name).restype = ctypes.c_int
        L.mcinv_last_error.argtypes = [vp]
        L.mcinv_last_error.restype = ctypes.c_char_p
        for name in ("mcinv_create", "mcinv_burnin", "mcinv_sample", "mcinv_estimate", "mcinv_sync",
                     "mcinv_get_state", "mcinv_set_state", "mcinv_reset_estimates", "mcinv_info",
                     "mcinv_profile", "mcinv_profile_read"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != MCINV_OK:
        msg = lib().mcinv_last_error(handle).decode(errors="replace")
        raise McinvError(status, msg)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def mcinv_default_options(**overrides) -> mcinv_options:
    opt = mcinv_options()
    lib().mcinv_default_options(ctypes.byref(opt))
    for k, v in overrides.items():
        setattr(opt, k, v)
    return opt


class Handle:
    """An mcinv_t plus the host arrays its options point to."""

    def __init__(self, ptr, n, K, is_complex, nR, nS, keep):
        self.ptr, self.n, self.K, self.is_complex = ptr, n, K, is_complex
        self.nR, self.nS = nR, nS
        self._keep = keep

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().mcinv_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def mcinv_create(n, row_ptr, col, val, *, K=1024, seed=0, chain_base=0, matrix_id=0, groups=0,
                 batch_cycles=0, acc=MCINV_ACC_BF16_TC, chains_per_cta=0, threads_per_cta=0,
                 ctas_per_slice=0, flags=0, stream="current", block_rows=None,
                 block_cols=None, partition=None) -> Handle:
    """mcinv_create, or mcinv_create_partitioned when `partition` (block_ptr, int64[nblocks+1])
    is given."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    is_complex = np.iscomplexobj(val)
    if is_complex:
        v = np.ascontiguousarray(val, dtype=np.complex128).view(np.float64)
        dt = MCINV_COMPLEX128
    else:
        v = np.ascontiguousarray(val, dtype=np.float64)
        dt = MCINV_REAL64
    opt = mcinv_default_options(K=K, seed=seed, chain_base=chain_base, matrix_id=matrix_id,
                                groups=groups, batch_cycles=batch_cycles, acc=acc,
                                chains_per_cta=chains_per_cta, threads_per_cta=threads_per_cta,
                                ctas_per_slice=ctas_per_slice, flags=flags)
    opt.stream = current_stream() if stream == "current" else stream
    keep = []
    nR = nS = 0
    if block_rows is not None:
        R = np.ascontiguousarray(block_rows, dtype=np.int64)
        S = np.ascontiguousarray(block_cols, dtype=np.int64)
        keep += [R, S]
        opt.block_rows = R.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        opt.block_cols = S.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        opt.n_block_rows, opt.n_block_cols = nR, nS = len(R), len(S)
    h = ctypes.c_void_p()
    if partition is None:
        _check(lib().mcinv_create(ctypes.byref(h), int(n), _ptr(row_ptr), _ptr(col), _ptr(v), dt,
                                  ctypes.byref(opt)))
    else:
        bp = np.ascontiguousarray(partition, dtype=np.int64)
        _check(lib().mcinv_create_partitioned(ctypes.byref(h), int(n), _ptr(row_ptr), _ptr(col), _ptr(v), dt,
                                              ctypes.byref(opt), int(len(bp) - 1), _ptr(bp)))
    return Handle(h, int(n), int(K), is_complex, nR, nS, keep)


def mcinv_burnin(h: Handle, cycles: int):
    _check(lib().mcinv_burnin(h.ptr, int(cycles)), h.ptr)


def mcinv_burnin_coupled(h: Handle, tol: float, max_cycles: int = 100_000) -> int:
    """Algorithm 1 steps 1-5: burn in until the coupled paths agree within tol; returns p."""
    p = ctypes.c_int64()
    _check(lib().mcinv_burnin_coupled(h.ptr, float(tol), int(max_cycles), ctypes.byref(p)), h.ptr)
    return int(p.value)


def mcinv_set_trace_weights(h: Handle, q_diag):
    q = np.ascontiguousarray(q_diag, dtype=np.float64)
    _check(lib().mcinv_set_trace_weights(h.ptr, _ptr(q)), h.ptr)


def mcinv_trace_mc_error(h: Handle) -> dict:
    """Geyer's Monte Carlo error of the trace: mean, var, ess, se."""
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().mcinv_trace_mc_error(h.ptr, *[ctypes.byref(x) for x in v]), h.ptr)
    return dict(zip(("mean", "var", "ess", "se"), (x.value for x in v)))


def mcinv_trace_series(h: Handle) -> np.ndarray:
    n = ctypes.c_int64()
    _check(lib().mcinv_trace_series(h.ptr, None, 0, ctypes.byref(n)), h.ptr)
    out = np.empty(n.value)
    _check(lib().mcinv_trace_series(h.ptr, _ptr(out), n.value, ctypes.byref(n)), h.ptr)
    return out


def mcinv_sample_until(h: Handle, rel_tol: float, check_every: int = 100, max_cycles: int = 1_000_000) -> int:
    c = ctypes.c_int64()
    _check(lib().mcinv_sample_until(h.ptr, float(rel_tol), int(check_every), int(max_cycles), ctypes.byref(c)), h.ptr)
    return int(c.value)


def mcinv_sample(h: Handle, cycles: int):
    _check(lib().mcinv_sample(h.ptr, int(cycles)), h.ptr)


def mcinv_sync(h: Handle):
    _check(lib().mcinv_sync(h.ptr), h.ptr)


def mcinv_estimate(h: Handle, kind: int, q_diag=None, out=None, se_out=None):
    """Returns (estimate, standard_error) as float64 / complex128 arrays."""
    if kind == MCINV_EST_DIAG:
        shape = (h.n,)
    elif kind == MCINV_EST_TRACE:
        shape = ()
    else:
        shape = (h.nR, h.nS)
    nv = 2 if h.is_complex else 1
    count = int(np.prod(shape)) * nv
    if out is None:
        out = np.empty(count, dtype=np.float64)
    if se_out is None:
        se_out = np.empty(count, dtype=np.float64)
    q = None if q_diag is None else np.ascontiguousarray(q_diag, dtype=np.float64)
    _check(lib().mcinv_estimate(h.ptr, int(kind), _ptr(q), _ptr(out), _ptr(se_out)), h.ptr)
    if h.is_complex:
        return out.view(np.complex128).reshape(shape), se_out.view(np.complex128).reshape(shape)
    return out.reshape(shape), se_out.reshape(shape)


def mcinv_get_state(h: Handle, chain0: int = 0, nchains: int | None = None):
    """Returns (z, w, cycle); z, w are [n][nchains] float64 or complex128."""
    nchains = h.K - chain0 if nchains is None else nchains
    nv = 2 if h.is_complex else 1
    z = np.empty(h.n * nchains * nv, dtype=np.float64)
    w = np.empty_like(z)
    cyc = ctypes.c_int64()
    st = lib().mcinv_get_state(h.ptr, int(chain0), int(nchains), _ptr(z), _ptr(w), ctypes.byref(cyc))
    if st not in (MCINV_OK, 3):
        _check(st, h.ptr)
    if h.is_complex:
        z, w = z.view(np.complex128), w.view(np.complex128)
    return z.reshape(h.n, nchains), w.reshape(h.n, nchains), int(cyc.value)


def mcinv_set_state(h: Handle, z, w, cycle: int):
    dt = np.complex128 if h.is_complex else np.float64
    z = np.ascontiguousarray(z, dtype=dt).reshape(h.n, h.K)
    w = np.ascontiguousarray(w, dtype=dt).reshape(h.n, h.K)
    _check(lib().mcinv_set_state(h.ptr, _ptr(z.view(np.float64)), _ptr(w.view(np.float64)), int(cycle)), h.ptr)


def mcinv_reset_estimates(h: Handle):
    _check(lib().mcinv_reset_estimates(h.ptr), h.ptr)


def mcinv_info(h: Handle) -> dict:
    info = mcinv_info_t()
    _check(lib().mcinv_info(h.ptr, ctypes.byref(info)), h.ptr)
    return info.as_dict()


def mcinv_profile(h: Handle, enable: bool):
    _check(lib().mcinv_profile(h.ptr, int(bool(enable))), h.ptr)


def mcinv_profile_read(h: Handle, kernel: int):
    """Returns (launches, milliseconds) recorded for one kernel class."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().mcinv_profile_read(h.ptr, int(kernel), ctypes.byref(n), ctypes.byref(ms)), h.ptr)
    return int(n.value), float(ms.value)


def mcinv_selftest_tc_gemm(A_bits, B_bits):
    """D = A B^T on the tensor cores; A_bits, B_bits: uint16 BF16 bit patterns [rows][inner]."""
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    assert A.shape[1] == B.shape[1]
    D = np.empty((A.shape[0], B.shape[0]), dtype=np.float32)
    _check(lib().mcinv_selftest_tc_gemm(A.shape[0], B.shape[0], A.shape[1], _ptr(A), _ptr(B), _ptr(D)))
    return D


def mcinv_block_accumulate_noalloc(M, N, inner, A_ptr, lda, B_ptr, ldb, scale_sq, sum_ptr, sq_ptr,
                                   stream=None):
    """One block-accumulation batch on caller device memory (integer addresses);
    the library allocates nothing.  Raises McinvError with the library's message."""
    err = ctypes.c_char_p()
    st = lib().mcinv_block_accumulate_noalloc(int(M), int(N), int(inner), ctypes.c_void_p(A_ptr), int(lda),
                                              ctypes.c_void_p(B_ptr), int(ldb), float(scale_sq),
                                              ctypes.c_void_p(sum_ptr), ctypes.c_void_p(sq_ptr),
                                              stream, ctypes.byref(err))
    if st != MCINV_OK:
        raise McinvError(st, (err.value or b"").decode(errors="replace"))


def mcinv_destroy(h: Handle):
    if h.ptr:
        lib().mcinv_destroy(h.ptr)
        h.ptr = None


def mcinv_last_error(h: Handle | None = None) -> str:
    return lib().mcinv_last_error(None if h is None else h.ptr).decode(errors="replace")


def mcinv_color_order(n: int, row_ptr, col):
    """The colour sweep order of C (host only): returns (order int32[n], ncolors)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    order = np.empty(int(n), dtype=np.int32)
    nc = ctypes.c_int32()
    st = lib().mcinv_color_order(int(n), rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                                 order.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nc))
    if st != MCINV_OK:
        raise McinvError(st, "mcinv_color_order failed")
    return order, int(nc.value)


def create_from_csr(csr, **kw) -> Handle:
    """mcinv_create from a workloads.CSR."""
    return mcinv_create(csr.n, csr.row_ptr, csr.col, csr.val, **kw)


# -- pool: many matrices advanced together, continuous batching -------------------------

def _pcheck(status, pool=None):
    if status != MCINV_OK:
        msg = lib().mcinv_pool_last_error(pool).decode(errors="replace")
        raise McinvError(status, msg)


class Pool:
    def __init__(self, ptr, K):
        self.ptr, self.K = ptr, K

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().mcinv_pool_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def mcinv_pool_default_options(**overrides) -> mcinv_pool_options:
    o = mcinv_pool_options()
    lib().mcinv_pool_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def mcinv_pool_create(*, K=256, seed=0, chain_base=0, mem_budget=1 << 32, max_slots=512, batch_cycles=8,
                      groups=32, fold_steps=0, chains_per_cta=0, threads_per_cta=0, flags=0,
                      stream="current") -> Pool:
    o = mcinv_pool_default_options(K=K, seed=seed, chain_base=chain_base, mem_budget=mem_budget,
                                   max_slots=max_slots, batch_cycles=batch_cycles, groups=groups,
                                   fold_steps=fold_steps, chains_per_cta=chains_per_cta,
                                   threads_per_cta=threads_per_cta, flags=flags)
    o.stream = current_stream() if stream == "current" else stream
    p = ctypes.c_void_p()
    _pcheck(lib().mcinv_pool_create(ctypes.byref(p), ctypes.byref(o)))
    return Pool(p, K)


def mcinv_pool_footprint(pool: Pool, n, nnz, want_inverse=True) -> int:
    b = ctypes.c_int64()
    _pcheck(lib().mcinv_pool_footprint(pool.ptr, int(n), int(nnz), int(bool(want_inverse)), ctypes.byref(b)), pool.ptr)
    return int(b.value)


def mcinv_pool_submit(pool: Pool, csr, matrix_id, burnin, samples, want_inverse=True) -> int:
    """Admit a real matrix; raises McinvError with status MCINV_E_NOMEM (4) if it does not fit now."""
    rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(csr.col, dtype=np.int32)
    val = np.ascontiguousarray(csr.val, dtype=np.float64)
    t = ctypes.c_int64()
    _pcheck(lib().mcinv_pool_submit(pool.ptr, csr.n, _ptr(rp), _ptr(col), _ptr(val), int(matrix_id),
                                    int(burnin), int(samples), int(bool(want_inverse)), ctypes.byref(t)),
            pool.ptr)
    return int(t.value)


def mcinv_pool_step(pool: Pool):
    _pcheck(lib().mcinv_pool_step(pool.ptr), pool.ptr)


def mcinv_pool_poll(pool: Pool, ticket) -> bool:
    d = ctypes.c_int32()
    _pcheck(lib().mcinv_pool_poll(pool.ptr, int(ticket), ctypes.byref(d)), pool.ptr)
    return bool(d.value)


def mcinv_pool_estimate(pool: Pool, ticket, kind, n, q_diag=None):
    shape = {MCINV_EST_DIAG: (n,), MCINV_EST_TRACE: (), MCINV_EST_BLOCK: (n, n)}[kind]
    count = int(np.prod(shape))
    out = np.empty(count)
    se = np.empty(count)
    q = None if q_diag is None else np.ascontiguousarray(q_diag, dtype=np.float64)
    _pcheck(lib().mcinv_pool_estimate(pool.ptr, int(ticket), int(kind), _ptr(q), _ptr(out), _ptr(se)), pool.ptr)
    return out.reshape(shape), se.reshape(shape)


def mcinv_pool_get_state(pool: Pool, ticket, n, chain0=0, nchains=None):
    nchains = pool.K - chain0 if nchains is None else nchains
    z = np.empty(n * nchains)
    w = np.empty(n * nchains)
    cyc = ctypes.c_int64()
    _pcheck(lib().mcinv_pool_get_state(pool.ptr, int(ticket), int(chain0), int(nchains), _ptr(z), _ptr(w),
                                       ctypes.byref(cyc)), pool.ptr)
    return z.reshape(n, nchains), w.reshape(n, nchains), int(cyc.value)


def mcinv_pool_release(pool: Pool, ticket):
    _pcheck(lib().mcinv_pool_release(pool.ptr, int(ticket)), pool.ptr)


def mcinv_pool_info(pool: Pool) -> dict:
    i = mcinv_pool_info_t()
    _pcheck(lib().mcinv_pool_info(pool.ptr, ctypes.byref(i)), pool.ptr)
    return i.as_dict()


def mcinv_pool_sync(pool: Pool):
    _pcheck(lib().mcinv_pool_sync(pool.ptr), pool.ptr)


def mcinv_pool_destroy(pool: Pool):
    if pool.ptr:
        lib().mcinv_pool_destroy(pool.ptr)
        pool.ptr = None


def mcinv_pool_last_error(pool: Pool | None = None) -> str:
    return lib().mcinv_pool_last_error(None if pool is None else pool.ptr).decode(errors="replace")


# -- server: requests on a pool, continuous batching ------------------------------------

class Server:
    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().mcinv_server_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def mcinv_server_create(*, stream=None, **pool_options) -> Server:
    o = mcinv_pool_default_options(**pool_options)
    o.stream = stream
    p = ctypes.c_void_p()
    st = lib().mcinv_server_create(ctypes.byref(p), ctypes.byref(o))
    if st != MCINV_OK:
        raise McinvError(st, lib().mcinv_pool_last_error(None).decode(errors="replace"))
    return Server(p)


def mcinv_server_submit(server: Server, csr, matrix_id, burnin, samples, kind, q_diag=None) -> int:
    rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(csr.col, dtype=np.int32)
    val = np.ascontiguousarray(csr.val, dtype=np.float64)
    q = None if q_diag is None else np.ascontiguousarray(q_diag, dtype=np.float64)
    rid = ctypes.c_int64()
    st = lib().mcinv_server_submit(server.ptr, csr.n, _ptr(rp), _ptr(col), _ptr(val), int(matrix_id), int(burnin),
                                   int(samples), int(kind), _ptr(q), ctypes.byref(rid))
    if st != MCINV_OK:
        raise McinvError(st, "submit rejected")
    return int(rid.value)


def mcinv_server_wait(server: Server, request, n, kind, timeout_s=600.0):
    """Returns (estimate, se, latency_ms)."""
    count = {MCINV_EST_DIAG: n, MCINV_EST_TRACE: 1, MCINV_EST_BLOCK: n * n}[kind]
    out = np.empty(count)
    se = np.empty(count)
    lat = ctypes.c_double()
    st = lib().mcinv_server_wait(server.ptr, int(request), float(timeout_s), _ptr(out), _ptr(se), ctypes.byref(lat))
    if st != MCINV_OK:
        raise McinvError(st, lib().mcinv_server_last_error(server.ptr).decode(errors="replace"))
    shape = {MCINV_EST_DIAG: (n,), MCINV_EST_TRACE: (), MCINV_EST_BLOCK: (n, n)}[kind]
    return out.reshape(shape), se.reshape(shape), float(lat.value)


def mcinv_server_stats(server: Server) -> dict:
    s = mcinv_server_stats_t()
    lib().mcinv_server_stats(server.ptr, ctypes.byref(s))
    return s.as_dict()


def mcinv_server_reset_stats(server: Server):
    lib().mcinv_server_reset_stats(server.ptr)


def mcinv_server_last_error(server: Server) -> str:
    return lib().mcinv_server_last_error(server.ptr).decode(errors="replace")


def mcinv_server_destroy(server: Server):
    if server.ptr:
        lib().mcinv_server_destroy(server.ptr)
        server.ptr = None
