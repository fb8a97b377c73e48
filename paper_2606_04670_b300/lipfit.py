"""Python binding of liblipfit.so (argument marshalling only; all arithmetic runs in the
library's CUDA kernels).

Module-level functions mirror the C ABI one to one (``lip_fit``, ``lip_eval``, ...),
taking raw pointers; ``LipFit`` wraps a handle for torch tensors on the GPU, following
the paper's package interface (Sec. 5: add, values, lipschitz_constant, clear,
setparams); ``LipEvalFn`` is the ``torch.autograd.Function`` whose backward is the
library's backward kernel.

There is no CPU fallback: if the compiled library is missing, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblipfit.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lipfit.h")

LIP_OK, LIP_ERR_ARG, LIP_ERR_NONFINITE, LIP_ERR_OOM, LIP_ERR_CUDA = 0, 1, 2, 3, 4
LIP_ERR_CAPACITY, LIP_ERR_TIMEOUT, LIP_ERR_UNSUPPORTED, LIP_ERR_NO_DEVICE, LIP_ERR_STATE = 5, 6, 7, 8, 9
LIP_L1, LIP_L2, LIP_LINF = 1, 2, 3
LIP_FP32, LIP_FP64, LIP_TC_BF16, LIP_TC_TF32, LIP_TC_FP16 = 0, 1, 2, 3, 4
LIP_NOALLOC_N_MAX = 32768
LIP_D_MAX = 32
LIP_LOCAL_KNOTS_MAX = 31
LIP_LOCAL_SAMPLE_MAX = 1 << 20
NORMS = {"L1": LIP_L1, "L2": LIP_L2, "Linf": LIP_LINF, "LINF": LIP_LINF,
         LIP_L1: LIP_L1, LIP_L2: LIP_L2, LIP_LINF: LIP_LINF}
PRECISIONS = {"fp32": LIP_FP32, "fp64": LIP_FP64, "tc_bf16": LIP_TC_BF16, "tc_tf32": LIP_TC_TF32,
              "tc_fp16": LIP_TC_FP16, LIP_FP32: LIP_FP32, LIP_FP64: LIP_FP64, LIP_TC_BF16: LIP_TC_BF16,
              LIP_TC_TF32: LIP_TC_TF32, LIP_TC_FP16: LIP_TC_FP16}


class lip_params(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("mon", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class lip_batch_set(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int32),
                ("norm", ctypes.c_int32), ("M", ctypes.c_double), ("mon", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("Q", ctypes.c_void_p), ("nq", ctypes.c_int64), ("g", ctypes.c_void_p), ("lo", ctypes.c_void_p),
                ("hi", ctypes.c_void_p), ("idx_up", ctypes.c_void_p), ("idx_lo", ctypes.c_void_p),
                ("tile_groups", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lip_batch_options(ctypes.Structure):
    _fields_ = [("tile_groups", ctypes.c_int32), ("items_per_block", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class LipError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {status_string(status)} ({status}): {detail}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run paper_2606_04670_b300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    H = ctypes.c_void_p
    sig = {
        "lip_fit": [P, P, i64, i32, f64, ctypes.POINTER(lip_params), P, ctypes.POINTER(H)],
        "lip_fit_host": [P, P, i64, i32, f64, ctypes.POINTER(lip_params), P, ctypes.POINTER(H)],
        "lip_reserve": [i64, i32, f64, ctypes.POINTER(lip_params), ctypes.POINTER(H)],
        "lip_add": [H, P, P, i64, P],
        "lip_add_host": [H, P, P, i64, P],
        "lip_clear": [H, P],
        "lip_set_M": [H, f64, P],
        "lip_eval": [H, P, i64, P, P, P, P, P, P],
        "lip_eval_host": [H, P, i64, P, P, P, P, P, P],
        "lip_eval_host_async": [H, P, i64, P, P, P, P, P, P],
        "lip_eval_k": [H, P, i64, i32, P, P, P, P, P, P, P],
        "lip_estimate_M": [H, ctypes.POINTER(f64), ctypes.POINTER(i64), ctypes.POINTER(i64), P],
        "lip_backward": [H, P, i64, P, P, P, P, P, P, i32, P],
        "lip_eval_batched": [H, P],
        "lip_autotune": [H, P, i64, i32, P, P, P, P, P],
        "lip_check": [H, P],
        "lip_set_tuning": [H, i32, i32, i32],
        "lip_get_tuning": [H, P, P, P, P, P],
        "lip_set_timing_events": [H, P, P],
        "lip_estimate_M_noalloc": [P, P, i64, i32, i32, P, P, P],
        "lip_batch_create": [ctypes.POINTER(lip_batch_set), i32, ctypes.POINTER(lip_batch_options), P,
                             ctypes.POINTER(H)],
        "lip_batch_eval": [H, P],
        "lip_batch_info": [H, P, P, P, P],
        "lip_batch_check": [H, P],
        "lip_batch_set_timing_events": [H, P, P],
        "lip_local_fit": [H, i32, i64, ctypes.c_uint64, P],
        "lip_local_fit_knots": [H, P, i32, P],
        "lip_local_knots": [H, P, P],
        "lip_local_table": [H, P, P, P, P],
        "lip_local_stats": [H, P, P],
        "lip_eval_local": [H, P, i64, P, P, P, P, P, P],
        "lip_eval_local_k": [H, P, i64, i32, P, P, P, P, P, P, P],
        "lip_smooth_objective": [H, f64, f64, P, ctypes.POINTER(f64), P, P],
        "lip_smooth": [H, f64, f64, i32, i32, f64, P, ctypes.POINTER(f64), ctypes.POINTER(i32),
                       ctypes.POINTER(i32), P],
        "lip_shard_scan": [H, P, i64, i64, P, P, P],
        "lip_shard_reeval": [H, P, i64, i64, P, P, P, P, P],
        "lip_shard_finish": [H, i64, P, P, P, P, P, P, P, P, P, P],
        "lip_estimate_M_part": [H, i32, i32, P, P],
        "lip_estimate_M_async": [H, P],
        "lip_estimate_M_result": [H, ctypes.POINTER(f64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "lip_set_tc_window": [H, i64],
        "lip_set_estimate_full": [H, i32],
        "lip_last_scan_work": [H, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "lip_last_estimate_work": [H, ctypes.POINTER(i64)],
        "lip_last_scan_stats": [H, ctypes.POINTER(i64)],
        "lip_add_async": [H, P, P, i64, P],
        "lip_add_host_async": [H, P, P, i64, P],
        "lip_debug_fail_alloc": [i64],
        "lip_debug_sqrt_fma": [P, P, i64, P],
        "lip_debug_scan_fault": [H, ctypes.c_uint64, i32],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lip_size.argtypes = [H]
    lib.lip_size.restype = i64
    lib.lip_free.argtypes = [H]
    lib.lip_free.restype = None
    lib.lip_batch_free.argtypes = [H]
    lib.lip_batch_free.restype = None
    lib.lip_status_string.argtypes = [ctypes.c_int]
    lib.lip_status_string.restype = ctypes.c_char_p
    lib.lip_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.lip_last_error.restype = ctypes.c_size_t
    lib.lip_last_error_detail.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.lip_last_error_detail.restype = ctypes.c_size_t
    lib.lip_version.restype = ctypes.c_char_p
    lib.lip_kernel_launches.restype = ctypes.c_uint64
    lib.lip_last_fallback.argtypes = [H]
    lib.lip_last_fallback.restype = ctypes.c_int64
    return lib


_lib = _load()


def library():
    return _lib


def header_symbols(path: str = HEADER) -> list:
    """Names of the functions that include/lipfit.h declares."""
    return sorted(set(re.findall(r"^LIP_API\s+[\w\s\*]+?\b(lip_\w+)\s*\(", open(path).read(), re.M)))


def status_string(s: int) -> str:
    return _lib.lip_status_string(int(s)).decode()


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    _lib.lip_last_error(buf, len(buf))
    return buf.value.decode()


def _check(status: int, where: str):
    if status != LIP_OK:
        raise LipError(status, where, last_error())


def make_params(norm=LIP_L2, precision=LIP_FP32, mon=None, w=None):
    """lip_params plus the host arrays it points to (kept alive by the returned tuple)."""
    mon_a = None if mon is None else np.ascontiguousarray(np.asarray(mon), dtype=np.int8)
    w_a = None if w is None else np.ascontiguousarray(np.asarray(w), dtype=np.float64)
    # unknown integers are passed through so that the library itself rejects them
    nv = NORMS.get(norm, norm) if isinstance(norm, (int, np.integer)) else NORMS[norm]
    pv = PRECISIONS.get(precision, precision) if isinstance(precision, (int, np.integer)) else PRECISIONS[precision]
    p = lip_params(int(nv), int(pv),
                   None if mon_a is None else mon_a.ctypes.data, None if w_a is None else w_a.ctypes.data)
    return p, (mon_a, w_a)


# ------------------------------------------------------------- raw ABI (same names)

def lip_fit(X_ptr, y_ptr, N, d, M, params, stream=0):
    h = ctypes.c_void_p()
    return _lib.lip_fit(X_ptr, y_ptr, N, d, M, ctypes.byref(params), stream, ctypes.byref(h)), h


def lip_fit_host(X_ptr, y_ptr, N, d, M, params, stream=0):
    h = ctypes.c_void_p()
    return _lib.lip_fit_host(X_ptr, y_ptr, N, d, M, ctypes.byref(params), stream, ctypes.byref(h)), h


def lip_reserve(capacity, d, M, params):
    h = ctypes.c_void_p()
    return _lib.lip_reserve(capacity, d, M, ctypes.byref(params), ctypes.byref(h)), h


def lip_add(h, X_ptr, y_ptr, n, stream=0):
    return _lib.lip_add(h, X_ptr, y_ptr, n, stream)


def lip_add_host(h, X_ptr, y_ptr, n, stream=0):
    return _lib.lip_add_host(h, X_ptr, y_ptr, n, stream)


def lip_add_async(h, X_ptr, y_ptr, n, stream=0):
    return _lib.lip_add_async(h, X_ptr, y_ptr, n, stream)


def lip_add_host_async(h, X_ptr, y_ptr, n, stream=0):
    return _lib.lip_add_host_async(h, X_ptr, y_ptr, n, stream)


def lip_set_tc_window(h, nbytes):
    return _lib.lip_set_tc_window(h, nbytes)


def lip_set_estimate_full(h, full):
    return _lib.lip_set_estimate_full(h, full)


def lip_clear(h, stream=0):
    return _lib.lip_clear(h, stream)


def lip_size(h):
    return _lib.lip_size(h)


def lip_set_M(h, M, stream=0):
    return _lib.lip_set_M(h, M, stream)


def lip_eval(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream)


def lip_eval_k(h, Q_ptr, nq, k, wk_ptr, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval_k(h, Q_ptr, nq, k, wk_ptr, g, lo, hi, idx_up, idx_lo, stream)


def lip_local_fit(h, nknots, sample_pairs, seed, stream=0):
    return _lib.lip_local_fit(h, nknots, sample_pairs, seed & (2**64 - 1), stream)


def lip_local_fit_knots(h, knots_ptr, nknots, stream=0):
    return _lib.lip_local_fit_knots(h, knots_ptr, nknots, stream)


def lip_local_knots(h):
    buf = (ctypes.c_double * LIP_LOCAL_KNOTS_MAX)()
    n = ctypes.c_int32()
    s = _lib.lip_local_knots(h, buf, ctypes.byref(n))
    return s, list(buf[:n.value]) if s == LIP_OK else []


def lip_local_table(h, d1, F, Mtab, stream=0):
    return _lib.lip_local_table(h, d1, F, Mtab, stream)


def lip_local_stats(h):
    over, mc = ctypes.c_int32(), ctypes.c_int32()
    s = _lib.lip_local_stats(h, ctypes.byref(over), ctypes.byref(mc))
    return s, over.value, mc.value


def lip_eval_local(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval_local(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream)


def lip_eval_local_k(h, Q_ptr, nq, k, wk_ptr, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval_local_k(h, Q_ptr, nq, k, wk_ptr, g, lo, hi, idx_up, idx_lo, stream)


def lip_smooth_objective(h, M, p, eps_ptr, grad_ptr, stream=0):
    f = ctypes.c_double()
    s = _lib.lip_smooth_objective(h, M, p, eps_ptr, ctypes.byref(f), grad_ptr, stream)
    return s, f.value


def lip_smooth(h, M, p, max_iter, history, gtol, eps_ptr, stream=0):
    f, it, ev = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    s = _lib.lip_smooth(h, M, p, max_iter, history, gtol, eps_ptr, ctypes.byref(f), ctypes.byref(it),
                        ctypes.byref(ev), stream)
    return s, f.value, it.value, ev.value


def lip_eval_host(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval_host(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream)


def lip_eval_host_async(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_eval_host_async(h, Q_ptr, nq, g, lo, hi, idx_up, idx_lo, stream)


def lip_estimate_M(h, stream=0):
    M, i, j = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    s = _lib.lip_estimate_M(h, ctypes.byref(M), ctypes.byref(i), ctypes.byref(j), stream)
    return s, M.value, i.value, j.value


def lip_estimate_M_async(h, stream=0):
    return _lib.lip_estimate_M_async(h, stream)


def lip_estimate_M_result(h):
    M, i, j = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    s = _lib.lip_estimate_M_result(h, ctypes.byref(M), ctypes.byref(i), ctypes.byref(j))
    return s, M.value, i.value, j.value


def lip_estimate_M_noalloc(X_ptr, y_ptr, N, d, norm, w_ptr, out_ptr, stream=0):
    """Handle-free estimate into device double[3] {M, i, j}; allocates nothing."""
    return _lib.lip_estimate_M_noalloc(X_ptr, y_ptr, N, d, norm, w_ptr, out_ptr, stream)


def lip_shard_scan(h, Q_ptr, nq, index_base, key_up, key_lo, stream=0):
    return _lib.lip_shard_scan(h, Q_ptr, nq, index_base, key_up, key_lo, stream)


def lip_shard_reeval(h, Q_ptr, nq, index_base, key_up, key_lo, hi64, lo64, stream=0):
    return _lib.lip_shard_reeval(h, Q_ptr, nq, index_base, key_up, key_lo, hi64, lo64, stream)


def lip_shard_finish(h, nq, key_up, key_lo, hi64, lo64, g, lo, hi, idx_up, idx_lo, stream=0):
    return _lib.lip_shard_finish(h, nq, key_up, key_lo, hi64, lo64, g, lo, hi, idx_up, idx_lo, stream)


def lip_estimate_M_part(h, part, nparts, stream=0):
    """(status, [M, i, j, key]) of one block-cyclic share of the estimate's pairs."""
    out = (ctypes.c_double * 4)()
    s = _lib.lip_estimate_M_part(h, part, nparts, out, stream)
    return s, list(out)


def lip_backward(h, Q_ptr, nq, idx_up, idx_lo, grad_g, grad_Q, grad_y, grad_M, deterministic=0, stream=0):
    return _lib.lip_backward(h, Q_ptr, nq, idx_up, idx_lo, grad_g, grad_Q, grad_y, grad_M, deterministic, stream)


def lip_autotune(h, Q_ptr, nq, reps=3, stream=0):
    """(status, tile_groups, splits, variant, ms) of the library's own autotuner."""
    tg, sp, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_double()
    s = _lib.lip_autotune(h, Q_ptr, nq, reps, ctypes.byref(tg), ctypes.byref(sp), ctypes.byref(v), ctypes.byref(ms),
                          stream)
    return s, tg.value, sp.value, v.value, ms.value


def lip_eval_batched(b, stream=0):
    return _lib.lip_eval_batched(b, stream)


def lip_last_error_detail():
    buf = ctypes.create_string_buffer(1024)
    _lib.lip_last_error_detail(buf, len(buf))
    return buf.value.decode()


def lip_set_tuning(h, tile_groups, splits, variant=-1):
    return _lib.lip_set_tuning(h, tile_groups, splits, variant)


def lip_get_tuning(h):
    v = [ctypes.c_int32() for _ in range(5)]
    s = _lib.lip_get_tuning(h, *[ctypes.byref(x) for x in v])
    return s, tuple(x.value for x in v)


def lip_set_timing_events(h, ev_before, ev_after):
    return _lib.lip_set_timing_events(h, ev_before, ev_after)


def lip_last_fallback(h):
    return int(_lib.lip_last_fallback(h))


def lip_kernel_launches():
    return int(_lib.lip_kernel_launches())


def lip_batch_create(sets, opt=None, stream=0):
    """sets: a ctypes array of lip_batch_set; opt: lip_batch_options or None."""
    h = ctypes.c_void_p()
    s = _lib.lip_batch_create(sets, len(sets), None if opt is None else ctypes.byref(opt), stream, ctypes.byref(h))
    return s, h


def lip_batch_eval(b, stream=0):
    return _lib.lip_batch_eval(b, stream)


def lip_batch_info(b):
    tp, tq, ni, gr = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    s = _lib.lip_batch_info(b, ctypes.byref(tp), ctypes.byref(tq), ctypes.byref(ni), ctypes.byref(gr))
    return s, tp.value, tq.value, ni.value, gr.value


def lip_batch_check(b, stream=0):
    return _lib.lip_batch_check(b, stream)


def lip_batch_free(b):
    _lib.lip_batch_free(b)


def lip_check(h, stream=0):
    return _lib.lip_check(h, stream)


def lip_free(h):
    _lib.lip_free(h)


def lip_status_string(s):
    return status_string(s)


def lip_last_error():
    return last_error()


def lip_version():
    return _lib.lip_version().decode()


def lip_debug_fail_alloc(n):
    """Tests only: the n-th device allocation from now on fails (0 = off)."""
    return _lib.lip_debug_fail_alloc(n)


def lip_debug_sqrt_fma(s_ptr, out_ptr, n, stream=0):
    """Tests only: the FMA-pipe square root of the scan variants 2-5, element by element."""
    return _lib.lip_debug_sqrt_fma(s_ptr, out_ptr, n, stream)


def lip_debug_scan_fault(h, wait_limit_ns, skip_tile):
    """Tests only: wait limit of the exact scan and the data tile it leaves out (-1 = none)."""
    return _lib.lip_debug_scan_fault(h, wait_limit_ns, skip_tile)


# ------------------------------------------------------------------ torch front end

def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


class LipFit:
    """A fitted data set on the GPU (Sec. 5: LipFit(reservedata, dim), add, values, ...).

    X [N, d] and y [N] are CUDA tensors (float32, or float64 with precision='fp64').
    norm: 'L1' | 'L2' | 'Linf'; mon: d entries in {-1,0,1} or None; w: d norm weights
    or None.  The data are copied into library-owned memory.
    """

    def __init__(self, X=None, y=None, M: float = 1.0, norm="L2", mon=None, w=None,
                 precision="fp32", capacity: Optional[int] = None, d: Optional[int] = None):
        torch = _torch()
        self.norm = NORMS[norm]
        self.precision = PRECISIONS[precision]
        self.dtype = torch.float64 if self.precision == LIP_FP64 else torch.float32
        self.mon = None if mon is None else np.asarray(mon, np.int8)
        self.w = None if w is None else np.asarray(w, np.float64)
        self._M = float(M)
        params, self._keep = make_params(self.norm, self.precision, self.mon, self.w)
        self.h = ctypes.c_void_p()
        if X is not None:
            X = self._dev(X)
            y = self._dev(y)
            self.d = int(X.shape[1])
            if capacity is None or capacity <= X.shape[0]:
                _check(_lib.lip_fit(X.data_ptr(), y.data_ptr(), X.shape[0], self.d, self._M,
                                    ctypes.byref(params), _stream_ptr(), ctypes.byref(self.h)), "lip_fit")
            else:
                _check(_lib.lip_reserve(capacity, self.d, self._M, ctypes.byref(params),
                                        ctypes.byref(self.h)), "lip_reserve")
                self.add(X, y)
        else:
            assert capacity is not None and d is not None, "give X, y or capacity and d"
            self.d = int(d)
            _check(_lib.lip_reserve(capacity, self.d, self._M, ctypes.byref(params),
                                    ctypes.byref(self.h)), "lip_reserve")

    def _dev(self, t):
        torch = _torch()
        if not torch.is_tensor(t):
            t = torch.as_tensor(np.asarray(t))
        return t.to(device="cuda", dtype=self.dtype).contiguous()

    # -- data (Sec. 5)
    def add(self, X, y):
        X, y = self._dev(X), self._dev(y)
        _check(_lib.lip_add(self.h, X.data_ptr(), y.data_ptr(), X.shape[0], _stream_ptr()), "lip_add")

    def add_host(self, X, y):
        """lip_add_host: X, y are host arrays (numpy or pinned CPU tensors) of the handle's type."""
        torch = _torch()

        def p(a):
            return a.data_ptr() if torch.is_tensor(a) else a.ctypes.data

        _check(_lib.lip_add_host(self.h, p(X), p(y), X.shape[0], _stream_ptr()), "lip_add_host")

    def add_async(self, X, y):
        """lip_add_async: no wait for the GPU; non-finite points are replaced on the device and
        reported by the next check() (LIP_ERR_NONFINITE)."""
        X, y = self._dev(X), self._dev(y)
        _check(_lib.lip_add_async(self.h, X.data_ptr(), y.data_ptr(), X.shape[0], _stream_ptr()), "lip_add_async")

    def add_host_async(self, X, y):
        """lip_add_host_async: X, y host arrays (pinned CPU tensors keep the copy asynchronous;
        they must stay alive until the stream has passed this call)."""
        torch = _torch()

        def p(a):
            return a.data_ptr() if torch.is_tensor(a) else a.ctypes.data

        _check(_lib.lip_add_host_async(self.h, p(X), p(y), X.shape[0], _stream_ptr()), "lip_add_host_async")

    def clear(self):
        _check(_lib.lip_clear(self.h, _stream_ptr()), "lip_clear")

    @property
    def N(self) -> int:
        return int(_lib.lip_size(self.h))

    @property
    def M(self) -> float:
        return self._M

    def set_M(self, M: float):
        _check(_lib.lip_set_M(self.h, float(M), _stream_ptr()), "lip_set_M")
        self._M = float(M)

    # -- evaluation
    def eval(self, Q, need=("g", "lo", "hi", "idx_up", "idx_lo")):
        """Dict of CUDA tensors g, lo, hi (H_lo, H_up) and idx_up, idx_lo for queries Q."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        out = {}
        for k in ("g", "lo", "hi"):
            out[k] = torch.empty(nq, device="cuda", dtype=self.dtype) if k in need else None
        for k in ("idx_up", "idx_lo"):
            out[k] = torch.empty(nq, device="cuda", dtype=torch.int32) if k in need else None
        _check(_lib.lip_eval(self.h, Q.data_ptr(), nq, _ptr(out["g"]), _ptr(out["lo"]), _ptr(out["hi"]),
                             _ptr(out["idx_up"]), _ptr(out["idx_lo"]), _stream_ptr()), "lip_eval")
        return {k: v for k, v in out.items() if v is not None}

    def eval_k(self, Q, k: int, wk):
        """k > 1 neighbours (Sec. 5): dict of g, lo, hi [nq] and idx_up, idx_lo [nq, k]."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        wk_a = np.ascontiguousarray(np.asarray(wk, np.float64))
        assert wk_a.shape == (k,)
        out = {key: torch.empty(nq, device="cuda", dtype=self.dtype) for key in ("g", "lo", "hi")}
        out.update({key: torch.empty((nq, k), device="cuda", dtype=torch.int32) for key in ("idx_up", "idx_lo")})
        _check(_lib.lip_eval_k(self.h, Q.data_ptr(), nq, int(k), wk_a.ctypes.data, out["g"].data_ptr(),
                               out["lo"].data_ptr(), out["hi"].data_ptr(), out["idx_up"].data_ptr(),
                               out["idx_lo"].data_ptr(), _stream_ptr()), "lip_eval_k")
        return out

    def values(self, Q):
        """g at the query points (Sec. 5: values(query, LC, model, k=1))."""
        return self.eval(Q, need=("g",))["g"]

    # ------------------------------------------- local Lipschitz constants (Sec. 4.3)
    def compute_local_lipschitz(self, nknots: int = 16, sample_pairs: int = 32768, seed: int = 0, knots=None):
        """Per-datum step functions M_k(t) (lip_local_fit, or lip_local_fit_knots with
        explicit knots); returns the knots in use."""
        if knots is None:
            _check(_lib.lip_local_fit(self.h, int(nknots), int(sample_pairs), int(seed) & (2**64 - 1),
                                      _stream_ptr()), "lip_local_fit")
        else:
            k = np.ascontiguousarray(np.asarray(knots, np.float64).reshape(-1))
            _check(_lib.lip_local_fit_knots(self.h, k.ctypes.data if k.size else None, int(k.size), _stream_ptr()),
                   "lip_local_fit_knots")
        return self.local_knots()

    def local_knots(self):
        s, k = lip_local_knots(self.h)
        _check(s, "lip_local_knots")
        return np.array(k, np.float64)

    def local_stats(self):
        """(overflow rows, longest candidate list) of the last table fit."""
        s, over, mc = lip_local_stats(self.h)
        _check(s, "lip_local_stats")
        return over, mc

    def local_table(self):
        """(d1 [N], F [N], Mtab [N, m+1]) as float64 CUDA tensors."""
        torch = _torch()
        m = self.local_knots().size
        N = self.N
        d1 = torch.empty(N, device="cuda", dtype=torch.float64)
        F = torch.empty(N, device="cuda", dtype=torch.float64)
        Mtab = torch.empty((N, m + 1), device="cuda", dtype=torch.float64)
        _check(_lib.lip_local_table(self.h, d1.data_ptr(), F.data_ptr(), Mtab.data_ptr(), _stream_ptr()),
               "lip_local_table")
        return d1, F, Mtab

    def eval_local(self, Q, need=("g", "lo", "hi", "idx_up", "idx_lo")):
        """Envelopes with the local constants (lip_eval_local): dict of CUDA tensors."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        out = {}
        for key in need:
            dt = torch.int32 if key.startswith("idx") else self.dtype
            out[key] = torch.empty(nq, device="cuda", dtype=dt)
        _check(_lib.lip_eval_local(self.h, Q.data_ptr(), nq, *[_ptr(out.get(k)) for k in ("g", "lo", "hi", "idx_up",
                                                                                           "idx_lo")],
                                   _stream_ptr()), "lip_eval_local")
        return out

    # --------------------------------------------------- penalty smoothing (Sec. 4.4)
    def smooth_objective(self, eps, M: float, p: float, grad: bool = True):
        """(Phi, grad) of Eq. (optim) at eps (float64 CUDA tensor [N])."""
        torch = _torch()
        eps = eps.to("cuda", torch.float64).contiguous()
        g = torch.empty(self.N, device="cuda", dtype=torch.float64) if grad else None
        s, f = lip_smooth_objective(self.h, float(M), float(p), eps.data_ptr(), _ptr(g), _stream_ptr())
        _check(s, "lip_smooth_objective")
        return f, g

    def smooth_lipschitz(self, M: float, p: float = 100.0, max_iter: int = 200, history: int = 10,
                         gtol: float = 1e-7):
        """Sec. 5 smooth_lipschitz(LC): minimise Eq. (optim) with L-BFGS, replace y by y + eps and
        the constant by M.  Returns (eps float64 CUDA tensor, Phi, iterations, evaluations)."""
        torch = _torch()
        eps = torch.empty(self.N, device="cuda", dtype=torch.float64)
        s, f, it, ev = lip_smooth(self.h, float(M), float(p), int(max_iter), int(history), float(gtol),
                                  eps.data_ptr(), _stream_ptr())
        _check(s, "lip_smooth")
        self._M = float(M)
        return eps, f, it, ev

    def eval_local_k(self, Q, k: int, wk):
        """k > 1 neighbours with the local constants: dict of g, lo, hi [nq], idx_up, idx_lo [nq, k]."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        wk_a = np.ascontiguousarray(np.asarray(wk, np.float64))
        assert wk_a.shape == (k,)
        out = {key: torch.empty(nq, device="cuda", dtype=self.dtype) for key in ("g", "lo", "hi")}
        out.update({key: torch.empty((nq, k), device="cuda", dtype=torch.int32) for key in ("idx_up", "idx_lo")})
        _check(_lib.lip_eval_local_k(self.h, Q.data_ptr(), nq, int(k), wk_a.ctypes.data, out["g"].data_ptr(),
                                     out["lo"].data_ptr(), out["hi"].data_ptr(), out["idx_up"].data_ptr(),
                                     out["idx_lo"].data_ptr(), _stream_ptr()), "lip_eval_local_k")
        return out

    def values_local(self, Q, k: int = 1, wk=None):
        """g with the local constants (Sec. 5: values_local(query, model, k))."""
        if k == 1 and wk is None:
            return self.eval_local(Q, need=("g",))["g"]
        return self.eval_local_k(Q, k, np.ones(k) / k if wk is None else wk)["g"]

    def eval_host(self, Q, out=None, wait=True):
        """lip_eval_host: Q and the outputs in host memory (numpy or pinned CPU tensors).
        wait=False: lip_eval_host_async, the outputs are valid once check() has returned
        (Q and out must stay alive until then)."""
        torch = _torch()
        if torch.is_tensor(Q):
            Qh = Q
            nq = Q.shape[0]
            qptr = Q.data_ptr()
        else:
            Qh = np.ascontiguousarray(Q, dtype=np.float64 if self.precision == LIP_FP64 else np.float32)
            nq = Qh.shape[0]
            qptr = Qh.ctypes.data
        if out is None:
            npdt = np.float64 if self.precision == LIP_FP64 else np.float32
            out = {k: np.empty(nq, npdt) for k in ("g", "lo", "hi")}
            out.update({k: np.empty(nq, np.int32) for k in ("idx_up", "idx_lo")})

        def p(a):
            if a is None:
                return None
            return a.data_ptr() if torch.is_tensor(a) else a.ctypes.data

        fn = _lib.lip_eval_host if wait else _lib.lip_eval_host_async
        _check(fn(self.h, qptr, nq, p(out.get("g")), p(out.get("lo")), p(out.get("hi")),
                  p(out.get("idx_up")), p(out.get("idx_lo")), _stream_ptr()), "lip_eval_host")
        return out

    # -- several GPUs (paper_2606_04670_b300.shard drives these around the collectives)
    def shard_scan(self, Q, index_base: int):
        """lip_shard_scan: packed keys (int64 CUDA tensors key_up, key_lo) of this handle's data,
        whose global indices start at index_base."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        ku = torch.empty(nq, device="cuda", dtype=torch.int64)
        kl = torch.empty(nq, device="cuda", dtype=torch.int64)
        _check(_lib.lip_shard_scan(self.h, Q.data_ptr(), nq, int(index_base), ku.data_ptr(), kl.data_ptr(),
                                   _stream_ptr()), "lip_shard_scan")
        return ku, kl

    def shard_reeval(self, Q, index_base: int, key_up, key_lo):
        """lip_shard_reeval: FP64 bounds (hi64, lo64) of the winners this handle holds, +-Inf
        elsewhere."""
        torch = _torch()
        Q = self._dev(Q)
        nq = Q.shape[0]
        hi = torch.empty(nq, device="cuda", dtype=torch.float64)
        lo = torch.empty(nq, device="cuda", dtype=torch.float64)
        _check(_lib.lip_shard_reeval(self.h, Q.data_ptr(), nq, int(index_base), key_up.data_ptr(), key_lo.data_ptr(),
                                     hi.data_ptr(), lo.data_ptr(), _stream_ptr()), "lip_shard_reeval")
        return hi, lo

    def shard_finish(self, key_up, key_lo, hi64, lo64):
        """lip_shard_finish: the outputs (g, lo, hi, idx_up, idx_lo) from merged keys and values."""
        torch = _torch()
        nq = key_up.shape[0]
        out = {k: torch.empty(nq, device="cuda", dtype=self.dtype) for k in ("g", "lo", "hi")}
        out.update({k: torch.empty(nq, device="cuda", dtype=torch.int32) for k in ("idx_up", "idx_lo")})
        _check(_lib.lip_shard_finish(self.h, nq, key_up.data_ptr(), key_lo.data_ptr(), hi64.data_ptr(),
                                     lo64.data_ptr(), out["g"].data_ptr(), out["lo"].data_ptr(), out["hi"].data_ptr(),
                                     out["idx_up"].data_ptr(), out["idx_lo"].data_ptr(), _stream_ptr()),
               "lip_shard_finish")
        return out

    def estimate_M_part(self, part: int, nparts: int):
        """lip_estimate_M_part: [M, i, j, key = M] of one block-cyclic share."""
        s, out = lip_estimate_M_part(self.h, int(part), int(nparts), _stream_ptr())
        _check(s, "lip_estimate_M_part")
        return out

    def lipschitz_constant(self):
        """(M_est, i, j) (Sec. 5: lipschitz_constant()), the FP64 definition's maximum and
        its lowest pair exactly; synchronises."""
        s, M, i, j = lip_estimate_M(self.h, _stream_ptr())
        _check(s, "lip_estimate_M")
        return M, i, j

    def lipschitz_constant_async(self):
        """Queue lipschitz_constant() on the current stream without waiting; the result is
        read by lipschitz_constant_result()."""
        _check(lip_estimate_M_async(self.h, _stream_ptr()), "lip_estimate_M_async")

    def lipschitz_constant_result(self):
        """(M_est, i, j) of the estimate lipschitz_constant_async() queued, after waiting
        for it."""
        s, M, i, j = lip_estimate_M_result(self.h)
        _check(s, "lip_estimate_M_result")
        return M, i, j

    def backward(self, Q, idx_up, idx_lo, grad_g, need_Q=True, need_y=True, need_M=True, deterministic=False):
        torch = _torch()
        Q = self._dev(Q)
        gg = grad_g.to(device="cuda", dtype=self.dtype).contiguous()
        gQ = torch.empty_like(Q) if need_Q else None
        gy = torch.zeros(self.N, device="cuda", dtype=self.dtype) if need_y else None
        gM = torch.empty(1, device="cuda", dtype=torch.float64) if need_M else None
        _check(_lib.lip_backward(self.h, Q.data_ptr(), Q.shape[0], idx_up.data_ptr(), idx_lo.data_ptr(),
                                 gg.data_ptr(), _ptr(gQ), _ptr(gy), _ptr(gM), int(bool(deterministic)),
                                 _stream_ptr()), "lip_backward")
        return gQ, gy, gM

    def check(self):
        _check(_lib.lip_check(self.h, _stream_ptr()), "lip_check")

    def last_estimate_work(self):
        """[tile pairs entered, (row, chunk) pairs evaluated, total (row, chunk) pairs] of
        the last pruned lip_estimate_M's screen; all -1 when it was not pruned."""
        out = (ctypes.c_int64 * 3)()
        _check(_lib.lip_last_estimate_work(self.h, out), "lip_last_estimate_work")
        return list(out)

    def last_scan_stats(self):
        """[evaluated (row, chunk) pairs, all of them, tiles copied, blocks x tiles,
        (warp, chunk) pairs past the warp-box test] of the last pruned scan; -1 entries when
        it was not pruned."""
        out = (ctypes.c_int64 * 5)()
        _check(_lib.lip_last_scan_stats(self.h, out), "lip_last_scan_stats")
        return list(out)

    def last_scan_work(self):
        """(evaluated, total) (32-query row, 32-point chunk) pairs of the last pruned scan
        (variants 6 / 7); (-1, -1) when the last scan was not pruned."""
        e, t = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.lip_last_scan_work(self.h, ctypes.byref(e), ctypes.byref(t)), "lip_last_scan_work")
        return e.value, t.value

    def set_estimate_full(self, full: bool = True):
        """lip_estimate_M with the full all-pairs kernel (True) or the default choice
        (False: the pruned form from N = 32768 where available); same result."""
        _check(_lib.lip_set_estimate_full(self.h, int(bool(full))), "lip_set_estimate_full")

    def set_estimate_form(self, form: str = "auto"):
        """lip_estimate_M's form: "auto" (the default: pruned from N = 32768 where
        available), "full" or "pruned" (wherever available); all give the same result."""
        code = {"auto": 0, "full": 1, "pruned": 2}[form]
        _check(_lib.lip_set_estimate_full(self.h, code), "lip_set_estimate_full")

    def set_tc_window(self, nbytes: int = 0):
        """Tensor-core handles: the data bytes a round's persistent CTAs may spread their
        sweeps over (0: the default)."""
        _check(_lib.lip_set_tc_window(self.h, int(nbytes)), "lip_set_tc_window")

    def last_fallback(self) -> int:
        return lip_last_fallback(self.h)

    def set_tuning(self, tile_groups: int = 0, splits: int = 0, variant: int = -1):
        _check(_lib.lip_set_tuning(self.h, int(tile_groups), int(splits), int(variant)), "lip_set_tuning")

    def set_timing_events(self, ev_before=None, ev_after=None):
        """torch.cuda.Event pair recorded around the scan kernel of every eval (None: off)."""
        for ev in (ev_before, ev_after):
            if ev is not None and not ev.cuda_event:
                ev.record()            # torch creates the CUDA event on first record
        a = None if ev_before is None else ev_before.cuda_event
        b = None if ev_after is None else ev_after.cuda_event
        _check(_lib.lip_set_timing_events(self.h, a, b), "lip_set_timing_events")

    def tuning(self):
        s, (tg, sp, last, rows, var) = lip_get_tuning(self.h)
        _check(s, "lip_get_tuning")
        return {"tile_groups": tg, "splits": sp, "last_splits": last, "queries_per_thread": rows, "variant": var}

    def close(self):
        if self.h:
            _lib.lip_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LipBatch:
    """Many independent data sets evaluated by one persistent launch (lip_batch_*).

    sets: list of dicts with keys X, y, Q (CUDA float32 tensors), M, norm, and optional
    mon, w.  Outputs are allocated here as CUDA tensors (``outputs[i]`` holds g, lo, hi,
    idx_up, idx_lo of set i) and refreshed in place by every ``eval``; refill
    ``sets[i]['Q']`` in place to evaluate new queries.  ``eval`` only enqueues work, so
    it can be captured in a torch.cuda.CUDAGraph.
    """

    def __init__(self, sets, tile_groups=0, items_per_block=0, waves=0, outputs=None):
        torch = _torch()
        self.sets = []
        self.outputs = []
        self._keep = []
        arr = (lip_batch_set * len(sets))()
        for k, st in enumerate(sets):
            X = st["X"].to(device="cuda", dtype=torch.float32).contiguous()
            y = st["y"].to(device="cuda", dtype=torch.float32).contiguous()
            Q = st["Q"].to(device="cuda", dtype=torch.float32).contiguous()
            nq = Q.shape[0]
            if outputs is not None:
                out = outputs[k]       # caller-owned CUDA tensors (e.g. views of one buffer)
            else:
                out = {"g": torch.empty(nq, device="cuda"), "lo": torch.empty(nq, device="cuda"),
                       "hi": torch.empty(nq, device="cuda"),
                       "idx_up": torch.empty(nq, device="cuda", dtype=torch.int32),
                       "idx_lo": torch.empty(nq, device="cuda", dtype=torch.int32)}
            mon = None if st.get("mon") is None else np.ascontiguousarray(st["mon"], np.int8)
            w = None if st.get("w") is None else np.ascontiguousarray(st["w"], np.float64)
            self._keep += [mon, w]
            nv = NORMS[st.get("norm", LIP_L2)]
            arr[k] = lip_batch_set(X.data_ptr(), y.data_ptr(), X.shape[0], X.shape[1], nv, float(st["M"]),
                                   None if mon is None else mon.ctypes.data, None if w is None else w.ctypes.data,
                                   Q.data_ptr() if nq else None, nq, out["g"].data_ptr(), out["lo"].data_ptr(),
                                   out["hi"].data_ptr(), out["idx_up"].data_ptr(), out["idx_lo"].data_ptr(),
                                   int(st.get("tile_groups", 0)), 0)
            self.sets.append({"X": X, "y": y, "Q": Q})
            self.outputs.append(out)
        opt = lip_batch_options(int(tile_groups), int(items_per_block), int(waves), 0)
        s, self.h = lip_batch_create(arr, opt, _stream_ptr())
        _check(s, "lip_batch_create")
        # the copies of X and y are made; keep Q and the outputs alive with the batch

    def eval(self):
        _check(_lib.lip_batch_eval(self.h, _stream_ptr()), "lip_batch_eval")

    def info(self):
        s, tp, tq, ni, gr = lip_batch_info(self.h)
        _check(s, "lip_batch_info")
        return {"total_pairs": tp, "total_queries": tq, "items": ni, "grid": gr}

    def check(self):
        _check(_lib.lip_batch_check(self.h, _stream_ptr()), "lip_batch_check")

    def set_timing_events(self, ev_before=None, ev_after=None):
        for ev in (ev_before, ev_after):
            if ev is not None and not ev.cuda_event:
                ev.record()
        _check(_lib.lip_batch_set_timing_events(self.h, None if ev_before is None else ev_before.cuda_event,
                                                None if ev_after is None else ev_after.cuda_event),
               "lip_batch_set_timing_events")

    def close(self):
        if self.h:
            _lib.lip_batch_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    torch = _torch()

    class LipEvalFn(torch.autograd.Function):
        """g(Q) with gradients for Q, y and M through the saved argmin/argmax.

        ``LipEvalFn.apply(Q, y, M, model)``: y and M are the tensors ``model`` was built
        from (y [N], M a 0-d or 1-element tensor); they only receive gradients.
        """

        @staticmethod
        def forward(ctx, Q, y, M, model):
            r = model.eval(Q, need=("g", "idx_up", "idx_lo"))
            ctx.model = model
            ctx.M_shape, ctx.M_dtype = M.shape, M.dtype
            ctx.save_for_backward(Q, r["idx_up"], r["idx_lo"])
            return r["g"]

        @staticmethod
        def backward(ctx, grad_g):
            Q, iu, il = ctx.saved_tensors
            m = ctx.model
            nQ, ny, nM = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            gQ, gy, gM = m.backward(Q, iu, il, grad_g, need_Q=nQ, need_y=ny, need_M=nM)
            gMo = gM.to(ctx.M_dtype).reshape(ctx.M_shape) if nM else None
            return gQ, gy, gMo, None

    return LipEvalFn


LipEvalFn = None
try:  # torch is optional for the raw ABI functions
    LipEvalFn = _make_autograd()
except Exception:  # pragma: no cover
    pass
