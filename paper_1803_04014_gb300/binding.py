"""ctypes binding of the tcgemm C ABI (include/tcgemm.h), same names as the C calls.

Argument marshalling only: every step runs in the CUDA library.  Matrix
arguments may be torch tensors (their ``data_ptr()`` is passed) or integer
device addresses; ``stream`` defaults to the current torch stream of the
current device.  A non-OK status raises ``TcError`` with the library's message
(``TC_PENDING`` from ``serve_poll`` is returned, not raised).  If the shared
library is missing the import of this module fails: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import builder as _build

TC_OK = 0
TC_PENDING = 1
TC_ERR_INVALID = -1
TC_ERR_UNSUPPORTED = -2
TC_ERR_OOM = -3
TC_ERR_CUDA = -4
TC_ERR_TIMEOUT = -5
TC_ERR_BUSY = -6

TC_F16, TC_BF16, TC_E4M3 = 0, 1, 2
TC_ROW_MAJOR, TC_COL_MAJOR = 0, 1
TC_MODE_F16, TC_MODE_BF16, TC_MODE_E4M3, TC_MODE_SPLIT3 = 0, 1, 2, 3

_STATUS_NAMES = {0: "TC_OK", 1: "TC_PENDING", -1: "TC_ERR_INVALID", -2: "TC_ERR_UNSUPPORTED",
                 -3: "TC_ERR_OOM", -4: "TC_ERR_CUDA", -5: "TC_ERR_TIMEOUT", -6: "TC_ERR_BUSY"}


class TcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tc_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("k", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("off_a", ctypes.c_int64), ("off_b", ctypes.c_int64), ("off_c", ctypes.c_int64),
                ("lda", ctypes.c_int32), ("ldb", ctypes.c_int32), ("ldc", ctypes.c_int32),
                ("reserved2", ctypes.c_int32)]


class tc_quantize_job(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("src", ctypes.c_void_p),
                ("ld_src", ctypes.c_int64), ("dst", ctypes.c_void_p), ("ld_dst", ctypes.c_int64),
                ("transpose", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tc_serve_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("num_streams", ctypes.c_int32), ("queue_capacity", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tc_request(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float)]


class tc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t_submit_us", ctypes.c_double),
                ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


_i32, _i64, _u64, _f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
_vp, _sz = ctypes.c_void_p, ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/tcgemm.h
SIGNATURES = {
    "tc_version": (ctypes.c_char_p, []),
    "tc_last_error": (ctypes.c_char_p, []),
    "tc_device_info": (_i32, [ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "tc_sync_status": (_i32, [_vp]),
    "tc_debug_stall_next_gemm": (_i32, [_i32]),
    "tc_quantize": (_i32, [_i32, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "tc_split": (_i32, [_i32, _i64, _i64, _vp, _i64, _i32, _vp, _vp, _i64, _vp]),
    "gemm_mixed": (_i32, [_i32, _i64, _i64, _i64, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _i64,
                          _vp, _vp, _vp]),
    "tc_split_scaled": (_i32, [_i32, _i64, _i64, _vp, _i64, _i32, _vp, _vp, _i64, _vp]),
    "tc_split_bf16x3": (_i32, [_i64, _i64, _vp, _i64, _i32, _vp, _vp, _vp, _i64, _vp]),
    "gemm_split_workspace_bytes": (_sz, [_i32, _i32, _i64, _i64, _i64]),
    "gemm_split_scaled": (_i32, [_i32, _i32, _i64, _i64, _i64, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp,
                                 _i64, _vp, _sz, _vp]),
    "gemm_split_bf16x3": (_i32, [_i64, _i64, _i64, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _i64, _vp,
                                 _sz, _vp]),
    "gemm_split_prepare": (_i32, [_i32, _i32, _i32, _i64, _i64, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _sz,
                                  _vp]),
    "gemm_split_run": (_i32, [_i32, _i32, _i32, _i64, _i64, _i64, _f32, _f32, _vp, _i64, _vp, _sz, _vp]),
    "gemm_split": (_i32, [_i32, _i32, _i64, _i64, _i64, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _i64,
                          _vp, _sz, _vp]),
    "gemm_sgemm": (_i32, [_i64, _i64, _i64, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32, _vp, _i64, _vp]),
    "gemm_batched_strided": (_i32, [_i32, _i64, _i32, _i32, _i32, _f32, _vp, _i64, _i32, _vp, _i64, _i32, _f32,
                                    _vp, _i64, _vp]),
    "gemm_grouped_plan_create": (_i32, [_i32, _i32, ctypes.POINTER(tc_problem), _i32, _i32,
                                        ctypes.POINTER(_vp)]),
    "gemm_grouped_plan_run": (_i32, [_vp, _vp, _vp, _vp, _f32, _f32, _i32, _vp]),
    "gemm_grouped_plan_destroy": (_i32, [_vp]),
    "gemm_grouped": (_i32, [_i32, _i32, ctypes.POINTER(tc_problem), _vp, _i32, _vp, _i32, _vp, _f32, _f32, _vp]),
    "gemm_grouped_noalloc": (_i32, [_i32, _i32, ctypes.POINTER(tc_problem), _vp, _i32, _vp, _i32, _vp, _f32, _f32,
                                    _vp]),
    "gemm_grouped_workspace_bytes": (_sz, [_i32, ctypes.POINTER(tc_problem)]),
    "gemm_grouped_ws": (_i32, [_i32, _i32, ctypes.POINTER(tc_problem), _vp, _i32, _vp, _i32, _vp, _f32, _f32, _vp,
                               _sz, _vp]),
    "tc_quantize_batch_workspace_bytes": (_sz, [_i32, ctypes.POINTER(tc_quantize_job)]),
    "tc_quantize_batch": (_i32, [_i32, _i32, ctypes.POINTER(tc_quantize_job), _vp, _sz, _vp]),
    "tc_quantize_batch_e4m3": (_i32, [_i32, ctypes.POINTER(tc_quantize_job), ctypes.POINTER(_vp), _vp, _sz, _vp]),
    "tc_autotune_gemm": (_i32, [_i32, _i64, _i64, _i64, _vp, ctypes.POINTER(ctypes.c_double)]),
    "gemm_grouped_plan_autotune": (_i32, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "tc_autotune_save": (_i32, [ctypes.c_char_p]),
    "tc_autotune_load": (_i32, [ctypes.c_char_p]),
    "tc_error_norm": (_i32, [_i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _i64, _i64, _i64, _vp, _i64, _i64,
                             _i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "tc_error_norm_workspace_bytes": (_sz, []),
    "tc_error_norm_dev": (_i32, [_i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _i64, _i64, _i64, _vp, _i64, _i64,
                                 _i64, _vp, _vp, _sz, _vp]),
    "serve_open": (_i32, [ctypes.POINTER(tc_serve_cfg), ctypes.POINTER(_vp)]),
    "serve_submit": (_i32, [_vp, ctypes.POINTER(tc_request), ctypes.POINTER(_u64)]),
    "serve_poll": (_i32, [_vp, _u64, ctypes.POINTER(tc_result)]),
    "serve_drain": (_i32, [_vp, _i64]),
    "serve_stats": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "serve_timing": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "serve_close": (_i32, [_vp]),
}

_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libtcgemm.so (building it first if allowed); raises if it cannot be loaded."""
    global _LIB
    lib = _LIB
    if lib is not None:   # set once, under the lock, fully configured
        return lib
    with _LOCK:
        if _LIB is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"tcgemm library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


_RAW_STREAM = None


def _current_stream_fn():
    """A function returning torch's current CUDA stream handle.  torch.cuda.current_stream()
    builds a Stream object (about 3 us per call on the Grace host); torch's own raw-stream
    query returns the handle alone.  It is used when present and agrees with the public API."""
    global _RAW_STREAM
    if _RAW_STREAM is None:
        import torch

        def public():
            return torch.cuda.current_stream().cuda_stream

        fn = public
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        get_dev = getattr(torch._C, "_cuda_getDevice", None)
        if raw is not None and get_dev is not None:
            def fast():
                return raw(get_dev())
            try:
                if fast() == public():
                    fn = fast
            except Exception:
                fn = public
        _RAW_STREAM = fn
    return _RAW_STREAM


def _stream(stream):
    if stream is None:
        return _current_stream_fn()()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str) -> int:
    if status not in (TC_OK, TC_PENDING):
        raise TcError(status, where, load().tc_last_error().decode())
    return status


def tc_version() -> str:
    return load().tc_version().decode()


def tc_last_error() -> str:
    return load().tc_last_error().decode()


def tc_device_info():
    sm, ma, mi = _i32(), _i32(), _i32()
    _check(load().tc_device_info(ctypes.byref(sm), ctypes.byref(ma), ctypes.byref(mi)), "tc_device_info")
    return sm.value, ma.value, mi.value


def tc_sync_status(stream=None) -> int:
    return _check(load().tc_sync_status(_stream(stream)), "tc_sync_status")


def tc_debug_stall_next_gemm(k_block):
    """Test hook: the next tensor-core GEMM of this thread withholds one k-block (see tcgemm_debug.h)."""
    return _check(load().tc_debug_stall_next_gemm(int(k_block)), "tc_debug_stall_next_gemm")


def tc_quantize(dt, rows, cols, src, ld_src, dst, ld_dst, transpose=0, scale_out=None, stream=None):
    return _check(load().tc_quantize(dt, rows, cols, _ptr(src), ld_src, _ptr(dst), ld_dst, int(transpose),
                                     _ptr(scale_out), _stream(stream)), "tc_quantize")


def tc_split(piece, rows, cols, src, ld_src, transpose, dst_hi, dst_lo, ld_dst, stream=None):
    return _check(load().tc_split(piece, rows, cols, _ptr(src), ld_src, int(transpose), _ptr(dst_hi),
                                  _ptr(dst_lo), ld_dst, _stream(stream)), "tc_split")


def gemm_mixed(dt, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, scale_a=None, scale_b=None, stream=None):
    return _check(load().gemm_mixed(dt, m, n, k, alpha, _ptr(A), lda, la, _ptr(B), ldb, lb, beta, _ptr(C), ldc,
                                    _ptr(scale_a), _ptr(scale_b), _stream(stream)), "gemm_mixed")


def tc_split_scaled(piece, rows, cols, src, ld_src, transpose, dst_hi, dst_lo, ld_dst, stream=None):
    return _check(load().tc_split_scaled(piece, rows, cols, _ptr(src), ld_src, int(transpose), _ptr(dst_hi),
                                         _ptr(dst_lo), ld_dst, _stream(stream)), "tc_split_scaled")


def tc_split_bf16x3(rows, cols, src, ld_src, transpose, dst0, dst1, dst2, ld_dst, stream=None):
    return _check(load().tc_split_bf16x3(rows, cols, _ptr(src), ld_src, int(transpose), _ptr(dst0), _ptr(dst1),
                                         _ptr(dst2), ld_dst, _stream(stream)), "tc_split_bf16x3")


def gemm_split_workspace_bytes(piece, nprod, m, n, k) -> int:
    return int(load().gemm_split_workspace_bytes(piece, nprod, m, n, k))


def gemm_split(piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, workspace=None,
               workspace_bytes=0, stream=None):
    return _check(load().gemm_split(piece, nprod, m, n, k, alpha, _ptr(A), lda, la, _ptr(B), ldb, lb, beta, _ptr(C),
                                    ldc, _ptr(workspace), int(workspace_bytes), _stream(stream)), "gemm_split")


def gemm_split_scaled(piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, workspace=None,
                      workspace_bytes=0, stream=None):
    return _check(load().gemm_split_scaled(piece, nprod, m, n, k, alpha, _ptr(A), lda, la, _ptr(B), ldb, lb, beta,
                                           _ptr(C), ldc, _ptr(workspace), int(workspace_bytes), _stream(stream)),
                  "gemm_split_scaled")


def gemm_split_bf16x3(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, workspace=None, workspace_bytes=0,
                      stream=None):
    return _check(load().gemm_split_bf16x3(m, n, k, alpha, _ptr(A), lda, la, _ptr(B), ldb, lb, beta, _ptr(C), ldc,
                                           _ptr(workspace), int(workspace_bytes), _stream(stream)),
                  "gemm_split_bf16x3")


def gemm_split_prepare(scheme, piece, nprod, m, n, k, A, lda, la, B, ldb, lb, workspace, workspace_bytes,
                       stream=None):
    """The pieces phase of a refined GEMM (scheme 0 gemm_split, 1 scaled, 2 BF16x3) into `workspace`."""
    return _check(load().gemm_split_prepare(scheme, piece, nprod, m, n, k, _ptr(A), lda, la, _ptr(B), ldb, lb,
                                            _ptr(workspace), int(workspace_bytes), _stream(stream)),
                  "gemm_split_prepare")


def gemm_split_run(scheme, piece, nprod, m, n, k, alpha, beta, C, ldc, workspace, workspace_bytes, stream=None):
    """The tensor-core phase of a refined GEMM, on the pieces gemm_split_prepare left in `workspace`."""
    return _check(load().gemm_split_run(scheme, piece, nprod, m, n, k, alpha, beta, _ptr(C), ldc, _ptr(workspace),
                                        int(workspace_bytes), _stream(stream)), "gemm_split_run")


def gemm_sgemm(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, stream=None):
    return _check(load().gemm_sgemm(m, n, k, alpha, _ptr(A), lda, la, _ptr(B), ldb, lb, beta, _ptr(C), ldc,
                                    _stream(stream)), "gemm_sgemm")


def gemm_batched_strided(dt, batch, m, n, k, alpha, A, stride_a, la, B, stride_b, lb, beta, C, stride_c,
                         stream=None):
    return _check(load().gemm_batched_strided(dt, batch, m, n, k, alpha, _ptr(A), stride_a, la, _ptr(B), stride_b,
                                              lb, beta, _ptr(C), stride_c, _stream(stream)), "gemm_batched_strided")


def problems_array(rows):
    """(count, 10)-like rows (m, n, k, off_a, off_b, off_c, lda, ldb, ldc) -> ctypes array of tc_problem."""
    arr = (tc_problem * len(rows))()
    for i, (m, n, k, oa, ob, oc, lda, ldb, ldc) in enumerate(rows):
        arr[i] = tc_problem(int(m), int(n), int(k), 0, int(oa), int(ob), int(oc), int(lda), int(ldb), int(ldc), 0)
    return arr


def gemm_grouped_plan_create(dt, problems, la, lb):
    plan = _vp()
    arr = problems if isinstance(problems, ctypes.Array) else problems_array(problems)
    _check(load().gemm_grouped_plan_create(dt, len(arr), arr, la, lb, ctypes.byref(plan)),
           "gemm_grouped_plan_create")
    return plan.value


def gemm_grouped_plan_run(plan, a_base, b_base, c_base, alpha, beta, use_graph=0, stream=None):
    return _check(load().gemm_grouped_plan_run(plan, _ptr(a_base), _ptr(b_base), _ptr(c_base), alpha, beta,
                                               int(use_graph), _stream(stream)), "gemm_grouped_plan_run")


def gemm_grouped_plan_destroy(plan):
    return _check(load().gemm_grouped_plan_destroy(plan), "gemm_grouped_plan_destroy")


def gemm_grouped(dt, problems, a_base, la, b_base, lb, c_base, alpha, beta, stream=None):
    arr = problems if isinstance(problems, ctypes.Array) else problems_array(problems)
    return _check(load().gemm_grouped(dt, len(arr), arr, _ptr(a_base), la, _ptr(b_base), lb, _ptr(c_base), alpha,
                                      beta, _stream(stream)), "gemm_grouped")


def gemm_grouped_noalloc(dt, problems, a_base, la, b_base, lb, c_base, alpha, beta, stream=None):
    """gemm_grouped without any device allocation (schedule in the library's static scratch)."""
    arr = problems if isinstance(problems, ctypes.Array) else problems_array(problems)
    return _check(load().gemm_grouped_noalloc(dt, len(arr), arr, _ptr(a_base), la, _ptr(b_base), lb, _ptr(c_base),
                                              alpha, beta, _stream(stream)), "gemm_grouped_noalloc")


def gemm_grouped_workspace_bytes(problems) -> int:
    arr = problems if isinstance(problems, ctypes.Array) else problems_array(problems)
    return int(load().gemm_grouped_workspace_bytes(len(arr), arr))


def gemm_grouped_ws(dt, problems, a_base, la, b_base, lb, c_base, alpha, beta, workspace, workspace_bytes,
                    stream=None):
    """gemm_grouped_noalloc with the schedule in caller-owned device memory."""
    arr = problems if isinstance(problems, ctypes.Array) else problems_array(problems)
    return _check(load().gemm_grouped_ws(dt, len(arr), arr, _ptr(a_base), la, _ptr(b_base), lb, _ptr(c_base), alpha,
                                         beta, _ptr(workspace), int(workspace_bytes), _stream(stream)),
                  "gemm_grouped_ws")


def quantize_jobs_array(jobs):
    """[(rows, cols, src, ld_src, dst, ld_dst, transpose)] -> ctypes array of tc_quantize_job."""
    arr = (tc_quantize_job * len(jobs))()
    for i, (rows, cols, src, ld_src, dst, ld_dst, tr) in enumerate(jobs):
        arr[i] = tc_quantize_job(int(rows), int(cols), _ptr(src), int(ld_src), _ptr(dst), int(ld_dst), int(tr), 0)
    return arr


def tc_quantize_batch_workspace_bytes(jobs) -> int:
    arr = jobs if isinstance(jobs, ctypes.Array) else quantize_jobs_array(jobs)
    return int(load().tc_quantize_batch_workspace_bytes(len(arr), arr))


def tc_quantize_batch(dt, jobs, workspace, workspace_bytes, stream=None):
    arr = jobs if isinstance(jobs, ctypes.Array) else quantize_jobs_array(jobs)
    return _check(load().tc_quantize_batch(dt, len(arr), arr, _ptr(workspace), int(workspace_bytes),
                                           _stream(stream)), "tc_quantize_batch")


def tc_quantize_batch_e4m3(jobs, scales, workspace, workspace_bytes, stream=None):
    """E4M3 roundings of many tensors, job j's scale into the device float scales[j] (tensors or
    device addresses)."""
    arr = jobs if isinstance(jobs, ctypes.Array) else quantize_jobs_array(jobs)
    ptrs = (_vp * len(arr))(*[_ptr(x) for x in scales])
    return _check(load().tc_quantize_batch_e4m3(len(arr), arr, ptrs, _ptr(workspace), int(workspace_bytes),
                                                _stream(stream)), "tc_quantize_batch_e4m3")


def tc_autotune_gemm(dt, m, n, k, stream=None):
    """Time gemm_mixed's configurations for this shape; returns the fastest time in ms."""
    ms = ctypes.c_double()
    _check(load().tc_autotune_gemm(dt, m, n, k, _stream(stream), ctypes.byref(ms)), "tc_autotune_gemm")
    return ms.value


def gemm_grouped_plan_autotune(plan, a_base, b_base, c_base, stream=None):
    """Time the plan's variants on its operands and keep the fastest; returns its time in ms."""
    ms = ctypes.c_double()
    _check(load().gemm_grouped_plan_autotune(plan, _ptr(a_base), _ptr(b_base), _ptr(c_base), _stream(stream),
                                             ctypes.byref(ms)), "gemm_grouped_plan_autotune")
    return ms.value


def tc_autotune_save(path):
    return _check(load().tc_autotune_save(str(path).encode()), "tc_autotune_save")


def tc_autotune_load(path):
    return _check(load().tc_autotune_load(str(path).encode()), "tc_autotune_load")


def tc_error_norm(m, n, C, ldc, Cref, ldr, ref_is_f64, A=None, a_rows=0, a_cols=0, lda=0, B=None, b_rows=0,
                  b_cols=0, ldb=0, stream=None):
    out = (ctypes.c_double * 4)()
    _check(load().tc_error_norm(m, n, _ptr(C), ldc, _ptr(Cref), ldr, int(ref_is_f64), _ptr(A), a_rows, a_cols, lda,
                                _ptr(B), b_rows, b_cols, ldb, out, _stream(stream)), "tc_error_norm")
    return tuple(out)


def tc_error_norm_workspace_bytes() -> int:
    return int(load().tc_error_norm_workspace_bytes())


def tc_error_norm_dev(m, n, C, ldc, Cref, ldr, ref_is_f64, A, a_rows, a_cols, lda, B, b_rows, b_cols, ldb, out_dev,
                      workspace, workspace_bytes, stream=None):
    """tc_error_norm into a device array of 4 doubles, enqueued without synchronising."""
    return _check(load().tc_error_norm_dev(m, n, _ptr(C), ldc, _ptr(Cref), ldr, int(ref_is_f64), _ptr(A), a_rows,
                                           a_cols, lda, _ptr(B), b_rows, b_cols, ldb, _ptr(out_dev), _ptr(workspace),
                                           int(workspace_bytes), _stream(stream)), "tc_error_norm_dev")


def serve_open(hbm_budget_bytes, max_inflight=16, num_streams=4, queue_capacity=1 << 16):
    cfg = tc_serve_cfg(int(hbm_budget_bytes), int(max_inflight), int(num_streams), int(queue_capacity), 0)
    srv = _vp()
    _check(load().serve_open(ctypes.byref(cfg), ctypes.byref(srv)), "serve_open")
    return srv.value


def serve_submit(server, mode, m, n, k, A, lda, B, ldb, C, ldc, alpha=1.0, beta=0.0):
    """Returns the ticket, or None when the queue is full (TC_ERR_BUSY)."""
    req = tc_request(int(mode), 0, int(m), int(n), int(k), _ptr(A), int(lda), _ptr(B), int(ldb), _ptr(C), int(ldc),
                     float(alpha), float(beta))
    t = _u64()
    st = load().serve_submit(server, ctypes.byref(req), ctypes.byref(t))
    if st == TC_ERR_BUSY:
        return None
    _check(st, "serve_submit")
    return t.value


def serve_poll(server, ticket):
    """None while pending, else a dict with the request's status and timestamps (microseconds)."""
    res = tc_result()
    st = _check(load().serve_poll(server, int(ticket), ctypes.byref(res)), "serve_poll")
    if st == TC_PENDING:
        return None
    return {"status": res.status, "t_submit_us": res.t_submit_us, "t_start_us": res.t_start_us,
            "t_done_us": res.t_done_us}


def serve_timing(server):
    """Cumulative scheduler time by phase (ns), launch groups, event queries and completed requests."""
    out = (_i64 * 6)()
    _check(load().serve_timing(server, out), "serve_timing")
    keys = ("retire_ns", "admit_ns", "launch_ns", "launch_groups", "event_queries", "completed")
    return dict(zip(keys, (int(v) for v in out)))


def serve_drain(server, timeout_ms=60_000):
    return _check(load().serve_drain(server, int(timeout_ms)), "serve_drain")


def serve_stats(server):
    out = (_i64 * 5)()
    _check(load().serve_stats(server, out), "serve_stats")
    return {"submitted": out[0], "completed": out[1], "peak_bytes": out[2], "peak_inflight": out[3],
            "budget_waits": out[4]}


def serve_close(server):
    return _check(load().serve_close(server), "serve_close")
