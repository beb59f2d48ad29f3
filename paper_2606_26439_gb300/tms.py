"""ctypes binding of libtms (C ABI declared in ``include/tms.h``).

Argument marshalling only: every step of the scoring path runs in the CUDA
library.  The raw entry points keep the C names (``tms_score_dense`` and so
on) and take integer device pointers; the thin helpers below take torch
CUDA tensors and pass their ``data_ptr()`` and the current stream.  There
is no CPU fallback -- if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

TMS_OK = 0
TMS_ERR_INVALID_ARG = -1
TMS_ERR_UNSUPPORTED = -2
TMS_ERR_CUDA = -3
TMS_ERR_DEVICE_FLAG = -5
TMS_ERR_TIMEOUT = -6
TMS_ERR_BUSY = -7

TMS_F16, TMS_BF16, TMS_F32 = 0, 1, 2

TMS_DEVERR_BAD_ID = 1
TMS_DEVERR_BAD_RANGE = 2
TMS_DEVERR_TIMEOUT = 4
TMS_DEVERR_BAD_CSR = 8

TMS_FAULT_HOLD_ACCUMULATOR = 1

#: every symbol include/tms.h declares
EXPORTS = ("tms_score_dense", "tms_tune_dense", "tms_score_dense_shared", "tms_tune_dense_shared",
           "tms_quantize_e4m3", "tms_score_fp8", "tms_tune_fp8", "tms_score_fp8_shared", "tms_tune_fp8_shared", "tms_build_pq_lut", "tms_score_pq", "tms_score_pq_f16",
           "tms_score_pq_tc_shared", "tms_topk", "tms_topk_workspace_size", "tms_topk_split", "tms_topk_split_noalloc", "tms_server_create",
           "tms_server_submit", "tms_server_wait", "tms_server_get_stats", "tms_server_destroy", "tms_get_device_error", "tms_debug_set", "tms_status_string",
           "tms_version", "tms_peak_shared_load", "tms_peak_hbm_read")

TMS_STORE_DENSE, TMS_STORE_PQ, TMS_STORE_FP8 = 0, 1, 2


class ServerConfig(ctypes.Structure):
    """Mirror of tms_server_config (include/tms.h)."""
    _fields_ = [
        ("doc_tokens", ctypes.c_void_p), ("dtype", ctypes.c_int), ("d", ctypes.c_int),
        ("n_tokens", ctypes.c_int64), ("doc_offsets", ctypes.c_void_p), ("doc_lengths", ctypes.c_void_p),
        ("n_docs", ctypes.c_int64),
        ("pq_codes", ctypes.c_void_p), ("pq_codebook", ctypes.c_void_p), ("pq_m", ctypes.c_int),
        ("pq_k", ctypes.c_int), ("pq_n_tokens", ctypes.c_int64), ("pq_offsets", ctypes.c_void_p),
        ("pq_lengths", ctypes.c_void_p), ("pq_n_docs", ctypes.c_int64),
        ("fp8_codes", ctypes.c_void_p), ("fp8_scales", ctypes.c_void_p), ("rescore_k", ctypes.c_int),
        ("nq", ctypes.c_int), ("topk", ctypes.c_int), ("max_batch_requests", ctypes.c_int),
        ("max_batch_candidates", ctypes.c_int64), ("max_pending", ctypes.c_int), ("max_pending_bytes", ctypes.c_int64),
        ("inject_error_batch", ctypes.c_int),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("enqueue_s", ctypes.c_double)]

_lib = None
_lock = threading.Lock()

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class TmsError(RuntimeError):
    def __init__(self, name, status):
        self.status = status
        super().__init__(f"{name} failed: {status_string(status)} ({status})")


def lib(build_if_missing: bool = True):
    """Load libtms.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libtms.so is missing and could not be built")
            L = ctypes.CDLL(path)
            L.tms_score_dense.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p]
            L.tms_tune_dense.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p,
                                         ctypes.POINTER(ctypes.c_int)]
            L.tms_score_dense_shared.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _i64, _p, _p]
            L.tms_tune_dense_shared.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _i64, _p, _p,
                                                ctypes.POINTER(ctypes.c_int)]
            L.tms_quantize_e4m3.argtypes = [_p, _i32, _i64, _i32, _p, _p, _p]
            L.tms_score_fp8.argtypes = [_p, _p, _i32, _i32, _i32, _p, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p]
            L.tms_tune_fp8.argtypes = [_p, _p, _i32, _i32, _i32, _p, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p,
                                       ctypes.POINTER(ctypes.c_int)]
            L.tms_score_fp8_shared.argtypes = [_p, _p, _i32, _i32, _i32, _p, _p, _i64, _p, _p, _i64, _p, _i64, _p, _p]
            L.tms_tune_fp8_shared.argtypes = [_p, _p, _i32, _i32, _i32, _p, _p, _i64, _p, _p, _i64, _p, _i64, _p, _p,
                                              ctypes.POINTER(ctypes.c_int)]
            L.tms_build_pq_lut.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i32, _i32, _p, _p]
            L.tms_score_pq.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p]
            L.tms_score_pq_f16.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _p, _i64, _p, _p]
            L.tms_score_pq_tc_shared.argtypes = [_p, _i32, _i32, _i32, _i32, _p, _i32, _i32, _p, _i64, _p, _p, _i64,
                                                 _p, _i64, _p, _p]
            L.tms_topk.argtypes = [_p, _p, _i32, _i32, _p, _p, _p]
            L.tms_topk_workspace_size.argtypes = [_i32, _i32, _i64, ctypes.POINTER(ctypes.c_int64)]
            L.tms_topk_split.argtypes = [_p, _p, _i32, _i32, _i64, _p, _p, _p, _i64, _p]
            L.tms_topk_split_noalloc.argtypes = [_p, _p, _i32, _i32, _i64, _p, _p, _p]
            L.tms_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
            L.tms_server_submit.argtypes = [_p, _i32, _p, _p, _i64, ctypes.POINTER(ctypes.c_uint64)]
            L.tms_server_wait.argtypes = [_p, ctypes.c_uint64, ctypes.c_double, _p, _p,
                                          ctypes.POINTER(ctypes.c_double)]
            L.tms_server_get_stats.argtypes = [_p, ctypes.POINTER(ServerStats)]
            L.tms_server_destroy.argtypes = [_p]
            L.tms_get_device_error.argtypes = [_p, ctypes.POINTER(ctypes.c_int)]
            L.tms_debug_set.argtypes = [_i64, _i32]
            L.tms_peak_shared_load.argtypes = [_i32, _p, ctypes.POINTER(ctypes.c_double)]
            L.tms_peak_hbm_read.argtypes = [_p, _i64, _i32, _p, ctypes.POINTER(ctypes.c_double)]
            L.tms_status_string.argtypes = [_i32]
            L.tms_status_string.restype = ctypes.c_char_p
            L.tms_version.argtypes = []
            for name in ("tms_score_dense", "tms_tune_dense", "tms_score_dense_shared", "tms_tune_dense_shared",
                         "tms_quantize_e4m3", "tms_score_fp8", "tms_tune_fp8", "tms_score_fp8_shared",
                         "tms_tune_fp8_shared", "tms_build_pq_lut", "tms_score_pq", "tms_score_pq_f16",
                         "tms_score_pq_tc_shared", "tms_topk", "tms_topk_workspace_size", "tms_topk_split",
                         "tms_topk_split_noalloc",
                         "tms_server_create", "tms_server_submit", "tms_server_wait", "tms_server_get_stats",
                         "tms_server_destroy", "tms_get_device_error", "tms_debug_set", "tms_version",
                         "tms_peak_shared_load", "tms_peak_hbm_read"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().tms_status_string(int(status)).decode()


def _check(name, status):
    if status != TMS_OK:
        raise TmsError(name, status)


# ------------------------------------------------------------ raw C ABI

def tms_score_dense(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths,
                    n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream) -> int:
    return lib().tms_score_dense(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets,
                                 doc_lengths, n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream)


def tms_score_dense_shared(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths,
                           n_docs, cand_ids, n_cand, out_scores, stream) -> int:
    return lib().tms_score_dense_shared(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets,
                                        doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream)


def tms_quantize_e4m3(x, dtype, rows, d, codes, scales, stream) -> int:
    return lib().tms_quantize_e4m3(x, dtype, rows, d, codes, scales, stream)


def tms_score_fp8(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets, doc_lengths,
                  n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream) -> int:
    return lib().tms_score_fp8(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                               doc_lengths, n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream)


def tms_score_fp8_shared(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                         doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream) -> int:
    return lib().tms_score_fp8_shared(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens,
                                      doc_offsets, doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream)


def tms_build_pq_lut(queries, qdtype, n_queries, nq, d, codebook, m, k, lut, stream) -> int:
    return lib().tms_build_pq_lut(queries, qdtype, n_queries, nq, d, codebook, m, k, lut, stream)


def tms_score_pq(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs,
                 cand_ids, cand_offsets, n_cand, out_scores, stream) -> int:
    return lib().tms_score_pq(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs,
                              cand_ids, cand_offsets, n_cand, out_scores, stream)


def tms_score_pq_f16(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs,
                     cand_ids, cand_offsets, n_cand, out_scores, stream) -> int:
    return lib().tms_score_pq_f16(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs,
                                  cand_ids, cand_offsets, n_cand, out_scores, stream)


def tms_score_pq_tc_shared(queries, qdtype, n_queries, nq, d, codebook, m, k, codes, n_tokens, doc_offsets,
                           doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream) -> int:
    return lib().tms_score_pq_tc_shared(queries, qdtype, n_queries, nq, d, codebook, m, k, codes, n_tokens,
                                        doc_offsets, doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream)


def tms_topk(scores, cand_offsets, n_queries, topk, out_scores, out_pos, stream) -> int:
    return lib().tms_topk(scores, cand_offsets, n_queries, topk, out_scores, out_pos, stream)


def tms_get_device_error(stream=None):
    """(status, flags) after draining ``stream``; clears the error word."""
    flags = ctypes.c_int(0)
    st = lib().tms_get_device_error(stream, ctypes.byref(flags))
    return st, flags.value


def tms_debug_set(wait_budget_cycles: int, fault: int) -> int:
    return lib().tms_debug_set(int(wait_budget_cycles), int(fault))


def peak_shared_load(iters=20000, stream=None) -> float:
    """Measured shared-memory load bandwidth of the device, GB/s (all SMs)."""
    g = ctypes.c_double()
    _check("tms_peak_shared_load", lib().tms_peak_shared_load(int(iters), _stream_ptr(stream), ctypes.byref(g)))
    return g.value


def peak_hbm_read(buf, reps=5, stream=None) -> float:
    """Measured HBM streaming-read bandwidth over the device tensor ``buf``, GB/s."""
    g = ctypes.c_double()
    nbytes = buf.numel() * buf.element_size()
    _check("tms_peak_hbm_read", lib().tms_peak_hbm_read(_dev(buf), nbytes - nbytes % 16, int(reps),
                                                        _stream_ptr(stream), ctypes.byref(g)))
    return g.value


def tms_version() -> int:
    return lib().tms_version()


# ------------------------------------------------- torch tensor helpers

def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    return {torch.float16: TMS_F16, torch.bfloat16: TMS_BF16, torch.float32: TMS_F32}[t.dtype]


def _stream_ptr(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dev(t, dtype=None):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def score_dense(queries, doc_tokens, doc_offsets, doc_lengths, cand_ids, cand_offsets, out=None,
                stream=None):
    """Dense MaxSim.  queries [n_queries][nq][d]; doc_tokens [n_tokens][d];
    cand_offsets int64 [n_queries + 1] (CUDA).  Returns out [n_cand] fp32."""
    torch = _torch()
    nQ, nq, d = queries.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty(n_cand, dtype=torch.float32, device=queries.device)
    _check("tms_score_dense", tms_score_dense(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(doc_tokens, queries.dtype), doc_tokens.shape[0],
        _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32), doc_offsets.shape[0],
        _dev(cand_ids, torch.int32), _dev(cand_offsets, torch.int64), n_cand, _dev(out, torch.float32),
        _stream_ptr(stream)))
    return out


def tune_dense(queries, doc_tokens, doc_offsets, doc_lengths, cand_ids, cand_offsets, out=None, stream=None):
    """tms_tune_dense: score_dense after timing the launch configurations;
    returns (scores, number of configurations timed)."""
    torch = _torch()
    nQ, nq, d = queries.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty(n_cand, dtype=torch.float32, device=queries.device)
    n = ctypes.c_int(0)
    _check("tms_tune_dense", lib().tms_tune_dense(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(doc_tokens, queries.dtype), doc_tokens.shape[0],
        _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32), doc_offsets.shape[0],
        _dev(cand_ids, torch.int32), _dev(cand_offsets, torch.int64), n_cand, _dev(out, torch.float32),
        _stream_ptr(stream), ctypes.byref(n)))
    return out, n.value


def score_dense_shared(queries, doc_tokens, doc_offsets, doc_lengths, cand_ids, out=None, stream=None):
    """Dense MaxSim of every query over ONE candidate list; out [n_queries][n_cand]."""
    torch = _torch()
    nQ, nq, d = queries.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty((nQ, n_cand), dtype=torch.float32, device=queries.device)
    _check("tms_score_dense_shared", tms_score_dense_shared(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(doc_tokens, queries.dtype), doc_tokens.shape[0],
        _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32), doc_offsets.shape[0],
        _dev(cand_ids, torch.int32), n_cand, _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def tune_dense_shared(queries, doc_tokens, doc_offsets, doc_lengths, cand_ids, out=None, stream=None):
    """tms_tune_dense_shared: score_dense_shared after timing the group sizes
    and launch configurations; returns (scores, configurations timed)."""
    torch = _torch()
    nQ, nq, d = queries.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty((nQ, n_cand), dtype=torch.float32, device=queries.device)
    n = ctypes.c_int(0)
    _check("tms_tune_dense_shared", lib().tms_tune_dense_shared(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(doc_tokens, queries.dtype), doc_tokens.shape[0],
        _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32), doc_offsets.shape[0],
        _dev(cand_ids, torch.int32), n_cand, _dev(out, torch.float32), _stream_ptr(stream), ctypes.byref(n)))
    return out, n.value


def quantize_e4m3(x, codes=None, scales=None, stream=None):
    """Per-row E4M3 codes (uint8, x's shape) and fp32 scales (x.shape[:-1])
    of a CUDA tensor x [..., d] (fp16 / bf16 / fp32)."""
    torch = _torch()
    d = x.shape[-1]
    rows = x.numel() // d if d else 0
    if codes is None:
        codes = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    if scales is None:
        scales = torch.empty(x.shape[:-1], dtype=torch.float32, device=x.device)
    _check("tms_quantize_e4m3", tms_quantize_e4m3(_dev(x), _dtype_code(x), rows, d, _dev(codes, torch.uint8),
                                                  _dev(scales, torch.float32), _stream_ptr(stream)))
    return codes, scales


def score_fp8(q_codes, q_scales, doc_codes, doc_scales, doc_offsets, doc_lengths, cand_ids, cand_offsets,
              out=None, stream=None):
    """MaxSim on the FP8 store.  q_codes [n_queries][nq][d] uint8, q_scales
    [n_queries][nq]; doc_codes [n_tokens][d] uint8, doc_scales [n_tokens]."""
    torch = _torch()
    nQ, nq, d = q_codes.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty(n_cand, dtype=torch.float32, device=q_codes.device)
    _check("tms_score_fp8", tms_score_fp8(
        _dev(q_codes, torch.uint8), _dev(q_scales, torch.float32), nQ, nq, d, _dev(doc_codes, torch.uint8),
        _dev(doc_scales, torch.float32), doc_codes.shape[0], _dev(doc_offsets, torch.int64),
        _dev(doc_lengths, torch.int32), doc_offsets.shape[0], _dev(cand_ids, torch.int32),
        _dev(cand_offsets, torch.int64), n_cand, _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def tune_fp8(q_codes, q_scales, doc_codes, doc_scales, doc_offsets, doc_lengths, cand_ids, cand_offsets,
             out=None, stream=None):
    """tms_tune_fp8: score_fp8 after timing the launch configurations;
    returns (scores, configurations timed)."""
    torch = _torch()
    nQ, nq, d = q_codes.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty(n_cand, dtype=torch.float32, device=q_codes.device)
    n = ctypes.c_int(0)
    _check("tms_tune_fp8", lib().tms_tune_fp8(
        _dev(q_codes, torch.uint8), _dev(q_scales, torch.float32), nQ, nq, d, _dev(doc_codes, torch.uint8),
        _dev(doc_scales, torch.float32), doc_codes.shape[0], _dev(doc_offsets, torch.int64),
        _dev(doc_lengths, torch.int32), doc_offsets.shape[0], _dev(cand_ids, torch.int32),
        _dev(cand_offsets, torch.int64), n_cand, _dev(out, torch.float32), _stream_ptr(stream), ctypes.byref(n)))
    return out, n.value


def tune_fp8_shared(q_codes, q_scales, doc_codes, doc_scales, doc_offsets, doc_lengths, cand_ids, out=None,
                    stream=None):
    """tms_tune_fp8_shared: score_fp8_shared after timing the group sizes and
    launch configurations; returns (scores, configurations timed)."""
    torch = _torch()
    nQ, nq, d = q_codes.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty((nQ, n_cand), dtype=torch.float32, device=q_codes.device)
    n = ctypes.c_int(0)
    _check("tms_tune_fp8_shared", lib().tms_tune_fp8_shared(
        _dev(q_codes, torch.uint8), _dev(q_scales, torch.float32), nQ, nq, d, _dev(doc_codes, torch.uint8),
        _dev(doc_scales, torch.float32), doc_codes.shape[0], _dev(doc_offsets, torch.int64),
        _dev(doc_lengths, torch.int32), doc_offsets.shape[0], _dev(cand_ids, torch.int32), n_cand,
        _dev(out, torch.float32), _stream_ptr(stream), ctypes.byref(n)))
    return out, n.value


def score_fp8_shared(q_codes, q_scales, doc_codes, doc_scales, doc_offsets, doc_lengths, cand_ids, out=None,
                     stream=None):
    """score_fp8 of every query over ONE candidate list; out [n_queries][n_cand]."""
    torch = _torch()
    nQ, nq, d = q_codes.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty((nQ, n_cand), dtype=torch.float32, device=q_codes.device)
    _check("tms_score_fp8_shared", tms_score_fp8_shared(
        _dev(q_codes, torch.uint8), _dev(q_scales, torch.float32), nQ, nq, d, _dev(doc_codes, torch.uint8),
        _dev(doc_scales, torch.float32), doc_codes.shape[0], _dev(doc_offsets, torch.int64),
        _dev(doc_lengths, torch.int32), doc_offsets.shape[0], _dev(cand_ids, torch.int32), n_cand,
        _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def build_pq_lut(queries, codebook, out=None, stream=None):
    """PQ table [n_queries][nq][m][k] fp32 from queries [n_queries][nq][d]."""
    torch = _torch()
    nQ, nq, d = queries.shape
    m, k, _ = codebook.shape
    if out is None:
        out = torch.empty((nQ, nq, m, k), dtype=torch.float32, device=queries.device)
    _check("tms_build_pq_lut", tms_build_pq_lut(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(codebook, torch.float32), m, k,
        _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def score_pq(lut, codes, doc_offsets, doc_lengths, cand_ids, cand_offsets, out=None, stream=None,
             f16_table=False):
    """Fused PQ MaxSim from a table [n_queries][nq][m][k] and codes [n_tokens][m].

    ``f16_table=True`` scores through the table rounded to fp16
    (tms_score_pq_f16)."""
    torch = _torch()
    nQ, nq, m, k = lut.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty(n_cand, dtype=torch.float32, device=lut.device)
    fn, name = (tms_score_pq_f16, "tms_score_pq_f16") if f16_table else (tms_score_pq, "tms_score_pq")
    _check(name, fn(
        _dev(lut, torch.float32), nQ, nq, m, k, _dev(codes, torch.uint8), codes.shape[0],
        _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32), doc_offsets.shape[0],
        _dev(cand_ids, torch.int32), _dev(cand_offsets, torch.int64), n_cand, _dev(out, torch.float32),
        _stream_ptr(stream)))
    return out


def score_pq_tc_shared(queries, codebook, codes, doc_offsets, doc_lengths, cand_ids, out=None, stream=None):
    """PQ MaxSim of queries [n_queries][nq][d] (fp16) sharing one candidate
    list, codes decompressed in shared memory and scored on the tensor cores:
    [n_queries][n_cand] fp32."""
    torch = _torch()
    nQ, nq, d = queries.shape
    m, k, _ = codebook.shape
    n_cand = cand_ids.shape[0]
    if out is None:
        out = torch.empty((nQ, n_cand), dtype=torch.float32, device=queries.device)
    _check("tms_score_pq_tc_shared", tms_score_pq_tc_shared(
        _dev(queries), _dtype_code(queries), nQ, nq, d, _dev(codebook, torch.float32), m, k,
        _dev(codes, torch.uint8), codes.shape[0], _dev(doc_offsets, torch.int64), _dev(doc_lengths, torch.int32),
        doc_offsets.shape[0], _dev(cand_ids, torch.int32), n_cand, _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def topk(scores, cand_offsets, k, out_scores=None, out_pos=None, stream=None):
    """Per-query top-k: ([n_queries][k] fp32 scores, [n_queries][k] int32 positions)."""
    torch = _torch()
    nQ = cand_offsets.shape[0] - 1
    if out_scores is None:
        out_scores = torch.empty((nQ, k), dtype=torch.float32, device=scores.device)
    if out_pos is None:
        out_pos = torch.empty((nQ, k), dtype=torch.int32, device=scores.device)
    _check("tms_topk", tms_topk(_dev(scores, torch.float32), _dev(cand_offsets, torch.int64), nQ, k,
                                _dev(out_scores, torch.float32), _dev(out_pos, torch.int32),
                                _stream_ptr(stream)))
    return out_scores, out_pos


def topk_workspace_size(n_queries, k, n_cand) -> int:
    """Bytes of device workspace tms_topk_split needs on the current device."""
    b = ctypes.c_int64()
    _check("tms_topk_workspace_size", lib().tms_topk_workspace_size(int(n_queries), int(k), int(n_cand),
                                                                    ctypes.byref(b)))
    return b.value


def topk_split(scores, cand_offsets, k, n_cand=None, out_scores=None, out_pos=None, workspace=None, stream=None):
    """tms_topk over slices of every list (same result as topk).  ``n_cand``:
    the host value of cand_offsets[-1] (default: the length of ``scores``);
    ``workspace``: a device tensor of at least topk_workspace_size bytes
    (allocated here when None)."""
    torch = _torch()
    nQ = cand_offsets.shape[0] - 1
    n_cand = scores.numel() if n_cand is None else int(n_cand)
    if out_scores is None:
        out_scores = torch.empty((nQ, k), dtype=torch.float32, device=scores.device)
    if out_pos is None:
        out_pos = torch.empty((nQ, k), dtype=torch.int32, device=scores.device)
    if workspace is None:
        workspace = torch.empty(max(16, topk_workspace_size(nQ, k, n_cand)), dtype=torch.uint8, device=scores.device)
    nbytes = workspace.numel() * workspace.element_size()
    _check("tms_topk_split", lib().tms_topk_split(_dev(scores, torch.float32), _dev(cand_offsets, torch.int64), nQ, k,
                                                  n_cand, _dev(out_scores, torch.float32), _dev(out_pos, torch.int32),
                                                  _dev(workspace), nbytes, _stream_ptr(stream)))
    return out_scores, out_pos


def topk_split_noalloc(scores, cand_offsets, k, n_cand=None, out_scores=None, out_pos=None, stream=None):
    """tms_topk_split with its scratch in the library's fixed device array
    (no workspace, no device allocation by the library; the output tensors
    are allocated here only when not given)."""
    torch = _torch()
    nQ = cand_offsets.shape[0] - 1
    n_cand = scores.numel() if n_cand is None else int(n_cand)
    if out_scores is None:
        out_scores = torch.empty((nQ, k), dtype=torch.float32, device=scores.device)
    if out_pos is None:
        out_pos = torch.empty((nQ, k), dtype=torch.int32, device=scores.device)
    _check("tms_topk_split_noalloc",
           lib().tms_topk_split_noalloc(_dev(scores, torch.float32), _dev(cand_offsets, torch.int64), nQ, k, n_cand,
                                        _dev(out_scores, torch.float32), _dev(out_pos, torch.int32),
                                        _stream_ptr(stream)))
    return out_scores, out_pos


def device_error(stream=None) -> int:
    """TMS_DEVERR_* flags raised since the last call (synchronises ``stream``)."""
    st, flags = tms_get_device_error(_stream_ptr(stream))
    if st not in (TMS_OK, TMS_ERR_DEVICE_FLAG):
        raise TmsError("tms_get_device_error", st)
    return flags


# --------------------------------------------------------------- serving

class Server:
    """Serving loop over a device-resident dense store (and optional PQ store
    and FP8 copy of the dense store): submit requests from the host, wait for
    their top-k.  The config's device tensors must outlive the server.

    ``pq``: (codes, codebook, offsets, lengths); ``fp8``: (codes, scales) of
    the dense store's tokens (quantize_e4m3), scored with an fp16 re-score
    of each request's ``rescore_k`` best candidates (0: FP8 scores)."""

    def __init__(self, doc_tokens, doc_offsets, doc_lengths, nq, topk, max_batch_requests,
                 max_batch_candidates, max_pending, pq=None, inject_error_batch=0, fp8=None, rescore_k=0,
                 max_pending_bytes=0):
        torch = _torch()
        cfg = ServerConfig()
        cfg.doc_tokens = _dev(doc_tokens)
        cfg.dtype = _dtype_code(doc_tokens)
        cfg.d = doc_tokens.shape[1]
        cfg.n_tokens = doc_tokens.shape[0]
        cfg.doc_offsets = _dev(doc_offsets, torch.int64)
        cfg.doc_lengths = _dev(doc_lengths, torch.int32)
        cfg.n_docs = doc_offsets.shape[0]
        if pq is not None:
            codes, codebook, offsets, lengths = pq
            cfg.pq_codes = _dev(codes, torch.uint8)
            cfg.pq_codebook = _dev(codebook, torch.float32)
            cfg.pq_m, cfg.pq_k = codebook.shape[0], codebook.shape[1]
            cfg.pq_n_tokens = codes.shape[0]
            cfg.pq_offsets = _dev(offsets, torch.int64)
            cfg.pq_lengths = _dev(lengths, torch.int32)
            cfg.pq_n_docs = offsets.shape[0]
        if fp8 is not None:
            codes, scales = fp8
            cfg.fp8_codes = _dev(codes, torch.uint8)
            cfg.fp8_scales = _dev(scales, torch.float32)
        cfg.rescore_k = rescore_k
        cfg.nq, cfg.topk = nq, topk
        cfg.max_batch_requests = max_batch_requests
        cfg.max_batch_candidates = max_batch_candidates
        cfg.max_pending = max_pending
        cfg.max_pending_bytes = max_pending_bytes
        cfg.inject_error_batch = inject_error_batch
        self.topk = topk
        self.qshape = (nq, cfg.d)
        self.qdtype = doc_tokens.dtype
        h = ctypes.c_void_p()
        _check("tms_server_create", lib().tms_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, query, cand_ids, store=TMS_STORE_DENSE):
        """query: host tensor [nq][d] of the store dtype; cand_ids: int32 numpy array."""
        import numpy as np
        q = query.contiguous()
        if tuple(q.shape) != self.qshape or q.dtype != self.qdtype or q.is_cuda:
            raise ValueError("query must be a host tensor of the store's dtype and shape [nq][d]")
        c = np.ascontiguousarray(cand_ids, dtype=np.int32)
        t = ctypes.c_uint64()
        _check("tms_server_submit", lib().tms_server_submit(self._h, store, q.data_ptr(), c.ctypes.data,
                                                            c.shape[0], ctypes.byref(t)))
        return t.value

    def wait(self, ticket, timeout_s=60.0):
        """(scores [topk] fp32, ids [topk] int32, latency seconds); raises TmsError on failure."""
        import numpy as np
        sc = np.empty(self.topk, np.float32)
        ids = np.empty(self.topk, np.int32)
        lat = ctypes.c_double()
        _check("tms_server_wait", lib().tms_server_wait(self._h, ticket, timeout_s, sc.ctypes.data, ids.ctypes.data,
                                                        ctypes.byref(lat)))
        return sc, ids, lat.value

    def stats(self):
        st = ServerStats()
        _check("tms_server_get_stats", lib().tms_server_get_stats(self._h, ctypes.byref(st)))
        return {"requests": st.requests, "batches": st.batches, "candidates": st.candidates,
                "rejected": st.rejected, "enqueue_s": st.enqueue_s}

    def close(self):
        if getattr(self, "_h", None):
            _check("tms_server_destroy", lib().tms_server_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
