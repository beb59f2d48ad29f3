"""FP64 CPU oracle for MaxSim / PQ-MaxSim / top-k (TileMaxSim, arxiv 2606.26439).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never calls it.

The arithmetic lives in ``maxsim_oracle.c``; this module only marshals numpy
arrays into it.  Each function names the definition it follows:

* :func:`dense_scores`       -- Eq. 1 (Section 2.1), MaxSim.
* :func:`pq_decompress_scores` -- Section 4.1, decompress then Eq. 1.
* :func:`pq_lut`             -- Section 4.2, the distance table T.
* :func:`pq_lut_scores`      -- Section 4.2 Phase 2, sum of table entries.
* :func:`topk`               -- Section 6.8, top-k after scoring.

Element types are passed as the stored bits: fp16 and bf16 arrays are
given as ``uint16`` bit patterns with an explicit dtype code, fp32 as ``float32``, and
fp64 as ``float64``.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

F16, BF16, F32, F64, E4M3 = 0, 1, 2, 3, 4

_lib = None
_lock = threading.Lock()

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build.build())
            lib.tmso_f16_to_f64.restype = ctypes.c_double
            lib.tmso_f16_to_f64.argtypes = [ctypes.c_uint16]
            lib.tmso_bf16_to_f64.restype = ctypes.c_double
            lib.tmso_bf16_to_f64.argtypes = [ctypes.c_uint16]
            lib.tmso_e4m3_to_f64.restype = ctypes.c_double
            lib.tmso_e4m3_to_f64.argtypes = [ctypes.c_uint8]
            lib.tmso_dense_scores_scaled.argtypes = [
                _p, _i32, _p, _i32, _i32, _p, _i32, _p, _i64, _p, _p, _i64, _p, _i64, _p]
            lib.tmso_dense_scores_scaled.restype = ctypes.c_int
            lib.tmso_e4m3_encode.argtypes = [ctypes.c_float]
            lib.tmso_e4m3_encode.restype = ctypes.c_uint8
            lib.tmso_quantize_e4m3.argtypes = [_p, _i32, _i64, _i32, _p, _p]
            lib.tmso_quantize_e4m3.restype = ctypes.c_int
            lib.tmso_max_threads.restype = ctypes.c_int
            lib.tmso_set_threads.argtypes = [ctypes.c_int]
            lib.tmso_dense_scores.argtypes = [
                _p, _i32, _i32, _i32, _p, _i32, _i64, _p, _p, _i64, _p, _i64, _p]
            lib.tmso_pq_decompress_scores.argtypes = [
                _p, _i32, _i32, _i32, _p, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _i64, _p]
            lib.tmso_pq_lut.argtypes = [_p, _i32, _i32, _i32, _p, _i32, _i32, _p]
            lib.tmso_pq_lut_scores.argtypes = [
                _p, _i32, _i32, _i32, _i32, _p, _i64, _p, _p, _i64, _p, _i64, _p]
            lib.tmso_topk.argtypes = [_p, _i64, _i32, _p, _p]
            for name in ("tmso_dense_scores", "tmso_pq_decompress_scores", "tmso_pq_lut",
                         "tmso_pq_lut_scores", "tmso_topk"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _typed(a: np.ndarray, dtype_code: int | None = None):
    """Return (contiguous array, oracle dtype code) for a stored-value array."""
    a = np.ascontiguousarray(a)
    if dtype_code is not None:
        return a, dtype_code
    if a.dtype == np.float16:
        return a.view(np.uint16), F16
    if a.dtype == np.float32:
        return a, F32
    if a.dtype == np.float64:
        return a, F64
    raise TypeError(f"pass uint16 bits with an explicit dtype code, not {a.dtype}")


def set_threads(n: int) -> None:
    _load().tmso_set_threads(int(n))


def max_threads() -> int:
    return int(_load().tmso_max_threads())


def f16_to_f64(bits: int) -> float:
    return float(_load().tmso_f16_to_f64(int(bits)))


def bf16_to_f64(bits: int) -> float:
    return float(_load().tmso_bf16_to_f64(int(bits)))


def e4m3_to_f64(bits: int) -> float:
    return float(_load().tmso_e4m3_to_f64(int(bits)))


def e4m3_encode(v: float) -> int:
    return int(_load().tmso_e4m3_encode(float(v)))


def quantize_e4m3(x, *, dtype=None):
    """Per-row E4M3 codes [rows][d] (uint8) and fp32 scales [rows]."""
    a, dt = _typed(x, dtype)
    rows, d = a.shape
    codes = np.empty((rows, d), np.uint8)
    scales = np.empty(rows, np.float32)
    if _load().tmso_quantize_e4m3(_ptr(a), dt, rows, d, _ptr(codes), _ptr(scales)):
        raise ValueError("oracle quantize_e4m3 rejected its arguments")
    return codes, scales


def dense_scores_scaled(queries, q_scales, tokens, t_scales, offsets, lengths, cand_ids, *,
                        qdtype=None, tdtype=None):
    """Eq. 1 on row-scaled stored values (a per-token scaled store, e.g. FP8
    E4M3 codes given as uint8 with dtype code E4M3); None scales mean 1."""
    q, qdt = _typed(queries, qdtype)
    t, tdt = _typed(tokens, tdtype)
    nq, d = q.shape
    qs = None if q_scales is None else _c(q_scales, np.float32)
    ts = None if t_scales is None else _c(t_scales, np.float32)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    cid = _c(cand_ids, np.int32)
    out = np.empty(cid.shape[0], np.float64)
    rc = _load().tmso_dense_scores_scaled(_ptr(q), qdt, None if qs is None else _ptr(qs), nq, d,
                                          _ptr(t), tdt, None if ts is None else _ptr(ts), t.shape[0],
                                          _ptr(off), _ptr(ln), off.shape[0], _ptr(cid), cid.shape[0], _ptr(out))
    if rc:
        raise ValueError("oracle dense_scores_scaled rejected its arguments")
    return out


def dense_scores(queries, tokens, offsets, lengths, cand_ids, *, qdtype=None, tdtype=None):
    """Eq. 1 for one query ``queries[nq][d]`` over ``cand_ids``."""
    q, qdt = _typed(queries, qdtype)
    t, tdt = _typed(tokens, tdtype)
    nq, d = q.shape
    assert t.ndim == 2 and t.shape[1] == d
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    cid = _c(cand_ids, np.int32)
    out = np.empty(cid.shape[0], np.float64)
    rc = _load().tmso_dense_scores(_ptr(q), qdt, nq, d, _ptr(t), tdt, t.shape[0],
                                   _ptr(off), _ptr(ln), off.shape[0],
                                   _ptr(cid), cid.shape[0], _ptr(out))
    if rc:
        raise ValueError("oracle dense_scores rejected its arguments")
    return out


def pq_decompress_scores(queries, codebook, codes, offsets, lengths, cand_ids, *, qdtype=None):
    """Section 4.1: rebuild each token from its centroids, then Eq. 1."""
    q, qdt = _typed(queries, qdtype)
    nq, d = q.shape
    cb = _c(codebook, np.float32)
    M, K, _ = cb.shape
    cd = _c(codes, np.uint8)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    cid = _c(cand_ids, np.int32)
    out = np.empty(cid.shape[0], np.float64)
    rc = _load().tmso_pq_decompress_scores(_ptr(q), qdt, nq, d, _ptr(cb), M, K,
                                           _ptr(cd), cd.shape[0], _ptr(off), _ptr(ln),
                                           off.shape[0], _ptr(cid), cid.shape[0], _ptr(out))
    if rc:
        raise ValueError("oracle pq_decompress_scores rejected its arguments")
    return out


def pq_lut(queries, codebook, *, qdtype=None):
    """Section 4.2: T[i][m][k] in double, shape [nq][M][K]."""
    q, qdt = _typed(queries, qdtype)
    nq, d = q.shape
    cb = _c(codebook, np.float32)
    M, K, _ = cb.shape
    lut = np.empty((nq, M, K), np.float64)
    rc = _load().tmso_pq_lut(_ptr(q), qdt, nq, d, _ptr(cb), M, K, _ptr(lut))
    if rc:
        raise ValueError("oracle pq_lut rejected its arguments")
    return lut


def pq_lut_scores(lut, codes, offsets, lengths, cand_ids):
    """Section 4.2 Phase 2 with a given table ``lut[nq][M][K]`` (fp16, fp32 or
    fp64; every entry read exactly, sums in double)."""
    lt = np.ascontiguousarray(lut)
    if lt.dtype == np.float16:
        ltype = F16
    elif lt.dtype == np.float32:
        ltype = F32
    else:
        lt = lt.astype(np.float64, copy=False)
        ltype = F64
    nq, M, K = lt.shape
    cd = _c(codes, np.uint8)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    cid = _c(cand_ids, np.int32)
    out = np.empty(cid.shape[0], np.float64)
    rc = _load().tmso_pq_lut_scores(_ptr(lt), ltype, nq, M, K, _ptr(cd), cd.shape[0],
                                    _ptr(off), _ptr(ln), off.shape[0],
                                    _ptr(cid), cid.shape[0], _ptr(out))
    if rc:
        raise ValueError("oracle pq_lut_scores rejected its arguments")
    return out


def topk(scores, k: int):
    """Top-k by (score desc, position asc), NaN last, padded with (-inf, -1)."""
    s = _c(scores, np.float64)
    out_s = np.empty(max(k, 0), np.float64)
    out_p = np.empty(max(k, 0), np.int64)
    rc = _load().tmso_topk(_ptr(s), s.shape[0], int(k), _ptr(out_s), _ptr(out_p))
    if rc:
        raise ValueError("oracle topk rejected its arguments")
    return out_s, out_p
