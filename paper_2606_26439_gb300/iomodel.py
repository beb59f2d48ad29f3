"""HBM byte and FLOP model of MaxSim scoring (TileMaxSim, arxiv 2606.26439).

These are the paper's analytical formulas, used by the benchmark to turn a
measured time into achieved GB/s and TFLOP/s:

* :func:`flops_paper` -- Section 2.3, Eq. "flops": B Nq Nd (2d + 1).
* :func:`flops_dot`   -- the 2 B Nq Nd d dot-product FLOPs the paper's
  profiling table (Section 6.7) divides by time.
* :func:`io_naive`    -- Section 2.3, Eq. "io_naive": Q, D and a written and
  re-read fp32 similarity matrix.
* :func:`io_fused`    -- Section 2.3, Eq. "io_flash" (output counted as
  B Nq 4 bytes, as the worked example there does).
* :func:`io_theorem1` -- Section 3.4, Theorem 1 (output counted as B 4 bytes,
  as the profiling and batch-scaling tables' GB/s figures do).
* :func:`io_pq_decompress`, :func:`io_pq_fused` -- Section 4.4 IO table.

For packed variable-length documents the build's *algorithmic* byte count
(:func:`dense_alg_bytes`, :func:`pq_alg_bytes`) replaces B Nd by the sum of
candidate lengths and adds the per-candidate metadata that the packed layout
must read: a 4-byte id, an 8-byte offset, a 4-byte length, plus the 4-byte
score written.  Over-fetch, padding and re-reads are not counted.
"""
from __future__ import annotations

import math

META_BYTES_PER_CAND = 4 + 8 + 4  # id, offset, length
SCORE_BYTES = 4


def flops_paper(B, nq, nd, d):
    return B * nq * nd * (2 * d + 1)


def flops_dot(B, nq, nd, d):
    return 2 * B * nq * nd * d


def io_naive(B, nq, nd, d, elem=2):
    return nq * d * elem + B * nd * d * elem + 2 * B * nq * nd * 4


def io_fused(B, nq, nd, d, elem=2):
    return nq * d * elem + B * nd * d * elem + B * nq * 4


def io_theorem1(B, nq, nd, d, bq=None, elem=2):
    bq = nq if bq is None else bq
    return (nq * d + math.ceil(nq / bq) * B * nd * d) * elem + B * 4


def io_pq_decompress(B, nq, nd, d, M, elem=2):
    return B * nd * (M + d * elem) + 2 * B * nq * nd * 4


def io_pq_fused(B, nq, nd, M, K):
    return nq * M * K * 4 + B * nd * M + B * nq * 4


def dense_alg_bytes(total_tokens, n_cand, n_queries, nq, d, elem):
    """Algorithmic HBM bytes of one dense scoring pass over packed documents:
    every candidate token read once, each query read once, metadata read and
    one fp32 score written per candidate."""
    return (total_tokens * d * elem + n_queries * nq * d * elem
            + n_cand * (META_BYTES_PER_CAND + SCORE_BYTES))


def fp8_alg_bytes(total_tokens, n_cand, n_queries, nq, d):
    """Algorithmic HBM bytes of one pass over the FP8 E4M3 store: d one-byte
    codes and one fp32 scale per candidate token, the same per query token,
    metadata read and one fp32 score written per candidate."""
    return (total_tokens * (d + 4) + n_queries * nq * (d + 4)
            + n_cand * (META_BYTES_PER_CAND + SCORE_BYTES))


def quantize_alg_bytes(rows, d, elem):
    """HBM bytes of quantizing rows x d elements of `elem` bytes to E4M3:
    read once, one-byte codes and one fp32 scale per row written."""
    return rows * (d * elem + d + 4)


def dense_alg_flops(total_tokens, nq, d):
    """Dot-product FLOPs of one dense pass: 2 Nq d per (query token, doc token)."""
    return 2 * total_tokens * nq * d


def pq_alg_bytes(total_tokens, n_cand, n_queries, nq, M, K):
    """Algorithmic HBM bytes of one fused PQ pass: codes read once, each
    query's fp32 table read once, metadata read and scores written."""
    return (total_tokens * M + n_queries * nq * M * K * 4
            + n_cand * (META_BYTES_PER_CAND + SCORE_BYTES))


def pq_lut_reads_bytes(total_tokens, nq, M):
    """Shared-memory table bytes one fused PQ pass gathers: Nq M fp32 entries
    per document token."""
    return total_tokens * nq * M * 4
