"""Seeded synthetic inputs shaped like the passage-retrieval workloads of the
TileMaxSim paper (arxiv 2606.26439, Section 6.1: Nq=32 query tokens, d=128,
L2-normalised token embeddings; variable-length documents packed row-wise).

This module only draws random numbers and lays them out.  It holds none of
the scoring arithmetic: both the CUDA library and the FP64 oracle consume
what it produces, and neither is imported here.

Two back ends produce the same *kind* of data:

* host (numpy ``Generator(PCG64)``) for the small cases the oracle scores
  in full;
* device (``torch.Generator`` on CUDA) for the multi-GB corpora of the
  benchmark, where host generation would take minutes.

Recipe (all seeds explicit):

* token / query embeddings: i.i.d. N(0, 1) per element, divided by the
  row's L2 norm, then cast to the storage dtype (fp16 / bf16 / fp32);
* document lengths: fixed, or uniform integers on [lo, hi] inclusive;
* packing: document i owns rows [offsets[i], offsets[i] + lengths[i]) of a
  [n_tokens][d] array, offsets the exclusive prefix sum of lengths;
* candidate lists: a uniformly random subset drawn without replacement, in
  draw order (unsorted), seeded by (seed, query index);
* PQ corpora: codebook C[M][K][dsub] i.i.d. N(0, 1); each token draws one
  centroid per subspace uniformly, adds N(0, noise^2) per element, and is
  encoded by the nearest centroid in L2 (ties to the lowest index).
"""
from __future__ import annotations

import numpy as np

try:  # torch is optional for the host generators
    import torch
except Exception:  # pragma: no cover
    torch = None


# ---------------------------------------------------------------- host side

def rng(seed, *stream) -> np.random.Generator:
    """Independent numpy generator for (seed, *stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *map(int, stream)])))


def lengths_fixed(n_docs: int, nd: int) -> np.ndarray:
    return np.full(n_docs, nd, np.int32)


def lengths_uniform(n_docs: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Uniform integers on [lo, hi], both ends included."""
    return rng(seed, 1).integers(lo, hi + 1, size=n_docs, dtype=np.int64).astype(np.int32)


def offsets_of(lengths: np.ndarray) -> np.ndarray:
    """Exclusive prefix sum: the first row of each packed document."""
    off = np.zeros(len(lengths), np.int64)
    if len(lengths) > 1:
        np.cumsum(lengths[:-1].astype(np.int64), out=off[1:])
    return off


def unit_rows(n: int, d: int, seed: int, stream: int = 0) -> np.ndarray:
    """n rows of i.i.d. Gaussians divided by their L2 norm (float64)."""
    x = rng(seed, 2, stream).standard_normal((n, d))
    norm = np.sqrt((x * x).sum(axis=1, keepdims=True))
    norm[norm == 0] = 1.0
    return x / norm


def cast(x: np.ndarray, dtype: str):
    """Cast float64 values to the storage dtype as a torch CPU tensor.

    dtype is one of "f16", "bf16", "f32"; rounding is round-to-nearest-even.
    """
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    return t.to({"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[dtype])


def candidates(n_docs: int, n_cand: int, seed: int, query_index: int = 0) -> np.ndarray:
    """n_cand distinct ids from [0, n_docs) in draw order."""
    if n_cand > n_docs:
        raise ValueError("more candidates than documents")
    return rng(seed, 3, query_index).choice(n_docs, size=n_cand, replace=False).astype(np.int32)


def dense_corpus(n_docs: int, lengths: np.ndarray, d: int, dtype: str, seed: int):
    """Packed corpus: (tokens [n_tokens][d] torch CPU tensor, offsets, lengths)."""
    lengths = np.asarray(lengths, np.int32)
    off = offsets_of(lengths)
    n_tok = int(lengths.astype(np.int64).sum())
    return cast(unit_rows(n_tok, d, seed, 1), dtype), off, lengths


def queries(n_queries: int, nq: int, d: int, dtype: str, seed: int):
    """Query tensor [n_queries][nq][d] (torch CPU)."""
    q = unit_rows(n_queries * nq, d, seed, 7).reshape(n_queries, nq, d)
    return cast(q, dtype)


def e4m3_codes(n: int, d: int, seed: int, stream: int = 0) -> np.ndarray:
    """n x d uniformly random finite E4M3 bit patterns (uint8; the two NaN
    patterns 0x7F and 0xFF are never drawn)."""
    c = rng(seed, 14, stream).integers(0, 254, size=(n, d))
    return (c + (c >= 127)).astype(np.uint8)


def row_scales(n: int, seed: int, stream: int = 0, lo: float = 0.5 / 448, hi: float = 2.0 / 448) -> np.ndarray:
    """n fp32 row scales drawn uniformly from [lo, hi)."""
    return rng(seed, 15, stream).uniform(lo, hi, n).astype(np.float32)


def pq_corpus(lengths: np.ndarray, M: int, K: int, dsub: int, seed: int, noise: float = 0.05):
    """PQ corpus on the host: (codebook [M][K][dsub] f32, codes [n_tokens][M] u8,
    reconstructed-from-noise token values [n_tokens][M*dsub] f32, offsets, lengths)."""
    lengths = np.asarray(lengths, np.int32)
    off = offsets_of(lengths)
    n_tok = int(lengths.astype(np.int64).sum())
    g = rng(seed, 4)
    cb = g.standard_normal((M, K, dsub)).astype(np.float32)
    pick = g.integers(0, K, size=(n_tok, M))
    x = cb[np.arange(M)[None, :], pick] + noise * g.standard_normal((n_tok, M, dsub)).astype(np.float32)
    codes = nearest_codes(x, cb)
    return cb, codes, x.reshape(n_tok, M * dsub).astype(np.float32), off, lengths


def nearest_codes(x: np.ndarray, cb: np.ndarray) -> np.ndarray:
    """Encode x[n][M][dsub] by the nearest centroid per subspace (host, float64)."""
    n, M, _ = x.shape
    codes = np.empty((n, M), np.uint8)
    for m in range(M):
        diff = x[:, m, None, :].astype(np.float64) - cb[m][None, :, :].astype(np.float64)
        codes[:, m] = np.argmin((diff * diff).sum(-1), axis=1)
    return codes


# -------------------------------------------------------------- device side

def _tdt(dtype: str):
    return {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[dtype]


def _gen(device, seed, *stream):
    g = torch.Generator(device=device)
    s = int(np.random.SeedSequence([int(seed), *map(int, stream)]).generate_state(1, np.uint64)[0] >> 1)
    g.manual_seed(s)
    return g


def device_unit_rows(n: int, d: int, dtype: str, seed: int, stream: int, device="cuda",
                     chunk_rows: int = 1 << 22, out=None):
    """n unit-norm Gaussian rows generated on the device, in chunks."""
    g = _gen(device, seed, 12, stream)
    if out is None:
        out = torch.empty((n, d), dtype=_tdt(dtype), device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        x = torch.randn((r1 - r0, d), generator=g, device=device, dtype=torch.float32)
        x /= x.norm(dim=1, keepdim=True).clamp_min(1e-30)
        out[r0:r1].copy_(x)
        del x
    return out


def device_dense_corpus(lengths: np.ndarray, d: int, dtype: str, seed: int, device="cuda"):
    """Packed corpus built on the device: (tokens, offsets, lengths) as CUDA tensors."""
    lengths = np.asarray(lengths, np.int32)
    off = offsets_of(lengths)
    n_tok = int(lengths.astype(np.int64).sum())
    tok = device_unit_rows(n_tok, d, dtype, seed, 1, device)
    return (tok, torch.from_numpy(off).to(device), torch.from_numpy(lengths).to(device))


def device_e4m3_store(lengths: np.ndarray, d: int, seed: int, device="cuda", chunk_rows: int = 1 << 22):
    """Packed random E4M3 store built on the device: (codes [n_tokens][d]
    uint8, scales [n_tokens] fp32, offsets, lengths) as CUDA tensors; codes
    uniform over the 254 finite patterns, scales uniform in [0.5, 2] / 448."""
    lengths = np.asarray(lengths, np.int32)
    off = offsets_of(lengths)
    n_tok = int(lengths.astype(np.int64).sum())
    g = _gen(device, seed, 16, 0)
    codes = torch.empty((n_tok, d), dtype=torch.uint8, device=device)
    for r0 in range(0, n_tok, chunk_rows):
        r1 = min(n_tok, r0 + chunk_rows)
        c = torch.randint(0, 254, (r1 - r0, d), generator=g, device=device, dtype=torch.int16)
        c += (c >= 127).to(torch.int16)
        codes[r0:r1].copy_(c)
        del c
    scales = torch.rand(n_tok, generator=g, device=device, dtype=torch.float32) * (1.5 / 448) + 0.5 / 448
    return codes, scales, torch.from_numpy(off).to(device), torch.from_numpy(lengths).to(device)


def device_candidates(n_docs: int, n_cand: int, seed: int, query_index: int, device="cuda"):
    """n_cand distinct ids from [0, n_docs) drawn on the device."""
    g = _gen(device, seed, 13, query_index)
    return torch.randperm(n_docs, generator=g, device=device)[:n_cand].to(torch.int32)


def device_pq_corpus(lengths: np.ndarray, M: int, K: int, dsub: int, seed: int,
                     noise: float = 0.05, device="cuda", chunk_rows: int = 1 << 21):
    """PQ corpus built on the device: (codebook f32 [M][K][dsub], codes u8
    [n_tokens][M], offsets, lengths) -- codes are nearest-centroid encodings."""
    lengths = np.asarray(lengths, np.int32)
    off = offsets_of(lengths)
    n_tok = int(lengths.astype(np.int64).sum())
    g = _gen(device, seed, 14)
    cb = torch.randn((M, K, dsub), generator=g, device=device, dtype=torch.float32)
    codes = torch.empty((n_tok, M), dtype=torch.uint8, device=device)
    cb_sq = (cb * cb).sum(-1)  # [M][K]
    for r0 in range(0, n_tok, chunk_rows):
        r1 = min(n_tok, r0 + chunk_rows)
        pick = torch.randint(0, K, (r1 - r0, M), generator=g, device=device)
        x = cb[torch.arange(M, device=device)[None, :], pick]
        x += noise * torch.randn(x.shape, generator=g, device=device, dtype=torch.float32)
        for m in range(M):
            # argmin_k ||x - c_k||^2 = argmin_k (||c_k||^2 - 2 x.c_k); ties -> first index
            dist = cb_sq[m][None, :] - 2.0 * (x[:, m, :] @ cb[m].T)
            codes[r0:r1, m] = torch.argmin(dist, dim=1).to(torch.uint8)
        del x, pick
    return cb, codes, torch.from_numpy(off).to(device), torch.from_numpy(lengths).to(device)
