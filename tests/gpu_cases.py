"""Shared builders for the GPU parity tests: seeded inputs from ``synth``,
the CUDA path through the C ABI, the oracle on the same stored values."""
from __future__ import annotations

import numpy as np

import oracle
import synth
from tests._common import oracle_view

EDGE_LENGTHS = [0, 1, 7, 8, 31, 32, 33, 127, 128, 129, 180, 255, 256, 257, 513]


def csr(cands):
    co = np.zeros(len(cands) + 1, np.int64)
    co[1:] = np.cumsum([len(c) for c in cands])
    flat = np.concatenate([np.asarray(c, np.int32) for c in cands]) if co[-1] else np.zeros(0, np.int32)
    return flat, co


def to_dev(*arrays):
    import torch
    out = []
    for a in arrays:
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        out.append(t.contiguous().cuda())
    return out


def gpu_dense(Q, tok, off, ln, cands):
    """Run tms_score_dense on the device; returns (scores numpy, error flags)."""
    import torch
    from paper_2606_26439_gb300 import tms
    flat, co = csr(cands)
    q_d, t_d, o_d, l_d, f_d, c_d = to_dev(Q, tok, off, ln, flat, co)
    out = torch.full((len(flat),), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_dense(q_d, t_d, o_d, l_d, f_d, c_d, out=out)
    torch.cuda.synchronize()
    flags = tms.device_error()
    return out.cpu().numpy(), flags


def oracle_dense_multi(Q, tok, off, ln, cands):
    qa, qdt = oracle_view(Q)
    ta, tdt = oracle_view(tok)
    res = [oracle.dense_scores(qa[i], ta, off, ln, c, qdtype=qdt, tdtype=tdt) for i, c in enumerate(cands)]
    return np.concatenate(res) if res else np.zeros(0)


def edge_corpus(d, dtype, seed, n_random=160):
    """Edge lengths + random U[1, 200] lengths; the last document is long so
    its row range ends exactly at the end of the token array."""
    g = np.random.default_rng(seed)
    lengths = np.array(EDGE_LENGTHS + list(g.integers(1, 201, n_random)) + [129], np.int32)
    n_docs = len(lengths)
    tok, off, ln = synth.dense_corpus(n_docs, lengths, d, dtype, seed)
    return tok, off, ln


def edge_candidates(n_docs, n_queries, seed):
    """Query 0: every document in shuffled order, duplicates and bad ids;
    further queries: random subsets (one empty list included)."""
    g = np.random.default_rng(seed + 99)
    c0 = list(g.permutation(n_docs)) + [0, 0, n_docs - 1]
    # bad ids scattered through the list, not only at its end
    for bad in (-1, -2, n_docs, 2 ** 31 - 1, -(2 ** 31)):
        c0.insert(int(g.integers(0, len(c0) + 1)), bad)
    cands = [np.array(c0, np.int32)]
    for qi in range(1, n_queries):
        n = 0 if qi == 2 else int(g.integers(1, n_docs))
        cands.append(synth.candidates(n_docs, n, seed, qi))
    return cands


def rows_of(off, lengths, ids):
    """Token rows of documents ``ids`` in order, as one index array."""
    lens = np.asarray(lengths, np.int64)[ids]
    starts = np.asarray(off, np.int64)[ids]
    if lens.sum() == 0:
        return np.zeros(0, np.int64)
    before = np.concatenate([[0], np.cumsum(lens)[:-1]])
    return np.repeat(starts - before, lens) + np.arange(int(lens.sum()), dtype=np.int64)


def gather_docs(rows_d, off, lengths, ids):
    """Host copy of the rows of documents ``ids`` of a device array, repacked
    (offsets, lengths) for the oracle.  ``ids`` = every document in order
    copies the array as it is."""
    import torch
    lens = np.asarray(lengths, np.int32)[ids]
    if len(ids) == len(lengths) and np.array_equal(ids, np.arange(len(lengths))):
        return rows_d.cpu(), np.asarray(off, np.int64), lens
    idx = torch.from_numpy(rows_of(off, lengths, ids)).to(rows_d.device)
    return rows_d[idx].cpu(), synth.offsets_of(lens), lens


def oracle_dense_list(q, tok_d, off, lengths, ids):
    """FP64 Eq. 1 of one query over a whole candidate list of a device corpus."""
    sub, sub_off, sub_len = gather_docs(tok_d, off, lengths, ids)
    qa, qdt = oracle_view(q)
    ta, tdt = oracle_view(sub)
    return oracle.dense_scores(qa, ta, sub_off, sub_len, np.arange(len(ids), dtype=np.int32), qdtype=qdt, tdtype=tdt)
