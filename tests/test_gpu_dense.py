"""Dense MaxSim on the GPU against the FP64 oracle (element by element).

Tolerances: 1e-3 relative for fp16/bf16 inputs, 1e-5 for fp32 (floor
Nq * 1e-3 for scores near zero), NaN exactly where the oracle has NaN and
equal infinities.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close, assert_topk_consistent, assert_topk_matches_oracle, oracle_view

pytestmark = pytest.mark.gpu

SHAPES = [(32, 128), (1, 64), (7, 72), (33, 200), (64, 384), (128, 128), (32, 768), (16, 8), (96, 256), (96, 576),
          (64, 512), (128, 576), (96, 832), (64, 1024), (128, 704), (96, 960), (128, 768), (96, 1024),
          (128, 1024)]


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("nq,d", SHAPES)
def test_dense_edge_grid(cuda_lib, dtype, nq, d):
    """Ragged and degenerate documents (0, 1, 7, ..., 513 tokens, a last
    document ending at the token array's end), duplicate and out-of-range
    ids, several queries in one launch (one with an empty list)."""
    from paper_2606_26439_gb300 import tms
    seed = 1000 + nq * 7 + d
    tok, off, ln = gc.edge_corpus(d, dtype, seed)
    n_queries = 3
    Q = synth.queries(n_queries, nq, d, dtype, seed)
    cands = gc.edge_candidates(len(ln), n_queries, seed)
    got, flags = gc.gpu_dense(Q, tok, off, ln, cands)
    want = gc.oracle_dense_multi(Q, tok, off, ln, cands)
    assert_scores_close(got, want, dtype, nq)
    assert flags & tms.TMS_DEVERR_BAD_ID
    assert not flags & tms.TMS_DEVERR_TIMEOUT
    assert not flags & tms.TMS_DEVERR_BAD_CSR


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
def test_dense_bad_row_range_is_nan_and_flagged(cuda_lib, dtype):
    from paper_2606_26439_gb300 import tms
    d, nq = 128, 32
    lengths = np.array([5, 9, 12], np.int32)
    tok, off, ln = synth.dense_corpus(3, lengths, d, dtype, 5)
    off = off.copy()
    ln = ln.copy()
    off[1] = 20          # rows 20..28 run past n_tokens = 26
    ln[2] = -3           # negative length
    Q = synth.queries(1, nq, d, dtype, 5)
    got, flags = gc.gpu_dense(Q, tok, off, ln, [np.array([0, 1, 2, 0], np.int32)])
    assert np.isnan(got[1]) and np.isnan(got[2])
    assert np.isfinite(got[0]) and got[3] == got[0]
    assert flags & tms.TMS_DEVERR_BAD_RANGE


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_dense_self_score_is_nq(cuda_lib, dtype):
    """Documents equal to the query: every score is sum_i ||q_i||^2 ~ Nq."""
    nq, d = 32, 128
    Q = synth.queries(1, nq, d, dtype, 17)
    tok = Q[0].clone()
    got, _ = gc.gpu_dense(Q, tok, np.array([0], np.int64), np.array([nq], np.int32), [np.array([0], np.int32)])
    qd = Q[0].double().numpy()
    assert got[0] == pytest.approx(float((qd * qd).sum()), rel=1e-3)


def test_dense_bitwise_repeatable(cuda_lib):
    """Fixed-order sums: two launches give bit-identical scores."""
    d, nq = 128, 32
    lengths = synth.lengths_uniform(3000, 32, 180, 3)
    tok, off, ln = synth.dense_corpus(3000, lengths, d, "f16", 3)
    Q = synth.queries(2, nq, d, "f16", 3)
    cands = [synth.candidates(3000, 2500, 3, 0), synth.candidates(3000, 1700, 3, 1)]
    a, _ = gc.gpu_dense(Q, tok, off, ln, cands)
    b, _ = gc.gpu_dense(Q, tok, off, ln, cands)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_dense_alone_equals_in_batch(cuda_lib):
    """A query scored alone or inside a multi-query launch gives the same
    bits (each score has one owner and a fixed summation order)."""
    d, nq = 128, 32
    lengths = synth.lengths_uniform(2000, 1, 200, 4)
    tok, off, ln = synth.dense_corpus(2000, lengths, d, "bf16", 4)
    Q = synth.queries(3, nq, d, "bf16", 4)
    cands = [synth.candidates(2000, n, 4, i) for i, n in enumerate((900, 1500, 300))]
    batch, _ = gc.gpu_dense(Q, tok, off, ln, cands)
    alone, _ = gc.gpu_dense(Q[1:2], tok, off, ln, [cands[1]])
    assert np.array_equal(batch[900:2400].view(np.uint32), alone.view(np.uint32))


def test_config1_full_parity_and_top10(cuda_lib):
    """Dense MaxSim, 1 query Nq=32, d=128, fp16, 10,000 documents of 128
    tokens, unit-normalised Gaussian embeddings, seed 0: every score and the
    top-10 against the oracle."""
    from paper_2606_26439_gb300 import tms
    import torch
    n_docs, nd, d, nq = 10000, 128, 128, 32
    tok, off, ln = synth.dense_corpus(n_docs, synth.lengths_fixed(n_docs, nd), d, "f16", 0)
    Q = synth.queries(1, nq, d, "f16", 0)
    cands = [np.arange(n_docs, dtype=np.int32)]
    got, flags = gc.gpu_dense(Q, tok, off, ln, cands)
    assert flags == 0
    want = gc.oracle_dense_multi(Q, tok, off, ln, cands)
    assert_scores_close(got, want, "f16", nq)
    s_d, co_d = gc.to_dev(got, np.array([0, n_docs], np.int64))
    for k in (10, 100):
        ts, tp = tms.topk(s_d, co_d, k)
        torch.cuda.synchronize()
        # the oracle's own top-k, runs of tolerance-tied scores merged
        assert_topk_matches_oracle(tp.cpu().numpy()[0], want, k, "f16", nq)


def _sampled_parity(tok_d, off, ln, Q, cands, flat_scores, dtype, n_sample, seed):
    """Oracle on a sample of candidates: copy the sampled documents' rows to
    the host, re-pack them, score them one by one."""
    import torch
    g = np.random.default_rng(seed)
    co = np.zeros(len(cands) + 1, np.int64)
    co[1:] = np.cumsum([len(c) for c in cands])
    pos = np.sort(g.choice(co[-1], size=min(n_sample, co[-1]), replace=False))
    qidx = np.searchsorted(co, pos, side="right") - 1
    flat = np.concatenate(cands)
    ids = flat[pos]
    lens = ln[ids]
    rows = np.concatenate([np.arange(off[i], off[i] + ln[i]) for i in ids])
    sub = tok_d[torch.from_numpy(rows).cuda()].cpu()
    sub_off = synth.offsets_of(lens)
    want = np.empty(len(pos))
    ta, tdt = oracle_view(sub)
    qa, qdt = oracle_view(Q)
    for qi in np.unique(qidx):
        sel = np.nonzero(qidx == qi)[0]
        want[sel] = oracle.dense_scores(qa[qi], ta, sub_off, lens, sel.astype(np.int32), qdtype=qdt, tdtype=tdt)
    assert_scores_close(flat_scores[pos], want, dtype, Q.shape[1])


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
def test_config2_full_size_sampled(cuda_lib, dtype):
    """500,000 documents, Nd ~ U[32, 180], d = 128, 16 queries x 100,000
    candidates in one launch (the benchmark's launch): 1,600 sampled scores
    against the oracle, every score finite."""
    import torch
    from paper_2606_26439_gb300 import tms
    n_docs, d, nq, n_queries, n_cand = 500_000, 128, 32, 16, 100_000
    lengths = synth.lengths_uniform(n_docs, 32, 180, 0)
    tok_d, off_d, ln_d = synth.device_dense_corpus(lengths, d, dtype, 0)
    Q = synth.queries(n_queries, nq, d, dtype, 0)
    cands = [synth.candidates(n_docs, n_cand, 0, q) for q in range(n_queries)]
    flat, co = gc.csr(cands)
    q_d, f_d, c_d = gc.to_dev(Q, flat, co)
    out = tms.score_dense(q_d, tok_d, off_d, ln_d, f_d, c_d)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    scores = out.cpu().numpy()
    assert np.isfinite(scores).all()
    off = synth.offsets_of(lengths)
    _sampled_parity(tok_d, off, lengths, Q, cands, scores, dtype, 1600, 1)
    # query 0: every one of its 100,000 scores and its top-10 / top-100
    # against the oracle's own scores of the whole list
    want0 = gc.oracle_dense_list(Q[0], tok_d, off, lengths, cands[0])
    assert_scores_close(scores[:n_cand], want0, dtype, nq)
    for k in (10, 100):
        ts, tp = tms.topk(out, c_d, k)
        torch.cuda.synchronize()
        assert_topk_matches_oracle(tp.cpu().numpy()[0], want0, k, dtype, nq)
    del tok_d
    torch.cuda.empty_cache()


@pytest.mark.slow
@pytest.mark.parametrize("d", [64, 256, 512, 768])
def test_config3_dimension_tiling_full_query(cuda_lib, d):
    """200,000 documents, Nd ~ U[32, 180], bf16, 32 queries each scoring all
    documents, in both schedules (per-query lists: tms_score_dense; one
    shared list: tms_score_dense_shared).  Query 0: all 200,000 scores and
    the top-100 against the oracle's own scores (tolerance ties merged);
    sampled parity on the other queries; each schedule's top-100 is exactly
    the top-100 of its own scores."""
    import torch
    from paper_2606_26439_gb300 import tms
    n_docs, nq, n_queries = 200_000, 32, 32
    lengths = synth.lengths_uniform(n_docs, 32, 180, 2)
    off = synth.offsets_of(lengths)
    tok_d, off_d, ln_d = synth.device_dense_corpus(lengths, d, "bf16", 2)
    Q = synth.queries(n_queries, nq, d, "bf16", 2)
    cands = [np.arange(n_docs, dtype=np.int32)] * n_queries
    flat, co = gc.csr(cands)
    q_d, f_d, c_d = gc.to_dev(Q, flat, co)
    per_query = tms.score_dense(q_d, tok_d, off_d, ln_d, f_d, c_d)
    shared = tms.score_dense_shared(q_d, tok_d, off_d, ln_d, f_d[:n_docs]).view(-1)
    tops = [tms.topk(x, c_d, 100) for x in (per_query, shared)]
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    s_pq, s_sh = per_query.cpu().numpy(), shared.cpu().numpy()
    _sampled_parity(tok_d, off, lengths, Q, cands, s_pq, "bf16", 640, 3)
    _sampled_parity(tok_d, off, lengths, Q, cands, s_sh, "bf16", 640, 4)
    want0 = gc.oracle_dense_list(Q[0], tok_d, off, lengths, cands[0])
    assert_scores_close(s_pq[:n_docs], want0, "bf16", nq)
    assert_scores_close(s_sh[:n_docs], want0, "bf16", nq)
    for scores, (ts, tp) in zip((s_pq, s_sh), tops):
        tsn, tpn = ts.cpu().numpy(), tp.cpu().numpy()
        assert_topk_matches_oracle(tpn[0], want0, 100, "bf16", nq)
        for qi in range(n_queries):
            row = scores[qi * n_docs:(qi + 1) * n_docs]
            ws, wp = oracle.topk(row.astype(np.float64), 100)
            assert np.array_equal(tpn[qi], wp)
            assert np.array_equal(tsn[qi], ws.astype(np.float32))
    del tok_d
    torch.cuda.empty_cache()
