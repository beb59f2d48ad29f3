"""Fused PQ scoring and the PQ distance table on the GPU against the oracle.

* table: within the fp32 rounding bound of the exact FP64 table;
* code gathering: bit-exact -- with an integer-valued table every sum is
  exact, so the GPU score must equal the oracle's exact table-sum score;
* scores: within 1e-3 relative of FP64 decompress-then-dot (fp16 queries).

The fp16-table variant (tms_score_pq_f16) runs every check too, with two of
its own: a table of multiples of 1/2 whose fp16 rounding includes exact ties
scores bit for bit like the oracle on the table rounded to nearest-even
fp16 (rounded sums stay exact in fp32), and a random table stays within the
fp32 summation bound of that rounded-table score.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close, assert_topk_matches_oracle, oracle_view

pytestmark = pytest.mark.gpu


def _gpu_lut(Q, cb):
    import torch
    from paper_2606_26439_gb300 import tms
    q_d, cb_d = gc.to_dev(Q, cb)
    lut = tms.build_pq_lut(q_d, cb_d)
    torch.cuda.synchronize()
    return lut


def _gpu_pq(lut_d, codes, off, ln, cands, f16=False):
    import torch
    from paper_2606_26439_gb300 import tms
    flat, co = gc.csr(cands)
    c_d, o_d, l_d, f_d, co_d = gc.to_dev(codes, off, ln, flat, co)
    out = torch.full((len(flat),), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_pq(lut_d, c_d, o_d, l_d, f_d, co_d, out=out, f16_table=f16)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tms.device_error()


@pytest.mark.parametrize("qdtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("nq,d,M,K", [(32, 128, 16, 256), (5, 64, 4, 16), (33, 256, 32, 128), (8, 96, 8, 100)])
def test_pq_lut_within_fp32_bound(cuda_lib, qdtype, nq, d, M, K):
    """|T_gpu - T_exact| <= 2 dsub u sum_t |q_t c_t| (u = 2^-24, fma chain)."""
    n_queries = 2
    Q = synth.queries(n_queries, nq, d, qdtype, 40 + M)
    cb = np.random.default_rng(M).standard_normal((M, K, d // M)).astype(np.float32)
    got = _gpu_lut(Q, cb).cpu().numpy()
    qa, qdt = oracle_view(Q)
    dsub = d // M
    for qi in range(n_queries):
        want = oracle.pq_lut(qa[qi], cb, qdtype=qdt)
        qd = np.abs(Q[qi].double().numpy()).reshape(nq, M, dsub)
        mag = np.einsum("imt,mkt->imk", qd, np.abs(cb.astype(np.float64)))
        bound = 2 * dsub * 2.0 ** -24 * mag + 1e-30
        assert np.all(np.abs(got[qi] - want) <= bound)


@pytest.mark.parametrize("M", [4, 8, 16, 32])
@pytest.mark.parametrize("nq", [1, 7, 8, 9, 32, 33])
def test_pq_gather_bit_exact_integer_table(cuda_lib, M, nq):
    """Integer-valued table: every partial sum is exact in fp32, so the GPU
    result must equal the exact score bit for bit (a wrong code byte, wrong
    subspace or wrong query token would change it)."""
    import torch
    K = 256 if M <= 16 else 128
    g = np.random.default_rng(M * 100 + nq)
    n_queries = 2
    T = g.integers(-1000, 1001, size=(n_queries, nq, M, K)).astype(np.float32)
    lengths = np.array(gc.EDGE_LENGTHS + list(g.integers(1, 150, 60)) + [77], np.int32)
    off = synth.offsets_of(lengths)
    codes = g.integers(0, K, size=(int(lengths.sum()), M)).astype(np.uint8)
    n_docs = len(lengths)
    cands = gc.edge_candidates(n_docs, n_queries, M + nq)
    lut_d = torch.from_numpy(T).cuda()
    got, flags = _gpu_pq(lut_d, codes, off, lengths, cands)
    want = np.concatenate([oracle.pq_lut_scores(T[qi], codes, off, lengths, c) for qi, c in enumerate(cands)])
    fin = np.isfinite(want)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(got[~fin & ~np.isnan(want)], want[~fin & ~np.isnan(want)])
    assert np.array_equal(got[fin].astype(np.float64), want[fin])


@pytest.mark.parametrize("f16", [False, True])
@pytest.mark.parametrize("nq", [32, 9])
def test_pq_scores_vs_decompress(cuda_lib, nq, f16):
    """GPU table (tms_build_pq_lut) + fused scoring vs FP64
    decompress-then-dot on the same fp16 queries and fp32 codebook."""
    M, K, dsub = 16, 256, 8
    d = M * dsub
    lengths = synth.lengths_uniform(400, 1, 180, 50)
    cb, codes, _, off, ln = synth.pq_corpus(lengths, M, K, dsub, 50)
    Q = synth.queries(3, nq, d, "f16", 50)
    cands = [synth.candidates(400, n, 50, i) for i, n in enumerate((400, 250, 37))]
    lut_d = _gpu_lut(Q, cb)
    got, flags = _gpu_pq(lut_d, codes, off, ln, cands, f16)
    assert flags == 0
    qa, qdt = oracle_view(Q)
    want = np.concatenate([oracle.pq_decompress_scores(qa[i], cb, codes, off, ln, c, qdtype=qdt)
                           for i, c in enumerate(cands)])
    if not f16:
        assert_scores_close(got, want, "f16", nq)
        return
    # fp16 table: each entry carries a relative rounding error <= 2^-11 on top
    # of the fp32 table error (<= 2 dsub 2^-24 sum_t |q_t c_t|) and the fp32
    # sums, so |err| <= (2^-11 + 2^-24 (2 dsub + M + nq + 2)) * A with
    # A = sum_i max_j sum_m sum_t |q_t| |c_t| -- a bound on the table's
    # magnitude, not on the score, which may nearly cancel.
    qabs = np.abs(Q.double().numpy())
    A = np.concatenate([oracle.pq_lut_scores(oracle.pq_lut(qabs[i], np.abs(cb), qdtype=oracle.F64), codes, off,
                                             ln, c) for i, c in enumerate(cands)])
    bound = (2.0 ** -11 + 2.0 ** -24 * (2 * dsub + M + nq + 2)) * A
    assert np.all(np.abs(got - want) <= bound)


@pytest.mark.parametrize("f16", [False, True])
def test_pq_edge_documents_and_flags(cuda_lib, f16):
    """Empty documents score -inf, bad ids NaN with the error flag raised."""
    from paper_2606_26439_gb300 import tms
    import torch
    M, K, nq = 16, 256, 32
    lengths = np.array([0, 3, 0, 5], np.int32)
    off = synth.offsets_of(lengths)
    codes = np.random.default_rng(1).integers(0, K, size=(8, M)).astype(np.uint8)
    T = np.random.default_rng(2).standard_normal((1, nq, M, K)).astype(np.float32)
    got, flags = _gpu_pq(torch.from_numpy(T).cuda(), codes, off, lengths,
                         [np.array([0, 1, 2, 3, -5, 4], np.int32)], f16)
    assert got[0] == -np.inf and got[2] == -np.inf
    assert np.isnan(got[4]) and np.isnan(got[5])
    assert np.isfinite(got[1]) and np.isfinite(got[3])
    assert flags & tms.TMS_DEVERR_BAD_ID


@pytest.mark.parametrize("f16", [False, True])
def test_pq_bitwise_repeatable(cuda_lib, f16):
    M, K, dsub = 16, 256, 8
    lengths = synth.lengths_uniform(800, 32, 300, 51)
    cb, codes, _, off, ln = synth.pq_corpus(lengths, M, K, dsub, 51)
    Q = synth.queries(2, 32, M * dsub, "f16", 51)
    cands = [synth.candidates(800, 800, 51, 0), synth.candidates(800, 300, 51, 1)]
    lut_d = _gpu_lut(Q, cb)
    a, _ = _gpu_pq(lut_d, codes, off, ln, cands, f16)
    b, _ = _gpu_pq(lut_d, codes, off, ln, cands, f16)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.slow
def test_config4_pq_full_size_all_forms(cuda_lib):
    """1,000,000 documents, Nd ~ U[32, 180], M = 16, K = 256, dsub = 8,
    Gaussian centroids + N(0, 0.05) noise, nearest-centroid codes; 64 fp16
    queries each over all documents -- the benchmark's launches of the fused
    PQ kernel with the fp32 table and the fp16 table, and of the tensor-core
    PQ kernel (codes decompressed in shared memory).  For each: 512 sampled
    scores across the 64 queries, and query 0's all 1,000,000 scores and
    top-10 / top-100 against FP64 decompress-then-dot (tolerance ties merged)."""
    import torch
    from paper_2606_26439_gb300 import tms
    n_docs, M, K, dsub, nq, n_queries = 1_000_000, 16, 256, 8, 32, 64
    d = M * dsub
    lengths = synth.lengths_uniform(n_docs, 32, 180, 4)
    off = synth.offsets_of(lengths)
    cb_d, codes_d, off_d, ln_d = synth.device_pq_corpus(lengths, M, K, dsub, 4)
    Q = synth.queries(n_queries, nq, d, "f16", 4)
    q_d = gc.to_dev(Q)[0]
    lut_d = tms.build_pq_lut(q_d, cb_d)
    ids = np.arange(n_docs, dtype=np.int32)
    flat, co = gc.csr([ids] * n_queries)
    f_d, co_d = gc.to_dev(flat, co)
    forms = {
        "fp32 table": tms.score_pq(lut_d, codes_d, off_d, ln_d, f_d, co_d),
        "fp16 table": tms.score_pq(lut_d, codes_d, off_d, ln_d, f_d, co_d, f16_table=True),
        "tensor cores": tms.score_pq_tc_shared(q_d, cb_d, codes_d, off_d, ln_d, f_d[:n_docs]).view(-1),
    }
    tops = {name: [tms.topk(x, co_d[:2], k) for k in (10, 100)] for name, x in forms.items()}
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    cb = cb_d.cpu().numpy()
    codes = codes_d.cpu().numpy()
    qa, qdt = oracle_view(Q)
    want0 = oracle.pq_decompress_scores(qa[0], cb, codes, off, lengths, ids, qdtype=qdt)
    g = np.random.default_rng(5)
    pos = np.sort(g.choice(len(flat), 512, replace=False))
    qidx = pos // n_docs
    di = flat[pos]
    sub_len = lengths[di]
    sub_codes = codes[gc.rows_of(off, lengths, di)]
    want = np.empty(len(pos))
    for qi in np.unique(qidx):
        sel = np.nonzero(qidx == qi)[0]
        want[sel] = oracle.pq_decompress_scores(qa[qi], cb, sub_codes, synth.offsets_of(sub_len), sub_len,
                                                sel.astype(np.int32), qdtype=qdt)
    for name, out in forms.items():
        scores = out.cpu().numpy()
        assert np.isfinite(scores).all(), name
        assert_scores_close(scores[pos], want, "f16", nq)
        assert_scores_close(scores[:n_docs], want0, "f16", nq)
        for k, (ts, tp) in zip((10, 100), tops[name]):
            assert_topk_matches_oracle(tp.cpu().numpy()[0], want0, k, "f16", nq)


def _ragged_pq_case(M, K, nq, seed, n_queries=2):
    g = np.random.default_rng(seed)
    lengths = np.array(gc.EDGE_LENGTHS + list(g.integers(1, 150, 60)) + [77], np.int32)
    off = synth.offsets_of(lengths)
    codes = g.integers(0, K, size=(int(lengths.sum()), M)).astype(np.uint8)
    cands = gc.edge_candidates(len(lengths), n_queries, seed)
    return g, lengths, off, codes, cands


@pytest.mark.parametrize("M", [16, 32])
@pytest.mark.parametrize("nq", [1, 7, 15, 16, 17, 32, 33, 128])
def test_pq_f16_half_integer_table_bit_exact(cuda_lib, M, nq):
    """Table entries are multiples of 1/2 up to 4000 in magnitude, so fp16
    rounding meets exact ties (x.5 in [1024, 2048), odd integers in
    [2048, 4096)).  Every rounded entry is a multiple of 1/2 and every sum
    stays exact in fp32, so the GPU must equal the oracle on the table
    rounded to nearest-even fp16 bit for bit (a truncating or
    ties-away rounding, a wrong query token or half of a word would not)."""
    import torch
    K = 256 if M == 16 else 128
    n_queries = 2
    g, lengths, off, codes, cands = _ragged_pq_case(M, K, nq, M * 1000 + nq)
    T = (g.integers(-8000, 8001, size=(n_queries, nq, M, K)) / 2).astype(np.float32)
    T16 = T.astype(np.float16)   # IEEE round to nearest, ties to even
    assert np.any(T16.astype(np.float32) != T)   # ties and roundings were met
    got, flags = _gpu_pq(torch.from_numpy(T).cuda(), codes, off, lengths, cands, f16=True)
    want = np.concatenate([oracle.pq_lut_scores(T16[qi], codes, off, lengths, c) for qi, c in enumerate(cands)])
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok].astype(np.float64), want[ok])


@pytest.mark.parametrize("M,K", [(16, 256), (32, 128), (16, 100)])
@pytest.mark.parametrize("nq", [9, 32])
def test_pq_f16_random_table_within_fp32_sum_bound(cuda_lib, M, K, nq):
    """Random fp32 table: the GPU score is the score of the fp16-rounded
    table up to fp32 summation, |err| <= 2^-24 (M + nq + 2) sum_i max_j
    sum_m |T16| -- far below one fp16 rounding step of one entry in most
    scores, so a table read in fp32 (not rounded) fails too."""
    import torch
    n_queries = 2
    g, lengths, off, codes, cands = _ragged_pq_case(M, K, nq, 7 * M + nq + K)
    T = (g.standard_normal((n_queries, nq, M, K)) * 0.7).astype(np.float32)
    T16 = T.astype(np.float16)
    got, flags = _gpu_pq(torch.from_numpy(T).cuda(), codes, off, lengths, cands, f16=True)
    want = np.concatenate([oracle.pq_lut_scores(T16[qi], codes, off, lengths, c) for qi, c in enumerate(cands)])
    want32 = np.concatenate([oracle.pq_lut_scores(T[qi], codes, off, lengths, c) for qi, c in enumerate(cands)])
    mag = np.concatenate([oracle.pq_lut_scores(np.abs(T16[qi]).astype(np.float64), codes, off, lengths, c)
                          for qi, c in enumerate(cands)])
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[~fin & ~np.isnan(want)], want[~fin & ~np.isnan(want)])
    bound = 2.0 ** -24 * (M + nq + 2) * mag[fin]
    assert np.all(np.abs(got[fin] - want[fin]) <= bound)
    # the rounding is really applied: the fp32-table score is outside the bound somewhere
    assert np.any(np.abs(got[fin] - want32[fin]) > bound)


def test_pq_f16_rejects_small_m(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    T = torch.zeros((1, 4, 8, 16), dtype=torch.float32, device="cuda")
    codes = torch.zeros((4, 8), dtype=torch.uint8, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    ln = torch.full((1,), 4, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.int32, device="cuda")
    co = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.score_pq(T, codes, off, ln, f, co, f16_table=True)
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED
