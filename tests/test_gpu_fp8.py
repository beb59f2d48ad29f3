"""FP8 E4M3 store on the GPU against the oracle.

* quantization (tms_quantize_e4m3): codes and scales bit-exact against the
  oracle's definition (fp32 amax / 448, fp32 division, nearest-even
  saturating E4M3);
* scoring (tms_score_fp8, tms_score_fp8_shared): within 1e-3 relative of
  FP64 Eq. 1 on the dequantized vectors, NaN / -inf exactly where the
  oracle has them.  Oracle inputs are the oracle's own quantization of
  seeded fp16 data, or seeded random codes -- never GPU output.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_topk_matches_oracle, assert_scores_close, oracle_view

pytestmark = pytest.mark.gpu


def _quantize_host(x):
    a, dt = oracle_view(x)
    shape = a.shape
    codes, scales = oracle.quantize_e4m3(a.reshape(-1, shape[-1]), dtype=dt)
    return codes.reshape(shape), scales.reshape(shape[:-1])


def _oracle_multi(qc, qs, tc, ts, off, ln, cands):
    res = [oracle.dense_scores_scaled(qc[i], qs[i], tc, ts, off, ln, c, qdtype=oracle.E4M3, tdtype=oracle.E4M3)
           for i, c in enumerate(cands)]
    return np.concatenate(res) if res else np.zeros(0)


def _gpu_fp8(qc, qs, tc, ts, off, ln, cands):
    import torch
    from paper_2606_26439_gb300 import tms
    flat, co = gc.csr(cands)
    d_in = gc.to_dev(qc, qs, tc, ts, off, ln, flat, co)
    out = torch.full((len(flat),), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_fp8(*d_in, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tms.device_error()


def _gpu_fp8_shared(qc, qs, tc, ts, off, ln, cand):
    import torch
    from paper_2606_26439_gb300 import tms
    d_in = gc.to_dev(qc, qs, tc, ts, off, ln, np.asarray(cand, np.int32))
    out = torch.full((qc.shape[0], len(cand)), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_fp8_shared(*d_in, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tms.device_error()


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("d", [16, 96, 128, 1024])
def test_quantize_bit_exact(cuda_lib, dtype, d):
    """Rows at magnitudes 1e-3 .. 1e3, a zero row, a one-hot row and rows
    with exact E4M3 ties: codes and scales equal the oracle's bit for bit."""
    from paper_2606_26439_gb300 import tms
    g = np.random.default_rng(d)
    x = synth.unit_rows(700, d, d, 3) * (10.0 ** g.uniform(-3, 3, size=(700, 1)))
    x[3] = 0.0
    x[4] = 0.0
    x[4, d // 2] = -2.5
    x[5, :] = 448.0 * np.linspace(-1, 1, d)          # many values between codes
    xt = synth.cast(x, dtype)
    want_c, want_s = _quantize_host(xt)
    x_d, = gc.to_dev(xt)
    codes, scales = tms.quantize_e4m3(x_d)
    codes, scales = codes.cpu().numpy(), scales.cpu().numpy()
    assert np.array_equal(scales.view(np.uint32), want_s.view(np.uint32))
    assert np.array_equal(codes, want_c)
    assert tms.device_error() == 0


def test_quantize_rejects_bad_width(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    x = torch.zeros((4, 24), dtype=torch.float16, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.quantize_e4m3(x)
    assert e.value.status == tms.TMS_ERR_INVALID_ARG


SHAPES = [(32, 128), (1, 16), (7, 48), (33, 256), (64, 384), (128, 128), (32, 768), (96, 256), (32, 1024),
          (128, 512)]


@pytest.mark.parametrize("nq,d", SHAPES)
def test_fp8_edge_grid(cuda_lib, nq, d):
    """Ragged and degenerate documents, duplicate and out-of-range ids,
    several queries (one with an empty list); store and queries quantized
    by the oracle from seeded fp16 rows."""
    from paper_2606_26439_gb300 import tms
    seed = 5000 + nq * 7 + d
    tok, off, ln = gc.edge_corpus(d, "f16", seed)
    Q = synth.queries(3, nq, d, "f16", seed)
    tc, ts = _quantize_host(tok)
    qc, qs = _quantize_host(Q)
    cands = gc.edge_candidates(len(ln), 3, seed)
    got, flags = _gpu_fp8(qc, qs, tc, ts, off, ln, cands)
    want = _oracle_multi(qc, qs, tc, ts, off, ln, cands)
    assert_scores_close(got, want, "e4m3", nq)
    assert flags & tms.TMS_DEVERR_BAD_ID
    assert not flags & (tms.TMS_DEVERR_TIMEOUT | tms.TMS_DEVERR_BAD_CSR)


def test_fp8_random_codes_wide_range(cuda_lib):
    """Uniformly random finite codes (magnitudes 2^-9 .. 448) and random
    scales: the E4M3 x E4M3 products span 2^-18 .. 2^17."""
    nq, d = 32, 128
    lengths = synth.lengths_uniform(400, 1, 200, 21)
    off = synth.offsets_of(lengths)
    n_tok = int(lengths.sum())
    tc, ts = synth.e4m3_codes(n_tok, d, 21, 1), synth.row_scales(n_tok, 21, 1)
    qc = synth.e4m3_codes(2 * nq, d, 21, 2).reshape(2, nq, d)
    qs = synth.row_scales(2 * nq, 21, 2).reshape(2, nq)
    cands = [synth.candidates(400, 400, 21, 0), synth.candidates(400, 150, 21, 1)]
    got, flags = _gpu_fp8(qc, qs, tc, ts, off, lengths, cands)
    assert flags == 0
    want = _oracle_multi(qc, qs, tc, ts, off, lengths, cands)
    assert_scores_close(got, want, "e4m3", nq)


def test_fp8_bad_row_range_is_nan_and_flagged(cuda_lib):
    from paper_2606_26439_gb300 import tms
    d, nq = 128, 32
    lengths = np.array([5, 9, 12], np.int32)
    off = synth.offsets_of(lengths).copy()
    tc, ts = synth.e4m3_codes(26, d, 3), synth.row_scales(26, 3)
    qc, qs = synth.e4m3_codes(nq, d, 4).reshape(1, nq, d), synth.row_scales(nq, 4).reshape(1, nq)
    ln = lengths.copy()
    off[1] = 20
    ln[2] = -3
    got, flags = _gpu_fp8(qc, qs, tc, ts, off, ln, [np.array([0, 1, 2, 0], np.int32)])
    assert np.isnan(got[1]) and np.isnan(got[2])
    assert np.isfinite(got[0]) and got[3] == got[0]
    assert flags & tms.TMS_DEVERR_BAD_RANGE


def test_fp8_bitwise_repeatable_and_alone_equals_batch(cuda_lib):
    d, nq = 128, 32
    lengths = synth.lengths_uniform(2000, 1, 200, 6)
    off = synth.offsets_of(lengths)
    n_tok = int(lengths.sum())
    tc, ts = synth.e4m3_codes(n_tok, d, 6), synth.row_scales(n_tok, 6)
    qc = synth.e4m3_codes(3 * nq, d, 6, 1).reshape(3, nq, d)
    qs = synth.row_scales(3 * nq, 6, 1).reshape(3, nq)
    cands = [synth.candidates(2000, n, 6, i) for i, n in enumerate((900, 1500, 300))]
    a, _ = _gpu_fp8(qc, qs, tc, ts, off, lengths, cands)
    b, _ = _gpu_fp8(qc, qs, tc, ts, off, lengths, cands)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    alone, _ = _gpu_fp8(qc[1:2], qs[1:2], tc, ts, off, lengths, [cands[1]])
    assert np.array_equal(a[900:2400].view(np.uint32), alone.view(np.uint32))


@pytest.mark.parametrize("n_queries,nq,d", [(2, 32, 128), (3, 7, 48), (9, 32, 128), (17, 16, 256), (12, 32, 768),
                                            (5, 32, 1024)])
def test_fp8_shared_parity(cuda_lib, n_queries, nq, d):
    from paper_2606_26439_gb300 import tms
    seed = 6000 + n_queries * 13 + d
    tok, off, ln = gc.edge_corpus(d, "f16", seed, n_random=60)
    Q = synth.queries(n_queries, nq, d, "f16", seed)
    tc, ts = _quantize_host(tok)
    qc, qs = _quantize_host(Q)
    cand = gc.edge_candidates(len(ln), 1, seed)[0]
    got, flags = _gpu_fp8_shared(qc, qs, tc, ts, off, ln, cand)
    want = np.stack([oracle.dense_scores_scaled(qc[i], qs[i], tc, ts, off, ln, cand, qdtype=oracle.E4M3,
                                                tdtype=oracle.E4M3) for i in range(n_queries)])
    assert_scores_close(got.ravel(), want.ravel(), "e4m3", nq)
    assert flags & tms.TMS_DEVERR_BAD_ID
    assert not flags & tms.TMS_DEVERR_TIMEOUT


def test_fp8_shared_refuses_wide_queries(cuda_lib):
    from paper_2606_26439_gb300 import tms
    qc, qs = synth.e4m3_codes(66, 64, 1).reshape(2, 33, 64), synth.row_scales(66, 1).reshape(2, 33)
    tc, ts = synth.e4m3_codes(9, 64, 2), synth.row_scales(9, 2)
    ln = np.array([2, 3, 4], np.int32)
    with pytest.raises(tms.TmsError) as e:
        _gpu_fp8_shared(qc, qs, tc, ts, synth.offsets_of(ln), ln, np.array([0, 1, 2], np.int32))
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED


@pytest.mark.slow
@pytest.mark.parametrize("shared", [False, True])
def test_fp8_full_size_sampled(cuda_lib, shared):
    """500,000 documents, Nd ~ U[32, 180], d = 128, random E4M3 store:
    16 queries x 100,000 candidates (per-query lists), or 16 queries over
    one 100,000-candidate list (shared); 1,600 sampled scores vs the oracle."""
    import torch
    from paper_2606_26439_gb300 import tms
    n_docs, d, nq, n_queries, n_cand = 500_000, 128, 32, 16, 100_000
    lengths = synth.lengths_uniform(n_docs, 32, 180, 0)
    tc_d, ts_d, off_d, ln_d = synth.device_e4m3_store(lengths, d, 0)
    qc = synth.e4m3_codes(n_queries * nq, d, 0, 5).reshape(n_queries, nq, d)
    qs = synth.row_scales(n_queries * nq, 0, 5).reshape(n_queries, nq)
    qc_d, qs_d = gc.to_dev(qc, qs)
    if shared:
        cands = [synth.candidates(n_docs, n_cand, 0, 0)] * n_queries
        c_d, = gc.to_dev(cands[0])
        out = tms.score_fp8_shared(qc_d, qs_d, tc_d, ts_d, off_d, ln_d, c_d).view(-1)
    else:
        cands = [synth.candidates(n_docs, n_cand, 0, q) for q in range(n_queries)]
        flat, co = gc.csr(cands)
        f_d, co_d = gc.to_dev(flat, co)
        out = tms.score_fp8(qc_d, qs_d, tc_d, ts_d, off_d, ln_d, f_d, co_d)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    scores = out.cpu().numpy()
    assert np.isfinite(scores).all()
    g = np.random.default_rng(1)
    pos = np.sort(g.choice(len(scores), 1600, replace=False))
    qidx = pos // n_cand
    flat = np.concatenate(cands)
    ids = flat[pos]
    off = synth.offsets_of(lengths)
    rows = torch.from_numpy(np.concatenate([np.arange(off[i], off[i] + lengths[i]) for i in ids])).cuda()
    sub_c, sub_s = tc_d[rows].cpu().numpy(), ts_d[rows].cpu().numpy()
    sub_len = lengths[ids]
    sub_off = synth.offsets_of(sub_len)
    want = np.empty(len(pos))
    for qi in np.unique(qidx):
        sel = np.nonzero(qidx == qi)[0]
        want[sel] = oracle.dense_scores_scaled(qc[qi], qs[qi], sub_c, sub_s, sub_off, sub_len, sel.astype(np.int32),
                                               qdtype=oracle.E4M3, tdtype=oracle.E4M3)
    assert_scores_close(scores[pos], want, "e4m3", nq)
    # query 0: its whole list of 100,000 scores and its top-10 against the
    # oracle's own scores (tolerance ties merged)
    sub_c, sub_off, sub_len = gc.gather_docs(tc_d, off, lengths, cands[0])
    sub_s, _, _ = gc.gather_docs(ts_d, off, lengths, cands[0])
    want0 = oracle.dense_scores_scaled(qc[0], qs[0], sub_c.numpy(), sub_s.numpy(), sub_off, sub_len,
                                       np.arange(n_cand, dtype=np.int32), qdtype=oracle.E4M3, tdtype=oracle.E4M3)
    assert_scores_close(scores[:n_cand], want0, "e4m3", nq)
    co_d = torch.tensor([0, n_cand], dtype=torch.int64, device="cuda")
    _, tp = tms.topk(out[:n_cand], co_d, 10)
    torch.cuda.synchronize()
    assert_topk_matches_oracle(tp.cpu().numpy()[0], want0, 10, "e4m3", nq)
    del tc_d
    torch.cuda.empty_cache()
