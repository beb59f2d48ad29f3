"""Autotuner (tms_tune_dense): times the tensor-core launch configurations
that fit a shape, keeps the fastest for later launches; scores are the
same bits whatever configuration runs, and equal the oracle's within the
usual tolerance."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,nq,d", [("f16", 32, 128), ("bf16", 64, 64), ("f16", 7, 200), ("f32", 32, 128)])
def test_tune_then_score_same_bits(cuda_lib, dtype, nq, d):
    import torch
    from paper_2606_26439_gb300 import tms
    seed = 900 + nq + d
    tok, off, ln = gc.edge_corpus(d, dtype, seed, n_random=300)
    Q = synth.queries(3, nq, d, dtype, seed)
    cands = gc.edge_candidates(len(ln), 3, seed)
    before, _ = gc.gpu_dense(Q, tok, off, ln, cands)   # default configuration
    flat, co = gc.csr(cands)
    q_d, t_d, o_d, l_d, f_d, c_d = gc.to_dev(Q, tok, off, ln, flat, co)
    tuned, n = tms.tune_dense(q_d, t_d, o_d, l_d, f_d, c_d)
    torch.cuda.synchronize()
    tms.device_error()
    assert n >= 1
    after, _ = gc.gpu_dense(Q, tok, off, ln, cands)    # the tuned configuration
    assert np.array_equal(before.view(np.uint32), tuned.cpu().numpy().view(np.uint32))
    assert np.array_equal(before.view(np.uint32), after.view(np.uint32))
    want = gc.oracle_dense_multi(Q, tok, off, ln, cands)
    assert_scores_close(after, want, dtype, nq)


@pytest.mark.parametrize("dtype,n_queries,d", [("bf16", 9, 64), ("f16", 6, 256), ("bf16", 3, 768)])
def test_tune_dense_shared_same_bits(cuda_lib, dtype, n_queries, d):
    """The shared-list tuner searches group sizes as well: the scores of the
    tuned launch, of the next tms_score_dense_shared and of the default are
    the same bits, and equal the oracle's within the tolerance."""
    import torch
    from paper_2606_26439_gb300 import tms
    seed = 950 + n_queries + d
    tok, off, ln = gc.edge_corpus(d, dtype, seed, n_random=120)
    Q = synth.queries(n_queries, 32, d, dtype, seed)
    cand = gc.edge_candidates(len(ln), 1, seed)[0]
    q_d, t_d, o_d, l_d, c_d = gc.to_dev(Q, tok, off, ln, cand)
    before = tms.score_dense_shared(q_d, t_d, o_d, l_d, c_d).cpu().numpy()
    tuned, n = tms.tune_dense_shared(q_d, t_d, o_d, l_d, c_d)
    after = tms.score_dense_shared(q_d, t_d, o_d, l_d, c_d)
    torch.cuda.synchronize()
    tms.device_error()
    assert n >= 1
    assert np.array_equal(before.view(np.uint32), tuned.cpu().numpy().view(np.uint32))
    assert np.array_equal(before.view(np.uint32), after.cpu().numpy().view(np.uint32))
    want = np.stack([gc.oracle_dense_multi(Q[i:i + 1], tok, off, ln, [cand]) for i in range(n_queries)])
    assert_scores_close(before.ravel(), want.ravel(), dtype, 32)


@pytest.mark.parametrize("shared", [False, True])
def test_tune_fp8_same_bits(cuda_lib, shared):
    """FP8 store tuners: tuned, next and default launches agree bit for bit
    and match FP64 Eq. 1 on the dequantized vectors."""
    import torch
    import oracle
    from paper_2606_26439_gb300 import tms
    from tests._common import oracle_view
    d, nq, n_queries = 128, 32, 5
    seed = 970 + int(shared)
    tok, off, ln = gc.edge_corpus(d, "f16", seed, n_random=120)
    Q = synth.queries(n_queries, nq, d, "f16", seed)
    ta, tdt = oracle_view(tok)
    qa, qdt = oracle_view(Q)
    tc, ts = oracle.quantize_e4m3(ta, dtype=tdt)
    qc, qs = oracle.quantize_e4m3(qa.reshape(-1, d), dtype=qdt)
    qc, qs = qc.reshape(n_queries, nq, d), qs.reshape(n_queries, nq)
    if shared:
        cand = gc.edge_candidates(len(ln), 1, seed)[0]
        dev_in = gc.to_dev(qc, qs, tc, ts, off, ln, cand)
        run = lambda: tms.score_fp8_shared(*dev_in)  # noqa: E731
        before = run().cpu().numpy()
        tuned, n = tms.tune_fp8_shared(*dev_in)
        want = np.stack([oracle.dense_scores_scaled(qc[i], qs[i], tc, ts, off, ln, cand, qdtype=oracle.E4M3,
                                                    tdtype=oracle.E4M3) for i in range(n_queries)])
    else:
        cands = gc.edge_candidates(len(ln), n_queries, seed)
        flat, co = gc.csr(cands)
        dev_in = gc.to_dev(qc, qs, tc, ts, off, ln, flat, co)
        run = lambda: tms.score_fp8(*dev_in)  # noqa: E731
        before = run().cpu().numpy()
        tuned, n = tms.tune_fp8(*dev_in)
        want = np.concatenate([oracle.dense_scores_scaled(qc[i], qs[i], tc, ts, off, ln, c, qdtype=oracle.E4M3,
                                                          tdtype=oracle.E4M3) for i, c in enumerate(cands)])
    after = run()
    torch.cuda.synchronize()
    tms.device_error()
    assert n >= 1
    t_bits = tuned.cpu().numpy().view(np.uint32)
    assert np.array_equal(t_bits, before.view(np.uint32))
    assert np.array_equal(t_bits, after.cpu().numpy().view(np.uint32))
    assert_scores_close(tuned.cpu().numpy().ravel(), want.ravel(), "e4m3", nq)
