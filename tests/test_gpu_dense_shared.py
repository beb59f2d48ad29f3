"""Shared-candidate schedule (tms_score_dense_shared): every query scores
one candidate list, queries stacked in groups in the tensor-core N
dimension.  Element-by-element parity with the FP64 oracle, same
tolerances as the per-query path."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close, oracle_view

pytestmark = pytest.mark.gpu


def _run_shared(Q, tok, off, ln, cand):
    import torch
    from paper_2606_26439_gb300 import tms
    q_d, t_d, o_d, l_d, c_d = gc.to_dev(Q, tok, off, ln, np.asarray(cand, np.int32))
    out = torch.full((Q.shape[0], len(cand)), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_dense_shared(q_d, t_d, o_d, l_d, c_d, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tms.device_error()


def _oracle_all(Q, tok, off, ln, cand):
    qa, qdt = oracle_view(Q)
    ta, tdt = oracle_view(tok)
    return np.stack([oracle.dense_scores(qa[i], ta, off, ln, cand, qdtype=qdt, tdtype=tdt)
                     for i in range(Q.shape[0])])


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("n_queries,nq,d", [(2, 32, 128), (3, 7, 72), (5, 32, 200), (8, 1, 64), (9, 32, 128),
                                            (17, 16, 256), (12, 32, 768), (11, 32, 512), (9, 32, 1024)])
def test_shared_parity_edge_corpus(cuda_lib, dtype, n_queries, nq, d):
    """Groups of 2/4/8 queries (a partial last group included), ragged and
    empty documents, duplicate and out-of-range ids; at d >= 512 the
    group-of-8 query tile is streamed with each dimension chunk."""
    from paper_2606_26439_gb300 import tms
    seed = 3000 + n_queries * 13 + d
    tok, off, ln = gc.edge_corpus(d, dtype, seed, n_random=60)
    Q = synth.queries(n_queries, nq, d, dtype, seed)
    cand = gc.edge_candidates(len(ln), 1, seed)[0]
    got, flags = _run_shared(Q, tok, off, ln, cand)
    want = _oracle_all(Q, tok, off, ln, cand)
    assert_scores_close(got.ravel(), want.ravel(), dtype, nq)
    assert flags & tms.TMS_DEVERR_BAD_ID
    assert not flags & tms.TMS_DEVERR_TIMEOUT


def test_shared_matches_per_query_path(cuda_lib):
    """The shared schedule and the per-query schedule score the same pairs
    to within the fp16 tolerance (they differ only in MMA grouping)."""
    d, nq, n_q = 128, 32, 6
    lengths = synth.lengths_uniform(1500, 32, 180, 8)
    tok, off, ln = synth.dense_corpus(1500, lengths, d, "f16", 8)
    Q = synth.queries(n_q, nq, d, "f16", 8)
    cand = synth.candidates(1500, 1200, 8, 0)
    shared, _ = _run_shared(Q, tok, off, ln, cand)
    per_q, _ = gc.gpu_dense(Q, tok, off, ln, [cand] * n_q)
    assert_scores_close(shared.ravel(), per_q.astype(np.float64), "f16", nq)


@pytest.mark.parametrize("dtype,nq", [("f32", 32), ("f16", 33)])
def test_shared_refuses_unsupported(cuda_lib, dtype, nq):
    from paper_2606_26439_gb300 import tms
    tok, off, ln = synth.dense_corpus(3, np.array([2, 3, 4], np.int32), 64, dtype, 1)
    Q = synth.queries(2, nq, 64, dtype, 1)
    with pytest.raises(tms.TmsError) as e:
        _run_shared(Q, tok, off, ln, np.array([0, 1, 2], np.int32))
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED
