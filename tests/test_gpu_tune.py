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
