"""The timeout path of the pipelined tensor-core kernels, on the GPU.

A wait that nothing will ever satisfy is made with the diagnostics hook
(tms_debug_set, TMS_FAULT_HOLD_ACCUMULATOR: CTA 0's MMA thread never signals
its first accumulator), with a short wait budget.  The launch must come back
on its own with TMS_DEVERR_TIMEOUT in the device error word -- the waiting
epilogue gives up, raises the CTA's abort flag, every role stops, in-flight
copies and MMAs land, tensor memory is freed -- and the context must stay
usable: the next launch without the fault matches the oracle on every score.
No GPU fault, trap or endless loop is involved: the stuck wait is bounded.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close, oracle_view

pytestmark = pytest.mark.gpu

BUDGET = 4_000_000  # SM cycles (about 2 ms): every pipeline wait gives up after it


@pytest.fixture
def debug_hook(cuda_lib):
    from paper_2606_26439_gb300 import tms
    tms.device_error()  # start from a clear error word
    yield tms
    assert tms.tms_debug_set(0, 0) == tms.TMS_OK


def _corpus(dtype, seed):
    lengths = synth.lengths_uniform(400, 1, 200, seed)
    tok, off, ln = synth.dense_corpus(400, lengths, 128, dtype, seed)
    Q = synth.queries(2, 32, 128, dtype, seed)
    cands = [synth.candidates(400, 400, seed, 0), synth.candidates(400, 250, seed, 1)]
    return tok, off, ln, Q, cands


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_dense_wait_runs_out_then_recovers(debug_hook, dtype):
    tms = debug_hook
    tok, off, ln, Q, cands = _corpus(dtype, 61)
    assert tms.tms_debug_set(BUDGET, tms.TMS_FAULT_HOLD_ACCUMULATOR) == tms.TMS_OK
    t0 = time.time()
    _, flags = gc.gpu_dense(Q, tok, off, ln, cands)
    assert time.time() - t0 < 60
    assert flags & tms.TMS_DEVERR_TIMEOUT
    assert tms.tms_debug_set(0, 0) == tms.TMS_OK
    got, flags = gc.gpu_dense(Q, tok, off, ln, cands)
    assert flags == 0
    assert_scores_close(got, gc.oracle_dense_multi(Q, tok, off, ln, cands), dtype, 32)


def test_fp8_wait_runs_out_then_recovers(debug_hook):
    """The FP8 store runs two CTAs per SM with half the tensor memory each:
    the aborted CTA must free its half for the next launch."""
    import torch
    tms = debug_hook
    tok, off, ln, Q, cands = _corpus("f16", 62)
    ta, tdt = oracle_view(tok)
    codes, scales = oracle.quantize_e4m3(ta, dtype=tdt)
    qa, qdt = oracle_view(Q)
    qc, qs = oracle.quantize_e4m3(qa.reshape(-1, 128), dtype=qdt)
    qc, qs = qc.reshape(2, 32, 128), qs.reshape(2, 32)
    flat, co = gc.csr(cands)
    c_d, s_d, o_d, l_d, f_d, co_d, qc_d, qs_d = gc.to_dev(codes, scales, off, ln, flat, co, qc, qs)
    assert tms.tms_debug_set(BUDGET, tms.TMS_FAULT_HOLD_ACCUMULATOR) == tms.TMS_OK
    tms.score_fp8(qc_d, qs_d, c_d, s_d, o_d, l_d, f_d, co_d)
    torch.cuda.synchronize()
    assert tms.device_error() & tms.TMS_DEVERR_TIMEOUT
    assert tms.tms_debug_set(0, 0) == tms.TMS_OK
    out = tms.score_fp8(qc_d, qs_d, c_d, s_d, o_d, l_d, f_d, co_d)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    want = np.concatenate([oracle.dense_scores_scaled(qc[i], qs[i], codes, scales,
                                                      off, ln, c, qdtype=oracle.E4M3, tdtype=oracle.E4M3)
                           for i, c in enumerate(cands)])
    assert_scores_close(out.cpu().numpy(), want, "e4m3", 32)


def test_short_budget_alone_is_harmless_when_waits_are_short(debug_hook):
    """A budget far above the pipeline's real waits (here ~50 ms) changes
    nothing: same bits as the default budget."""
    tms = debug_hook
    tok, off, ln, Q, cands = _corpus("f16", 63)
    ref, _ = gc.gpu_dense(Q, tok, off, ln, cands)
    assert tms.tms_debug_set(100_000_000, 0) == tms.TMS_OK
    got, flags = gc.gpu_dense(Q, tok, off, ln, cands)
    assert flags == 0
    assert np.array_equal(ref.view(np.uint32), got.view(np.uint32))
