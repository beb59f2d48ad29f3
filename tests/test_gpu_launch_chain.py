"""Back-to-back launches on one stream with no synchronisation between them.

Every scoring and top-k kernel is launched with programmatic stream
serialization: it may be scheduled while the previous kernel is finishing
and must touch global memory only after griddepcontrol.wait.  These chains
reuse one score buffer (and one PQ table) across iterations, so a kernel
that read its input too early would see the previous iteration's values
and one that wrote too early would corrupt what the previous kernel is
still reading (a write-after-read across launches).  Nothing else runs
between the launches, so each top-k reads the score buffer that the next
iteration's scoring launch overwrites; every iteration's top-k, and the
last scores, must equal the same work run alone with a synchronisation
after every launch, bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _dense_inputs(dev, n_docs=20_000, n_iter=12, n_cand=6_000):
    import torch
    lens = synth.lengths_uniform(n_docs, 1, 180, 70)
    tok, off, ln = synth.device_dense_corpus(lens, 128, "f16", 70, dev)
    qs = [synth.queries(2, 32, 128, "f16", 100 + i).to(dev) for i in range(n_iter)]
    cands = [torch.from_numpy(np.concatenate([synth.candidates(n_docs, n_cand, 200 + i, j) for j in range(2)])
                              .astype(np.int32)).to(dev) for i in range(n_iter)]
    co = torch.tensor([0, n_cand, 2 * n_cand], dtype=torch.int64, device=dev)
    return tok, off, ln, qs, cands, co


def test_dense_then_topk_chain_matches_synchronised_runs(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    tok, off, ln, qs, cands, co = _dense_inputs(dev)
    n_iter, k = len(qs), 16
    n_cand = int(co[-1])
    out = torch.empty(n_cand, dtype=torch.float32, device=dev)       # shared by every iteration
    ws = torch.empty(max(16, tms.topk_workspace_size(2, k, n_cand)), dtype=torch.uint8, device=dev)
    ts = torch.empty((n_iter, 2, k), dtype=torch.float32, device=dev)
    tp = torch.empty((n_iter, 2, k), dtype=torch.int32, device=dev)
    ts2 = torch.empty_like(ts)
    tp2 = torch.empty_like(tp)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for i in range(n_iter):
            tms.score_dense(qs[i], tok, off, ln, cands[i], co, out=out, stream=s)
            tms.topk(out, co, k, ts[i], tp[i], stream=s)
            tms.topk_split(out, co, k, n_cand, ts2[i], tp2[i], ws, stream=s)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    for i in range(n_iter):
        alone = tms.score_dense(qs[i], tok, off, ln, cands[i], co)
        torch.cuda.synchronize()
        a_s, a_p = tms.topk(alone, co, k)
        torch.cuda.synchronize()
        if i == n_iter - 1:
            assert torch.equal(out.view(torch.int32), alone.view(torch.int32))
        assert torch.equal(tp[i], a_p) and torch.equal(ts[i].view(torch.int32), a_s.view(torch.int32)), i
        assert torch.equal(tp2[i], a_p) and torch.equal(ts2[i].view(torch.int32), a_s.view(torch.int32)), i


def test_pq_table_scoring_topk_chain_matches_synchronised_runs(cuda_lib):
    """One PQ table buffer rewritten every iteration while the previous
    iteration's scoring and top-k launches are still queued ahead of it."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    M, K, dsub, n_docs, n_iter, k = 16, 256, 8, 8_000, 8, 16  # k * 4 B: every ts[i] 16-byte aligned
    lens = synth.lengths_uniform(n_docs, 1, 120, 71)
    cb, codes, _, off, ln = synth.pq_corpus(lens, M, K, dsub, 71)
    cb_d = torch.from_numpy(cb).to(dev)
    codes_d = torch.from_numpy(codes).to(dev)
    off_d, ln_d = torch.from_numpy(off).to(dev), torch.from_numpy(ln).to(dev)
    qs = [synth.queries(1, 32, M * dsub, "f32", 300 + i).to(dev) for i in range(n_iter)]
    ids = torch.arange(n_docs, dtype=torch.int32, device=dev)
    co = torch.tensor([0, n_docs], dtype=torch.int64, device=dev)
    lut = torch.empty((1, 32, M, K), dtype=torch.float32, device=dev)   # shared by every iteration
    out = torch.empty(n_docs, dtype=torch.float32, device=dev)          # shared by every iteration
    ts = torch.empty((n_iter, 1, k), dtype=torch.float32, device=dev)
    tp = torch.empty((n_iter, 1, k), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for i in range(n_iter):
            tms.build_pq_lut(qs[i], cb_d, out=lut, stream=s)
            tms.score_pq(lut, codes_d, off_d, ln_d, ids, co, out=out, stream=s)
            tms.topk(out, co, k, ts[i], tp[i], stream=s)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    for i in range(n_iter):
        lut_i = tms.build_pq_lut(qs[i], cb_d)
        torch.cuda.synchronize()
        alone = tms.score_pq(lut_i, codes_d, off_d, ln_d, ids, co)
        torch.cuda.synchronize()
        a_s, a_p = tms.topk(alone, co, k)
        torch.cuda.synchronize()
        if i == n_iter - 1:
            assert torch.equal(out.view(torch.int32), alone.view(torch.int32))
        assert torch.equal(tp[i], a_p) and torch.equal(ts[i].view(torch.int32), a_s.view(torch.int32)), i
