"""PQ MaxSim on the tensor cores (tms_score_pq_tc_shared): codes decompressed
in shared memory, scored by Eq. 1 on fp16 rows, queries sharing one list.

* bit-exact: a codebook of multiples of 1/8 (exact in fp16) and integer
  queries make every product and sum exact in fp32, so the GPU must equal
  the oracle's FP64 decompress-then-dot bit for bit -- a wrong code byte,
  subspace, swizzle unit, query row or padding row would change it;
* bound: on Gaussian codebooks, within the fp16 rounding of the centroids
  (2^-11 relative per element) plus fp32 summation, against FP64
  decompress-then-dot (Section 4.1) on the fp32 codebook;
* the full-size config-4 case sampled at 1e-3 per score.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_scores_close, oracle_view

pytestmark = pytest.mark.gpu

M, DSUB, D = 16, 8, 128


def _gpu(Q, cb, codes, off, ln, cand):
    import torch
    from paper_2606_26439_gb300 import tms
    q_d, cb_d, c_d, o_d, l_d, f_d = gc.to_dev(Q, cb, codes, off, ln, cand)
    out = torch.full((Q.shape[0], len(cand)), 12345.0, dtype=torch.float32, device="cuda")
    tms.score_pq_tc_shared(q_d, cb_d, c_d, o_d, l_d, f_d, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tms.device_error()


def _edge_case(K, seed, n_random=80):
    g = np.random.default_rng(seed)
    lengths = np.array(gc.EDGE_LENGTHS + list(g.integers(1, 200, n_random)) + [129], np.int32)
    off = synth.offsets_of(lengths)
    codes = g.integers(0, K, size=(int(lengths.sum()), M)).astype(np.uint8)
    n_docs = len(lengths)
    cand = np.concatenate([g.permutation(n_docs), [0, 0, n_docs - 1, -1, n_docs, 2 ** 31 - 1]]).astype(np.int32)
    return g, lengths, off, codes, cand


def _oracle(Q, cb, codes, off, ln, cand):
    qa, qdt = oracle_view(Q)
    return np.stack([oracle.pq_decompress_scores(qa[i], cb, codes, off, ln, cand, qdtype=qdt)
                     for i in range(Q.shape[0])])


@pytest.mark.parametrize("n_queries,nq", [(1, 32), (2, 1), (3, 17), (5, 32), (8, 32), (9, 7)])
@pytest.mark.parametrize("K", [256, 100])
def test_pq_tc_bit_exact(cuda_lib, n_queries, nq, K):
    import torch
    from paper_2606_26439_gb300 import tms
    g, lengths, off, codes, cand = _edge_case(K, 100 * n_queries + nq + K)
    cb = (g.integers(-32, 33, size=(M, K, DSUB)) / 8).astype(np.float32)
    Q = torch.from_numpy(g.integers(-4, 5, size=(n_queries, nq, D)).astype(np.float16))
    got, flags = _gpu(Q, cb, codes, off, lengths, cand)
    want = _oracle(Q, cb, codes, off, lengths, cand)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok].astype(np.float64), want[ok])
    assert flags & tms.TMS_DEVERR_BAD_ID


@pytest.mark.parametrize("n_queries", [4, 6])
def test_pq_tc_within_fp16_centroid_bound(cuda_lib, n_queries):
    """|err| <= (2^-11 + 2^-24 (2 D + Nq + 2)) A, A = sum_i max_j sum_t |q_t| |c_t|
    (the bound on the table's magnitude, not on the score)."""
    lengths = synth.lengths_uniform(300, 1, 180, 60)
    cb, codes, _, off, ln = synth.pq_corpus(lengths, M, 256, DSUB, 60)
    nq = 32
    Q = synth.queries(n_queries, nq, D, "f16", 60)
    cand = synth.candidates(300, 300, 60, 0)
    got, flags = _gpu(Q, cb, codes, off, ln, cand)
    assert flags == 0
    want = _oracle(Q, cb, codes, off, ln, cand)
    qabs = np.abs(Q.double().numpy())
    A = np.stack([oracle.pq_decompress_scores(qabs[i], np.abs(cb), codes, off, ln, cand, qdtype=oracle.F64)
                  for i in range(n_queries)])
    bound = (2.0 ** -11 + 2.0 ** -24 * (2 * D + nq + 2)) * A
    assert np.all(np.abs(got - want) <= bound)


def test_pq_tc_bitwise_repeatable_and_group_independent(cuda_lib):
    """The same query scores the same bits in any group and any position of
    the batch (groups of 2 and of 4; one owner per score)."""
    lengths = synth.lengths_uniform(200, 1, 180, 61)
    cb, codes, _, off, ln = synth.pq_corpus(lengths, M, 256, DSUB, 61)
    Q = synth.queries(7, 32, D, "f16", 61)
    cand = synth.candidates(200, 200, 61, 0)
    a, _ = _gpu(Q, cb, codes, off, ln, cand)
    b, _ = _gpu(Q, cb, codes, off, ln, cand)
    c, _ = _gpu(Q[3:5], cb, codes, off, ln, cand)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(a[3:5].view(np.uint32), c.view(np.uint32))


def test_pq_tc_rejects_unsupported(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    cb = torch.zeros((8, 256, 16), dtype=torch.float32, device="cuda")    # m = 8
    codes = torch.zeros((4, 8), dtype=torch.uint8, device="cuda")
    q = torch.zeros((1, 32, 128), dtype=torch.float16, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    ln = torch.full((1,), 4, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.score_pq_tc_shared(q, cb, codes, off, ln, f)
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED
    cb16 = torch.zeros((16, 256, 8), dtype=torch.float32, device="cuda")
    codes16 = torch.zeros((4, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(tms.TmsError) as e:   # nq > 32
        tms.score_pq_tc_shared(torch.zeros((1, 33, 128), dtype=torch.float16, device="cuda"), cb16, codes16,
                               off, ln, f)
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED
    with pytest.raises(tms.TmsError) as e:   # bf16 queries
        tms.score_pq_tc_shared(q.to(torch.bfloat16), cb16, codes16, off, ln, f)
    assert e.value.status == tms.TMS_ERR_UNSUPPORTED
