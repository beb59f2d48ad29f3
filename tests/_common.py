"""Helpers shared by the tests: views of torch tensors as oracle inputs and
the parity tolerances.

Tolerances (per score, relative, with an absolute floor of Nq * 1e-3 times
the relative tolerance for scores near zero):
  * fp16 / bf16 inputs: 1e-3;
  * fp32 inputs:        1e-5;
  * FP8 E4M3 store:     1e-3 against Eq. 1 on the dequantized vectors (the
    E4M3 products are exact in fp32; the error is the fp32 sums and the
    two scale multiplications).
The floor matters only for scores whose magnitude is below Nq * 1e-3; on
unit-normalised data the scores are O(Nq * 0.2).
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL = {"f16": 1e-3, "bf16": 1e-3, "f32": 1e-5, "e4m3": 1e-3}


def oracle_view(t):
    """(numpy array, oracle dtype code) for a torch CPU tensor."""
    import torch
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.float16:
        return t.view(torch.int16).numpy().view(np.uint16), oracle.F16
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16), oracle.BF16
    if t.dtype == torch.float32:
        return t.numpy(), oracle.F32
    if t.dtype == torch.float64:
        return t.numpy(), oracle.F64
    raise TypeError(t.dtype)


def oracle_dense(q, tokens, offsets, lengths, cand_ids):
    qa, qdt = oracle_view(q)
    ta, tdt = oracle_view(tokens)
    return oracle.dense_scores(qa, ta, offsets, lengths, cand_ids, qdtype=qdt, tdtype=tdt)


def assert_scores_close(got, want, dtype: str, nq: int):
    """Element-wise parity: NaN where the oracle has NaN, equal infinities,
    and |got - want| <= rtol * max(|want|, nq * 1e-3) elsewhere."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), "NaN pattern differs"
    inf_w = np.isinf(want)
    assert np.array_equal(got[inf_w], want[inf_w]), "infinite scores differ"
    fin = ~(nan_w | inf_w)
    rtol = RTOL[dtype]
    bound = rtol * np.maximum(np.abs(want[fin]), nq * 1e-3)
    err = np.abs(got[fin] - want[fin])
    if err.size:
        worst = int(np.argmax(err / bound))
        assert np.all(err <= bound), (
            f"max rel-err {err[worst] / max(abs(want[fin][worst]), 1e-30):.3e} "
            f"at {worst}: got {got[fin][worst]!r} want {want[fin][worst]!r}")


def assert_topk_consistent(got_s, got_p, scores_ref, k: int, tol_abs):
    """Top-k parity against reference scores: the returned positions must be
    a valid top-k of ``scores_ref`` up to ties within ``tol_abs``.

    * every returned position is distinct and in range (or -1 padding);
    * the returned list is sorted by the GPU's own scores (desc);
    * a reference score outside the returned set is never larger than the
      k-th reference score in the set by more than tol_abs (no candidate
      that clearly belongs was dropped).
    """
    got_p = np.asarray(got_p)
    n = len(scores_ref)
    valid = got_p[got_p >= 0]
    assert len(valid) == min(k, n)
    assert len(np.unique(valid)) == len(valid)
    ref = np.asarray(scores_ref, np.float64)
    ref_nan_last = np.where(np.isnan(ref), -np.inf, ref)
    chosen = ref_nan_last[valid]
    if len(valid) < n and len(valid) > 0:
        mask = np.ones(n, bool)
        mask[valid] = False
        assert ref_nan_last[mask].max() <= chosen.min() + tol_abs


def _tau(s, rtol, nq):
    return rtol * np.maximum(np.abs(s), nq * 1e-3)


def _tied(a, b, rtol, nq):
    """Elementwise: a and b equal within the parity tolerance of each (both
    NaN, or the same infinity, count as equal)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    both_nan = np.isnan(a) & np.isnan(b)
    same_inf = np.isinf(a) & np.isinf(b) & (a == b)
    fin = np.isfinite(a) & np.isfinite(b)
    with np.errstate(invalid="ignore"):
        close = fin & (np.abs(a - b) <= _tau(a, rtol, nq) + _tau(b, rtol, nq))
    return both_nan | same_inf | close


def assert_topk_matches_oracle(got_pos, want, k: int, dtype: str, nq: int) -> int:
    """Top-k parity against the oracle's own scores, tolerance ties merged.

    ``want`` holds the oracle's scores of the whole list (NaN for bad
    candidates); ``got_pos`` the GPU's top-k positions.  With the oracle's
    ranking o (score desc, position asc, NaN last) and tau(s) = rtol *
    max(|s|, nq * 1e-3) (rtol of ``dtype``):
      * got_pos holds min(k, n) distinct positions of the list, then -1;
      * rank by rank, the GPU's pick and the oracle's candidate are tied
        within tolerance (|s - o_r| <= tau(s) + tau(o_r)): inside a run of
        tolerance-tied oracle scores the GPU may order differently, never
        across runs;
      * no candidate left out beats the weakest pick by more than the
        tolerance (no run is cut except at its tied boundary).
    Returns how many ranks hold exactly the oracle's position.
    """
    import oracle
    rtol = RTOL[dtype]
    want = np.asarray(want, np.float64)
    got_pos = np.asarray(got_pos, np.int64)
    n = len(want)
    m = min(k, n)
    assert got_pos.shape == (k,)
    assert np.all(got_pos[m:] == -1), "padding past the list's length"
    picks = got_pos[:m]
    assert np.all((picks >= 0) & (picks < n)), "position out of range"
    assert len(np.unique(picks)) == m, "repeated position"
    _, opos = oracle.topk(want, k)
    o = want[opos[:m]]
    s = want[picks]
    bad = np.nonzero(~_tied(s, o, rtol, nq))[0]
    assert bad.size == 0, (f"rank {bad[0]}: GPU pick {picks[bad[0]]} (oracle score {s[bad[0]]!r}) is not tied "
                           f"with the oracle's rank-{bad[0]} candidate {opos[bad[0]]} ({o[bad[0]]!r})")
    if m < n:
        rest = np.ones(n, bool)
        rest[picks] = False
        low = np.where(np.isnan(s), -np.inf, s)
        weakest = low.min()
        out = np.where(np.isnan(want[rest]), -np.inf, want[rest])
        if np.isfinite(weakest):
            with np.errstate(invalid="ignore"):
                over = out - weakest - _tau(out, rtol, nq) - _tau(weakest, rtol, nq)
            assert not np.any(over > 0), f"a left-out candidate beats the weakest pick by {over.max():.3e}"
        else:
            assert not np.any(out > weakest), "a left-out candidate beats a -inf / NaN pick"
    return int(np.sum(picks == opos[:m]))
