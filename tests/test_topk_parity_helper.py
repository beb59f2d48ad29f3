"""CPU checks of the tie-merged top-k comparison used by the GPU parity
tests: it accepts the oracle's own ranking and swaps inside a tolerance tie,
and it rejects the mistakes a top-k kernel could make (a dropped winner, a
swap across a clear gap, a repeated position, wrong padding)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests._common import assert_topk_matches_oracle


def _scores():
    g = np.random.default_rng(3)
    s = 6.0 + g.standard_normal(500)
    s[10] = 20.0          # a clear winner
    s[11] = 19.0          # a clear second
    s[20], s[21] = 15.0, 15.0 + 1e-4   # a tolerance tie (1e-3 relative of 15 is 0.015)
    s[30] = np.nan
    return s


def test_accepts_oracle_ranking():
    s = _scores()
    _, p = oracle.topk(s, 10)
    assert assert_topk_matches_oracle(p, s, 10, "f16", 32) == 10


def test_accepts_swap_inside_tie():
    s = _scores()
    _, p = oracle.topk(s, 10)
    p = p.copy()
    i, j = list(p).index(21), list(p).index(20)
    p[i], p[j] = p[j], p[i]
    assert assert_topk_matches_oracle(p, s, 10, "f16", 32) == 8


@pytest.mark.parametrize("mistake", ["drop_winner", "swap_gap", "repeat", "pad", "fp32_tolerance"])
def test_rejects_mistakes(mistake):
    s = _scores()
    _, p = oracle.topk(s, 10)
    p = p.copy()
    dtype = "f16"
    if mistake == "drop_winner":
        p[0] = int(np.argsort(s)[250])   # a middling candidate instead of the winner
    elif mistake == "swap_gap":
        p[0], p[1] = p[1], p[0]          # 20 vs 19: far outside the tolerance
    elif mistake == "repeat":
        p[5] = p[4]
    elif mistake == "pad":
        p[9] = -1
    elif mistake == "fp32_tolerance":
        s[21] = 15.0 + 1e-3              # tied at 1e-3, not at 1e-5
        _, p = oracle.topk(s, 10)
        p = p.copy()
        i, j = list(p).index(21), list(p).index(20)
        p[i], p[j] = p[j], p[i]
        dtype = "f32"
    with pytest.raises(AssertionError):
        assert_topk_matches_oracle(p, s, 10, dtype, 32)


def test_short_list_and_nan_last():
    s = np.array([1.0, np.nan, 3.0, -np.inf])
    _, p = oracle.topk(s, 6)
    assert list(p) == [2, 0, 3, 1, -1, -1]
    assert assert_topk_matches_oracle(p, s, 6, "f16", 4) == 4
    with pytest.raises(AssertionError):
        assert_topk_matches_oracle(np.array([2, 0, 1, 3, -1, -1]), s, 6, "f16", 4)
