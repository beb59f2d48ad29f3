"""Top-k on the GPU: bit-exact against the oracle's sort on the same fp32
scores (ties by lower position, NaN last, -inf before NaN, padding)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


def _run(lists, k):
    import torch
    from paper_2606_26439_gb300 import tms
    co = np.zeros(len(lists) + 1, np.int64)
    co[1:] = np.cumsum([len(x) for x in lists])
    flat = np.concatenate(lists).astype(np.float32) if co[-1] else np.zeros(1, np.float32)
    s_d, co_d = gc.to_dev(flat, co)
    ts, tp = tms.topk(s_d, co_d, k)
    torch.cuda.synchronize()
    return ts.cpu().numpy(), tp.cpu().numpy()


def _check(lists, k):
    ts, tp = _run(lists, k)
    for qi, x in enumerate(lists):
        ws, wp = oracle.topk(np.asarray(x, np.float32).astype(np.float64), k)
        assert np.array_equal(tp[qi], wp), (qi, tp[qi][:20], wp[:20])
        same = (ts[qi].astype(np.float64) == ws) | (np.isnan(ts[qi]) & np.isnan(ws))
        assert same.all()


@pytest.mark.parametrize("k", [1, 10, 100, 1024])
def test_topk_random_with_ties_nan_inf(cuda_lib, k):
    g = np.random.default_rng(k)
    lists = []
    for n in (0, 1, 5, k - 1 if k > 1 else 2, k, k + 1, 3000, 100_000):
        x = np.round(g.standard_normal(n) * 4, 1).astype(np.float32)  # many exact ties
        x[g.random(n) < 0.02] = -np.inf
        x[g.random(n) < 0.02] = np.nan
        x[g.random(n) < 0.01] = -0.0
        lists.append(x)
    _check(lists, k)


def test_topk_all_equal_takes_lowest_positions(cuda_lib):
    _check([np.full(5000, 3.25, np.float32), np.full(70, -np.inf, np.float32)], 10)


def test_topk_all_nan(cuda_lib):
    _check([np.full(40, np.nan, np.float32)], 16)


def test_topk_million_scores(cuda_lib):
    g = np.random.default_rng(9)
    lists = [g.standard_normal(1_000_000).astype(np.float32) + 7 for _ in range(3)]
    _check(lists, 100)
