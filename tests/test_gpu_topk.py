"""Top-k on the GPU: bit-exact against the oracle's sort on the same fp32
scores (ties by lower position, NaN last, -inf before NaN, padding).  The
split form (tms_topk_split: per-slice top-k into a workspace, then a merge)
runs every case too and must equal the oracle and tms_topk bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


def _run(lists, k, split=False):
    import torch
    from paper_2606_26439_gb300 import tms
    co = np.zeros(len(lists) + 1, np.int64)
    co[1:] = np.cumsum([len(x) for x in lists])
    flat = np.concatenate(lists).astype(np.float32) if co[-1] else np.zeros(1, np.float32)
    s_d, co_d = gc.to_dev(flat, co)
    if split:
        ws = torch.full((max(16, tms.topk_workspace_size(len(lists), k, int(co[-1]))),), 0x5A, dtype=torch.uint8,
                        device="cuda")   # stale contents must not matter
        ts, tp = tms.topk_split(s_d, co_d, k, n_cand=int(co[-1]), workspace=ws)
    else:
        ts, tp = tms.topk(s_d, co_d, k)
    torch.cuda.synchronize()
    assert tms.device_error() == 0
    return ts.cpu().numpy(), tp.cpu().numpy()


def _check(lists, k):
    ts, tp = _run(lists, k)
    ts2, tp2 = _run(lists, k, split=True)
    assert np.array_equal(tp, tp2) and np.array_equal(ts.view(np.uint32), ts2.view(np.uint32))
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


@pytest.mark.parametrize("k", [1, 10, 100, 1024])
def test_topk_split_few_long_lists(cuda_lib, k):
    """The split form's case: few lists, long enough to be cut into many
    slices (ties, NaN and -inf spread over every slice, slice lengths not
    multiples of anything, an empty list and a list shorter than k)."""
    from paper_2606_26439_gb300 import tms
    g = np.random.default_rng(100 + k)
    lists = []
    for n in (250_000, 100_003, 0, max(1, k // 2), 131_071):
        x = np.round(g.standard_normal(n) * 3, 1).astype(np.float32)
        x[g.random(n) < 0.01] = -np.inf
        x[g.random(n) < 0.01] = np.nan
        lists.append(x)
    assert tms.topk_workspace_size(len(lists), k, sum(len(x) for x in lists)) > 0   # really split
    _check(lists, k)


def test_topk_split_all_nan_and_all_equal_across_slices(cuda_lib):
    _check([np.full(200_000, np.nan, np.float32), np.full(150_000, 1.5, np.float32)], 100)


def test_topk_split_workspace_contract(cuda_lib):
    """Too small or misaligned a workspace is refused before anything runs;
    one list of a few scores needs none."""
    import torch
    from paper_2606_26439_gb300 import tms
    n = 300_000
    need = tms.topk_workspace_size(1, 10, n)
    assert need > 0 and tms.topk_workspace_size(1, 10, 500) == 0
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    co = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    ts = torch.empty((1, 10), dtype=torch.float32, device="cuda")
    tp = torch.empty((1, 10), dtype=torch.int32, device="cuda")
    small = torch.empty(need - 8, dtype=torch.uint8, device="cuda")
    st = tms.lib().tms_topk_split(s.data_ptr(), co.data_ptr(), 1, 10, n, ts.data_ptr(), tp.data_ptr(),
                                  small.data_ptr(), need - 8, None)
    assert st == tms.TMS_ERR_INVALID_ARG
    big = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    st = tms.lib().tms_topk_split(s.data_ptr(), co.data_ptr(), 1, 10, n, ts.data_ptr(), tp.data_ptr(),
                                  big.data_ptr() + 8, need, None)
    assert st == tms.TMS_ERR_INVALID_ARG
    st = tms.lib().tms_topk_split(s.data_ptr(), co.data_ptr(), 1, 10, n, ts.data_ptr(), tp.data_ptr(),
                                  big.data_ptr(), need, None)
    assert st == tms.TMS_OK
    torch.cuda.synchronize()
    assert list(tp.cpu().numpy()[0]) == list(range(10))


def test_topk_bad_csr_is_flagged_not_read(cuda_lib):
    """A negative start or a decreasing pair sets TMS_DEVERR_BAD_CSR; the
    list reads as empty (negative start) or clamped (decreasing end)."""
    import torch
    from paper_2606_26439_gb300 import tms
    s = torch.arange(100, dtype=torch.float32, device="cuda")
    for split in (False, True):
        co = torch.tensor([-5, 40, 30, 100], dtype=torch.int64, device="cuda")
        tms.device_error()
        if split:
            ts, tp = tms.topk_split(s, co, 3, n_cand=100)
        else:
            ts, tp = tms.topk(s, co, 3)
        torch.cuda.synchronize()
        assert tms.device_error() & tms.TMS_DEVERR_BAD_CSR
        tp = tp.cpu().numpy()
        assert list(tp[0]) == [-1, -1, -1]          # negative start: empty
        assert list(tp[1]) == [-1, -1, -1]          # 40 > 30: clamped to empty
        assert list(tp[2]) == [69, 68, 67]          # [30, 100): positions within the list
