"""tms_topk_split_noalloc: the split top-k for callers that cannot allocate
device memory (a plugin whose host application owns every device buffer,
or a serving path that makes no cudaMalloc after start-up), with its
scratch in the library's fixed 4 MiB device array.  Called through the C
ABI with raw device pointers and compared with tms_topk_split on the same
scores: positions and scores must be identical (integer results, exact).
Two calls in a row with different shapes check that what the first call
leaves in the shared array never reaches the second.  The file is named so
that pytest collects it last."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _scores(n_queries, per, seed, device):
    """Scores with many exact ties (values on a coarse grid), a few -inf and
    NaN, lists of uneven length in CSR form."""
    import torch
    rng = np.random.default_rng(seed)
    lens = rng.integers(per // 2, per + 1, size=n_queries)
    co = np.zeros(n_queries + 1, np.int64)
    co[1:] = np.cumsum(lens)
    s = (rng.integers(0, 4096, size=int(co[-1])) / 64.0).astype(np.float32)
    s[rng.integers(0, len(s), size=7)] = -np.inf
    s[rng.integers(0, len(s), size=5)] = np.nan
    return torch.from_numpy(s).to(device), torch.from_numpy(co).to(device), int(co[-1])


def _noalloc(lib, scores, co, n_queries, k, n_cand):
    import torch
    out_s = torch.full((n_queries, k), 7.0, dtype=torch.float32, device=scores.device)
    out_p = torch.full((n_queries, k), -7, dtype=torch.int32, device=scores.device)
    st = lib.tms_topk_split_noalloc(scores.data_ptr(), co.data_ptr(), n_queries, k, n_cand, out_s.data_ptr(),
                                    out_p.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out_s, out_p


def test_noalloc_topk_matches_split_topk_on_two_calls(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    for n_queries, per, k, seed in [(16, 100_000, 10, 1), (5, 60_000, 100, 2)]:
        scores, co, n_cand = _scores(n_queries, per, seed, dev)
        st, got_s, got_p = _noalloc(cuda_lib, scores, co, n_queries, k, n_cand)
        assert st == tms.TMS_OK, tms.status_string(st)
        want_s, want_p = tms.topk_split(scores, co, k, n_cand=n_cand)
        torch.cuda.synchronize()
        assert tms.device_error() == 0
        assert torch.equal(got_p, want_p)
        assert torch.equal(got_s.view(torch.int32), want_s.view(torch.int32))


def test_noalloc_topk_refuses_more_than_its_array(cuda_lib):
    import torch
    from paper_2606_26439_gb300 import tms
    n_queries, k = 300, 1024
    n_cand = n_queries * 10_000
    need = tms.topk_workspace_size(n_queries, k, n_cand)
    assert need > 4 * 1024 * 1024
    dev = torch.device("cuda")
    scores = torch.zeros(16, dtype=torch.float32, device=dev)
    co = torch.zeros(n_queries + 1, dtype=torch.int64, device=dev)
    st, _, _ = _noalloc(cuda_lib, scores, co, n_queries, k, n_cand)
    assert st == tms.TMS_ERR_UNSUPPORTED
