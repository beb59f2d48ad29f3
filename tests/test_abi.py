"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/tms.h declares, and rejects invalid arguments on the host before
touching the device."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_2606_26439_gb300 import build as tms_build
from paper_2606_26439_gb300 import tms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared():
    """Every function declared by the headers under include/."""
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(tms_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return tms.lib()


def test_library_built_in_tree(lib):
    assert os.path.dirname(tms_build.LIB) == os.path.join(ROOT, "paper_2606_26439_gb300")
    assert os.path.exists(tms_build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert set(names) == set(tms.EXPORTS), names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert tms.status_string(tms.TMS_OK) == "ok"
    assert "invalid" in tms.status_string(tms.TMS_ERR_INVALID_ARG)
    assert tms.status_string(-99) == "unknown status"
    assert tms.tms_version() >= 100


NULL = None
DUMMY = 0x1000  # 16-byte aligned non-null address; never dereferenced by the host checks


@pytest.mark.parametrize("nq,d,dtype", [(0, 128, 0), (129, 128, 0), (32, 0, 0), (32, 12, 0),
                                        (32, 1032, 0), (32, 128, 7)])
def test_dense_rejects_bad_shapes(lib, nq, d, dtype):
    st = tms.tms_score_dense(DUMMY, dtype, 1, nq, d, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG


def test_dense_rejects_misaligned_and_null(lib):
    st = tms.tms_score_dense(DUMMY + 4, 0, 1, 32, 128, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG
    st = tms.tms_score_dense(DUMMY, 0, 1, 32, 128, NULL, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG
    st = tms.tms_score_dense(DUMMY, 0, 0, 32, 128, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG


def test_dense_empty_candidate_list_is_noop(lib):
    # n_cand == 0: valid, nothing to launch
    st = tms.tms_score_dense(DUMMY, 0, 1, 32, 128, DUMMY, 10, DUMMY, DUMMY, 1, NULL, DUMMY, 0, NULL, NULL)
    assert st == tms.TMS_OK


@pytest.mark.parametrize("m,k", [(3, 256), (16, 300), (64, 256), (16, 0)])
def test_pq_rejects_bad_shapes(lib, m, k):
    st = tms.tms_score_pq(DUMMY, 1, 32, m, k, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st in (tms.TMS_ERR_INVALID_ARG, tms.TMS_ERR_UNSUPPORTED)


@pytest.mark.parametrize("m,k,want", [(4, 256, "unsupported"), (8, 256, "unsupported"), (16, 0, "invalid"),
                                      (32, 256, "unsupported")])
def test_pq_f16_rejects_before_any_device_call(lib, m, k, want):
    """The fp16-table variant takes m in {16, 32} with m * k <= 4096."""
    st = tms.tms_score_pq_f16(DUMMY, 1, 32, m, k, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL)
    assert st == (tms.TMS_ERR_UNSUPPORTED if want == "unsupported" else tms.TMS_ERR_INVALID_ARG)


@pytest.mark.parametrize("args,want", [
    (dict(qdtype=7), "invalid"),                       # not a dtype
    (dict(qdtype=tms.TMS_BF16), "unsupported"),       # fp16 queries only
    (dict(nq=33), "unsupported"),                      # shared lists: nq <= 32
    (dict(m=8, d=64), "unsupported"),                  # M = 16 only
    (dict(d=100), "invalid"),                          # d % m != 0
    (dict(k=257), "invalid"),
    (dict(queries=DUMMY + 8), "invalid"),              # misaligned
    (dict(n_cand=0, cand_ids=None, out=None), "ok"),   # nothing to launch
])
def test_pq_tc_shared_host_checks(lib, args, want):
    a = dict(queries=DUMMY, qdtype=tms.TMS_F16, n_queries=4, nq=32, d=128, codebook=DUMMY, m=16, k=256,
             codes=DUMMY, n_tokens=10, offsets=DUMMY, lengths=DUMMY, n_docs=1, cand_ids=DUMMY, n_cand=1, out=DUMMY)
    a.update(args)
    st = tms.tms_score_pq_tc_shared(a["queries"], a["qdtype"], a["n_queries"], a["nq"], a["d"], a["codebook"], a["m"],
                                    a["k"], a["codes"], a["n_tokens"], a["offsets"], a["lengths"], a["n_docs"],
                                    a["cand_ids"], a["n_cand"], a["out"], NULL)
    assert st == {"invalid": tms.TMS_ERR_INVALID_ARG, "unsupported": tms.TMS_ERR_UNSUPPORTED, "ok": tms.TMS_OK}[want]


def test_pq_lut_rejects_indivisible_d(lib):
    st = tms.tms_build_pq_lut(DUMMY, 0, 1, 32, 100, DUMMY, 16, 256, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG


@pytest.mark.parametrize("k", [0, 1025])
def test_topk_rejects_bad_k(lib, k):
    st = tms.tms_topk(DUMMY, DUMMY, 1, k, DUMMY, DUMMY, NULL)
    assert st == tms.TMS_ERR_INVALID_ARG


def test_get_device_error_rejects_null(lib):
    assert lib.tms_get_device_error(None, ctypes.POINTER(ctypes.c_int)()) == tms.TMS_ERR_INVALID_ARG


def test_server_rejects_bad_config(lib):
    """Config checks happen before any device call (runs without a GPU)."""
    cfg = tms.ServerConfig()
    h = ctypes.c_void_p()
    assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG
    cfg.doc_tokens, cfg.doc_offsets, cfg.doc_lengths = DUMMY, DUMMY, DUMMY
    cfg.dtype, cfg.d, cfg.n_tokens, cfg.n_docs = tms.TMS_F16, 128, 100, 10
    cfg.nq, cfg.topk, cfg.max_batch_requests, cfg.max_batch_candidates, cfg.max_pending = 32, 10, 8, 1000, 16
    for field, bad in (("nq", 0), ("topk", 1025), ("max_batch_requests", 0), ("max_pending", 0), ("d", 12),
                       ("dtype", tms.TMS_F32), ("inject_error_batch", -1), ("max_pending_bytes", -1)):
        good = getattr(cfg, field)
        setattr(cfg, field, bad)
        assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG, field
        setattr(cfg, field, good)
    cfg.rescore_k = 20  # a re-score without an FP8 store
    assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG
    cfg.fp8_codes = DUMMY  # FP8 store without scales
    assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG
    cfg.fp8_scales = DUMMY
    for field, bad in (("rescore_k", 5), ("rescore_k", 1025), ("d", 120)):  # < topk, > 1024, d % 16 != 0
        good = getattr(cfg, field)
        setattr(cfg, field, bad)
        assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG, (field, bad)
        setattr(cfg, field, good)
    cfg.fp8_codes, cfg.fp8_scales, cfg.rescore_k = None, None, 0
    cfg.pq_codes, cfg.pq_codebook, cfg.pq_offsets, cfg.pq_lengths = DUMMY, DUMMY, DUMMY, DUMMY
    cfg.pq_n_tokens, cfg.pq_n_docs, cfg.pq_k = 100, 10, 256
    cfg.pq_m = 12  # unsupported subspace count
    assert lib.tms_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_server_destroy(None) == tms.TMS_ERR_INVALID_ARG
    assert "admission" in tms.status_string(tms.TMS_ERR_BUSY)


def test_tune_dense_rejects_like_score_dense(lib):
    n = ctypes.c_int(-1)
    st = lib.tms_tune_dense(DUMMY, 0, 1, 0, 128, DUMMY, 10, DUMMY, DUMMY, 1, DUMMY, DUMMY, 1, DUMMY, NULL,
                            ctypes.byref(n))
    assert st == tms.TMS_ERR_INVALID_ARG and n.value == 0


def test_debug_set_checks_and_restores(lib):
    """tms_debug_set refuses a negative budget and unknown faults; (0, 0)
    restores the defaults (no device needed)."""
    assert tms.tms_debug_set(-1, 0) == tms.TMS_ERR_INVALID_ARG
    assert tms.tms_debug_set(0, 7) == tms.TMS_ERR_INVALID_ARG
    assert tms.tms_debug_set(1000, tms.TMS_FAULT_HOLD_ACCUMULATOR) == tms.TMS_OK
    assert tms.tms_debug_set(0, 0) == tms.TMS_OK


def test_peak_probes_reject_bad_arguments(lib):
    """The measurement calls check their arguments on the host."""
    g = ctypes.c_double()
    assert lib.tms_peak_shared_load(0, None, ctypes.byref(g)) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_peak_shared_load(10, None, None) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_peak_hbm_read(None, 1 << 20, 1, None, ctypes.byref(g)) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_peak_hbm_read(DUMMY + 8, 1 << 20, 1, None, ctypes.byref(g)) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_peak_hbm_read(DUMMY, 1000, 1, None, ctypes.byref(g)) == tms.TMS_ERR_INVALID_ARG
    assert lib.tms_peak_hbm_read(DUMMY, 1 << 20, 0, None, ctypes.byref(g)) == tms.TMS_ERR_INVALID_ARG
