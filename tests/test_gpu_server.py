"""Serving loop (tms_server_*): continuous batching of requests over a
device-resident dense store, PQ store and FP8 copy of the dense store.

* parity: every request's top-k against the FP64 oracle's scores of its
  own candidates (dense: Eq. 1; PQ: decompress-then-dot), within the 1e-3
  tolerance, positions a valid top-k up to tolerance ties;
* FP8 store: with a re-score, the returned scores are the oracle's fp16
  scores of the returned documents and the set is a valid top-k of the
  whole list under those scores (the shortlist kept every document that
  belongs); without one, the scores are Eq. 1 on the E4M3 values (the
  store written by the oracle's quantizer from the same fp16 tokens);
* a request's result is bitwise the same alone (batches of one) and mixed
  with others in large batches;
* admission by pending budget, a host-injected batch failure, bounded
  waits and unknown tickets;
* candidate ids outside the store are refused at submit, on the host;
* submit and wait from different threads at once (the ticket map grows and
  rehashes meanwhile), and two waiters on one ticket: one gets the result.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_cases as gc
from tests._common import assert_topk_consistent, oracle_view

pytestmark = pytest.mark.gpu

NQ, D, TOPK, M, K, DSUB = 32, 128, 10, 16, 256, 8
RESCORE = 40


@pytest.fixture(scope="module")
def stores(cuda_lib):
    import torch
    lengths = synth.lengths_uniform(600, 1, 200, 70)
    tok, off, ln = synth.dense_corpus(600, lengths, D, "f16", 70)
    plen = synth.lengths_uniform(500, 1, 180, 71)
    cb, codes, _, poff, pln = synth.pq_corpus(plen, M, K, DSUB, 71)
    dev = gc.to_dev(tok, off, ln, codes, cb, poff, pln)
    ta, tdt = oracle_view(tok)
    f8c, f8s = oracle.quantize_e4m3(ta, dtype=tdt)
    f8 = gc.to_dev(f8c, f8s)
    torch.cuda.synchronize()
    return dict(tok=tok, off=off, ln=ln, cb=cb, codes=codes, poff=poff, pln=pln, dev=dev, f8c=f8c, f8s=f8s, f8=f8)


def _server(stores, **kw):
    from paper_2606_26439_gb300 import tms
    tok_d, off_d, ln_d, codes_d, cb_d, poff_d, pln_d = stores["dev"]
    args = dict(nq=NQ, topk=TOPK, max_batch_requests=64, max_batch_candidates=200_000, max_pending=256,
                fp8=tuple(stores["f8"]), rescore_k=RESCORE)
    args.update(kw)
    return tms.Server(tok_d, off_d, ln_d, pq=(codes_d, cb_d, poff_d, pln_d), **args)


def _requests(n, seed, n_stores=2):
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        store = int(g.integers(0, n_stores))
        n_docs = 500 if store == 1 else 600
        size = int(g.choice([0, 1, 7, 10, 33, 250, n_docs]))
        cands = g.choice(n_docs, size, replace=False).astype(np.int32)
        q = synth.queries(1, NQ, D, "f16", seed * 1000 + i)[0]
        reqs.append((store, q, cands))
    return reqs


def _oracle_scores(stores, store, q, cands):
    qa, qdt = oracle_view(q)
    if store == 0:
        ta, tdt = oracle_view(stores["tok"])
        return oracle.dense_scores(qa, ta, stores["off"], stores["ln"], cands, qdtype=qdt, tdtype=tdt)
    return oracle.pq_decompress_scores(qa, stores["cb"], stores["codes"], stores["poff"], stores["pln"], cands,
                                       qdtype=qdt)


def test_server_parity_with_oracle(stores):
    reqs = _requests(40, 1)
    with _server(stores) as srv:
        tickets = [srv.submit(q, c, store) for store, q, c in reqs]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["requests"] == len(reqs) and st["rejected"] == 0
    assert st["batches"] >= 1 and st["enqueue_s"] > 0.0
    for (store, q, cands), (sc, ids, lat) in zip(reqs, results):
        want = _oracle_scores(stores, store, q, cands)
        n_valid = min(TOPK, len(cands))
        assert np.all(ids[n_valid:] == -1) and np.all(np.isneginf(sc[n_valid:]))
        if len(cands) == 0:
            continue
        # map the returned ids back to positions of the list (first occurrence)
        pos = np.array([int(np.nonzero(cands == i)[0][0]) for i in ids[:n_valid]])
        tol = 2e-3 * max(1.0, np.nanmax(np.abs(want)))
        assert_topk_consistent(sc[:n_valid], pos, want, TOPK, tol)
        fin = np.isfinite(want[pos])
        assert np.all(np.abs(sc[:n_valid][fin] - want[pos][fin]) <= 1e-3 * np.maximum(np.abs(want[pos][fin]),
                                                                                       NQ * 1e-3))
        assert lat > 0


def test_alone_equals_mixed(stores):
    reqs = _requests(48, 2, n_stores=3)
    with _server(stores, max_batch_requests=1) as srv:   # every request alone
        alone = [srv.wait(srv.submit(q, c, s))[:2] for s, q, c in reqs]
    with _server(stores, max_batch_requests=64) as srv:  # all submitted at once, batched
        tickets = [srv.submit(q, c, s) for s, q, c in reqs]
        mixed = [srv.wait(t)[:2] for t in tickets]
        assert srv.stats()["batches"] < len(reqs)
    for (sa, ia), (sm, im) in zip(alone, mixed):
        assert np.array_equal(sa.view(np.uint32), sm.view(np.uint32))
        assert np.array_equal(ia, im)


def test_admission_budget(stores):
    from paper_2606_26439_gb300 import tms
    reqs = _requests(30, 3)
    with _server(stores, max_pending=2, max_batch_requests=1) as srv:
        tickets, busy = [], 0
        for s, q, c in reqs:
            try:
                tickets.append(srv.submit(q, c, s))
            except tms.TmsError as e:
                assert e.status == tms.TMS_ERR_BUSY
                busy += 1
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["rejected"] == busy and st["requests"] == len(tickets)
    assert len(tickets) >= 2


def test_admission_by_device_bytes(stores):
    """A byte budget for admitted-but-unfinished requests (query + 8 bytes
    per candidate): past it submit answers BUSY, a request larger than the
    whole budget is refused outright, and admitted work still completes."""
    from paper_2606_26439_gb300 import tms
    q = synth.queries(1, NQ, D, "f16", 31)[0]
    qbytes = NQ * D * 2
    cands = np.random.default_rng(31).integers(0, 600, 500).astype(np.int32)
    one = qbytes + 8 * len(cands)
    with _server(stores, max_batch_requests=1, max_pending_bytes=3 * one) as srv:
        with pytest.raises(tms.TmsError) as e:      # alone over the budget
            srv.submit(q, np.zeros(3 * one // 8, np.int32))
        assert e.value.status == tms.TMS_ERR_UNSUPPORTED
        tickets, busy = [], 0
        for _ in range(40):
            try:
                tickets.append(srv.submit(q, cands))
            except tms.TmsError as err:
                assert err.status == tms.TMS_ERR_BUSY
                busy += 1
        assert busy > 0 and len(tickets) >= 3
        results = [srv.wait(t) for t in tickets]
        assert all(np.array_equal(r[1], results[0][1]) for r in results)
        st = srv.stats()
        assert st["rejected"] == busy and st["requests"] == len(tickets)
        srv.wait(srv.submit(q, cands))   # the budget is free again


def test_injected_batch_failure_is_reported(stores):
    from paper_2606_26439_gb300 import tms
    reqs = _requests(6, 4)
    with _server(stores, max_batch_requests=1, inject_error_batch=2) as srv:
        statuses = []
        for s, q, c in reqs:
            try:
                srv.wait(srv.submit(q, c, s))
                statuses.append(tms.TMS_OK)
            except tms.TmsError as e:
                statuses.append(e.status)
    assert statuses[1] == tms.TMS_ERR_CUDA
    assert all(st == tms.TMS_OK for i, st in enumerate(statuses) if i != 1)


def test_bounded_wait_unknown_ticket_and_oversize(stores):
    from paper_2606_26439_gb300 import tms
    big = np.random.default_rng(5).integers(0, 600, 150_000).astype(np.int32)
    q = synth.queries(1, NQ, D, "f16", 5)[0]
    with _server(stores) as srv:
        with pytest.raises(tms.TmsError) as e:
            srv.wait(12345)
        assert e.value.status == tms.TMS_ERR_INVALID_ARG
        with pytest.raises(tms.TmsError) as e:
            srv.submit(q, np.zeros(200_001, np.int32))
        assert e.value.status == tms.TMS_ERR_UNSUPPORTED
        tickets = [srv.submit(q, big) for _ in range(8)]
        with pytest.raises(tms.TmsError) as e:
            srv.wait(tickets[-1], timeout_s=0.0)
        assert e.value.status == tms.TMS_ERR_TIMEOUT
        for t in tickets:                 # still waitable after a timeout
            srv.wait(t)


def _fp8_oracle_scores(stores, q, cands):
    qa, qdt = oracle_view(q[None])
    qc, qs = oracle.quantize_e4m3(qa.reshape(NQ, D), dtype=qdt)
    return oracle.dense_scores_scaled(qc, qs, stores["f8c"], stores["f8s"], stores["off"], stores["ln"], cands,
                                      qdtype=oracle.E4M3, tdtype=oracle.E4M3)


@pytest.mark.parametrize("rescore", [RESCORE, 0])
def test_server_fp8_store(stores, rescore):
    """FP8 requests: with a re-score the results are exact fp16 scores of a
    valid top-k; without one they are the FP8 scores of a valid top-k."""
    from paper_2606_26439_gb300 import tms
    g = np.random.default_rng(7 + rescore)
    reqs = []
    for i in range(30):
        size = int(g.choice([0, 1, 9, 10, 11, 40, 41, 300, 600]))
        cands = g.choice(600, size, replace=False).astype(np.int32)
        reqs.append((synth.queries(1, NQ, D, "f16", 900 + i)[0], cands))
    with _server(stores, rescore_k=rescore) as srv:
        results = [srv.wait(srv.submit(q, c, tms.TMS_STORE_FP8)) for q, c in reqs]
    for (q, cands), (sc, ids, _) in zip(reqs, results):
        n_valid = min(TOPK, len(cands))
        assert np.all(ids[n_valid:] == -1) and np.all(np.isneginf(sc[n_valid:]))
        if len(cands) == 0:
            continue
        want = _oracle_scores(stores, 0, q, cands) if rescore else _fp8_oracle_scores(stores, q, cands)
        pos = np.array([int(np.nonzero(cands == i)[0][0]) for i in ids[:n_valid]])
        tol = 2e-3 * max(1.0, np.nanmax(np.abs(want)))
        assert_topk_consistent(sc[:n_valid], pos, want, TOPK, tol)
        fin = np.isfinite(want[pos])
        assert np.array_equal(np.isnan(sc[:n_valid]), np.isnan(want[pos]))
        assert np.all(np.abs(sc[:n_valid][fin] - want[pos][fin]) <= 1e-3 * np.maximum(np.abs(want[pos][fin]),
                                                                                       NQ * 1e-3))


def test_server_fp8_rescore_uses_fp16_scores(stores):
    """A re-scored FP8 request returns the same scores and ids as the same
    request to the dense store whenever the dense top-k is inside the FP8
    shortlist -- here a list no longer than the shortlist, so always."""
    from paper_2606_26439_gb300 import tms
    q = synth.queries(1, NQ, D, "f16", 77)[0]
    cands = np.random.default_rng(77).choice(600, RESCORE, replace=False).astype(np.int32)
    with _server(stores) as srv:
        s8, i8, _ = srv.wait(srv.submit(q, cands, tms.TMS_STORE_FP8))
        sd, idd, _ = srv.wait(srv.submit(q, cands, tms.TMS_STORE_DENSE))
    assert np.array_equal(s8.view(np.uint32), sd.view(np.uint32))
    assert np.array_equal(i8, idd)


def test_bad_ids_refused_on_host(stores):
    """An id outside [0, n_docs) of the request's store is refused by submit
    with TMS_ERR_INVALID_ARG: nothing is admitted, nothing reaches the
    device, and the device error word stays clear."""
    from paper_2606_26439_gb300 import tms
    q = synth.queries(1, NQ, D, "f16", 41)[0]
    tms.device_error()  # start from a clear word
    with _server(stores) as srv:
        for store, bad in ((tms.TMS_STORE_DENSE, 600), (tms.TMS_STORE_DENSE, -1), (tms.TMS_STORE_PQ, 500),
                           (tms.TMS_STORE_PQ, -7), (tms.TMS_STORE_FP8, 600), (tms.TMS_STORE_FP8, 2 ** 31 - 1)):
            cands = np.array([3, 4, bad, 5], np.int32)
            with pytest.raises(tms.TmsError) as e:
                srv.submit(q, cands, store)
            assert e.value.status == tms.TMS_ERR_INVALID_ARG
        # PQ ids up to 499 are valid on the PQ store, 500..599 only on the dense one
        srv.wait(srv.submit(q, np.array([0, 499], np.int32), tms.TMS_STORE_PQ))
        srv.wait(srv.submit(q, np.array([0, 599], np.int32), tms.TMS_STORE_DENSE))
        st = srv.stats()
    assert st["requests"] == 2 and st["rejected"] == 0
    assert tms.device_error() == 0


def test_submit_while_waiting(stores):
    """One thread submits 600 requests while the main thread waits for each
    ticket as soon as it exists: the server's ticket map grows (and rehashes)
    while waiters hold their lookups.  Every result equals the same request
    run alone."""
    import threading
    reqs = []
    g = np.random.default_rng(43)
    for i in range(600):
        store = i % 3
        n_docs = 500 if store == 1 else 600
        cands = g.choice(n_docs, int(g.integers(1, 60)), replace=False).astype(np.int32)
        reqs.append((store, synth.queries(1, NQ, D, "f16", 43_000 + i)[0], cands))
    with _server(stores, max_batch_requests=1) as srv:
        alone = [srv.wait(srv.submit(q, c, s))[:2] for s, q, c in reqs[:60]]
    tickets = [None] * len(reqs)
    ready = [threading.Event() for _ in reqs]
    errors = []
    with _server(stores, max_batch_requests=64, max_pending=1024) as srv:
        def producer():
            try:
                for i, (s, q, c) in enumerate(reqs):
                    tickets[i] = srv.submit(q, c, s)
                    ready[i].set()
            except Exception as e:  # surfaced below
                errors.append(e)
                for ev in ready:
                    ev.set()
        th = threading.Thread(target=producer)
        th.start()
        results = []
        for i in range(len(reqs)):
            assert ready[i].wait(60)
            assert not errors, errors
            results.append(srv.wait(tickets[i])[:2])
        th.join()
    assert not errors, errors
    for (sa, ia), (sm, im) in zip(alone, results[:60]):
        assert np.array_equal(sa.view(np.uint32), sm.view(np.uint32))
        assert np.array_equal(ia, im)
    for (s, q, c), (sm, im) in zip(reqs, results):
        n_valid = min(TOPK, len(c))
        assert np.all(np.isin(im[:n_valid], c)) and np.all(im[n_valid:] == -1)


def test_two_waiters_one_ticket(stores):
    """Two threads wait on the same ticket: one takes the result, the other
    is told the ticket is no longer known (a result is handed out once)."""
    import threading
    from paper_2606_26439_gb300 import tms
    q = synth.queries(1, NQ, D, "f16", 45)[0]
    big = np.random.default_rng(45).integers(0, 600, 150_000).astype(np.int32)
    with _server(stores) as srv:
        blockers = [srv.submit(q, big) for _ in range(4)]   # keep the GPU busy for a while
        t = srv.submit(q, np.arange(50, dtype=np.int32))
        outcome = []

        def waiter():
            try:
                srv.wait(t)
                outcome.append("ok")
            except tms.TmsError as e:
                outcome.append(e.status)
        ths = [threading.Thread(target=waiter) for _ in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for b in blockers:
            srv.wait(b)
    assert sorted(outcome, key=str) == sorted(["ok", tms.TMS_ERR_INVALID_ARG], key=str)
