#!/usr/bin/env python3
"""Benchmark of the MaxSim scoring path on GB300.

Workload (the headline): dense MaxSim at scale -- 500,000 packed documents
with Nd ~ uniform integer [32, 180], d = 128, fp16 unit-normalised
Gaussian embeddings (13.6 GB resident in HBM, far larger than the 129 MB
L2, so no flush is needed between steps); 16 queries of Nq = 32 tokens,
each scoring its own random 100,000-document candidate subset.  One step
= one tms_score_dense launch over all 16 x 100,000 candidates plus the
top-10 per query by tms_topk_split (per-slice top-k into a workspace
allocated once, then a per-query merge: two launches).  Metric: documents
scored per second.

Also reported (N = 1 only): config 1 (one query over 10,000 documents of
128 tokens, three corpus copies rotated so that L2 holds none of the copy a
launch reads), measured ceilings (shared-memory load and HBM read
bandwidth), the same workload in bf16, fp32 and on the
FP8 E4M3 store (per-token scales), dimension tiling at d = 64/256/512/768
(200,000 docs, 32 queries over all of them, bf16, top-100; per-query and
shared-candidate schedules), the FP8 store at 1,000,000 docs with 64
queries over all of them (throughput, error and top-10 overlap against the
fp16 scorer, with and without an fp16 re-score of the FP8 top-100),
fused PQ (1,000,000 docs, M = 16, K = 256, 64 queries over all of them:
fp32 table, fp16 table, and codes decompressed in shared memory on the
tensor cores), the serving loop on a mixed dense + PQ request stream
(p50 / p99 latency and docs/s, batched against one request per launch),
and the served FP8 form (batched, fp16 re-score of each request's top 100)
against one fp16 request per launch, with top-10 overlap.  The headline
line also carries the per-step time distribution (median, p10, p90 over
the K steps) and the oracle's rate on all host cores and on one thread.

The oracle leg of the secondary rows: for one query per configuration
(config 1 in full; query 0's 100,000 candidates per dtype of config 2;
query 0 over all 200,000 documents per d of config 3; query 0 over all
1,000,000 documents for PQ and for the FP8 store) the FP64 oracle scores the
whole list on the host cores.  Its time is reported (docs/s, cores), and
the GPU's scores and top-k of that query are compared with it: relative
error (max, mean) and top-k overlap -- for the FP8 store against the oracle
of the fp16 corpus it was quantized from, i.e. the store's whole error.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tms|reference]

``--impl reference`` times the FP64 CPU oracle on this host's cores on
bounded samples of the same workload (the one reference this project has).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2606_26439_gb300 import iomodel  # noqa: E402

N_DOCS, LO, HI, D, NQ, N_QUERIES, N_CAND, TOPK = 500_000, 32, 180, 128, 32, 16, 100_000, 10
METRIC = "docs scored/sec"
WORKLOAD = ("dense MaxSim at scale: 500,000 docs, Nd~U[32,180], d=128, packed; "
            "16 queries Nq=32 x 100,000-doc random candidate subsets; top-10")
KERNEL_SRC = os.path.join(ROOT, "paper_2606_26439_gb300", "csrc", "tms_dense_tc.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dense_tc_kernel_500k_docs_fp16.txt")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["tms", "reference"], default="tms")
    p.add_argument("--no-rows", action="store_true", help="skip the secondary workloads")
    p.add_argument("--workload", choices=["headline", "small"], default="headline",
                   help="small: 100,000 docs, 1 query x 100,000 candidates (sized for ncu captures)")
    p.add_argument("--profile-case", choices=["fp8_small", "f32_small", "d64_small", "pq_small", "pq16_small", "pqtc_small",
                                              "shared_small", "shared64_small", "shared768_small"],
                   default=None,
                   help="run only one small secondary kernel (sized for ncu captures) and print its timing")
    args = p.parse_args()
    if args.workload == "small":
        global N_DOCS, N_QUERIES, WORKLOAD
        N_DOCS, N_QUERIES = 100_000, 1
        WORKLOAD = ("dense MaxSim, small profiling case: 100,000 docs, Nd~U[32,180], d=128, packed; "
                    "1 query Nq=32 x 100,000 candidates; top-10")
        args.no_rows = True
    return args


# ------------------------------------------------------------------ helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def kernel_sha():
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic_per_token():
    """DRAM bytes per processed document token for the dense kernel, from the
    committed ncu summary -- None if absent or taken on another source."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != kernel_sha():
            return None
        return float(kv["dram_bytes_per_token"])
    except Exception:
        return None


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[3:7]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "tms" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX)


def replica_rate(units, ms, ws):
    """Whole-job rate of independent replicas: the units every rank
    processed divided by the slowest rank's time.  Returns (units/s, max ms)."""
    import torch.distributed as dist
    total = _reduce(float(units), ws, dist.ReduceOp.SUM)
    ms_max = _reduce(ms, ws, dist.ReduceOp.MAX)
    return total / (ms_max * 1e-3), ms_max


# --------------------------------------------------------------- workloads

def headline_inputs(seed=0):
    lengths = synth.lengths_uniform(N_DOCS, LO, HI, seed)
    cands = [synth.candidates(N_DOCS, N_CAND, seed, q) for q in range(N_QUERIES)]
    return lengths, cands


def cpu_sample(lengths, cands, n_sample, seed=1):
    """Host copy of a bounded sample of the headline workload: the first
    n_sample candidates of query 0, their documents generated on the host
    with the same recipe (same lengths, same distribution)."""
    ids = cands[0][:n_sample]
    sub_len = lengths[ids]
    import torch
    tok, off, ln = synth.dense_corpus(len(ids), sub_len, D, "f16", seed)
    Q = synth.queries(1, NQ, D, "f16", seed)
    q = Q[0].view(torch.int16).numpy().view(np.uint16)
    t = tok.view(torch.int16).numpy().view(np.uint16)
    return q, t, off, ln, np.arange(len(ids), dtype=np.int32)


def time_oracle(lengths, cands, target_s, threads=None):
    """Docs/s of the FP64 oracle on this host's cores (calibrated sample),
    on `threads` threads (default: all)."""
    import oracle
    cores = oracle.max_threads()
    oracle.set_threads(threads or cores)
    try:
        q, t, off, ln, c = cpu_sample(lengths, cands, 300)
        t0 = time.perf_counter()
        oracle.dense_scores(q, t, off, ln, c, qdtype=oracle.F16, tdtype=oracle.F16)
        rate = len(c) / (time.perf_counter() - t0)
        n = int(max(300, min(N_CAND, rate * target_s)))
        q, t, off, ln, c = cpu_sample(lengths, cands, n)
        t0 = time.perf_counter()
        oracle.dense_scores(q, t, off, ln, c, qdtype=oracle.F16, tdtype=oracle.F16)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return n / dt, n, dt, threads or cores


def rows_of(off, lengths, ids):
    """Token rows of documents ``ids`` in order, as one index array."""
    lens = np.asarray(lengths, np.int64)[ids]
    starts = np.asarray(off, np.int64)[ids]
    before = np.concatenate([[0], np.cumsum(lens)[:-1]])
    return np.repeat(starts - before, lens) + np.arange(int(lens.sum()), dtype=np.int64)


def host_docs(rows_d, off, lengths, ids):
    """Host copy of documents ``ids`` of a device row array, repacked for the
    oracle: (rows as numpy, offsets, lengths)."""
    import torch
    lens = np.asarray(lengths, np.int32)[ids]
    if len(ids) == len(lengths) and np.array_equal(ids, np.arange(len(lengths))):
        sub, sub_off = rows_d.cpu(), np.asarray(off, np.int64)
    else:
        sub = rows_d[torch.from_numpy(rows_of(off, lengths, ids)).to(rows_d.device)].cpu()
        sub_off = synth.offsets_of(lens)
    if sub.dtype in (torch.float16, torch.bfloat16):
        sub = sub.view(torch.int16).numpy().view(np.uint16)
    else:
        sub = sub.numpy()
    return sub, sub_off, lens


def _odt(dtype):
    import oracle
    return {"f16": oracle.F16, "bf16": oracle.BF16, "f32": oracle.F32}[dtype]


def oracle_dense_query(q, dtype, tok_d, off, lengths, ids):
    """The oracle leg: FP64 Eq. 1 of one query (host tensor [nq][d]) over a
    whole candidate list of a device corpus, on all host cores.  Returns
    (scores, seconds of oracle arithmetic)."""
    import oracle
    import torch
    sub, sub_off, lens = host_docs(tok_d, off, lengths, ids)
    qh = q.contiguous()
    qa = qh.view(torch.int16).numpy().view(np.uint16) if qh.dtype in (torch.float16, torch.bfloat16) else qh.numpy()
    t0 = time.perf_counter()
    want = oracle.dense_scores(qa, sub, sub_off, lens, np.arange(len(ids), dtype=np.int32),
                               qdtype=_odt(dtype), tdtype=_odt(dtype))
    return want, time.perf_counter() - t0


def quality_vs_oracle(got, want, gpu_top, k):
    """GPU scores of one query against the oracle's scores of the same list:
    relative error (floor Nq 1e-3, the parity tests' rule), the overlap of the
    GPU's top-k (positions from tms_topk) with the oracle's own top-k, and
    how many ranks hold the same position."""
    import oracle
    got = np.asarray(got, np.float64)
    fin = np.isfinite(want)
    rel = np.abs(got[fin] - want[fin]) / np.maximum(np.abs(want[fin]), NQ * 1e-3)
    _, wp = oracle.topk(want, k)
    gp = np.asarray(gpu_top)[:k]
    return {"rel_err_max": float(rel.max()), "rel_err_mean": float(rel.mean()),
            f"top{k}_overlap": len(set(gp.tolist()) & set(wp.tolist())) / k,
            f"top{k}_same_rank": int(np.sum(gp == wp))}


def oracle_timing(n_docs, seconds):
    import oracle
    return {"docs": int(n_docs), "seconds": seconds, "docs_per_s": n_docs / seconds, "cores": oracle.max_threads()}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    lengths, cands = headline_inputs()
    # calibrate so that warmup + steps stay within ~2 minutes
    q, t, off, ln, c = cpu_sample(lengths, cands, 200)
    t0 = time.perf_counter()
    oracle.dense_scores(q, t, off, ln, c, qdtype=oracle.F16, tdtype=oracle.F16)
    rate = len(c) / (time.perf_counter() - t0)
    per_step_s = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    n = int(max(16, min(N_CAND, rate * per_step_s)))
    q, t, off, ln, c = cpu_sample(lengths, cands, n)
    for _ in range(args.warmup):
        oracle.dense_scores(q, t, off, ln, c, qdtype=oracle.F16, tdtype=oracle.F16)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dense_scores(q, t, off, ln, c, qdtype=oracle.F16, tdtype=oracle.F16)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = n / dt
    sample = f"first {n} candidates of query 0 per step (Nq=32, d=128, fp16 stored values, FP64 arithmetic)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "docs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (plain C + OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "docs/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "docs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def dense_workload(dtype, lengths, cands, device):
    import torch
    tok_d, off_d, ln_d = synth.device_dense_corpus(lengths, D, dtype, 0, device)
    Q = synth.queries(N_QUERIES, NQ, D, dtype, 0)
    flat = np.concatenate(cands).astype(np.int32)
    co = np.zeros(N_QUERIES + 1, np.int64)
    co[1:] = np.cumsum([len(c) for c in cands])
    return dict(tok=tok_d, off=off_d, ln=ln_d, Q=Q, q=Q.to(device), flat=flat, co=co,
                f=torch.from_numpy(flat).to(device), c=torch.from_numpy(co).to(device),
                tokens=int(lengths[flat].astype(np.int64).sum()))


def topk_workspace(n_cand, device):
    """The split top-k's workspace for the headline launch, allocated once."""
    import torch
    from paper_2606_26439_gb300 import tms
    return torch.empty(max(16, tms.topk_workspace_size(N_QUERIES, TOPK, n_cand)), dtype=torch.uint8, device=device)


def time_dense(w, steps, warmup, stream):
    """Device-resident steps: (ms per step, dense-kernel ms per launch,
    scores, per-step ms -- consecutive step-boundary events on the stream)."""
    import torch
    from paper_2606_26439_gb300 import tms
    out = torch.empty(len(w["flat"]), dtype=torch.float32, device=w["q"].device)
    ts = torch.empty((N_QUERIES, TOPK), dtype=torch.float32, device=w["q"].device)
    tp = torch.empty((N_QUERIES, TOPK), dtype=torch.int32, device=w["q"].device)
    ws = topk_workspace(len(w["flat"]), w["q"].device)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        tms.score_dense(w["q"], w["tok"], w["off"], w["ln"], w["f"], w["c"], out=out, stream=stream)
        if evs is not None:
            evs[1].record(stream)
        tms.topk_split(out, w["c"], TOPK, n_cand=len(w["flat"]), out_scores=ts, out_pos=tp, workspace=ws,
                       stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            sev[i].record(stream)
            step(kev[i])
        sev[steps].record(stream)
    torch.cuda.synchronize()
    total = sev[0].elapsed_time(sev[steps])
    kern = [a.elapsed_time(b) for a, b in kev]
    per_step = [sev[i].elapsed_time(sev[i + 1]) for i in range(steps)]
    return total / steps, statistics.mean(kern), out, per_step


def time_dense_e2e(w, steps, warmup, stream):
    """End to end through the public API from pinned host buffers: per step
    H2D of the queries, candidate ids and CSR offsets, both launches, and
    D2H of all scores and the top-k."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = w["q"].device
    hq = w["Q"].contiguous().pin_memory()
    hf = torch.from_numpy(w["flat"]).pin_memory()
    hc = torch.from_numpy(w["co"]).pin_memory()
    q = torch.empty_like(hq, device=dev)
    f = torch.empty_like(hf, device=dev)
    c = torch.empty_like(hc, device=dev)
    out = torch.empty(len(w["flat"]), dtype=torch.float32, device=dev)
    ts = torch.empty((N_QUERIES, TOPK), dtype=torch.float32, device=dev)
    tp = torch.empty((N_QUERIES, TOPK), dtype=torch.int32, device=dev)
    hs = torch.empty(len(w["flat"]), dtype=torch.float32).pin_memory()
    hts = torch.empty((N_QUERIES, TOPK), dtype=torch.float32).pin_memory()
    htp = torch.empty((N_QUERIES, TOPK), dtype=torch.int32).pin_memory()
    ws = topk_workspace(len(w["flat"]), dev)

    def step():
        q.copy_(hq, non_blocking=True)
        f.copy_(hf, non_blocking=True)
        c.copy_(hc, non_blocking=True)
        tms.score_dense(q, w["tok"], w["off"], w["ln"], f, c, out=out, stream=stream)
        tms.topk_split(out, c, TOPK, n_cand=len(w["flat"]), out_scores=ts, out_pos=tp, workspace=ws, stream=stream)
        hs.copy_(out, non_blocking=True)
        hts.copy_(ts, non_blocking=True)
        htp.copy_(tp, non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
    torch.cuda.synchronize()
    h2d = hq.numel() * hq.element_size() + hf.numel() * 4 + hc.numel() * 8
    d2h = hs.numel() * 4 + hts.numel() * 4 + htp.numel() * 4
    return e0.elapsed_time(e1) / steps, h2d, d2h


def time_launch(fn, stream, reps, warmup=2):
    """Mean CUDA-event time (ms) of `fn` launched `reps` times on `stream`."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def fp8_store_row(stream, hbm_peak):
    """1,000,000 docs (Nd~U[32,180], d=128) quantized to the FP8 store; 64
    fp16 queries, each over every document, in the shared schedule.
    Throughput of the FP8 pass, and its quality against the fp16 tensor-core
    scorer on the same documents (itself within 1e-3 of FP64 in the parity
    tests): relative score error over all 64M scores, overlap of the top-10,
    and the overlap after re-scoring the FP8 top-100 with the fp16 scorer.
    Query 0 is also scored over all documents by the FP64 oracle: the FP8
    scores' error and top-10 overlap against it (raw and re-scored)."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    n, nQ, k_short = 1_000_000, 64, 100
    lens = synth.lengths_uniform(n, LO, HI, 4)
    tok, off, ln = synth.device_dense_corpus(lens, D, "f16", 4, dev)
    Q = synth.queries(nQ, NQ, D, "f16", 4).to(dev)
    tc, tsc = tms.quantize_e4m3(tok)
    qc, qsc = tms.quantize_e4m3(Q)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    co = torch.arange(0, (nQ + 1) * n, n, dtype=torch.int64, device=dev)
    s8 = torch.empty((nQ, n), dtype=torch.float32, device=dev)
    s16 = torch.empty((nQ, n), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(2):
            tms.score_fp8_shared(qc, qsc, tc, tsc, off, ln, ids, out=s8, stream=stream)
        tms.score_dense_shared(Q, tok, off, ln, ids, out=s16, stream=stream)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = 3
    with torch.cuda.stream(stream):
        e[0].record(stream)
        for _ in range(reps):
            tms.score_fp8_shared(qc, qsc, tc, tsc, off, ln, ids, out=s8, stream=stream)
        e[1].record(stream)
        for _ in range(reps):
            tms.score_dense_shared(Q, tok, off, ln, ids, out=s16, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    ms8 = e[0].elapsed_time(e[1]) / reps
    ms16 = e[1].elapsed_time(e[2]) / reps
    tok_total = int(lens.astype(np.int64).sum())
    # quality against the fp16 scorer
    rel = ((s8 - s16).abs() / s16.abs().clamp_min(1e-6))
    t8s, t8p = tms.topk(s8.view(-1), co, k_short)
    t16s, t16p = tms.topk(s16.view(-1), co, TOPK)
    torch.cuda.synchronize()
    top10_8 = t8p[:, :TOPK].cpu().numpy()
    top10_16 = t16p.cpu().numpy()
    overlap = float(np.mean([len(set(a) & set(b)) / TOPK for a, b in zip(top10_8, top10_16)]))
    # two-stage: re-score the FP8 top-100 (positions are document ids here) in fp16
    short = t8p.reshape(-1).contiguous()
    sco = torch.arange(0, (nQ + 1) * k_short, k_short, dtype=torch.int64, device=dev)
    rs = tms.score_dense(Q, tok, off, ln, short, sco)
    rts, rtp = tms.topk(rs, sco, TOPK)
    torch.cuda.synchronize()
    short_np = short.view(nQ, k_short).cpu().numpy()
    top10_rs = np.take_along_axis(short_np, rtp.cpu().numpy().astype(np.int64), axis=1)
    overlap_rs = float(np.mean([len(set(a) & set(b)) / TOPK for a, b in zip(top10_rs, top10_16)]))
    # the oracle leg: query 0 over all 1,000,000 documents in FP64 on the fp16
    # corpus the store was quantized from
    want0, secs = oracle_dense_query(Q[0].cpu(), "f16", tok, synth.offsets_of(lens), lens, np.arange(n))
    rescored = quality_vs_oracle(s16[0].cpu().numpy(), want0, top10_rs[0], TOPK)
    vs_oracle = {"fp8": quality_vs_oracle(s8[0].cpu().numpy(), want0, top10_8[0], TOPK),
                 "fp8_rescored_top100": {k: v for k, v in rescored.items() if k.startswith("top")},
                 "fp16": quality_vs_oracle(s16[0].cpu().numpy(), want0, top10_16[0], TOPK)}
    fl = iomodel.dense_alg_flops(tok_total * nQ, NQ, D)
    row = {"vs_fp64_oracle_query0": vs_oracle, "oracle_query0": oracle_timing(n, secs),
           "docs_per_s": nQ * n / (ms8 * 1e-3), "kernel_ms": ms8, "fp16_shared_kernel_ms": ms16,
           "speedup_vs_fp16": ms16 / ms8, "tflops": fl / (ms8 * 1e-3) / 1e12,
           "store_reads_gbs": tok_total * (D + 4) * (nQ // 8) / (ms8 * 1e-3) / 1e9,
           "rel_err_vs_fp16_mean": float(rel.mean()), "rel_err_vs_fp16_max": float(rel.max()),
           "top10_overlap_vs_fp16": overlap, "top10_overlap_rescored_top100": overlap_rs}
    del tok, tc, tsc, s8, s16, rel
    torch.cuda.empty_cache()
    return row


def config1_row(stream, hbm_peak):
    """Config 1: one query (Nq=32, d=128, fp16) over 10,000 documents of
    exactly 128 tokens (unit-normalised Gaussian, seed 0): every score and
    the top-10.  328 MB of tokens, a few times the L2, so three identical
    copies of the corpus are rotated between launches and the copy a launch
    reads was last touched two launches (~650 MB of traffic) earlier.  Each
    step (tms_score_dense + tms_topk: one CTA selects from the 10,000
    scores, faster here than slices plus a merge) is timed between events
    at the step boundaries, and the scoring launch alone in a second pass;
    median and p10/p90 over 200 of each.  The oracle scores the same query in full
    on the host cores (its timing and the GPU's parity against it)."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    n, nd = 10_000, 128
    lengths = synth.lengths_fixed(n, nd)
    tok, off, ln = synth.dense_corpus(n, lengths, D, "f16", 0)
    Q = synth.queries(1, NQ, D, "f16", 0)
    copies = [tok.to(dev) for _ in range(3)]
    off_d, ln_d, q_d = torch.from_numpy(off).to(dev), torch.from_numpy(ln).to(dev), Q.to(dev)
    f = torch.arange(n, dtype=torch.int32, device=dev)
    c = torch.tensor([0, n], dtype=torch.int64, device=dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    ts = torch.empty((1, TOPK), dtype=torch.float32, device=dev)
    tp = torch.empty((1, TOPK), dtype=torch.int32, device=dev)
    reps = 200
    mk = lambda: torch.cuda.Event(enable_timing=True)
    sev = [mk() for _ in range(reps + 1)]                 # step boundaries
    kev = [(mk(), mk()) for _ in range(reps)]             # the scoring launch alone
    with torch.cuda.stream(stream):
        for i in range(6):
            tms.score_dense(q_d, copies[i % 3], off_d, ln_d, f, c, out=out, stream=stream)
            tms.topk(out, c, TOPK, ts, tp, stream=stream)
        # steps: an event at each step boundary only, so that the top-k
        # launch follows the scoring launch directly
        for i in range(reps):
            sev[i].record(stream)
            tms.score_dense(q_d, copies[i % 3], off_d, ln_d, f, c, out=out, stream=stream)
            tms.topk(out, c, TOPK, ts, tp, stream=stream)
        sev[reps].record(stream)
        for i in range(reps):
            kev[i][0].record(stream)
            tms.score_dense(q_d, copies[i % 3], off_d, ln_d, f, c, out=out, stream=stream)
            kev[i][1].record(stream)
        tms.topk(out, c, TOPK, ts, tp, stream=stream)
    torch.cuda.synchronize()
    assert tms.device_error(stream) == 0
    step = np.array([sev[i].elapsed_time(sev[i + 1]) for i in range(reps)])
    kern = np.array([a.elapsed_time(b) for a, b in kev])
    alg = iomodel.dense_alg_bytes(n * nd, n, 1, NQ, D, 2)
    kmed = float(np.median(kern))
    row = {"workload": "config 1: 1 query Nq=32, d=128, fp16, 10,000 docs x 128 tokens, every score + top-10",
           "docs_per_s": n / (float(np.median(step)) * 1e-3),
           "step_ms": {"median": float(np.median(step)), "p10": float(np.percentile(step, 10)),
                       "p90": float(np.percentile(step, 90))},
           "kernel_ms_median": kmed, "achieved_gbs": alg / (kmed * 1e-3) / 1e9,
           "frac_hbm_measured": alg / (kmed * 1e-3) / 1e9 / hbm_peak,
           "frac_hbm_nominal_8tbs": alg / (kmed * 1e-3) / 1e9 / 8000.0,
           "l2": "3 corpus copies rotated (984 MB > 129 MB L2)"}
    got = out.cpu().numpy()
    gtop = tp.cpu().numpy()[0]
    want, secs = oracle_dense_query(Q[0], "f16", tok, off, lengths, np.arange(n))
    row["oracle"] = oracle_timing(n, secs)
    row["vs_oracle"] = quality_vs_oracle(got, want, gtop, TOPK)
    del copies
    torch.cuda.empty_cache()
    return row


def peaks_row(stream):
    """Measured ceilings: shared-memory load bandwidth (conflict-free 128-bit
    loads, all SMs) and HBM streaming-read bandwidth (4 GB buffer)."""
    import torch
    from paper_2606_26439_gb300 import tms
    lds = tms.peak_shared_load(20000, stream=stream)
    buf = torch.empty(1 << 32, dtype=torch.uint8, device="cuda")
    buf.fill_(1)
    rd = tms.peak_hbm_read(buf, reps=5, stream=stream)
    del buf
    torch.cuda.empty_cache()
    return {"lds_gbs": lds, "hbm_read_gbs": rd}


def serving_row():
    """Serving loop on a mix like config 5: 1,000,000 fp16 documents and
    1,000,000 PQ documents (M=16, K=256) resident; requests of 32 query
    tokens, each on one store (even odds), candidate lists log-uniform in
    [1,000, 100,000] (ids drawn uniformly), top-10, Poisson arrivals.  For
    each arrival rate: p50 / p99 latency (submit to result) and docs/s with
    continuous batching, and with one request per launch (the plain
    per-request baseline, same kernels)."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    n_docs = 1_000_000
    tok, off, ln = synth.device_dense_corpus(synth.lengths_uniform(n_docs, LO, HI, 5), D, "f16", 5, dev)
    cb, codes, poff, pln = synth.device_pq_corpus(synth.lengths_uniform(n_docs, LO, HI, 6), 16, 256, 8, 6,
                                                  device=dev)
    g = np.random.default_rng(7)
    pool = []
    for i in range(512):
        n = int(np.exp(g.uniform(np.log(1_000), np.log(100_000))))
        pool.append((int(g.integers(0, 2)), synth.queries(1, NQ, D, "f16", 100 + i)[0],
                     g.integers(0, n_docs, n).astype(np.int32)))
    mean_cands = float(np.mean([len(p[2]) for p in pool]))

    def run(rate, batched, duration=3.0):
        with tms.Server(tok, off, ln, nq=NQ, topk=TOPK, max_batch_requests=256 if batched else 1,
                        max_batch_candidates=4_000_000, max_pending=1 << 20, pq=(codes, cb, poff, pln)) as srv:
            return serve_poisson(srv, pool, rate, duration)

    out = {"mean_candidates": mean_cands}
    for rate in (1000, 4000):
        out[f"{rate}_qps"] = {"demand_docs_per_s": rate * mean_cands, "batched": run(rate, True),
                              "one_per_launch": run(rate, False)}
    del codes
    torch.cuda.empty_cache()
    out_fp8 = serving_fp8_row(tok, off, ln)
    del tok
    torch.cuda.empty_cache()
    return out, out_fp8


def serve_poisson(srv, pool, rate, duration, store_of=None):
    """Submit pool requests (cycling) at Poisson arrivals of `rate` per
    second for `duration` seconds from a second thread, wait for each in
    order; p50 / p99 latency (submit to result) and docs/s over the wall
    time until the last result.  Pool entries are (query, cands) sent to
    `store_of`, or (store, query, cands) when it is None."""
    import threading
    n_req = int(rate * duration)
    gaps = np.random.default_rng(11).exponential(1.0 / rate, n_req)
    tickets = [None] * n_req
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        due = 0.0
        for i in range(n_req):
            due += gaps[i]
            delay = t0 + due - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            e = pool[i % len(pool)]
            store, q, c = (store_of,) + tuple(e) if store_of is not None else e
            tickets[i] = (srv.submit(q, c, store), len(c))
            ready.release()

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    lat, docs = [], 0
    for i in range(n_req):
        ready.acquire()
        t, n = tickets[i]
        _, _, l = srv.wait(t, timeout_s=600.0)
        lat.append(l)
        docs += n
    wall = time.perf_counter() - t_start
    th.join()
    st = srv.stats()
    lat = np.array(lat) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "docs_per_s": docs / wall, "requests": n_req, "batches": st["batches"],
            "host_enqueue_us_per_batch": 1e6 * st["enqueue_s"] / max(1, st["batches"])}


def serving_fp8_row(tok, off, ln):
    """The served, batched FP8 form against plain per-request fp16 scoring:
    the 1,000,000-document fp16 store of the serving row and its FP8 E4M3
    copy (quantized on the device), dense requests only (32 query tokens,
    lists log-uniform in [1,000, 100,000], top-10, Poisson arrivals).
    FP8: batched (up to 256 requests per launch), each request's 100 best
    FP8 candidates re-scored in fp16.  Plain: one fp16 request per launch.
    Batched fp16 is reported beside them.  Top-10 overlap of the FP8 form
    (with and without the re-score) against the fp16 top-10 of the same
    requests, over 256 of them."""
    import torch
    from paper_2606_26439_gb300 import tms
    n_docs = off.shape[0]
    f8c, f8s = tms.quantize_e4m3(tok)
    g = np.random.default_rng(17)
    pool = []
    for i in range(512):
        n = int(np.exp(g.uniform(np.log(1_000), np.log(100_000))))
        pool.append((synth.queries(1, NQ, D, "f16", 5000 + i)[0], g.integers(0, n_docs, n).astype(np.int32)))
    mean_cands = float(np.mean([len(p[1]) for p in pool]))

    def server(batched, rescore_k=100):
        return tms.Server(tok, off, ln, nq=NQ, topk=TOPK, max_batch_requests=256 if batched else 1,
                          max_batch_candidates=4_000_000, max_pending=1 << 20, fp8=(f8c, f8s), rescore_k=rescore_k)

    out = {"mean_candidates": mean_cands, "rescore_k": 100}
    # top-10 overlap against the fp16 scorer
    with server(True) as srv, server(True, rescore_k=0) as raw:
        ov, ov_raw = [], []
        for q, c in pool[:256]:
            _, ref, _ = srv.wait(srv.submit(q, c, tms.TMS_STORE_DENSE))
            _, got, _ = srv.wait(srv.submit(q, c, tms.TMS_STORE_FP8))
            _, got_raw, _ = raw.wait(raw.submit(q, c, tms.TMS_STORE_FP8))
            ref_set = set(ref[ref >= 0].tolist())
            ov.append(len(ref_set & set(got[got >= 0].tolist())) / max(1, len(ref_set)))
            ov_raw.append(len(ref_set & set(got_raw[got_raw >= 0].tolist())) / max(1, len(ref_set)))
    out["top10_overlap_rescored"] = float(np.mean(ov))
    out["top10_overlap_rescored_min"] = float(np.min(ov))
    out["top10_overlap_fp8_only"] = float(np.mean(ov_raw))
    for rate in (4000, 7000, 10000):
        row = {"demand_docs_per_s": rate * mean_cands}
        for name, batched, store in (("fp8_batched_rescored", True, tms.TMS_STORE_FP8),
                                     ("fp16_one_per_launch", False, tms.TMS_STORE_DENSE),
                                     ("fp16_batched", True, tms.TMS_STORE_DENSE)):
            with server(batched) as srv:
                row[name] = serve_poisson(srv, pool, rate, 3.0, store)
        out[f"{rate}_qps"] = row
    del f8c, f8s
    torch.cuda.empty_cache()
    return out


def secondary_rows(lengths, cands, stream, hbm_peak, sm_mhz):
    """bf16/fp32 of the headline workload, dimension tiling, fused PQ."""
    import torch
    from paper_2606_26439_gb300 import tms
    rows = {}
    dev = torch.device("cuda")
    peaks = peaks_row(stream)
    rows["measured_peaks"] = peaks
    rows["config1"] = config1_row(stream, hbm_peak)
    off0 = synth.offsets_of(lengths)

    def vs_oracle_q0(w, dtype, out):
        """Oracle leg for query 0 of a config-2 launch: its 100,000 scores and
        top-10 against the FP64 oracle, and the oracle's own timing."""
        _, tp = tms.topk(out, w["c"], TOPK)
        want, secs = oracle_dense_query(w["Q"][0], dtype, w["tok"], off0, lengths, cands[0])
        q = quality_vs_oracle(out[:N_CAND].cpu().numpy(), want, tp.cpu().numpy()[0], TOPK)
        return want, {"oracle_query0": oracle_timing(N_CAND, secs), "vs_oracle_query0": q}

    for dtype, steps in (("bf16", 50), ("f32", 10)):
        w = dense_workload(dtype, lengths, cands, dev)
        ms, kms, out, _ = time_dense(w, steps, 3, stream)
        elem = 2 if dtype == "bf16" else 4
        alg = iomodel.dense_alg_bytes(w["tokens"], len(w["flat"]), N_QUERIES, NQ, D, elem)
        rows[f"dense_{dtype}"] = {
            "docs_per_s": len(w["flat"]) / (ms * 1e-3), "ms_per_step": ms, "kernel_ms": kms,
            "achieved_gbs": alg / (kms * 1e-3) / 1e9, "frac_hbm": alg / (kms * 1e-3) / 1e9 / hbm_peak,
            "frac_hbm_read_peak": alg / (kms * 1e-3) / 1e9 / peaks["hbm_read_gbs"]}
        rows[f"dense_{dtype}"].update(vs_oracle_q0(w, dtype, out)[1])
        del w, out
        torch.cuda.empty_cache()
    # the headline after the autotuner picked its launch configuration
    w = dense_workload("f16", lengths, cands, dev)
    _, n_cfg = tms.tune_dense(w["q"], w["tok"], w["off"], w["ln"], w["f"], w["c"], stream=stream)
    ms, kms, _, _ = time_dense(w, 30, 3, stream)
    alg = iomodel.dense_alg_bytes(w["tokens"], len(w["flat"]), N_QUERIES, NQ, D, 2)
    rows["dense_f16_autotuned"] = {"docs_per_s": len(w["flat"]) / (ms * 1e-3), "ms_per_step": ms, "kernel_ms": kms,
                                   "configs_timed": n_cfg, "achieved_gbs": alg / (kms * 1e-3) / 1e9,
                                   "frac_hbm": alg / (kms * 1e-3) / 1e9 / hbm_peak}
    # the headline's fp16 scores of query 0 against the oracle (the FP8 row reuses them)
    out16 = tms.score_dense(w["q"], w["tok"], w["off"], w["ln"], w["f"], w["c"], stream=stream)
    torch.cuda.synchronize()
    want16, q16 = vs_oracle_q0(w, "f16", out16)
    rows["dense_f16"] = q16
    del w, out16
    torch.cuda.empty_cache()
    # FP8 E4M3 store of the headline workload (quantized on the device)
    w = dense_workload("f16", lengths, cands, dev)
    n_tok = w["tok"].shape[0]
    tc, tsc = tms.quantize_e4m3(w["tok"])
    qc, qsc = tms.quantize_e4m3(w["q"])
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        e[0].record(stream)
        tms.quantize_e4m3(w["tok"], tc, tsc, stream=stream)
        e[1].record(stream)
    torch.cuda.synchronize()
    quant_ms = e[0].elapsed_time(e[1])
    del w["tok"]
    torch.cuda.empty_cache()
    out = torch.empty(len(w["flat"]), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            tms.score_fp8(qc, qsc, tc, tsc, w["off"], w["ln"], w["f"], w["c"], out=out, stream=stream)
    torch.cuda.synchronize()
    reps = 20
    with torch.cuda.stream(stream):
        e[0].record(stream)
        for _ in range(reps):
            tms.score_fp8(qc, qsc, tc, tsc, w["off"], w["ln"], w["f"], w["c"], out=out, stream=stream)
        e[1].record(stream)
    torch.cuda.synchronize()
    kms = e[0].elapsed_time(e[1]) / reps
    alg = iomodel.fp8_alg_bytes(w["tokens"], len(w["flat"]), N_QUERIES, NQ, D)
    qbytes = iomodel.quantize_alg_bytes(n_tok, D, 2)
    _, tp8 = tms.topk(out, w["c"], TOPK)
    # the same launch after tms_tune_fp8 chose its configuration
    _, n_cfg8 = tms.tune_fp8(qc, qsc, tc, tsc, w["off"], w["ln"], w["f"], w["c"], out=out, stream=stream)
    tuned_ms = time_launch(lambda: tms.score_fp8(qc, qsc, tc, tsc, w["off"], w["ln"], w["f"], w["c"], out=out,
                                                 stream=stream), stream, reps)
    rows["fp8_e4m3"] = {"docs_per_s": len(w["flat"]) / (kms * 1e-3), "kernel_ms": kms,
                        "achieved_gbs": alg / (kms * 1e-3) / 1e9, "frac_hbm": alg / (kms * 1e-3) / 1e9 / hbm_peak,
                        "quantize_corpus_ms": quant_ms, "quantize_gbs": qbytes / (quant_ms * 1e-3) / 1e9,
                        "autotuned": {"kernel_ms": tuned_ms, "configs_timed": n_cfg8,
                                      "frac_hbm": alg / (tuned_ms * 1e-3) / 1e9 / hbm_peak,
                                      "speedup_vs_default": kms / tuned_ms},
                        # FP8 scores of query 0 against the FP64 oracle of the fp16 corpus they were
                        # quantized from: quantization error included (the FP8 store's quality)
                        "vs_fp64_oracle_query0": quality_vs_oracle(out[:N_CAND].cpu().numpy(), want16,
                                                                   tp8.cpu().numpy()[0], TOPK)}
    del w, tc, tsc, qc, qsc, out
    torch.cuda.empty_cache()
    rows["fp8_e4m3_shared_1m"] = fp8_store_row(stream, hbm_peak)
    del want16
    rows["serving_mix_1m_dense_1m_pq"], rows["serving_fp8_vs_fp16_1m"] = serving_row()
    # dimension tiling: 200K docs, 32 queries over all docs, bf16, top-100, in
    # the per-query schedule and the shared-list schedule; query 0 of each
    # against the oracle (all 200,000 scores and the top-100)
    n3 = 200_000
    len3 = synth.lengths_uniform(n3, LO, HI, 2)
    off3 = synth.offsets_of(len3)
    tok3 = int(len3.astype(np.int64).sum())
    for d in (64, 256, 512, 768):
        tok, off, ln = synth.device_dense_corpus(len3, d, "bf16", 2, dev)
        Qh = synth.queries(32, NQ, d, "bf16", 2)
        Q = Qh.to(dev)
        f = torch.arange(n3, dtype=torch.int32, device=dev).repeat(32)
        c = torch.arange(0, 33 * n3, n3, dtype=torch.int64, device=dev)
        out = torch.empty(32 * n3, dtype=torch.float32, device=dev)
        out_sh = torch.empty((32, n3), dtype=torch.float32, device=dev)
        ts = torch.empty((32, 100), dtype=torch.float32, device=dev)
        tp = torch.empty((32, 100), dtype=torch.int32, device=dev)
        ts_sh, tp_sh = torch.empty_like(ts), torch.empty_like(tp)
        with torch.cuda.stream(stream):
            for _ in range(3):
                tms.score_dense(Q, tok, off, ln, f, c, out=out, stream=stream)
                tms.score_dense_shared(Q, tok, off, ln, f[:n3], out=out_sh, stream=stream)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        with torch.cuda.stream(stream):
            e[0].record(stream)
            for _ in range(3):
                tms.score_dense(Q, tok, off, ln, f, c, out=out, stream=stream)
            e[1].record(stream)
            tms.topk(out, c, 100, ts, tp, stream=stream)
            e[2].record(stream)
            for _ in range(5):
                tms.score_dense_shared(Q, tok, off, ln, f[:n3], out=out_sh, stream=stream)
            e[3].record(stream)
            tms.topk(out_sh.view(-1), c, 100, ts_sh, tp_sh, stream=stream)
            e[4].record(stream)
        torch.cuda.synchronize()
        kms = e[0].elapsed_time(e[1]) / 3
        kms_sh = e[2].elapsed_time(e[3]) / 5
        alg = iomodel.dense_alg_bytes(tok3 * 32, 32 * n3, 32, NQ, d, 2)
        fl = iomodel.dense_alg_flops(tok3 * 32, NQ, d)
        want0, secs = oracle_dense_query(Qh[0], "bf16", tok, off3, len3, np.arange(n3))
        rows[f"dtile_bf16_d{d}"] = {"docs_per_s": 32 * n3 / (kms * 1e-3), "kernel_ms": kms,
                                   "topk100_ms": e[1].elapsed_time(e[2]),
                                   "achieved_gbs": alg / (kms * 1e-3) / 1e9,
                                   "frac_hbm": alg / (kms * 1e-3) / 1e9 / hbm_peak,
                                   "vs_oracle_query0": quality_vs_oracle(out[:n3].cpu().numpy(), want0,
                                                                         tp.cpu().numpy()[0], 100),
                                   "oracle_query0": oracle_timing(n3, secs)}
        if d in (64, 768):
            # the same launches after the autotuner chose their configuration
            # (the shared-list tuner also chooses the query group size)
            if d == 64:
                _, n_cfg = tms.tune_dense(Q, tok, off, ln, f, c, out=out, stream=stream)
                t_ms = time_launch(lambda: tms.score_dense(Q, tok, off, ln, f, c, out=out, stream=stream), stream, 3)
                rows_tuned = {"kernel_ms": t_ms, "configs_timed": n_cfg, "speedup_vs_default": kms / t_ms,
                              "frac_hbm": alg / (t_ms * 1e-3) / 1e9 / hbm_peak}
            _, n_cfg_sh = tms.tune_dense_shared(Q, tok, off, ln, f[:n3], out=out_sh, stream=stream)
            t_sh = time_launch(lambda: tms.score_dense_shared(Q, tok, off, ln, f[:n3], out=out_sh, stream=stream),
                               stream, 5)
            rows_tuned_sh = {"kernel_ms": t_sh, "configs_timed": n_cfg_sh, "speedup_vs_default": kms_sh / t_sh,
                             "tflops": fl / (t_sh * 1e-3) / 1e12}
        rows[f"dtile_shared_bf16_d{d}"] = {"docs_per_s": 32 * n3 / (kms_sh * 1e-3), "kernel_ms": kms_sh,
                                          "topk100_ms": e[3].elapsed_time(e[4]),
                                          "tflops": fl / (kms_sh * 1e-3) / 1e12,
                                          "corpus_reads_gbs": tok3 * d * 2 / (kms_sh * 1e-3) / 1e9,
                                          "vs_oracle_query0": quality_vs_oracle(out_sh[0].cpu().numpy(), want0,
                                                                                tp_sh.cpu().numpy()[0], 100)}
        if d in (64, 768):
            rows[f"dtile_shared_bf16_d{d}"]["autotuned"] = rows_tuned_sh
            if d == 64:
                rows[f"dtile_bf16_d{d}"]["autotuned"] = rows_tuned
        del tok, off, ln, Q, f, out, out_sh
        torch.cuda.empty_cache()
    # fused PQ: 1M docs, M=16, K=256, dsub=8, 64 fp16 queries over all docs
    n4, M, K, dsub, nQ4 = 1_000_000, 16, 256, 8, 64
    len4 = synth.lengths_uniform(n4, LO, HI, 4)
    cb, codes, off, ln = synth.device_pq_corpus(len4, M, K, dsub, 4, device=dev)
    Q = synth.queries(nQ4, NQ, M * dsub, "f16", 4).to(dev)
    f = torch.arange(n4, dtype=torch.int32, device=dev).repeat(nQ4)
    c = torch.arange(0, (nQ4 + 1) * n4, n4, dtype=torch.int64, device=dev)
    out = torch.empty(nQ4 * n4, dtype=torch.float32, device=dev)
    lut = torch.empty((nQ4, NQ, M, K), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        tms.build_pq_lut(Q, cb, out=lut, stream=stream)
        tms.score_pq(lut, codes, off, ln, f, c, out=out, stream=stream)
    torch.cuda.synchronize()
    out16 = torch.empty_like(out)
    with torch.cuda.stream(stream):
        tms.score_pq(lut, codes, off, ln, f, c, out=out16, stream=stream, f16_table=True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    reps = 2
    with torch.cuda.stream(stream):
        e[0].record(stream)
        for _ in range(reps):
            tms.build_pq_lut(Q, cb, out=lut, stream=stream)
        e[1].record(stream)
        for _ in range(reps):
            tms.score_pq(lut, codes, off, ln, f, c, out=out, stream=stream)
        e[2].record(stream)
        for _ in range(reps):
            tms.score_pq(lut, codes, off, ln, f, c, out=out16, stream=stream, f16_table=True)
        e[3].record(stream)
    torch.cuda.synchronize()
    lut_ms = e[0].elapsed_time(e[1]) / reps
    pq_ms = e[1].elapsed_time(e[2]) / reps
    pq16_ms = e[2].elapsed_time(e[3]) / reps
    rel = ((out16 - out).abs() / out.abs().clamp_min(NQ * 1e-3)).max().item()
    tok4 = int(len4.astype(np.int64).sum()) * nQ4
    alg = iomodel.pq_alg_bytes(tok4, nQ4 * n4, nQ4, NQ, M, K)
    lds = iomodel.pq_lut_reads_bytes(tok4, NQ, M)
    lds_peak = peaks["lds_gbs"]  # measured: conflict-free 128-bit shared-memory loads, all SMs
    lds_nominal = 152 * 128 * (sm_mhz or 1900.0) * 1e6 / 1e9
    rows["pq_m16_k256"] = {"docs_per_s": nQ4 * n4 / (pq_ms * 1e-3), "kernel_ms": pq_ms, "lut_ms": lut_ms,
                           "achieved_gbs": alg / (pq_ms * 1e-3) / 1e9,
                           "frac_hbm": alg / (pq_ms * 1e-3) / 1e9 / hbm_peak,
                           "lds_gbs": lds / (pq_ms * 1e-3) / 1e9, "lds_peak_gbs": lds_peak,
                           "lds_peak_kind": "measured (tms_peak_shared_load)",
                           "frac_lds": lds / (pq_ms * 1e-3) / 1e9 / lds_peak,
                           "frac_lds_nominal": lds / (pq_ms * 1e-3) / 1e9 / lds_nominal}
    # the same queries with the codes decompressed in shared memory and scored
    # on the tensor cores (one shared list: every document)
    ids = torch.arange(n4, dtype=torch.int32, device=dev)
    out_tc = torch.empty((nQ4, n4), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        tms.score_pq_tc_shared(Q, cb, codes, off, ln, ids, out=out_tc, stream=stream)
        e[0].record(stream)
        for _ in range(reps):
            tms.score_pq_tc_shared(Q, cb, codes, off, ln, ids, out=out_tc, stream=stream)
        e[1].record(stream)
    torch.cuda.synchronize()
    tc_ms = e[0].elapsed_time(e[1]) / reps
    rel_tc = ((out_tc.view(-1) - out).abs() / out.abs().clamp_min(NQ * 1e-3)).max().item()
    tc_flops = iomodel.dense_alg_flops(tok4, NQ, M * dsub)
    rows["pq_m16_k256_tensor_core"] = {"docs_per_s": nQ4 * n4 / (tc_ms * 1e-3), "kernel_ms": tc_ms,
                                       "speedup_vs_fp32_table": pq_ms / tc_ms,
                                       "max_rel_diff_vs_fp32_table": rel_tc,
                                       "tflops": tc_flops / (tc_ms * 1e-3) / 1e12,
                                       "codes_reads_gbs": tok4 // nQ4 * M * ((nQ4 + 3) // 4) / (tc_ms * 1e-3) / 1e9}
    out_tc_q0 = out_tc[0].clone()
    del out_tc
    # the oracle leg: query 0 over all 1,000,000 documents, FP64 decompress-then-dot
    import oracle
    cb_h, codes_h = cb.cpu().numpy(), codes.cpu().numpy()
    Qh = Q.cpu().contiguous()
    t0 = time.perf_counter()
    want0 = oracle.pq_decompress_scores(Qh[0].view(torch.int16).numpy().view(np.uint16), cb_h, codes_h,
                                        synth.offsets_of(len4), len4, np.arange(n4, dtype=np.int32),
                                        qdtype=oracle.F16)
    pq_oracle_s = time.perf_counter() - t0
    del codes_h
    c1 = c[:2]
    pq_vs = {}
    for name, scores in (("fp32_table", out), ("fp16_table", out16), ("tensor_core", out_tc_q0)):
        _, tpq = tms.topk(scores, c1, TOPK)
        pq_vs[name] = quality_vs_oracle(scores[:n4].cpu().numpy(), want0, tpq.cpu().numpy()[0], TOPK)
    rows["pq_m16_k256"]["vs_oracle_query0"] = pq_vs["fp32_table"]
    rows["pq_m16_k256"]["oracle_query0"] = oracle_timing(n4, pq_oracle_s)
    rows["pq_m16_k256_tensor_core"]["vs_oracle_query0"] = pq_vs["tensor_core"]
    # the same pass through the fp16 table: half the shared-memory bytes per lookup
    lds16 = lds // 2
    rows["pq_m16_k256_f16_table"] = {"docs_per_s": nQ4 * n4 / (pq16_ms * 1e-3), "kernel_ms": pq16_ms,
                                     "speedup_vs_fp32_table": pq_ms / pq16_ms,
                                     "max_rel_diff_vs_fp32_table": rel,
                                     "lds_gbs": lds16 / (pq16_ms * 1e-3) / 1e9, "lds_peak_gbs": lds_peak,
                                     "frac_lds": lds16 / (pq16_ms * 1e-3) / 1e9 / lds_peak,
                                     "vs_oracle_query0": pq_vs["fp16_table"]}
    return rows


def run_tms(args, ws, rank, local):
    import torch
    from paper_2606_26439_gb300 import tms
    torch.cuda.set_device(local)
    tms.lib(build_if_missing=True)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    hbm_peak, _, peak_kind = measured_peaks()
    lengths, cands = headline_inputs()
    w = dense_workload("f16", lengths, cands, dev)
    n_docs_step = len(w["flat"])

    # headline: device-resident, CUDA events, clocks sampled during the run
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ms, kms, out, per_step = time_dense(w, args.steps, args.warmup, stream)
    clk = clocks.stop()
    assert tms.device_error(stream) == 0, "device error flags raised during the benchmark"
    assert bool(torch.isfinite(out).all())
    barrier(ws)
    value, ms_max = replica_rate(n_docs_step, ms, ws)
    kms_max = max_over_ranks(kms, ws)

    e2e_ms, h2d, d2h = time_dense_e2e(w, max(10, args.steps // 4), max(3, args.warmup), stream)
    e2e_value, e2e_ms = replica_rate(n_docs_step, e2e_ms, ws)

    alg = iomodel.dense_alg_bytes(w["tokens"], n_docs_step, N_QUERIES, NQ, D, 2)
    achieved = alg / (kms_max * 1e-3) / 1e9
    tpt = recorded_traffic_per_token()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": (tpt * w["tokens"] if tpt else None),
                "peak_kind": f"of {peak_kind} (copy bandwidth)", "alg_bytes_per_launch": alg,
                "kernel": "tms::dense::dense_tc_kernel<1>", "kernel_ms": kms_max}

    line = {
        "metric": METRIC, "value": value, "unit": "docs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_docs": N_DOCS, "n_queries": N_QUERIES, "nq": NQ, "d": D,
                   "cand_per_query": N_CAND, "topk": TOPK, "tokens_per_step": w["tokens"],
                   "l2": f"inputs larger than L2 ({w['tok'].numel() * 2 / 1e9:.1f} GB fp16 corpus, "
                         f"{w['tokens'] * D * 2 / 1e9:.1f} GB read per step)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "docs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "step_ms": {"median": float(np.median(per_step)), "p10": float(np.percentile(per_step, 10)),
                    "p90": float(np.percentile(per_step, 90)), "n": len(per_step)},
        "gpu_launches": (2 + (tms.topk_workspace_size(N_QUERIES, TOPK, n_docs_step) > 0)) * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    del w, out
    torch.cuda.empty_cache()
    if ws == 1 and rank == 0 and args.workload == "headline":
        rate, n, dt, cores = time_oracle(lengths, cands, 15.0)
        rate1, n1, dt1, _ = time_oracle(lengths, cands, 5.0, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "docs/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {n} candidates of query 0 ({dt:.1f} s, FP64, fp16 stored values)",
                                "one_thread": {"value": rate1, "unit": "docs/s",
                                               "sample": f"first {n1} candidates of query 0 ({dt1:.1f} s)"}}
        if not args.no_rows:
            try:
                line["rows"] = secondary_rows(lengths, cands, stream, hbm_peak, clk["sm_mhz"])
            except Exception as exc:  # the headline line is still printed
                import traceback
                line["rows_error"] = "".join(traceback.format_exception_only(type(exc), exc)).strip()
                traceback.print_exc()
    if rank == 0:
        print(json.dumps(line), flush=True)


def profile_case(args):
    """One secondary kernel on a small case (100,000 documents, a few GB):
    fp8_small -- FP8 store, 1 query x 100,000 candidates; f32_small -- fp32
    (split TF32), the same; d64_small -- bf16 d=64, the same; pq_small --
    PQ M=16 K=256, 8 queries over all documents (pq16_small: the same
    through the fp16 table; pqtc_small: decompressed in shared memory,
    tensor cores); shared_small / shared64_small / shared768_small -- bf16
    d=256 / 64 / 768, 8 queries over all documents in the shared schedule
    (20,000 documents at d=768: 3.3 GB)."""
    import torch
    from paper_2606_26439_gb300 import tms
    dev = torch.device("cuda")
    n = 100_000
    lens = synth.lengths_uniform(n, LO, HI, 9)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    if args.profile_case in ("f32_small", "d64_small"):
        dt, d = ("f32", 128) if args.profile_case == "f32_small" else ("bf16", 64)
        tok, off, ln = synth.device_dense_corpus(lens, d, dt, 9, dev)
        q = synth.queries(1, NQ, d, dt, 9).to(dev)
        co = torch.tensor([0, n], dtype=torch.int64, device=dev)
        run = lambda: tms.score_dense(q, tok, off, ln, ids, co)  # noqa: E731
        units = n
    elif args.profile_case == "fp8_small":
        tok, off, ln = synth.device_dense_corpus(lens, D, "f16", 9, dev)
        tc, ts = tms.quantize_e4m3(tok)
        del tok
        qc, qs = tms.quantize_e4m3(synth.queries(1, NQ, D, "f16", 9).to(dev))
        co = torch.tensor([0, n], dtype=torch.int64, device=dev)
        run = lambda: tms.score_fp8(qc, qs, tc, ts, off, ln, ids, co)  # noqa: E731
        units = n
    elif args.profile_case in ("pq_small", "pq16_small", "pqtc_small"):
        cb, codes, off, ln = synth.device_pq_corpus(lens, 16, 256, 8, 9, device=dev)
        q = synth.queries(8, NQ, 128, "f16", 9).to(dev)
        lut = tms.build_pq_lut(q, cb)
        f = ids.repeat(8)
        co = torch.arange(0, 9 * n, n, dtype=torch.int64, device=dev)
        half = args.profile_case == "pq16_small"
        if args.profile_case == "pqtc_small":
            run = lambda: tms.score_pq_tc_shared(q, cb, codes, off, ln, ids)  # noqa: E731
        else:
            run = lambda: tms.score_pq(lut, codes, off, ln, f, co, f16_table=half)  # noqa: E731
        units = 8 * n
    else:
        d = {"shared_small": 256, "shared64_small": 64, "shared768_small": 768}[args.profile_case]
        if d == 768:
            n = 20_000
            lens = lens[:n]
            ids = ids[:n]
        tok, off, ln = synth.device_dense_corpus(lens, d, "bf16", 9, dev)
        q = synth.queries(8, NQ, d, "bf16", 9).to(dev)
        run = lambda: tms.score_dense_shared(q, tok, off, ln, ids)  # noqa: E731
        units = 8 * n
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    assert tms.device_error() == 0
    print(json.dumps({"profile_case": args.profile_case, "kernel_ms": ms, "docs_per_s": units / (ms * 1e-3)}),
          flush=True)


def main():
    args = parse_args()
    if args.profile_case:
        profile_case(args)
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_tms(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
