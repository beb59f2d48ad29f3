// tms_server.cu -- the serving loop: continuous batching of MaxSim requests
// over a device-resident corpus (a dense store, optionally a PQ store and an
// FP8 copy of the dense store).
//
// One worker thread per server.  Each turn it takes every pending request
// that fits the batch buffers (FIFO), stages their queries and candidate
// lists in pinned memory, and enqueues, per store on its own stream: the
// host-to-device copies, the scoring -- tms_score_dense (dense requests),
// tms_build_pq_lut + tms_score_pq (PQ requests), or tms_quantize_e4m3 +
// tms_score_fp8 followed by an exact fp16 re-score of each request's
// shortlist (FP8 requests) -- tms_topk, and the device-to-host copy of the
// top-k.  The HBM-bound dense and FP8 scoring and the shared-memory-bound
// PQ scoring of a batch overlap on their streams.  Two
// buffer slots alternate, so while the GPU runs one batch the
// worker completes the previous one and stages the next: requests that
// arrive during a launch go into the following one (continuous batching).
// Batch composition never changes a result: every score has one owner and
// a fixed summation order, and the top-k of a request reads only its own
// scores.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {

namespace server {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int store = 0;
    std::vector<uint8_t> query;
    std::vector<int32_t> cands;
    std::vector<float> scores;
    std::vector<int32_t> ids;
    int64_t bytes = 0;  // device bytes claimed in the batch buffers (admission)
    tms_status status = TMS_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

using RequestPtr = std::shared_ptr<Request>;

constexpr int kStores = 3;  // dense, PQ, FP8

// Buffers of one batch in flight, per store (0 dense, 1 PQ, 2 FP8).
struct Slot {
    void* h_q[kStores] = {};
    int32_t* h_c[kStores] = {};
    int64_t* h_co[kStores] = {};
    float* h_ts[kStores] = {};
    int32_t* h_tp[kStores] = {};
    void* d_q[kStores] = {};
    int32_t* d_c[kStores] = {};
    int64_t* d_co[kStores] = {};
    float* d_sc[kStores] = {};
    float* d_ts[kStores] = {};
    int32_t* d_tp[kStores] = {};
    float* d_lut = nullptr;
    // FP8 requests: quantized queries, the shortlist (top rescore_k
    // positions), its CSR offsets and ids, and its fp16 scores
    uint8_t* d_qc = nullptr;
    float* d_qs = nullptr;
    float* d_rts = nullptr;
    int32_t* d_rtp = nullptr;
    int32_t* h_rtp = nullptr;
    int64_t* d_cor = nullptr;
    int32_t* d_cr = nullptr;
    float* d_scr = nullptr;
    cudaEvent_t done[kStores] = {};
    std::vector<RequestPtr> reqs[kStores];
    tms_status status = TMS_OK;
};

}  // namespace server

}  // namespace tms

struct tms_server {
    tms_server_config cfg;
    int device = 0;
    size_t qbytes = 0;  // bytes of one query
    cudaStream_t stream[tms::server::kStores] = {};  // dense, PQ, FP8
    tms::server::Slot slots[2];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<tms::server::RequestPtr> pending;
    std::unordered_map<uint64_t, tms::server::RequestPtr> live;  // admitted, result not yet taken
    uint64_t next_ticket = 1;
    int unfinished = 0;
    int64_t unfinished_bytes = 0;
    bool stop = false;
    uint64_t batch_ordinal = 0;
    tms_server_stats stats{};
    std::thread worker;
};

namespace tms {

namespace server {

inline bool cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return true;
    (void)cudaGetLastError();
    return false;
}

bool has_store(const tms_server_config& c, int st) {
    return st == 0 || (st == 1 && c.pq_codes) || (st == 2 && c.fp8_codes);
}

bool alloc_slot(tms_server* s, Slot& sl) {
    const tms_server_config& c = s->cfg;
    const size_t nb = static_cast<size_t>(c.max_batch_requests);
    const size_t nc = static_cast<size_t>(c.max_batch_candidates);
    for (int st = 0; st < kStores; ++st) {
        if (!has_store(c, st)) continue;
        if (!cuda_ok(cudaMallocHost(&sl.h_q[st], nb * s->qbytes)) ||
            !cuda_ok(cudaMallocHost(reinterpret_cast<void**>(&sl.h_c[st]), nc * 4)) ||
            !cuda_ok(cudaMallocHost(reinterpret_cast<void**>(&sl.h_co[st]), (nb + 1) * 8)) ||
            !cuda_ok(cudaMallocHost(reinterpret_cast<void**>(&sl.h_ts[st]), nb * c.topk * 4)) ||
            !cuda_ok(cudaMallocHost(reinterpret_cast<void**>(&sl.h_tp[st]), nb * c.topk * 4)) ||
            !cuda_ok(cudaMalloc(&sl.d_q[st], nb * s->qbytes)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_c[st]), nc * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_co[st]), (nb + 1) * 8)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_sc[st]), nc * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_ts[st]), nb * c.topk * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_tp[st]), nb * c.topk * 4)))
            return false;
    }
    if (c.pq_codes &&
        !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_lut),
                            nb * static_cast<size_t>(c.nq) * c.pq_m * c.pq_k * 4)))
        return false;
    if (c.fp8_codes) {
        const size_t rk = static_cast<size_t>(c.rescore_k > 0 ? c.rescore_k : 1);
        if (!cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_qc), nb * c.nq * c.d)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_qs), nb * c.nq * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_rts), nb * rk * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_rtp), nb * rk * 4)) ||
            !cuda_ok(cudaMallocHost(reinterpret_cast<void**>(&sl.h_rtp), nb * rk * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_cor), (nb + 1) * 8)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_cr), nb * rk * 4)) ||
            !cuda_ok(cudaMalloc(reinterpret_cast<void**>(&sl.d_scr), nb * rk * 4)))
            return false;
    }
    for (int st = 0; st < kStores; ++st)
        if (!cuda_ok(cudaEventCreateWithFlags(&sl.done[st], cudaEventDisableTiming))) return false;
    return true;
}

void free_slot(Slot& sl) {
    for (int st = 0; st < kStores; ++st) {
        cudaFreeHost(sl.h_q[st]);
        cudaFreeHost(sl.h_c[st]);
        cudaFreeHost(sl.h_co[st]);
        cudaFreeHost(sl.h_ts[st]);
        cudaFreeHost(sl.h_tp[st]);
        cudaFree(sl.d_q[st]);
        cudaFree(sl.d_c[st]);
        cudaFree(sl.d_co[st]);
        cudaFree(sl.d_sc[st]);
        cudaFree(sl.d_ts[st]);
        cudaFree(sl.d_tp[st]);
    }
    cudaFree(sl.d_lut);
    cudaFree(sl.d_qc);
    cudaFree(sl.d_qs);
    cudaFree(sl.d_rts);
    cudaFree(sl.d_rtp);
    cudaFreeHost(sl.h_rtp);
    cudaFree(sl.d_cor);
    cudaFree(sl.d_cr);
    cudaFree(sl.d_scr);
    for (int st = 0; st < kStores; ++st)
        if (sl.done[st]) cudaEventDestroy(sl.done[st]);
    (void)cudaGetLastError();
}

// FP8 requests: the CSR offsets of the shortlists, cor[i] = sum over
// requests j < i of min(list length, rk), computed on the device from the
// batch's own offsets (one CTA, nb <= 4096: four requests per thread, a
// warp scan, then a scan of the warp totals).
constexpr int kCsrThreads = 1024;
__global__ void __launch_bounds__(kCsrThreads) shortlist_csr(const int64_t* __restrict__ co, int nb, int rk,
                                                             int64_t* __restrict__ cor) {
    __shared__ int64_t warp_tot[kCsrThreads / 32];
    griddep_wait();
    griddep_launch_dependents();
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t v[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = 4 * t + j;
        const int64_t n = i < nb ? co[i + 1] - co[i] : 0;
        v[j] = n < rk ? n : rk;
        sum += v[j];
    }
    int64_t incl = sum;  // inclusive scan of the per-thread sums within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t x = warp_tot[lane], y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        warp_tot[lane] = y - x;  // exclusive: everything before warp `lane`
    }
    __syncthreads();
    int64_t run = warp_tot[w] + incl - sum;  // everything before this thread's first request
    if (t == 0) cor[0] = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = 4 * t + j;
        run += v[j];
        if (i < nb) cor[i + 1] = run;
    }
}

// FP8 requests: the ids of request i's shortlist -- the first cor[i+1] -
// cor[i] positions of its top-rescore_k (all valid: a list shorter than
// rescore_k contributes all of its candidates) -- packed at cor[i].
__global__ void shortlist_ids(const int32_t* __restrict__ pos, int rk, const int64_t* __restrict__ co,
                              const int64_t* __restrict__ cor, const int32_t* __restrict__ cands, int nb,
                              int32_t* __restrict__ out) {
    griddep_wait();
    griddep_launch_dependents();
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(nb) * rk) return;
    const int i = static_cast<int>(idx / rk);
    const int j = static_cast<int>(idx - static_cast<int64_t>(i) * rk);
    if (j >= cor[i + 1] - cor[i]) return;
    const int32_t p = pos[idx];
    out[cor[i] + j] = p >= 0 ? cands[co[i] + p] : -1;
}

// Stage a batch into `sl` and enqueue its work; the result lands in the
// slot's pinned buffers when every sl.done event completes.
void launch(tms_server* s, Slot& sl, std::vector<RequestPtr>& batch) {
    const tms_server_config& c = s->cfg;
    for (auto& v : sl.reqs) v.clear();
    for (auto& r : batch) sl.reqs[r->store].push_back(r);
    sl.status = TMS_OK;
    const bool inject = c.inject_error_batch > 0 && s->batch_ordinal == static_cast<uint64_t>(c.inject_error_batch);
    for (int st = 0; st < kStores && !inject; ++st) {
        const int nb = static_cast<int>(sl.reqs[st].size());
        if (nb == 0) continue;
        int64_t total = 0;
        sl.h_co[st][0] = 0;
        for (int i = 0; i < nb; ++i) {
            const Request& r = *sl.reqs[st][i];
            std::memcpy(static_cast<uint8_t*>(sl.h_q[st]) + i * s->qbytes, r.query.data(), s->qbytes);
            if (!r.cands.empty()) std::memcpy(sl.h_c[st] + total, r.cands.data(), r.cands.size() * 4);
            total += static_cast<int64_t>(r.cands.size());
            sl.h_co[st][i + 1] = total;
        }
        tms_status rc = TMS_OK;
        if (!cuda_ok(cudaMemcpyAsync(sl.d_q[st], sl.h_q[st], nb * s->qbytes, cudaMemcpyHostToDevice, s->stream[st])) ||
            !cuda_ok(cudaMemcpyAsync(sl.d_c[st], sl.h_c[st], total * 4, cudaMemcpyHostToDevice, s->stream[st])) ||
            !cuda_ok(cudaMemcpyAsync(sl.d_co[st], sl.h_co[st], (nb + 1) * 8, cudaMemcpyHostToDevice, s->stream[st])))
            rc = TMS_ERR_CUDA;
        if (rc == TMS_OK && st == 0)
            rc = tms_score_dense(sl.d_q[st], c.dtype, nb, c.nq, c.d, c.doc_tokens, c.n_tokens, c.doc_offsets,
                                 c.doc_lengths, c.n_docs, sl.d_c[st], sl.d_co[st], total, sl.d_sc[st], s->stream[st]);
        if (rc == TMS_OK && st == 1) {
            rc = tms_build_pq_lut(sl.d_q[st], c.dtype, nb, c.nq, c.d, c.pq_codebook, c.pq_m, c.pq_k, sl.d_lut,
                                  s->stream[st]);
            if (rc == TMS_OK)
                rc = tms_score_pq(sl.d_lut, nb, c.nq, c.pq_m, c.pq_k, c.pq_codes, c.pq_n_tokens, c.pq_offsets,
                                  c.pq_lengths, c.pq_n_docs, sl.d_c[st], sl.d_co[st], total, sl.d_sc[st], s->stream[st]);
        }
        const bool rescore = st == 2 && c.rescore_k > 0;
        if (rc == TMS_OK && st == 2) {
            rc = tms_quantize_e4m3(sl.d_q[st], c.dtype, static_cast<int64_t>(nb) * c.nq, c.d, sl.d_qc, sl.d_qs,
                                   s->stream[st]);
            if (rc == TMS_OK)
                rc = tms_score_fp8(sl.d_qc, sl.d_qs, nb, c.nq, c.d, c.fp8_codes, c.fp8_scales, c.n_tokens,
                                   c.doc_offsets, c.doc_lengths, c.n_docs, sl.d_c[st], sl.d_co[st], total, sl.d_sc[st],
                                   s->stream[st]);
            if (rc == TMS_OK && rescore) {
                // shortlist: the rescore_k best FP8 scores of each request,
                // scored again on the dense store
                const int rk = c.rescore_k;
                rc = tms_topk(sl.d_sc[st], sl.d_co[st], nb, rk, sl.d_rts, sl.d_rtp, s->stream[st]);
                // the shortlists' CSR is built on the device; the host keeps
                // only their total (the re-score call's n_cand)
                int64_t total_r = 0;
                for (int i = 0; i < nb; ++i) {
                    const int64_t n = static_cast<int64_t>(sl.reqs[st][i]->cands.size());
                    total_r += n < rk ? n : rk;
                }
                if (rc == TMS_OK) {
                    if (!cuda_ok(launch_dependent(shortlist_csr, dim3(1), dim3(kCsrThreads), 0, s->stream[st],
                                                  sl.d_co[st], nb, rk, sl.d_cor)))
                        rc = TMS_ERR_CUDA;
                }
                if (rc == TMS_OK) {
                    const int64_t n = static_cast<int64_t>(nb) * rk;
                    if (!cuda_ok(launch_dependent(shortlist_ids, dim3(static_cast<unsigned>((n + 255) / 256)),
                                                  dim3(256), 0, s->stream[st], sl.d_rtp, rk, sl.d_co[st], sl.d_cor,
                                                  sl.d_c[st], nb, sl.d_cr)))
                        rc = TMS_ERR_CUDA;
                }
                if (rc == TMS_OK)
                    rc = tms_score_dense(sl.d_q[st], c.dtype, nb, c.nq, c.d, c.doc_tokens, c.n_tokens, c.doc_offsets,
                                         c.doc_lengths, c.n_docs, sl.d_cr, sl.d_cor, total_r, sl.d_scr,
                                         s->stream[st]);
                if (rc == TMS_OK &&
                    !cuda_ok(cudaMemcpyAsync(sl.h_rtp, sl.d_rtp, static_cast<size_t>(nb) * rk * 4,
                                             cudaMemcpyDeviceToHost, s->stream[st])))
                    rc = TMS_ERR_CUDA;
            }
        }
        if (rc == TMS_OK) {
            if (rescore)
                rc = tms_topk(sl.d_scr, sl.d_cor, nb, c.topk, sl.d_ts[st], sl.d_tp[st], s->stream[st]);
            else
                rc = tms_topk(sl.d_sc[st], sl.d_co[st], nb, c.topk, sl.d_ts[st], sl.d_tp[st], s->stream[st]);
        }
        if (rc == TMS_OK &&
            (!cuda_ok(cudaMemcpyAsync(sl.h_ts[st], sl.d_ts[st], static_cast<size_t>(nb) * c.topk * 4,
                                      cudaMemcpyDeviceToHost, s->stream[st])) ||
             !cuda_ok(cudaMemcpyAsync(sl.h_tp[st], sl.d_tp[st], static_cast<size_t>(nb) * c.topk * 4,
                                      cudaMemcpyDeviceToHost, s->stream[st]))))
            rc = TMS_ERR_CUDA;
        if (rc != TMS_OK) sl.status = rc;
    }
    if (inject) sl.status = TMS_ERR_CUDA;
    for (int st = 0; st < kStores; ++st)
        if (s->stream[st] && !cuda_ok(cudaEventRecord(sl.done[st], s->stream[st]))) sl.status = TMS_ERR_CUDA;
}

// Wait for a slot's batch and hand each request its result.
void complete(tms_server* s, Slot& sl) {
    const tms_server_config& c = s->cfg;
    for (int st = 0; st < kStores; ++st)
        if (s->stream[st] && !cuda_ok(cudaEventSynchronize(sl.done[st])) && sl.status == TMS_OK)
            sl.status = TMS_ERR_CUDA;
    const Clock::time_point now = Clock::now();
    uint64_t n = 0, cands = 0;
    int64_t bytes = 0;
    for (int st = 0; st < kStores; ++st) {
        const bool rescore = st == 2 && c.rescore_k > 0;
        for (size_t i = 0; i < sl.reqs[st].size(); ++i) {
            Request& r = *sl.reqs[st][i];
            r.status = sl.status;
            r.scores.assign(c.topk, -INFINITY);
            r.ids.assign(c.topk, -1);
            if (sl.status == TMS_OK) {
                const float* ts = sl.h_ts[st] + i * c.topk;
                const int32_t* tp = sl.h_tp[st] + i * c.topk;
                const int32_t* rp = rescore ? sl.h_rtp + i * static_cast<size_t>(c.rescore_k) : nullptr;
                const int64_t n_list = static_cast<int64_t>(r.cands.size());
                const int64_t n_short = rescore ? (n_list < c.rescore_k ? n_list : c.rescore_k) : n_list;
                for (int j = 0; j < c.topk; ++j) {
                    r.scores[j] = ts[j];
                    int64_t p = (tp[j] >= 0 && tp[j] < n_short) ? tp[j] : -1;  // position in the scored list
                    if (rescore && p >= 0) p = rp[p];                             // shortlist -> request's list
                    r.ids[j] = (p >= 0 && p < n_list) ? r.cands[p] : -1;
                }
            }
            r.t_done = now;
            cands += r.cands.size();
            bytes += r.bytes;
            ++n;
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int st = 0; st < kStores; ++st)
            for (auto& r : sl.reqs[st]) r->done = true;
        s->unfinished -= static_cast<int>(n);
        s->unfinished_bytes -= bytes;
        s->stats.requests += n;
        s->stats.candidates += cands;
    }
    for (auto& v : sl.reqs) v.clear();
    s->cv_done.notify_all();
}

void worker_main(tms_server* s) {
    cudaSetDevice(s->device);
    bool inflight[2] = {false, false};
    int cur = 0;
    for (;;) {
        std::vector<RequestPtr> batch;
        bool quit = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const bool busy = inflight[cur ^ 1];
            if (!busy) s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            int64_t cands = 0;
            while (!s->pending.empty() && static_cast<int>(batch.size()) < s->cfg.max_batch_requests) {
                const RequestPtr& r = s->pending.front();
                const int64_t n = static_cast<int64_t>(r->cands.size());
                if (!batch.empty() && cands + n > s->cfg.max_batch_candidates) break;
                cands += n;
                batch.push_back(r);
                s->pending.pop_front();
            }
            if (!batch.empty()) {
                ++s->batch_ordinal;
                ++s->stats.batches;
            }
            quit = batch.empty() && !busy && s->stop;
        }
        if (quit) break;
        if (!batch.empty()) {
            const Clock::time_point t0 = Clock::now();
            launch(s, s->slots[cur], batch);
            const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.enqueue_s += dt;
        }
        if (inflight[cur ^ 1]) {
            complete(s, s->slots[cur ^ 1]);
            inflight[cur ^ 1] = false;
        }
        if (!batch.empty()) {
            inflight[cur] = true;
            cur ^= 1;
        }
    }
}

bool config_ok(const tms_server_config& c) {
    if (c.dtype != TMS_F16 && c.dtype != TMS_BF16) return false;
    if (!c.doc_tokens || !c.doc_offsets || !c.doc_lengths || c.n_docs < 1 || c.n_tokens < 1) return false;
    if (c.d < 8 || c.d > 1024 || c.d % 8 != 0) return false;
    if (c.nq < 1 || c.nq > 128 || c.topk < 1 || c.topk > 1024) return false;
    if (c.max_batch_requests < 1 || c.max_batch_requests > 4096 || c.max_batch_candidates < 1 ||
        c.max_batch_candidates >= (int64_t(1) << 31) || c.max_pending < 1 || c.max_pending_bytes < 0 ||
        c.inject_error_batch < 0)
        return false;
    if (c.pq_codes) {
        if (!c.pq_codebook || !c.pq_offsets || !c.pq_lengths || c.pq_n_docs < 1 || c.pq_n_tokens < 1) return false;
        if (c.pq_m != 4 && c.pq_m != 8 && c.pq_m != 16 && c.pq_m != 32) return false;
        if (c.pq_k < 1 || c.pq_k > 256 || c.pq_m * c.pq_k > 4096 || c.d % c.pq_m != 0) return false;
    }
    if (c.fp8_codes) {
        if (!c.fp8_scales || c.d < 16 || c.d % 16 != 0) return false;
        if (c.rescore_k != 0 && (c.rescore_k < c.topk || c.rescore_k > 1024)) return false;
    } else if (c.rescore_k != 0) {
        return false;
    }
    return true;
}

void destroy(tms_server* s) {
    for (auto& sl : s->slots) free_slot(sl);
    for (int st = 0; st < kStores; ++st)
        if (s->stream[st]) cudaStreamDestroy(s->stream[st]);
    (void)cudaGetLastError();
    delete s;
}

}  // namespace server

}  // namespace tms

extern "C" tms_status tms_server_create(const tms_server_config* cfg, tms_server** out) {
    using namespace tms::server;
    if (!cfg || !out || !config_ok(*cfg)) return TMS_ERR_INVALID_ARG;
    tms_server* s = new (std::nothrow) tms_server();
    if (!s) return TMS_ERR_CUDA;
    s->cfg = *cfg;
    s->qbytes = static_cast<size_t>(cfg->nq) * cfg->d * 2;
    if (!cuda_ok(cudaGetDevice(&s->device)) ||
        !cuda_ok(cudaStreamCreateWithFlags(&s->stream[0], cudaStreamNonBlocking)) ||
        (cfg->pq_codes && !cuda_ok(cudaStreamCreateWithFlags(&s->stream[1], cudaStreamNonBlocking))) ||
        (cfg->fp8_codes && !cuda_ok(cudaStreamCreateWithFlags(&s->stream[2], cudaStreamNonBlocking))) ||
        !alloc_slot(s, s->slots[0]) || !alloc_slot(s, s->slots[1])) {
        destroy(s);
        return TMS_ERR_CUDA;
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        destroy(s);
        return TMS_ERR_CUDA;
    }
    *out = s;
    return TMS_OK;
}

extern "C" tms_status tms_server_submit(tms_server* s, tms_store store, const void* query, const int32_t* cand_ids,
                                        int64_t n_cand, uint64_t* ticket) {
    using namespace tms::server;
    if (!s || !query || !ticket || n_cand < 0 || (n_cand > 0 && !cand_ids)) return TMS_ERR_INVALID_ARG;
    if (store != TMS_STORE_DENSE && store != TMS_STORE_PQ && store != TMS_STORE_FP8) return TMS_ERR_INVALID_ARG;
    if ((store == TMS_STORE_PQ && !s->cfg.pq_codes) || (store == TMS_STORE_FP8 && !s->cfg.fp8_codes))
        return TMS_ERR_UNSUPPORTED;
    if (n_cand > s->cfg.max_batch_candidates) return TMS_ERR_UNSUPPORTED;
    // Ids are checked here, next to the copy, so a bad id never reaches the
    // device (where it would score NaN and set a bit of the process-wide
    // device error word that another caller would then read as its own).
    const int64_t n_ids = store == TMS_STORE_PQ ? s->cfg.pq_n_docs : s->cfg.n_docs;
    for (int64_t i = 0; i < n_cand; ++i)
        if (cand_ids[i] < 0 || cand_ids[i] >= n_ids) return TMS_ERR_INVALID_ARG;
    const int64_t bytes = static_cast<int64_t>(s->qbytes) + 8 * n_cand;
    if (s->cfg.max_pending_bytes > 0 && bytes > s->cfg.max_pending_bytes) return TMS_ERR_UNSUPPORTED;
    auto r = std::make_shared<Request>();
    r->store = store;
    r->bytes = bytes;
    r->query.assign(static_cast<const uint8_t*>(query), static_cast<const uint8_t*>(query) + s->qbytes);
    r->cands.assign(cand_ids, cand_ids + n_cand);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return TMS_ERR_INVALID_ARG;
        if (s->unfinished >= s->cfg.max_pending ||
            (s->cfg.max_pending_bytes > 0 && s->unfinished_bytes + bytes > s->cfg.max_pending_bytes)) {
            ++s->stats.rejected;
            return TMS_ERR_BUSY;
        }
        r->ticket = s->next_ticket++;
        s->pending.push_back(r);
        s->live.emplace(r->ticket, r);
        ++s->unfinished;
        s->unfinished_bytes += bytes;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return TMS_OK;
}

extern "C" tms_status tms_server_wait(tms_server* s, uint64_t ticket, double timeout_s, float* out_scores,
                                      int32_t* out_ids, double* latency_s) {
    using namespace tms::server;
    if (!s || !out_scores || !out_ids || !(timeout_s >= 0.0)) return TMS_ERR_INVALID_ARG;
    RequestPtr r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        const auto it = s->live.find(ticket);
        if (it == s->live.end()) return TMS_ERR_INVALID_ARG;
        r = it->second;
        const auto limit = std::chrono::duration<double>(timeout_s > 1e6 ? 1e6 : timeout_s);
        if (!s->cv_done.wait_for(lk, limit, [&] { return r->done; })) return TMS_ERR_TIMEOUT;
        // The lock was released while waiting: submit may have rehashed the
        // map (invalidating `it`) and another waiter on the same ticket may
        // have taken the result.  Erase by key; only one waiter wins.
        if (s->live.erase(ticket) == 0) return TMS_ERR_INVALID_ARG;
    }
    std::memcpy(out_scores, r->scores.data(), r->scores.size() * 4);
    std::memcpy(out_ids, r->ids.data(), r->ids.size() * 4);
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    return r->status;
}

extern "C" tms_status tms_server_get_stats(tms_server* s, tms_server_stats* out) {
    if (!s || !out) return TMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return TMS_OK;
}

extern "C" tms_status tms_server_destroy(tms_server* s) {
    using namespace tms::server;
    if (!s) return TMS_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy(s);
    return TMS_OK;
}
