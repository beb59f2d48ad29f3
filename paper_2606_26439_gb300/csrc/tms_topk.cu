// tms_topk.cu -- per-query top-k after scoring (Section 6.8, end-to-end retrieval latency).
//
// The select step (one 1024-thread CTA over n elements):
//   1. scores map to order-preserving 32-bit keys (NaN after every number,
//      -0 == +0; key 0 is kept for workspace padding, below NaN);
//   2. a byte-wise radix select (four histogram passes, warp-private
//      histograms filled with match_any so equal digits cost one update)
//      finds the k-th largest key T and how many keys equal to T belong
//      to the top-k; a list of up to 12 x 1024 keys is read once and kept
//      in registers for all passes, a longer one is re-read per pass with
//      eight loads in flight per thread;
//   3. one pass in element order keeps every key > T and the first keys ==
//      T, using a block-wide ordered scan -- the lowest positions, because
//      equal keys always appear in ascending position order; when every
//      key equal to T is kept (no tie across the cut) the pass keeps every
//      key >= T in any order, without the scan;
//   4. a bitonic sort orders the <= k survivors by (key desc, position asc).
//
// tms_topk: one CTA per query selects from the whole list.
// tms_topk_split: S CTAs per query each select the top-k of one contiguous
// slice of the list into the caller's workspace (k sorted entries, padded
// with key 0), then one CTA per query selects from the S x k entries.  The
// order (key desc, position asc) is total, so every member of the list's
// top-k is in its slice's top-k, and the merge sees equal keys in ascending
// position (slices are in position order, each slice sorted): the result is
// bit-identical to tms_topk.  Deterministic and exact: it depends only on
// the scores.
#include <algorithm>
#include <map>
#include <mutex>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {
namespace topk {

constexpr int kThreads = 1024;  // four quarters of 256 threads: the histogram sums below rely on it
constexpr int kWarps = kThreads / 32;
constexpr int kMaxK = 1024;
constexpr int kMaxSlices = 64;

__device__ __forceinline__ uint32_t score_key(float x) {
    if (x != x) return 1u;  // NaN: after every number (the smallest number's key is 0x007fffff)
    if (x == 0.0f) x = 0.0f;
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// A survivor: key in the high word, ~position in the low word, so that one
// unsigned comparison orders by (key desc, position asc).
__device__ __forceinline__ unsigned long long pack(uint32_t key, uint32_t pos) {
    return (static_cast<unsigned long long>(key) << 32) | static_cast<unsigned long long>(0xffffffffu - pos);
}
__device__ __forceinline__ uint32_t key_of(unsigned long long e) { return static_cast<uint32_t>(e >> 32); }
__device__ __forceinline__ uint32_t pos_of(unsigned long long e) {
    return 0xffffffffu - static_cast<uint32_t>(e & 0xffffffffull);
}

struct Smem {
    uint32_t whist[kWarps][256];
    uint32_t hist[256];
    unsigned long long sel[kMaxK];
    int scan_buf[33];
    uint32_t digit;
    int need;
    int eq;  // keys equal to the k-th largest (set by the last radix pass)
    int count;
};

// Elements a thread reads ahead of processing them, so that their loads
// overlap instead of each waiting in turn; a list of at most
// kResident * kThreads elements is instead read once and kept in registers
// for every pass.
constexpr int kAhead = 8;
constexpr int kResident = 12;

// Exclusive scan of one int per thread over the CTA; returns the prefix and
// writes the total to *total.  `buf` holds kWarps + 1 ints.
__device__ __forceinline__ int block_exclusive_scan(int v, int* buf, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) buf[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = buf[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        buf[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31) buf[32] = wi;
    }
    __syncthreads();
    const int res = buf[warp] + inc - v;
    *total = buf[32];
    __syncthreads();
    return res;
}

// The select step over n elements (element i: key key_at(i), position
// pos_at(i); elements with equal keys must come in ascending position
// order).  Leaves the min(k, n) survivors sorted by (key desc, position
// asc) in sm.sel[0 .. count) and returns count.  Every thread of the CTA
// calls it.  RES: n <= kResident * kThreads, keys held in registers.
template <bool RES, class KeyAt, class PosAt>
__device__ int select_sorted(int n, int k, KeyAt key_at, PosAt pos_at, Smem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int A = RES ? kResident : kAhead;  // elements per thread per step
    uint32_t prefix = 0, mask = 0;
    int need = min(k, n);  // how many of the keys matching prefix/mask still to take
    const bool select_all = n <= k;
    uint32_t rkeys[RES ? kResident : 1];
    if constexpr (RES) {
#pragma unroll
        for (int u = 0; u < kResident; ++u) {
            const int i = u * kThreads + threadIdx.x;
            rkeys[u] = i < n ? key_at(i) : 0u;
        }
    }
    if (!select_all) {
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < kWarps * 256; b += kThreads) (&sm.whist[0][0])[b] = 0;
            __syncthreads();
            for (int base = 0; base < n; base += A * kThreads) {
                uint32_t keys[A];
#pragma unroll
                for (int u = 0; u < A; ++u) {
                    const int i = base + u * kThreads + threadIdx.x;
                    if constexpr (RES) keys[u] = rkeys[u];
                    else keys[u] = i < n ? key_at(i) : 0u;
                }
#pragma unroll
                for (int u = 0; u < A; ++u) {
                    if (RES && u * kThreads >= n) break;  // the same for the whole CTA
                    const int i = base + u * kThreads + threadIdx.x;
                    const uint32_t key = keys[u];
                    const bool match = i < n && ((key & mask) == prefix);
                    const unsigned active = __ballot_sync(0xffffffffu, match);
                    if (match) {
                        const uint32_t dgt = (key >> shift) & 255u;
                        const unsigned peers = __match_any_sync(active, dgt);
                        if (lane == __ffs(peers) - 1) sm.whist[warp][dgt] += __popc(peers);
                    }
                }
            }
            __syncthreads();
            // The largest digit whose suffix count (keys with that digit or
            // a larger one) reaches `need`: thread t < 256 holds the count
            // of digit 255 - t, an inclusive scan over the first 8 warps
            // gives the suffix counts, and the one thread whose bin crosses
            // `need` records the digit and what is still needed below it.
            if (threadIdx.x == 0) {
                sm.digit = 0;
                sm.need = need;
                sm.eq = -1;
            }
            // the 32 warp histograms summed in two steps: four quarters of
            // 8 warps in parallel (each quarter's sum left in its first
            // warp's row), then the four quarter sums
            {
                const int qtr = threadIdx.x >> 8;
                const int dgt = 255 - (threadIdx.x & 255);
                uint32_t t = 0;
#pragma unroll
                for (int w = 0; w < kWarps / 4; ++w) t += sm.whist[qtr * (kWarps / 4) + w][dgt];
                sm.whist[qtr * (kWarps / 4)][dgt] = t;  // only this thread reads or writes column dgt of the quarter
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                const int dgt = 255 - threadIdx.x;
                int tot = 0;
#pragma unroll
                for (int qtr = 0; qtr < 4; ++qtr) tot += static_cast<int>(sm.whist[qtr * (kWarps / 4)][dgt]);
                int inc = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += v;
                }
                if (lane == 31) sm.scan_buf[warp] = inc;
                sm.hist[dgt] = static_cast<uint32_t>(inc);  // within-warp suffix count, completed below
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                const int dgt = 255 - threadIdx.x;
                int before = 0;  // keys with a digit above this warp's bins
                for (int w = 0; w < warp; ++w) before += sm.scan_buf[w];
                const int incl = before + static_cast<int>(sm.hist[dgt]);
                const int tot = static_cast<int>(sm.hist[dgt]) -
                                (lane > 0 ? static_cast<int>(sm.hist[dgt + 1]) : 0);  // this digit's count
                const int excl = incl - tot;
                if (incl >= need && excl < need) {
                    sm.digit = static_cast<uint32_t>(dgt);
                    sm.need = need - excl;
                    sm.eq = tot;  // after the last pass: the keys equal to T
                }
            }
            __syncthreads();
            prefix |= sm.digit << shift;
            mask |= 255u << shift;
            need = sm.need;
            __syncthreads();
        }
    }
    // prefix is now the k-th largest key T (when !select_all); `need` keys
    // equal to T are taken, lowest positions first.  When every key equal
    // to T is taken (always, unless T is tied across the cut) no ranking is
    // needed: the survivors are the same set whatever order they arrive in,
    // and the sort below fixes their order.
    const bool all_eq = select_all || sm.eq == need;
    if (threadIdx.x == 0) sm.count = 0;
    __syncthreads();
    if (all_eq) {
        for (int base = 0; base < n; base += A * kThreads) {
            uint32_t keys[A];
#pragma unroll
            for (int u = 0; u < A; ++u) {
                const int i = base + u * kThreads + threadIdx.x;
                if constexpr (RES) keys[u] = rkeys[u];
                else keys[u] = i < n ? key_at(i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < A; ++u) {
                if (RES && u * kThreads >= n) break;
                const int i = base + u * kThreads + threadIdx.x;
                if (i < n && (select_all || keys[u] >= prefix)) {
                    const int slot = atomicAdd(&sm.count, 1);
                    if (slot < kMaxK) sm.sel[slot] = pack(keys[u], pos_at(i));
                }
            }
        }
    } else {
        int taken_eq = 0;
        for (int base = 0; base < n; base += kThreads) {
            const int i = base + threadIdx.x;
            const bool in = i < n;
            const uint32_t key = in ? key_at(i) : 0u;
            const bool gt = in && key > prefix;
            const bool eq = in && key == prefix;
            int eq_total = 0;
            const int rank = block_exclusive_scan(eq ? 1 : 0, sm.scan_buf, &eq_total);
            const bool take = gt || (eq && taken_eq + rank < need);
            if (take) {
                const int slot = atomicAdd(&sm.count, 1);
                if (slot < kMaxK) sm.sel[slot] = pack(key, pos_at(i));
            }
            taken_eq += eq_total;
        }
    }
    __syncthreads();
    const int cnt = min(sm.count, kMaxK);
    // pad to the sort width with zero entries (below every real entry)
    int width = 1;
    while (width < cnt) width <<= 1;
    for (int i = cnt + threadIdx.x; i < width; i += kThreads) sm.sel[i] = 0ull;
    __syncthreads();
    // bitonic sort, descending
    for (int size = 2; size <= width; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < width; i += kThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = sm.sel[i], b = sm.sel[j];
                    if (desc ? (a < b) : (a > b)) {
                        sm.sel[i] = b;
                        sm.sel[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    return cnt;
}

// select_sorted with the keys held in registers when the list is short
// enough (n is the same for the whole CTA).
template <class KeyAt, class PosAt>
__device__ int select_any(int n, int k, KeyAt key_at, PosAt pos_at, Smem& sm) {
    return n <= kResident * kThreads ? select_sorted<true>(n, k, key_at, pos_at, sm)
                                     : select_sorted<false>(n, k, key_at, pos_at, sm);
}

// The list [c0, c1) of query q, checked: a negative start or a decreasing
// pair is a CSR error -- flagged (when err is given), and the list read as
// empty (negative start) or clamped to its start, never read below it.
__device__ __forceinline__ void query_list(const int64_t* cand_offsets, int q, unsigned int* err, int64_t* c0,
                                           int64_t* c1) {
    int64_t a = cand_offsets[q], b = cand_offsets[q + 1];
    if (a < 0 || b < a) {
        if (err != nullptr && threadIdx.x == 0) atomicOr(err, TMS_DEVERR_BAD_CSR);
        if (a < 0) a = b = 0;
        if (b < a) b = a;
    }
    *c0 = a;
    *c1 = b;
}

// Row q of the output: the survivors' scores and positions, (-inf, -1)
// past them and for padding entries (key 0).
__device__ __forceinline__ void write_out(const Smem& sm, int cnt, int k, const float* list, float* out_s,
                                          int32_t* out_p) {
    for (int r = threadIdx.x; r < k; r += kThreads) {
        float sc = -INFINITY;
        int pos = -1;
        if (r < cnt && key_of(sm.sel[r]) != 0u) {
            pos = static_cast<int>(pos_of(sm.sel[r]));
            sc = list[pos];
        }
        out_s[r] = sc;
        out_p[r] = pos;
    }
}

__device__ __forceinline__ int list_len(int64_t c0, int64_t c1) {
    return static_cast<int>((c1 - c0) > 0x7fffffff ? 0x7fffffff : (c1 - c0));
}

__global__ void __launch_bounds__(kThreads, 1)
    topk_kernel(const float* __restrict__ scores, const int64_t* __restrict__ cand_offsets, int k,
                float* __restrict__ out_scores, int32_t* __restrict__ out_pos, unsigned int* err) {
    __shared__ Smem sm;
    griddep_wait();
    griddep_launch_dependents();
    const int q = blockIdx.x;
    int64_t c0, c1;
    query_list(cand_offsets, q, err, &c0, &c1);
    const float* s = scores + c0;
    const int cnt = select_any(
        list_len(c0, c1), k, [&](int i) { return score_key(s[i]); }, [](int i) { return static_cast<uint32_t>(i); },
        sm);
    write_out(sm, cnt, k, s, out_scores + static_cast<int64_t>(q) * k, out_pos + static_cast<int64_t>(q) * k);
}

// Slice `blockIdx.x % S` of query `blockIdx.x / S`: its top-k (sorted,
// padded with zero entries to k) at ws[(q * S + slice) * k ...].
__global__ void __launch_bounds__(kThreads, 1)
    topk_slice_kernel(const float* __restrict__ scores, const int64_t* __restrict__ cand_offsets, int k, int S,
                      unsigned long long* __restrict__ ws, unsigned int* err) {
    __shared__ Smem sm;
    griddep_wait();
    griddep_launch_dependents();
    const int q = blockIdx.x / S;
    const int sl = blockIdx.x - q * S;
    int64_t c0, c1;
    query_list(cand_offsets, q, sl == 0 ? err : nullptr, &c0, &c1);
    const int64_t len = list_len(c0, c1);
    const int64_t a = len * sl / S, b = len * (sl + 1) / S;  // slice [a, b) of the list
    const float* s = scores + c0 + a;
    const int cnt = select_any(
        static_cast<int>(b - a), k, [&](int i) { return score_key(s[i]); },
        [&](int i) { return static_cast<uint32_t>(a + i); }, sm);
    unsigned long long* dst = ws + static_cast<int64_t>(blockIdx.x) * k;
    for (int r = threadIdx.x; r < k; r += kThreads) dst[r] = r < cnt ? sm.sel[r] : 0ull;
}

// Query blockIdx.x: the top-k of its S x k slice entries.
__global__ void __launch_bounds__(kThreads, 1)
    topk_merge_kernel(const float* __restrict__ scores, const int64_t* __restrict__ cand_offsets, int k, int S,
                      const unsigned long long* __restrict__ ws, float* __restrict__ out_scores,
                      int32_t* __restrict__ out_pos) {
    __shared__ Smem sm;
    griddep_wait();
    griddep_launch_dependents();
    const int q = blockIdx.x;
    int64_t c0, c1;
    query_list(cand_offsets, q, nullptr, &c0, &c1);
    const unsigned long long* e = ws + static_cast<int64_t>(q) * S * k;
    const int cnt = select_any(
        S * k, k, [&](int i) { return key_of(e[i]); }, [&](int i) { return pos_of(e[i]); }, sm);
    write_out(sm, cnt, k, scores + c0, out_scores + static_cast<int64_t>(q) * k,
              out_pos + static_cast<int64_t>(q) * k);
}

// Slices per query of tms_topk_split: about two CTAs per SM in all, lists
// of a few thousand scores per slice at least, at most kMaxSlices.
int slices(int sm_count, int n_queries, int k, int64_t n_cand) {
    const int64_t avg = n_cand / n_queries;
    const int64_t by_grid = (2 * static_cast<int64_t>(sm_count) + n_queries - 1) / n_queries;
    const int64_t by_len = avg / std::max<int64_t>(2048, 4 * static_cast<int64_t>(k));
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({static_cast<int64_t>(kMaxSlices), by_grid, by_len})));
}

bool args_ok(const float* scores, const int64_t* cand_offsets, int n_queries, int k, const float* out_scores,
             const int32_t* out_pos) {
    return n_queries >= 1 && k >= 1 && k <= kMaxK && scores && cand_offsets && out_scores && out_pos &&
           aligned16(cand_offsets) && aligned16(out_scores) && aligned16(out_pos) &&
           (reinterpret_cast<uintptr_t>(scores) & 3u) == 0;
}

}  // namespace topk
}  // namespace tms

extern "C" tms_status tms_topk(const float* scores, const int64_t* cand_offsets, int n_queries, int topk,
                               float* out_scores, int32_t* out_pos, cudaStream_t stream) {
    using namespace tms;
    if (!topk::args_ok(scores, cand_offsets, n_queries, topk, out_scores, out_pos)) return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    return launch_status(launch_dependent(topk::topk_kernel, dim3(static_cast<unsigned>(n_queries)),
                                          dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, out_scores,
                                          out_pos, dev.err));
}

extern "C" tms_status tms_topk_workspace_size(int n_queries, int topk, int64_t n_cand, int64_t* bytes) {
    using namespace tms;
    if (n_queries < 1 || topk < 1 || topk > topk::kMaxK || n_cand < 0 || bytes == nullptr) return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    const int S = topk::slices(dev.sm_count, n_queries, topk, n_cand);
    *bytes = S > 1 ? static_cast<int64_t>(n_queries) * S * topk * 8 : 0;
    return TMS_OK;
}

extern "C" tms_status tms_topk_split(const float* scores, const int64_t* cand_offsets, int n_queries, int topk,
                                     int64_t n_cand, float* out_scores, int32_t* out_pos, void* workspace,
                                     int64_t workspace_bytes, cudaStream_t stream) {
    using namespace tms;
    if (!topk::args_ok(scores, cand_offsets, n_queries, topk, out_scores, out_pos) || n_cand < 0 ||
        workspace_bytes < 0)
        return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    const int S = topk::slices(dev.sm_count, n_queries, topk, n_cand);
    if (S == 1) {
        return launch_status(launch_dependent(topk::topk_kernel, dim3(static_cast<unsigned>(n_queries)),
                                              dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, out_scores,
                                              out_pos, dev.err));
    }
    const int64_t need = static_cast<int64_t>(n_queries) * S * topk * 8;
    if (workspace == nullptr || !aligned16(workspace) || workspace_bytes < need) return TMS_ERR_INVALID_ARG;
    auto* ws = static_cast<unsigned long long*>(workspace);
    st = launch_status(launch_dependent(topk::topk_slice_kernel, dim3(static_cast<unsigned>(n_queries * S)),
                                        dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, S, ws, dev.err));
    if (st != TMS_OK) return st;
    return launch_status(launch_dependent(topk::topk_merge_kernel, dim3(static_cast<unsigned>(n_queries)),
                                          dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, S, ws,
                                          out_scores, out_pos));
}

// ---------------------------------------------------------------------------
// tms_topk_split_noalloc: tms_topk_split for callers that cannot allocate
// device memory.  The slice entries go to one fixed array in the library's
// own device memory instead of a caller workspace; it exists once per GPU
// that loads the library, for the life of the process.
namespace tms {
namespace topk {

constexpr int64_t kNoAllocScratchBytes = int64_t(4) << 20;  // 4 MiB
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];

// The device address of g_noalloc_scratch on the current device.  Host code
// sees the array's name only as a host-side stand-in, so the address is
// looked up with cudaGetSymbolAddress the first time a device asks (that
// device current) and remembered per device ordinal.
tms_status noalloc_scratch(int ordinal, unsigned long long** out) {
    static std::mutex m;
    static std::map<int, unsigned long long*> addr;
    std::lock_guard<std::mutex> lk(m);
    auto it = addr.find(ordinal);
    if (it == addr.end()) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return TMS_ERR_CUDA;
        }
        it = addr.emplace(ordinal, static_cast<unsigned long long*>(p)).first;
    }
    *out = it->second;
    return TMS_OK;
}

}  // namespace topk
}  // namespace tms

extern "C" tms_status tms_topk_split_noalloc(const float* scores, const int64_t* cand_offsets, int n_queries,
                                             int topk, int64_t n_cand, float* out_scores, int32_t* out_pos,
                                             cudaStream_t stream) {
    using namespace tms;
    if (!topk::args_ok(scores, cand_offsets, n_queries, topk, out_scores, out_pos) || n_cand < 0)
        return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    const int S = topk::slices(dev.sm_count, n_queries, topk, n_cand);
    if (S == 1) {  // one CTA per query: no scratch at all
        return launch_status(launch_dependent(topk::topk_kernel, dim3(static_cast<unsigned>(n_queries)),
                                              dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, out_scores,
                                              out_pos, dev.err));
    }
    const int64_t need = static_cast<int64_t>(n_queries) * S * topk * 8;
    if (need > topk::kNoAllocScratchBytes) return TMS_ERR_UNSUPPORTED;
    unsigned long long* ws = nullptr;
    st = topk::noalloc_scratch(dev.ordinal, &ws);
    if (st != TMS_OK) return st;
    // Every slice writes all k of its entries (padding included), so nothing
    // from an earlier call is ever read.
    st = launch_status(launch_dependent(topk::topk_slice_kernel, dim3(static_cast<unsigned>(n_queries * S)),
                                        dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, S, ws, dev.err));
    if (st != TMS_OK) return st;
    return launch_status(launch_dependent(topk::topk_merge_kernel, dim3(static_cast<unsigned>(n_queries)),
                                          dim3(topk::kThreads), 0, stream, scores, cand_offsets, topk, S, ws,
                                          out_scores, out_pos));
}
