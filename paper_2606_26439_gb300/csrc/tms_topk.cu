// tms_topk.cu -- per-query top-k after scoring (Section 6.8, end-to-end retrieval latency).
//
// One 1024-thread CTA per query:
//   1. scores map to order-preserving 32-bit keys (NaN lowest, -0 == +0);
//   2. a byte-wise radix select (four histogram passes, warp-private
//      histograms filled with match_any so equal digits cost one update)
//      finds the k-th largest key T and how many keys equal to T belong
//      to the top-k;
//   3. one pass in position order keeps every key > T and the first
//      (lowest-position) keys == T, using a block-wide ordered scan;
//   4. a bitonic sort orders the <= k survivors by (key desc, position asc)
//      and they are written with their original float value.
// Deterministic and exact: the result depends only on the scores.
#include <algorithm>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {
namespace topk {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxK = 1024;

__device__ __forceinline__ uint32_t score_key(float x) {
    if (x != x) return 0u;  // NaN sorts after everything
    if (x == 0.0f) x = 0.0f;
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Exclusive scan of one int per thread over the CTA; returns the prefix and
// writes the total to *total.  `buf` holds kWarps ints.
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

__global__ void __launch_bounds__(kThreads, 1)
    topk_kernel(const float* __restrict__ scores, const int64_t* __restrict__ cand_offsets, int n_queries, int k,
                float* __restrict__ out_scores, int32_t* __restrict__ out_pos, unsigned int* err) {
    __shared__ uint32_t whist[kWarps][256];
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long sel[kMaxK];
    __shared__ int scan_buf[33];
    __shared__ uint32_t s_digit;
    __shared__ int s_need;
    __shared__ int s_count;
    const int q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // A list must lie inside the scores buffer: a negative start or a
    // decreasing pair is a CSR error -- flagged, and the list read as empty
    // (a negative start) or clamped to its start (never read below it).
    int64_t c0 = cand_offsets[q], c1 = cand_offsets[q + 1];
    if (c0 < 0 || c1 < c0) {
        if (threadIdx.x == 0) atomicOr(err, TMS_DEVERR_BAD_CSR);
        if (c0 < 0) c0 = c1 = 0;
        if (c1 < c0) c1 = c0;
    }
    const int n = static_cast<int>((c1 - c0) > 0x7fffffff ? 0x7fffffff : (c1 - c0));
    const float* s = scores + c0;

    uint32_t prefix = 0, mask = 0;
    int need = min(k, n);  // how many of the keys matching prefix/mask still to take
    const bool select_all = n <= k;
    if (!select_all) {
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < kWarps * 256; b += kThreads) (&whist[0][0])[b] = 0;
            __syncthreads();
            for (int base = 0; base < n; base += kThreads) {
                const int i = base + threadIdx.x;
                const bool in = i < n;
                const uint32_t key = in ? score_key(s[i]) : 0u;
                const bool match = in && ((key & mask) == prefix);
                const unsigned active = __ballot_sync(0xffffffffu, match);
                if (match) {
                    const uint32_t dgt = (key >> shift) & 255u;
                    const unsigned peers = __match_any_sync(active, dgt);
                    if (lane == __ffs(peers) - 1) whist[warp][dgt] += __popc(peers);
                }
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                uint32_t tot = 0;
                for (int w = 0; w < kWarps; ++w) tot += whist[w][threadIdx.x];
                hist[threadIdx.x] = tot;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                // largest digit whose suffix count reaches `need`
                int acc = 0;
                int dgt = 255;
                for (; dgt >= 0; --dgt) {
                    if (acc + static_cast<int>(hist[dgt]) >= need) break;
                    acc += static_cast<int>(hist[dgt]);
                }
                s_digit = static_cast<uint32_t>(dgt < 0 ? 0 : dgt);
                s_need = need - acc;
            }
            __syncthreads();
            prefix |= s_digit << shift;
            mask |= 255u << shift;
            need = s_need;
            __syncthreads();
        }
    }
    // prefix is now the k-th largest key T (when !select_all); `need` keys
    // equal to T are taken, lowest positions first.
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    int taken_eq = 0;
    for (int base = 0; base < n; base += kThreads) {
        const int i = base + threadIdx.x;
        const bool in = i < n;
        const uint32_t key = in ? score_key(s[i]) : 0u;
        const bool gt = in && (select_all || key > prefix);
        const bool eq = in && !select_all && key == prefix;
        int eq_total = 0;
        const int rank = block_exclusive_scan(eq ? 1 : 0, scan_buf, &eq_total);
        const bool take = gt || (eq && taken_eq + rank < need);
        if (take) {
            const int slot = atomicAdd(&s_count, 1);
            if (slot < kMaxK)
                sel[slot] = (static_cast<unsigned long long>(key) << 32) |
                            static_cast<unsigned long long>(0xffffffffu - static_cast<uint32_t>(i));
        }
        taken_eq += eq_total;
    }
    __syncthreads();
    const int cnt = min(s_count, kMaxK);
    // pad to the sort width with zero keys (below every real entry)
    int width = 1;
    while (width < cnt) width <<= 1;
    for (int i = cnt + threadIdx.x; i < width; i += kThreads) sel[i] = 0ull;
    __syncthreads();
    // bitonic sort, descending
    for (int size = 2; size <= width; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < width; i += kThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = sel[i], b = sel[j];
                    if (desc ? (a < b) : (a > b)) {
                        sel[i] = b;
                        sel[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < k; r += kThreads) {
        float sc = -INFINITY;
        int pos = -1;
        if (r < cnt) {
            pos = static_cast<int>(0xffffffffu - static_cast<uint32_t>(sel[r] & 0xffffffffull));
            sc = s[pos];
        }
        out_scores[static_cast<int64_t>(q) * k + r] = sc;
        out_pos[static_cast<int64_t>(q) * k + r] = pos;
    }
}

}  // namespace topk
}  // namespace tms

extern "C" tms_status tms_topk(const float* scores, const int64_t* cand_offsets, int n_queries, int topk,
                               float* out_scores, int32_t* out_pos, cudaStream_t stream) {
    using namespace tms;
    if (n_queries < 1 || topk < 1 || topk > topk::kMaxK) return TMS_ERR_INVALID_ARG;
    if (!scores || !cand_offsets || !out_scores || !out_pos || !aligned16(cand_offsets) ||
        !aligned16(out_scores) || !aligned16(out_pos) || (reinterpret_cast<uintptr_t>(scores) & 3u))
        return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    topk::topk_kernel<<<static_cast<unsigned>(n_queries), topk::kThreads, 0, stream>>>(scores, cand_offsets, n_queries,
                                                                                        topk, out_scores, out_pos, dev.err);
    return launch_status(cudaGetLastError());
}
