// tms_fp8.cu -- the FP8 E4M3 token store: per-row quantization and MaxSim
// scoring of E4M3 codes with one fp32 scale per row.
//
// A stored row stands for the vector scale * decode(codes).  Scoring runs
// the tensor-core kernel of tms_dense_tc.cuh with tcgen05.mma kind::f8f6f4
// (E4M3 x E4M3, fp32 accumulation): the 128-byte chunks, swizzle and
// descriptors are byte-for-byte those of the fp16 path, a chunk just holds
// 128 elements, so each document row costs half the HBM bytes and half the
// MMAs.  The document row's scale multiplies its similarities before the
// max; the query token's scale multiplies the column max before the sum
// (both scales are >= 0, so this equals Eq. 1 on the dequantized vectors).
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "tms_dense_tc.cuh"

namespace tms {

namespace fp8 {

constexpr int kQuantWarps = 8;
constexpr int kMaxGroups = 8;  // d <= 1024: d / 4 groups of 4 elements over 32 lanes

template <int DT>
__device__ __forceinline__ float4 load4(const void* x, int64_t e) {
    if (DT == TMS_F32) return *reinterpret_cast<const float4*>(static_cast<const float*>(x) + e);
    const uint2 u = *reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(x) + e);
    float2 lo, hi;
    if (DT == TMS_F16) {
        lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    } else {
        lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    }
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ uint32_t encode(float v, float s) {
    if (s == 0.f) return 0u;
    return static_cast<uint32_t>(__nv_cvt_float_to_fp8(__fdiv_rn(v, s), __NV_SATFINITE, __NV_E4M3));
}

// One warp per row: amax over the row (fp32), s = amax / 448, code =
// E4M3(x / s) rounded to nearest even with saturation; both divisions are
// IEEE fp32.  Lane l holds groups l, l + 32, ... of 4 elements.
template <int DT>
__global__ void __launch_bounds__(kQuantWarps * 32)
    quantize_kernel(const void* __restrict__ x, int64_t rows, int d, uint8_t* __restrict__ codes,
                    float* __restrict__ scales) {
    const int lane = threadIdx.x & 31;
    const int ng = d >> 2;
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * kQuantWarps + (threadIdx.x >> 5); r < rows;
         r += static_cast<int64_t>(gridDim.x) * kQuantWarps) {
        float4 v[kMaxGroups];
        float amax = 0.f;
#pragma unroll
        for (int g = 0; g < kMaxGroups; ++g) {
            const int gi = lane + 32 * g;
            if (gi < ng) {
                v[g] = load4<DT>(x, r * d + 4 * gi);
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[g].x), fabsf(v[g].y)), fmaxf(fabsf(v[g].z), fabsf(v[g].w))));
            }
        }
        amax = warp_max(amax);
        const float s = __fdiv_rn(amax, 448.f);
#pragma unroll
        for (int g = 0; g < kMaxGroups; ++g) {
            const int gi = lane + 32 * g;
            if (gi < ng) {
                const uint32_t w = encode(v[g].x, s) | (encode(v[g].y, s) << 8) | (encode(v[g].z, s) << 16) |
                                   (encode(v[g].w, s) << 24);
                *reinterpret_cast<uint32_t*>(codes + r * d + 4 * gi) = w;
            }
        }
        if (lane == 0) scales[r] = s;
    }
}

inline bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// Host checks shared by both scoring entry points; fills the common Args.
tms_status prepare(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq, int d,
                   const uint8_t* doc_codes, const float* doc_scales, int64_t n_tokens, const int64_t* doc_offsets,
                   const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids, int64_t n_cand,
                   float* out_scores, DeviceInfo* dev, dense::Args* a) {
    if (n_queries < 1 || n_queries > 4096 || nq < 1 || nq > 128 || d < 16 || d > 1024 || d % 16 != 0)
        return TMS_ERR_INVALID_ARG;
    if (n_tokens < 0 || n_tokens >= (int64_t(1) << 31) || n_docs < 0 || n_cand < 0 ||
        n_cand >= (int64_t(1) << 31))
        return TMS_ERR_INVALID_ARG;
    if (!q_codes || !q_scales || !aligned16(q_codes) || !aligned4(q_scales)) return TMS_ERR_INVALID_ARG;
    if (n_cand > 0 && (!cand_ids || !out_scores || !aligned16(cand_ids) || !aligned16(out_scores)))
        return TMS_ERR_INVALID_ARG;
    if (n_docs > 0 && (!doc_offsets || !doc_lengths || !aligned16(doc_offsets) || !aligned16(doc_lengths)))
        return TMS_ERR_INVALID_ARG;
    if (n_tokens > 0 && (!doc_codes || !doc_scales || !aligned16(doc_codes) || !aligned16(doc_scales)))
        return TMS_ERR_INVALID_ARG;
    tms_status st = current_device(dev);
    if (st != TMS_OK) return st;
    *a = dense::Args{};
    a->offsets = doc_offsets;
    a->lengths = doc_lengths;
    a->cand_ids = cand_ids;
    a->out = out_scores;
    a->q_scales = q_scales;
    a->t_scales = doc_scales;
    a->err = dev->err;
    a->budget = debug_wait_budget();
    a->fault = debug_fault();
    a->n_docs = n_docs;
    a->n_tokens = n_tokens;
    a->n_cand = n_cand;
    a->n_queries = n_queries;
    a->nq = nq;
    a->nchunks = (d + dense::chunk_elems(dense::kE4M3) - 1) / dense::chunk_elems(dense::kE4M3);
    return TMS_OK;
}

}  // namespace fp8

}  // namespace tms

extern "C" tms_status tms_quantize_e4m3(const void* x, tms_dtype dtype, int64_t rows, int d, uint8_t* codes,
                                        float* scales, cudaStream_t stream) {
    using namespace tms;
    if (dtype != TMS_F16 && dtype != TMS_BF16 && dtype != TMS_F32) return TMS_ERR_INVALID_ARG;
    if (rows < 0 || d < 16 || d > 1024 || d % 16 != 0) return TMS_ERR_INVALID_ARG;
    if (rows == 0) return TMS_OK;
    if (!x || !codes || !scales || !aligned16(x) || !aligned16(codes) || !fp8::aligned4(scales))
        return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    const int64_t want = (rows + fp8::kQuantWarps - 1) / fp8::kQuantWarps;
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(want, int64_t(dev.sm_count) * 8));
    const unsigned threads = fp8::kQuantWarps * 32;
    switch (dtype) {
        case TMS_F16: fp8::quantize_kernel<TMS_F16><<<grid, threads, 0, stream>>>(x, rows, d, codes, scales); break;
        case TMS_BF16: fp8::quantize_kernel<TMS_BF16><<<grid, threads, 0, stream>>>(x, rows, d, codes, scales); break;
        default: fp8::quantize_kernel<TMS_F32><<<grid, threads, 0, stream>>>(x, rows, d, codes, scales); break;
    }
    return launch_status(cudaGetLastError());
}

namespace tms {
namespace fp8 {

// tms_score_fp8 / tms_tune_fp8: the same checks, then launch (or tune).
tms_status score(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq, int d,
                 const uint8_t* doc_codes, const float* doc_scales, int64_t n_tokens, const int64_t* doc_offsets,
                 const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids, const int64_t* cand_offsets,
                 int64_t n_cand, float* out_scores, cudaStream_t stream, bool tune, int* n_configs) {
    if (n_configs) *n_configs = 0;
    if (!cand_offsets || !aligned16(cand_offsets)) return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    dense::Args a;
    tms_status st = prepare(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                            doc_lengths, n_docs, cand_ids, n_cand, out_scores, &dev, &a);
    if (st != TMS_OK || n_cand == 0) return st;
    a.cand_offsets = cand_offsets;
    a.n_flat = n_cand;
    a.group = 0;
    a.bpc = (nq + 31) / 32;
    a.qbox = 32 * a.bpc;
    if (tune)
        return dense::tune_tc<1, false, dense::kE4M3>(dev, q_codes, TMS_F16, n_queries, nq, d, doc_codes, n_tokens, a,
                                                      stream, n_configs);
    return dense::launch_tc<1, false, dense::kE4M3>(dev, q_codes, TMS_F16, n_queries, nq, d, doc_codes, n_tokens, a,
                                                    stream);
}

// tms_score_fp8_shared / tms_tune_fp8_shared.
tms_status score_shared(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq, int d,
                        const uint8_t* doc_codes, const float* doc_scales, int64_t n_tokens,
                        const int64_t* doc_offsets, const int32_t* doc_lengths, int64_t n_docs,
                        const int32_t* cand_ids, int64_t n_cand, float* out_scores, cudaStream_t stream, bool tune,
                        int* n_configs) {
    if (n_configs) *n_configs = 0;
    DeviceInfo dev;
    dense::Args a;
    tms_status st = prepare(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                            doc_lengths, n_docs, cand_ids, n_cand, out_scores, &dev, &a);
    if (st != TMS_OK) return st;
    if (nq > 32) return TMS_ERR_UNSUPPORTED;
    if (n_cand == 0) return TMS_OK;
    a.cand_offsets = nullptr;
    return dense::shared_run<dense::kE4M3>(dev, q_codes, TMS_F16, n_queries, nq, d, doc_codes, n_tokens, a, stream,
                                           tune, n_configs);
}

}  // namespace fp8
}  // namespace tms

extern "C" tms_status tms_score_fp8(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq, int d,
                                    const uint8_t* doc_codes, const float* doc_scales, int64_t n_tokens,
                                    const int64_t* doc_offsets, const int32_t* doc_lengths, int64_t n_docs,
                                    const int32_t* cand_ids, const int64_t* cand_offsets, int64_t n_cand,
                                    float* out_scores, cudaStream_t stream) {
    return tms::fp8::score(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                           doc_lengths, n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream, false, nullptr);
}

extern "C" tms_status tms_tune_fp8(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq, int d,
                                   const uint8_t* doc_codes, const float* doc_scales, int64_t n_tokens,
                                   const int64_t* doc_offsets, const int32_t* doc_lengths, int64_t n_docs,
                                   const int32_t* cand_ids, const int64_t* cand_offsets, int64_t n_cand,
                                   float* out_scores, cudaStream_t stream, int* n_configs) {
    return tms::fp8::score(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                           doc_lengths, n_docs, cand_ids, cand_offsets, n_cand, out_scores, stream, true, n_configs);
}

extern "C" tms_status tms_score_fp8_shared(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq,
                                           int d, const uint8_t* doc_codes, const float* doc_scales,
                                           int64_t n_tokens, const int64_t* doc_offsets, const int32_t* doc_lengths,
                                           int64_t n_docs, const int32_t* cand_ids, int64_t n_cand,
                                           float* out_scores, cudaStream_t stream) {
    return tms::fp8::score_shared(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                                  doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream, false, nullptr);
}

extern "C" tms_status tms_tune_fp8_shared(const uint8_t* q_codes, const float* q_scales, int n_queries, int nq,
                                          int d, const uint8_t* doc_codes, const float* doc_scales,
                                          int64_t n_tokens, const int64_t* doc_offsets, const int32_t* doc_lengths,
                                          int64_t n_docs, const int32_t* cand_ids, int64_t n_cand,
                                          float* out_scores, cudaStream_t stream, int* n_configs) {
    return tms::fp8::score_shared(q_codes, q_scales, n_queries, nq, d, doc_codes, doc_scales, n_tokens, doc_offsets,
                                  doc_lengths, n_docs, cand_ids, n_cand, out_scores, stream, true, n_configs);
}
