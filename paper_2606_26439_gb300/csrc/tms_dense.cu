// tms_dense.cu -- dense MaxSim entry points for fp16 / bf16 / fp32 rows.
//
// fp16 / bf16 run the tensor-core kernel of tms_dense_tc.cuh; fp32 runs an
// exact-fp32 CUDA-core kernel (one warp per candidate, lanes = query tokens,
// a 64-element chunk of the query row in registers).
#include "tms_dense_tc.cuh"

namespace tms {

namespace dense {

// ------------------------------------------------------------------ fp32

constexpr int kF32Warps = 8;
constexpr int kF32Chunk = 64;

// Exact-fp32 MaxSim: one warp per candidate, lane i = query token
// (blocks of 32), a 64-wide chunk of the query row in registers, each
// document row broadcast to the warp.  Dot products accumulate in fp32
// over all dimension chunks before the max.
__global__ void __launch_bounds__(kF32Warps * 32)
    dense_f32_kernel(const float* __restrict__ queries, const float* __restrict__ tokens, const Args a, int d) {
    extern __shared__ float qs[];  // [32][d + 4]
    griddep_wait();
    griddep_launch_dependents();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int pitch = d + 4;
    if (blockIdx.x == 0 && threadIdx.x == 0 && __ldg(a.cand_offsets + a.n_queries) != a.n_cand)
        atomicOr(a.err, TMS_DEVERR_BAD_CSR);
    for (int q = 0; q < a.n_queries; ++q) {
        int64_t c0 = __ldg(a.cand_offsets + q), c1 = __ldg(a.cand_offsets + q + 1);
        c0 = c0 < 0 ? 0 : (c0 > a.n_cand ? a.n_cand : c0);
        c1 = c1 < c0 ? c0 : (c1 > a.n_cand ? a.n_cand : c1);
        for (int ib = 0; ib < a.nq; ib += 32) {
            __syncthreads();
            for (int e = threadIdx.x; e < 32 * d; e += blockDim.x) {
                const int i = e / d, t = e - i * d;
                qs[i * pitch + t] = (ib + i < a.nq) ? queries[(static_cast<int64_t>(q) * a.nq + ib + i) * d + t] : 0.f;
            }
            __syncthreads();
            for (int64_t c = c0 + static_cast<int64_t>(blockIdx.x) * kF32Warps + warp; c < c1;
                 c += static_cast<int64_t>(gridDim.x) * kF32Warps) {
                const int id = __ldg(a.cand_ids + c);
                int64_t off = 0;
                int len = 0;
                int status = 0;
                if (id < 0 || id >= a.n_docs) {
                    status = 1;
                } else {
                    off = __ldg(a.offsets + id);
                    len = __ldg(a.lengths + id);
                    if (len < 0 || off < 0 || off + len > a.n_tokens) status = 2;
                }
                if (status != 0 || len == 0) {
                    if (ib == 0 && lane == 0) {
                        if (status) {
                            a.out[c] = __int_as_float(0x7fc00000);
                            atomicOr(a.err, status == 1 ? TMS_DEVERR_BAD_ID : TMS_DEVERR_BAD_RANGE);
                        } else {
                            a.out[c] = -INFINITY;
                        }
                    }
                    continue;
                }
                float best = -INFINITY;
                for (int j0 = 0; j0 < len; j0 += 32) {
                    float acc[32];
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) acc[jj] = 0.f;
                    for (int kc = 0; kc < d; kc += kF32Chunk) {
                        float qr[kF32Chunk];
                        const float4* qrow = reinterpret_cast<const float4*>(qs + lane * pitch + kc);
#pragma unroll
                        for (int u = 0; u < kF32Chunk / 4; ++u) {
                            const float4 v = (kc + 4 * u < d) ? qrow[u] : make_float4(0.f, 0.f, 0.f, 0.f);
                            qr[4 * u] = v.x;
                            qr[4 * u + 1] = v.y;
                            qr[4 * u + 2] = v.z;
                            qr[4 * u + 3] = v.w;
                        }
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            if (j0 + jj < len) {
                                const float4* xr =
                                    reinterpret_cast<const float4*>(tokens + (off + j0 + jj) * d + kc);
#pragma unroll
                                for (int u = 0; u < kF32Chunk / 4; ++u) {
                                    if (kc + 4 * u < d) {
                                        const float4 x = __ldg(xr + u);
                                        acc[jj] = fmaf(qr[4 * u], x.x, acc[jj]);
                                        acc[jj] = fmaf(qr[4 * u + 1], x.y, acc[jj]);
                                        acc[jj] = fmaf(qr[4 * u + 2], x.z, acc[jj]);
                                        acc[jj] = fmaf(qr[4 * u + 3], x.w, acc[jj]);
                                    }
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj)
                        if (j0 + jj < len) best = fmaxf(best, acc[jj]);
                }
                float v = (ib + lane < a.nq) ? best : 0.f;
                v = warp_sum(v);
                if (lane == 0) a.out[c] = (ib == 0) ? v : a.out[c] + v;
            }
        }
    }
}

}  // namespace dense

}  // namespace tms

namespace tms {
namespace {

// tms_score_dense, or (tune) tms_tune_dense: the same checks and launch,
// the tensor-core configurations timed first.
tms_status score_dense(const void* queries, tms_dtype dtype, int n_queries, int nq, int d, const void* doc_tokens,
                       int64_t n_tokens, const int64_t* doc_offsets, const int32_t* doc_lengths, int64_t n_docs,
                       const int32_t* cand_ids, const int64_t* cand_offsets, int64_t n_cand, float* out_scores,
                       cudaStream_t stream, bool tune, int* n_timed) {
    if (n_timed) *n_timed = 0;
    if (dtype != TMS_F16 && dtype != TMS_BF16 && dtype != TMS_F32) return TMS_ERR_INVALID_ARG;
    if (n_queries < 1 || n_queries > 4096 || nq < 1 || nq > 128 || d < 8 || d > 1024 || d % 8 != 0)
        return TMS_ERR_INVALID_ARG;
    if (n_tokens < 0 || n_tokens >= (int64_t(1) << 31) || n_docs < 0 || n_cand < 0 ||
        n_cand >= (int64_t(1) << 31))
        return TMS_ERR_INVALID_ARG;
    if (!queries || !cand_offsets || !aligned16(queries) || !aligned16(cand_offsets)) return TMS_ERR_INVALID_ARG;
    if (n_cand > 0 && (!cand_ids || !out_scores || !aligned16(cand_ids) || !aligned16(out_scores)))
        return TMS_ERR_INVALID_ARG;
    if (n_docs > 0 && (!doc_offsets || !doc_lengths || !aligned16(doc_offsets) || !aligned16(doc_lengths)))
        return TMS_ERR_INVALID_ARG;
    if (n_tokens > 0 && (!doc_tokens || !aligned16(doc_tokens))) return TMS_ERR_INVALID_ARG;
    if (n_cand == 0) return TMS_OK;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;

    dense::Args a{};
    a.offsets = doc_offsets;
    a.lengths = doc_lengths;
    a.cand_ids = cand_ids;
    a.cand_offsets = cand_offsets;
    a.out = out_scores;
    a.err = dev.err;
    a.budget = debug_wait_budget();
    a.fault = debug_fault();
    a.n_docs = n_docs;
    a.n_tokens = n_tokens;
    a.n_cand = n_cand;
    a.n_flat = n_cand;
    a.group = 0;
    a.n_queries = n_queries;
    a.nq = nq;
    a.bpc = (nq + 31) / 32;
    a.qbox = 32 * a.bpc;

    if (dtype == TMS_F32) {
        // split TF32 on the tensor cores; the exact CUDA-core kernel below
        // covers the shapes whose query tile does not fit
        a.nchunks = (d + dense::chunk_elems(dense::kTF32) - 1) / dense::chunk_elems(dense::kTF32);
        st = tune ? dense::tune_tc<1, false, dense::kTF32>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens,
                                                           a, stream, n_timed)
                  : dense::launch_tc<1, false, dense::kTF32>(dev, queries, dtype, n_queries, nq, d, doc_tokens,
                                                             n_tokens, a, stream);
        if (st != TMS_ERR_UNSUPPORTED) return st;
        const int smem = 32 * (d + 4) * 4;
        if (smem > dev.max_smem_optin) return TMS_ERR_UNSUPPORTED;
        if (cudaFuncSetAttribute(dense::dense_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return launch_status(cudaErrorInvalidValue);
        const int64_t want = (n_cand + dense::kF32Warps - 1) / dense::kF32Warps;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(int64_t(dev.sm_count) * 4, want));
        return launch_status(launch_dependent(dense::dense_f32_kernel, dim3(static_cast<unsigned>(grid)),
                                              dim3(dense::kF32Warps * 32), static_cast<size_t>(smem), stream,
                                              static_cast<const float*>(queries),
                                              static_cast<const float*>(doc_tokens), a, d));
    }
    a.nchunks = (d + dense::chunk_elems(dense::kF16) - 1) / dense::chunk_elems(dense::kF16);
    return tune ? dense::tune_tc<1, false, dense::kF16>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a,
                                                        stream, n_timed)
                : dense::launch_tc<1, false, dense::kF16>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens,
                                                          a, stream);
}

}  // namespace
}  // namespace tms

extern "C" tms_status tms_score_dense(const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                                      const void* doc_tokens, int64_t n_tokens, const int64_t* doc_offsets,
                                      const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                                      const int64_t* cand_offsets, int64_t n_cand, float* out_scores,
                                      cudaStream_t stream) {
    return tms::score_dense(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths, n_docs,
                            cand_ids, cand_offsets, n_cand, out_scores, stream, false, nullptr);
}

extern "C" tms_status tms_tune_dense(const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                                     const void* doc_tokens, int64_t n_tokens, const int64_t* doc_offsets,
                                     const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                                     const int64_t* cand_offsets, int64_t n_cand, float* out_scores,
                                     cudaStream_t stream, int* n_configs) {
    return tms::score_dense(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths, n_docs,
                            cand_ids, cand_offsets, n_cand, out_scores, stream, true, n_configs);
}

namespace tms {
namespace {

tms_status score_dense_shared(const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                              const void* doc_tokens, int64_t n_tokens, const int64_t* doc_offsets,
                              const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids, int64_t n_cand,
                              float* out_scores, cudaStream_t stream, bool tune, int* n_configs) {
    if (n_configs) *n_configs = 0;
    if (dtype != TMS_F16 && dtype != TMS_BF16 && dtype != TMS_F32) return TMS_ERR_INVALID_ARG;
    if (n_queries < 1 || n_queries > 4096 || nq < 1 || nq > 128 || d < 8 || d > 1024 || d % 8 != 0)
        return TMS_ERR_INVALID_ARG;
    if (dtype == TMS_F32 || nq > 32) return TMS_ERR_UNSUPPORTED;
    if (n_tokens < 0 || n_tokens >= (int64_t(1) << 31) || n_docs < 0 || n_cand < 0) return TMS_ERR_INVALID_ARG;
    if (!queries || !aligned16(queries)) return TMS_ERR_INVALID_ARG;
    if (n_cand > 0 && (!cand_ids || !out_scores || !aligned16(cand_ids) || !aligned16(out_scores)))
        return TMS_ERR_INVALID_ARG;
    if (n_docs > 0 && (!doc_offsets || !doc_lengths || !aligned16(doc_offsets) || !aligned16(doc_lengths)))
        return TMS_ERR_INVALID_ARG;
    if (n_tokens > 0 && (!doc_tokens || !aligned16(doc_tokens))) return TMS_ERR_INVALID_ARG;
    if (n_cand == 0) return TMS_OK;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    dense::Args a{};
    a.offsets = doc_offsets;
    a.lengths = doc_lengths;
    a.cand_ids = cand_ids;
    a.cand_offsets = nullptr;
    a.out = out_scores;
    a.err = dev.err;
    a.budget = debug_wait_budget();
    a.fault = debug_fault();
    a.n_docs = n_docs;
    a.n_tokens = n_tokens;
    a.n_cand = n_cand;
    a.n_queries = n_queries;
    a.nq = nq;
    a.nchunks = (d + dense::chunk_elems(dense::kF16) - 1) / dense::chunk_elems(dense::kF16);
    return dense::shared_run<dense::kF16>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a, stream, tune,
                                          n_configs);
}

}  // namespace
}  // namespace tms

extern "C" tms_status tms_score_dense_shared(const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                                             const void* doc_tokens, int64_t n_tokens, const int64_t* doc_offsets,
                                             const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                                             int64_t n_cand, float* out_scores, cudaStream_t stream) {
    return tms::score_dense_shared(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths,
                                   n_docs, cand_ids, n_cand, out_scores, stream, false, nullptr);
}

extern "C" tms_status tms_tune_dense_shared(const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                                            const void* doc_tokens, int64_t n_tokens, const int64_t* doc_offsets,
                                            const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                                            int64_t n_cand, float* out_scores, cudaStream_t stream, int* n_configs) {
    return tms::score_dense_shared(queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, doc_offsets, doc_lengths,
                                   n_docs, cand_ids, n_cand, out_scores, stream, true, n_configs);
}
