// tms_pq.cu -- fused PQ MaxSim on GB300 (sm_103a).
//
// Phase 1 (Section 4.2): the distance table
//     T[q][i][m][k] = q_i[m*dsub : (m+1)*dsub] . C[m][k]
// one thread per entry, fp32 fused multiply-adds in ascending t.
//
// Phase 2 (Section 4.2): score = sum_i max_j sum_m T[i][m][code_{j,m}],
// straight from the uint8 codes; no token is ever decompressed.
//
// On GB300 this phase is bound by shared-memory gathers, not HBM: a token
// costs 16 code bytes of HBM but Nq * M table reads.  The kernel is built
// around the gathers:
//   * the table of 8 query tokens (a "chunk", 128 KB for M = 16, K = 256)
//     lives in shared memory in the layout
//         word ((m / 4) * K + k) * 32 + (m % 4) * 8 + i,
//     and lane (g = lane / 8, i = lane % 8) of a warp looks up subspace
//     m = 4 s + g of query token i at step s.  Whatever the four codes a
//     warp instruction uses, its 32 addresses fall in 32 distinct banks
//     (the bank is (m % 4) * 8 + i), so every gather is one wavefront;
//   * each lane sums its 4 (of 16) subspaces for 4 tokens, and a two-step
//     transposed shuffle reduction turns that into the full dot of token
//     (4 j + g) with query token i -- 3 shuffles per 4 tokens;
//   * the running max stays in registers; tokens past the document end
//     re-use the last token (a duplicate cannot change a max);
//   * chunks are processed one after another over the CTA's candidates,
//     and out_scores itself carries the running sum over chunks, added in
//     ascending chunk order by the same CTA -- deterministic, no atomics,
//     no scratch memory.
#include <algorithm>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {
namespace pq {

constexpr int kWarps = 16;
constexpr int kQC = 8;  // query tokens per chunk

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }

template <typename QT>
__global__ void lut_kernel(const QT* __restrict__ queries, int d, const float* __restrict__ codebook, int M, int K,
                           float* __restrict__ lut, int64_t total) {
    griddep_wait();
    griddep_launch_dependents();
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int k = static_cast<int>(idx % K);
    const int m = static_cast<int>((idx / K) % M);
    const int64_t row = idx / (static_cast<int64_t>(K) * M);  // q * nq + i
    const int dsub = d / M;
    const QT* qv = queries + row * d + m * dsub;
    const float* cv = codebook + (static_cast<int64_t>(m) * K + k) * dsub;
    float acc = 0.f;
    for (int t = 0; t < dsub; ++t) acc = fmaf(to_f32(qv[t]), __ldg(cv + t), acc);
    lut[idx] = acc;
}

struct Args {
    const float* lut;
    const uint8_t* codes;
    const int64_t* offsets;
    const int32_t* lengths;
    const int32_t* cand_ids;
    const int64_t* cand_offsets;
    float* out;
    unsigned int* err;
    int64_t n_docs;
    int64_t n_tokens;
    int64_t n_cand;
    int n_queries;
    int nq;
    int K;
    long long budget;  // SM cycles a wait may last (<= 0: kWaitBudgetCycles)
};

// Codes of one token as M/4 32-bit words (M bytes, 4-byte aligned rows).
template <int M>
struct CodeRow {
    uint32_t w[M / 4];
};

template <int M>
__device__ __forceinline__ CodeRow<M> load_codes(const uint8_t* row) {
    CodeRow<M> c;
    if constexpr (M == 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row));
        c.w[0] = v.x;
        c.w[1] = v.y;
        c.w[2] = v.z;
        c.w[3] = v.w;
    } else if constexpr (M == 32) {
        const uint4 v0 = __ldg(reinterpret_cast<const uint4*>(row));
        const uint4 v1 = __ldg(reinterpret_cast<const uint4*>(row) + 1);
        c.w[0] = v0.x; c.w[1] = v0.y; c.w[2] = v0.z; c.w[3] = v0.w;
        c.w[4] = v1.x; c.w[5] = v1.y; c.w[6] = v1.z; c.w[7] = v1.w;
    } else if constexpr (M == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(row));
        c.w[0] = v.x;
        c.w[1] = v.y;
    } else {
        c.w[0] = __ldg(reinterpret_cast<const uint32_t*>(row));
    }
    return c;
}

// Partial dot of this lane's subspaces {g, g+4, ...} for one token.
template <int M>
__device__ __forceinline__ float lane_partial(const float* lut_lane, const CodeRow<M>& c, uint32_t sel, int K) {
    float p = 0.f;
#pragma unroll
    for (int s = 0; s < M / 4; ++s) {
        const uint32_t code = __byte_perm(c.w[s], 0u, sel);  // byte g of word s
        p += lut_lane[(s * K + static_cast<int>(code)) * 32];
    }
    return p;
}

template <int M>
__global__ void __launch_bounds__(kWarps * 32, 1) score_kernel(const Args a) {
    extern __shared__ float lut_s[];  // [M/4][K][4][8]
    __shared__ int next_local;
    griddep_wait();
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3;  // subspace group
    const int i = lane & 7;   // query token within the chunk
    const uint32_t sel = 0x4440u | static_cast<uint32_t>(g);
    const float* lut_lane = lut_s + lane;
    const int K = a.K;
    const int nchunks = (a.nq + kQC - 1) / kQC;
    const int words = kQC * M * K;

    if (blockIdx.x == 0 && threadIdx.x == 0 && __ldg(a.cand_offsets + a.n_queries) != a.n_cand)
        atomicOr(a.err, TMS_DEVERR_BAD_CSR);

    for (int q = 0; q < a.n_queries; ++q) {
        int64_t c0 = __ldg(a.cand_offsets + q), c1 = __ldg(a.cand_offsets + q + 1);
        c0 = c0 < 0 ? 0 : (c0 > a.n_cand ? a.n_cand : c0);
        c1 = c1 < c0 ? c0 : (c1 > a.n_cand ? a.n_cand : c1);
        // this CTA's candidates of query q: c0 + blockIdx.x + j * gridDim.x
        if (c0 + blockIdx.x >= c1) continue;
        const int64_t n_local = (c1 - c0 - blockIdx.x + gridDim.x - 1) / gridDim.x;
        for (int ch = 0; ch < nchunks; ++ch) {
            __syncthreads();
            // table chunk -> shared memory, transposed to [m/4][k][m%4][i]
            const float* src = a.lut + static_cast<int64_t>(q) * a.nq * M * K;
            for (int w = threadIdx.x; w < words; w += blockDim.x) {
                const int ii = w & 7;
                const int ml = (w >> 3) & 3;
                const int rest = w >> 5;
                const int kk = rest % K;
                const int mh = rest / K;
                const int qi = ch * kQC + ii;
                lut_s[w] = (qi < a.nq) ? __ldg(src + (static_cast<int64_t>(qi) * M + mh * 4 + ml) * K + kk) : 0.f;
            }
            if (threadIdx.x == 0) next_local = 0;
            __syncthreads();
            for (;;) {
                int li = 0;
                if (lane == 0) li = atomicAdd(&next_local, 1);
                li = __shfl_sync(0xffffffffu, li, 0);
                if (li >= n_local) break;
                const int64_t f = c0 + blockIdx.x + static_cast<int64_t>(li) * gridDim.x;
                const int id = __ldg(a.cand_ids + f);
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
                    if (ch == 0 && lane == 0) {
                        if (status) {
                            a.out[f] = __int_as_float(0x7fc00000);
                            atomicOr(a.err, status == 1 ? TMS_DEVERR_BAD_ID : TMS_DEVERR_BAD_RANGE);
                        } else {
                            a.out[f] = -INFINITY;
                        }
                    }
                    continue;
                }
                const uint8_t* base = a.codes + off * M;
                const int last = len - 1;
                float rmax = -INFINITY;
                CodeRow<M> c[4];
#pragma unroll
                for (int tt = 0; tt < 4; ++tt) c[tt] = load_codes<M>(base + static_cast<int64_t>(min(tt, last)) * M);
                for (int j = 0; j < len; j += 4) {
                    // prefetch the next four tokens' codes
                    CodeRow<M> nc[4];
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt)
                        nc[tt] = load_codes<M>(base + static_cast<int64_t>(min(j + 4 + tt, last)) * M);
                    float p[4];
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt) p[tt] = lane_partial<M>(lut_lane, c[tt], sel, K);
                    // transposed reduction over the 4 subspace groups:
                    // lane (g, i) ends with token 4j + g's full dot with query token i
                    const bool up16 = (lane & 16) != 0;
                    float k0 = up16 ? p[2] : p[0];
                    float k1 = up16 ? p[3] : p[1];
                    const float s0 = up16 ? p[0] : p[2];
                    const float s1 = up16 ? p[1] : p[3];
                    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
                    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
                    const bool up8 = (lane & 8) != 0;
                    float kk = up8 ? k1 : k0;
                    const float ss = up8 ? k0 : k1;
                    kk += __shfl_xor_sync(0xffffffffu, ss, 8);
                    rmax = fmaxf(rmax, kk);
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt) c[tt] = nc[tt];
                }
                rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, 8));
                rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, 16));
                float v = (ch * kQC + i < a.nq) ? rmax : 0.f;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                if (lane == 0) a.out[f] = (ch == 0) ? v : a.out[f] + v;
            }
        }
    }
}


// ---------------------------------------------------------------------------
// Staged variant for M in {16, 32}: every warp streams its documents' code
// rows into a private double-buffered shared-memory piece buffer with
// cp.async.bulk (TMA) and reads them back as broadcast 128-bit loads, so the
// gather loop never waits on global memory.  While a piece is scored, the
// warp has already issued the copy of the next piece (of this document or of
// the next one, whose metadata was fetched one document ahead).
//
// Gathers are 128-bit: the table chunk is laid out in 256-byte rows
//     byte ((s / 2) * KS + k) * 256 + (s % 2) * 128 + (m % 4) * 32 + i * E
// for subspace m = 4 s + (m % 4), code k and query token i (KS = 4096 / M
// rows per block; E = 4 bytes and 8 query tokens for the fp32 table, E = 2
// and 16 query tokens for the fp16 one).  Lane (r = lane / 2, ip = lane % 2)
// scores document token j + r of a group of sixteen against the query
// tokens of 16-byte slot ip of a 32-byte section: 4 ip .. 4 ip + 3 for the
// fp32 table, 8 ip .. 8 ip + 7 for the fp16 one.  Each lane sums all M
// subspaces of its own token, in an order rotated by g = r % 4: at inner
// step t of subspace group s it reads subspace 4 s + (t + g) % 4.  One byte
// permute builds the offset (the code byte times 256 plus the lane offset
// ((t + g) % 4) * 32 + ip * 16); in each quarter-warp the four values of g
// meet four different 32-byte sections and the two values of ip the two
// slots, so the 8 lanes cover all 32 banks (one wavefront per quarter-warp)
// whatever the codes are.  No cross-lane reduction is needed per token: a
// lane holds the whole dot of its token and keeps the running max of its
// query tokens in registers; the lanes of one slot are combined once per
// document.  fp32 entries are added pairwise with add.rn.f32x2 (two IEEE
// fp32 additions in one instruction).
//
// fp16 table (H16): each entry is rounded to the nearest fp16 when the chunk
// is staged and added to an fp32 accumulator exactly widened
// (add.rn.f32.f16); a 128 KB chunk then serves 16 query tokens and every
// gather returns 8 entries.
constexpr int kPieceBytes = 2048;  // per buffer: 128 tokens at M = 16

template <int M>
__device__ __forceinline__ CodeRow<M> smem_codes(const uint8_t* row) {
    CodeRow<M> c;
    const uint4 v = *reinterpret_cast<const uint4*>(row);
    c.w[0] = v.x;
    c.w[1] = v.y;
    c.w[2] = v.z;
    c.w[3] = v.w;
    if constexpr (M == 32) {
        const uint4 u = *reinterpret_cast<const uint4*>(row + 16);
        c.w[4] = u.x;
        c.w[5] = u.y;
        c.w[6] = u.z;
        c.w[7] = u.w;
    }
    return c;
}

// acc0 += lo half of w, acc1 += hi half of w (fp16 widened exactly, one
// fp32 rounding per add)
__device__ __forceinline__ void add_f16x2(float& acc0, float& acc1, uint32_t w) {
    asm("{\n\t.reg .f16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.f16 %0, lo, %0;\n\tadd.rn.f32.f16 %1, hi, %1;\n\t}"
        : "+f"(acc0), "+f"(acc1)
        : "r"(w));
}

// 16-byte shared-memory load at shared-window address addr + OFF
template <int OFF>
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr), "n"(OFF));
    return v;
}

// acc (two fp32 in one 64-bit register, x low) += (x, y), element-wise
__device__ __forceinline__ void add_f32x2(unsigned long long& acc, uint32_t x, uint32_t y) {
    asm("{\n\t.reg .b64 e;\n\tmov.b64 e, {%1, %2};\n\tadd.rn.f32x2 %0, %0, e;\n\t}"
        : "+l"(acc)
        : "r"(x), "r"(y));
}

// All M table entries of one token for this lane: subspace group sg, inner
// step t reads subspace 4 sg + (t + g) % 4 at the shared-window address
// tbl + block offset of sg + code * 256 + lane offset; f consumes each
// 16-byte gather in order.
template <int M, int KS, int SG = 0, typename F>
__device__ __forceinline__ void gather_groups(const CodeRow<M>& c, uint32_t tbl, const uint32_t (&lane_off)[4],
                                              const uint32_t (&sel)[4], F&& f) {
    if constexpr (SG < M / 4) {
        constexpr int kOff = (SG >> 1) * KS * 256 + (SG & 1) * 128;
#pragma unroll
        for (int t = 0; t < 4; ++t) f(lds128<kOff>(tbl + __byte_perm(c.w[SG], lane_off[t], sel[t])));
        gather_groups<M, KS, SG + 1>(c, tbl, lane_off, sel, static_cast<F&&>(f));
    }
}

struct PendingMeta {
    int64_t li;  // local candidate index (>= n_local: none)
    int id;
    int64_t off;
    int len;
};

// Table bytes of the staged variant: the last block holds 256 rows so that
// a code >= k still reads inside the allocation.
__host__ __device__ constexpr int staged_table_bytes(int M) { return ((M / 8 - 1) * (4096 / M) + 256) * 256; }

template <int M, bool H16>
__global__ void __launch_bounds__(kWarps * 32, 1) score_kernel_staged(const Args a, int lut_bytes) {
    griddep_wait();
    griddep_launch_dependents();
    constexpr int kPiece = kPieceBytes / M;  // tokens per piece
    constexpr int KS = 4096 / M;             // table rows per block
    constexpr int QC = H16 ? 16 : kQC;       // query tokens per chunk
    extern __shared__ __align__(128) uint8_t smem_raw[];
    float* lut_s = reinterpret_cast<float*>(smem_raw);
    const uint32_t tbl_sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
    uint8_t* bufs = smem_raw + lut_bytes;  // [kWarps][2][kPieceBytes]
    __shared__ uint64_t bars[kWarps][2];
    __shared__ int next_local;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    constexpr int QL = H16 ? 8 : 4;                    // query tokens per lane
    const int r = lane >> 1;                           // token of the group of sixteen
    const int g = r & 3;                               // rotation of the subspace order
    const int ip = lane & 1;                           // 16-byte slot: query tokens QL ip .. QL ip + QL - 1
    const int qt = QL * ip;
    // byte permute per inner step t: result byte 0 = lane offset, byte 1 =
    // code byte (t + g) % 4 of the group's word, bytes 2-3 = 0
    uint32_t lane_off[4], sel[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const uint32_t mm = static_cast<uint32_t>((t + g) & 3);
        lane_off[t] = mm * 32 + static_cast<uint32_t>(ip * 16);
        sel[t] = 0x6504u | (mm << 4);
    }
    const int K = a.K;
    const int nchunks = (a.nq + QC - 1) / QC;
    uint8_t* wbuf = bufs + warp * 2 * kPieceBytes;
    uint64_t* wbar = bars[warp];

    if (threadIdx.x == 0) {
        for (int w = 0; w < kWarps; ++w) {
            mbar_init(&bars[w][0], 1);
            mbar_init(&bars[w][1], 1);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && __ldg(a.cand_offsets + a.n_queries) != a.n_cand)
        atomicOr(a.err, TMS_DEVERR_BAD_CSR);
    uint32_t issued = 0, consumed = 0;  // pieces of this warp (buffer = count & 1)

    for (int q = 0; q < a.n_queries; ++q) {
        int64_t c0 = __ldg(a.cand_offsets + q), c1 = __ldg(a.cand_offsets + q + 1);
        c0 = c0 < 0 ? 0 : (c0 > a.n_cand ? a.n_cand : c0);
        c1 = c1 < c0 ? c0 : (c1 > a.n_cand ? a.n_cand : c1);
        if (c0 + blockIdx.x >= c1) continue;
        const int64_t n_local = (c1 - c0 - blockIdx.x + gridDim.x - 1) / gridDim.x;
        for (int ch = 0; ch < nchunks; ++ch) {
            __syncthreads();
            // Table chunk -> shared memory.  A warp fills 8 rows x one 128-byte
            // half (slo) per task; lane (ii, ml) reads 8 consecutive codes of
            // table row (query token, subspace) -- whole sectors -- and each
            // store instruction writes 32 consecutive words.  Rows of codes >= k
            // and query tokens >= nq are filled with zeros.
            {
                const float* src = a.lut + static_cast<int64_t>(q) * a.nq * M * K;
                const int ii = lane & 7;
                const int ml = lane >> 3;
                const int tasks = (lut_bytes / 256 / 8) * 2;
                for (int task = warp; task < tasks; task += kWarps) {
                    const int slo = task & 1;
                    const int rho0 = (task >> 1) * 8;               // KS is a multiple of 8
                    const int shi = min(rho0 / KS, M / 8 - 1);
                    const int kk0 = rho0 - shi * KS;
                    const int m = 4 * (2 * shi + slo) + ml;
                    float* dst = lut_s + rho0 * 64 + slo * 32 + ml * 8 + ii;
                    if constexpr (H16) {  // query tokens 2 ii and 2 ii + 1, rounded to nearest fp16
                        const int qi = ch * QC + 2 * ii;
                        const float* r0 = src + (static_cast<int64_t>(qi) * M + m) * K;
                        const float* r1 = r0 + static_cast<int64_t>(M) * K;
                        const bool ok0 = qi < a.nq, ok1 = qi + 1 < a.nq;
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            const int kk = kk0 + x;
                            const float t0 = (ok0 && kk < K) ? __ldg(r0 + kk) : 0.f;
                            const float t1 = (ok1 && kk < K) ? __ldg(r1 + kk) : 0.f;
                            const __half2 h = __floats2half2_rn(t0, t1);
                            dst[x * 64] = *reinterpret_cast<const float*>(&h);
                        }
                    } else {
                        const int qi = ch * QC + ii;
                        const float* r0 = src + (static_cast<int64_t>(qi) * M + m) * K;
                        const bool ok0 = qi < a.nq;
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            const int kk = kk0 + x;
                            dst[x * 64] = (ok0 && kk < K) ? __ldg(r0 + kk) : 0.f;
                        }
                    }
                }
            }
            if (threadIdx.x == 0) next_local = 0;
            __syncthreads();

            auto grab = [&]() -> int64_t {
                int li = 0;
                if (lane == 0) li = atomicAdd(&next_local, 1);
                return __shfl_sync(0xffffffffu, li, 0);
            };
            auto fetch = [&](int64_t li) {  // issue the metadata loads of candidate li
                PendingMeta m;
                m.li = li;
                m.id = -1;
                m.off = 0;
                m.len = 0;
                if (li < n_local) {
                    const int64_t f = c0 + blockIdx.x + li * gridDim.x;
                    m.id = __ldg(a.cand_ids + f);
                    if (m.id >= 0 && m.id < a.n_docs) {
                        m.off = __ldg(a.offsets + m.id);
                        m.len = __ldg(a.lengths + m.id);
                    }
                }
                return m;
            };
            // next valid document: (f, off, len) with f = -1 at the end;
            // empty and invalid candidates met on the way are written here.
            PendingMeta pend = fetch(grab());
            auto take = [&](int64_t& f, int64_t& off, int& len) {
                for (;;) {
                    if (pend.li >= n_local) {
                        f = -1;
                        return;
                    }
                    const PendingMeta cur = pend;
                    pend = fetch(grab());
                    f = c0 + blockIdx.x + cur.li * gridDim.x;
                    int status = 0;
                    if (cur.id < 0 || cur.id >= a.n_docs)
                        status = 1;
                    else if (cur.len < 0 || cur.off < 0 || cur.off + cur.len > a.n_tokens)
                        status = 2;
                    if (status == 0 && cur.len > 0) {
                        off = cur.off;
                        len = cur.len;
                        return;
                    }
                    if (ch == 0 && lane == 0) {
                        if (status) {
                            a.out[f] = __int_as_float(0x7fc00000);
                            atomicOr(a.err, status == 1 ? TMS_DEVERR_BAD_ID : TMS_DEVERR_BAD_RANGE);
                        } else {
                            a.out[f] = -INFINITY;
                        }
                    }
                }
            };
            auto issue = [&](int64_t off, int start, int cnt) {
                const int b = issued & 1;
                if (lane == 0) {
                    fence_proxy_async_smem();
                    const uint32_t bytes = static_cast<uint32_t>(cnt * M);
                    mbar_arrive_expect_tx(&wbar[b], bytes);
                    bulk_load(wbuf + b * kPieceBytes, a.codes + (off + start) * M, bytes, &wbar[b]);
                }
                ++issued;
            };

            int64_t f, off;
            int len = 0;
            take(f, off, len);
            if (f >= 0) issue(off, 0, min(kPiece, len));
            bool ok = true;
            while (f >= 0 && ok) {
                int64_t nf = -1, noff = 0;
                int nlen = 0;
                float rmax[QL];
#pragma unroll
                for (int u = 0; u < QL; ++u) rmax[u] = -INFINITY;
                for (int start = 0; start < len; start += kPiece) {
                    const int cnt = min(kPiece, len - start);
                    if (start + kPiece < len) {
                        issue(off, start + kPiece, min(kPiece, len - start - kPiece));
                    } else {
                        take(nf, noff, nlen);
                        if (nf >= 0) issue(noff, 0, min(kPiece, nlen));
                    }
                    const int b = consumed & 1;
                    const bool got = mbar_wait(&wbar[b], (consumed >> 1) & 1, &abort_flag, a.err, a.budget);
                    ++consumed;
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        break;
                    }
                    const uint8_t* base = wbuf + b * kPieceBytes;
                    const int last = cnt - 1;
                    // this lane's token j + r (a duplicate of the last token past the
                    // end cannot change a max); the next group's codes load early
                    CodeRow<M> c = smem_codes<M>(base + min(r, last) * M);
                    for (int j = 0; j < cnt; j += 16) {
                        const CodeRow<M> cn = smem_codes<M>(base + min(j + 16 + r, last) * M);
                        float acc[QL];
                        if constexpr (H16) {
#pragma unroll
                            for (int u = 0; u < QL; ++u) acc[u] = 0.f;
                            gather_groups<M, KS>(c, tbl_sa, lane_off, sel, [&](const uint4& e) {
                                add_f16x2(acc[0], acc[1], e.x);
                                add_f16x2(acc[2], acc[3], e.y);
                                add_f16x2(acc[4], acc[5], e.z);
                                add_f16x2(acc[6], acc[7], e.w);
                            });
                        } else {
                            unsigned long long p01 = 0ull, p23 = 0ull;  // (acc0, acc1), (acc2, acc3)
                            gather_groups<M, KS>(c, tbl_sa, lane_off, sel, [&](const uint4& e) {
                                add_f32x2(p01, e.x, e.y);
                                add_f32x2(p23, e.z, e.w);
                            });
                            acc[0] = __uint_as_float(static_cast<uint32_t>(p01));
                            acc[1] = __uint_as_float(static_cast<uint32_t>(p01 >> 32));
                            acc[2] = __uint_as_float(static_cast<uint32_t>(p23));
                            acc[3] = __uint_as_float(static_cast<uint32_t>(p23 >> 32));
                        }
#pragma unroll
                        for (int u = 0; u < QL; ++u) rmax[u] = fmaxf(rmax[u], acc[u]);
                        c = cn;
                    }
                    __syncwarp();
                }
                if (!ok) break;
                // max over the sixteen token lanes of each slot, then the sum over
                // this chunk's query tokens (u ascending, then the two slots)
                float v = 0.f;
#pragma unroll
                for (int u = 0; u < QL; ++u) {
                    float m = rmax[u];
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
                    v += (ch * QC + qt + u < a.nq) ? m : 0.f;
                }
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                if (lane == 0) a.out[f] = (ch == 0) ? v : a.out[f] + v;
                f = nf;
                off = noff;
                len = nlen;
            }
            // a timed-out warp lets its copies land before anything reuses the buffers
            while (consumed < issued) {
                const int b = consumed & 1;
                const long long t0 = clock64();
                while (!mbar_try_wait(&wbar[b], (consumed >> 1) & 1) && clock64() - t0 < kWaitBudgetCycles) {
                }
                ++consumed;
            }
        }
    }
}

}  // namespace pq
}  // namespace tms

extern "C" tms_status tms_build_pq_lut(const void* queries, tms_dtype qdtype, int n_queries, int nq, int d,
                                       const float* codebook, int m, int k, float* lut, cudaStream_t stream) {
    using namespace tms;
    if (qdtype != TMS_F16 && qdtype != TMS_BF16 && qdtype != TMS_F32) return TMS_ERR_INVALID_ARG;
    if (n_queries < 1 || nq < 1 || nq > 128 || d < 1 || m < 1 || m > 64 || k < 1 || k > 256 || d % m != 0)
        return TMS_ERR_INVALID_ARG;
    if (!queries || !codebook || !lut || !aligned16(queries) || !aligned16(codebook) || !aligned16(lut))
        return TMS_ERR_INVALID_ARG;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    const int64_t total = static_cast<int64_t>(n_queries) * nq * m * k;
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    const dim3 grid(static_cast<unsigned>(blocks)), block(threads);
    if (qdtype == TMS_F16)
        return launch_status(launch_dependent(pq::lut_kernel<__half>, grid, block, 0, stream,
                                              static_cast<const __half*>(queries), d, codebook, m, k, lut, total));
    if (qdtype == TMS_BF16)
        return launch_status(launch_dependent(pq::lut_kernel<__nv_bfloat16>, grid, block, 0, stream,
                                              static_cast<const __nv_bfloat16*>(queries), d, codebook, m, k, lut,
                                              total));
    return launch_status(launch_dependent(pq::lut_kernel<float>, grid, block, 0, stream,
                                          static_cast<const float*>(queries), d, codebook, m, k, lut, total));
}

namespace tms {
namespace pq {

// Shared host checks and launch of tms_score_pq / tms_score_pq_f16.
tms_status score(const float* lut, int n_queries, int nq, int m, int k, const uint8_t* codes, int64_t n_tokens,
                 const int64_t* doc_offsets, const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                 const int64_t* cand_offsets, int64_t n_cand, float* out_scores, bool half, cudaStream_t stream) {
    if (n_queries < 1 || n_queries > 4096 || nq < 1 || nq > 128 || k < 1 || k > 256) return TMS_ERR_INVALID_ARG;
    if (m != 4 && m != 8 && m != 16 && m != 32) return TMS_ERR_UNSUPPORTED;
    if (m * k > 4096 || (half && m < 16)) return TMS_ERR_UNSUPPORTED;
    if (n_tokens < 0 || n_docs < 0 || n_cand < 0 || n_cand >= (int64_t(1) << 31)) return TMS_ERR_INVALID_ARG;
    if (!lut || !cand_offsets || !aligned16(lut) || !aligned16(cand_offsets)) return TMS_ERR_INVALID_ARG;
    if (n_cand > 0 && (!cand_ids || !out_scores || !aligned16(cand_ids) || !aligned16(out_scores)))
        return TMS_ERR_INVALID_ARG;
    if (n_docs > 0 && (!doc_offsets || !doc_lengths || !aligned16(doc_offsets) || !aligned16(doc_lengths)))
        return TMS_ERR_INVALID_ARG;
    if (n_tokens > 0 && (!codes || !aligned16(codes))) return TMS_ERR_INVALID_ARG;
    if (n_cand == 0) return TMS_OK;
    DeviceInfo dev;
    tms_status st = current_device(&dev);
    if (st != TMS_OK) return st;
    Args a{};
    a.lut = lut;
    a.codes = codes;
    a.offsets = doc_offsets;
    a.lengths = doc_lengths;
    a.cand_ids = cand_ids;
    a.cand_offsets = cand_offsets;
    a.out = out_scores;
    a.err = dev.err;
    a.budget = debug_wait_budget();
    a.n_docs = n_docs;
    a.n_tokens = n_tokens;
    a.n_cand = n_cand;
    a.n_queries = n_queries;
    a.nq = nq;
    a.K = k;
    // The last subspace group is sized for 256 codes so that a code >= k
    // still indexes inside the allocation.
    const int smem = ((m / 4 - 1) * k + 256) * 32 * 4;
    const int tbl_st = staged_table_bytes(m >= 16 ? m : 16);
    const int smem_st = tbl_st + kWarps * 2 * kPieceBytes;  // staged variant: table + piece buffers
    if ((m >= 16 ? smem_st : smem) > dev.max_smem_optin) return TMS_ERR_UNSUPPORTED;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(dev.sm_count, n_cand)));
    const unsigned threads = kWarps * 32;
    auto staged = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_st);
        if (e == cudaSuccess) e = launch_dependent(kernel, dim3(grid), dim3(threads), smem_st, stream, a, tbl_st);
        return e;
    };
    auto plain = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = launch_dependent(kernel, dim3(grid), dim3(threads), smem, stream, a);
        return e;
    };
    cudaError_t e;
    if (m == 4)
        e = plain(score_kernel<4>);
    else if (m == 8)
        e = plain(score_kernel<8>);
    else if (m == 16)
        e = half ? staged(score_kernel_staged<16, true>) : staged(score_kernel_staged<16, false>);
    else
        e = half ? staged(score_kernel_staged<32, true>) : staged(score_kernel_staged<32, false>);
    if (e != cudaSuccess) return launch_status(e);
    return launch_status(cudaGetLastError());
}

}  // namespace pq
}  // namespace tms

extern "C" tms_status tms_score_pq(const float* lut, int n_queries, int nq, int m, int k, const uint8_t* codes,
                                   int64_t n_tokens, const int64_t* doc_offsets, const int32_t* doc_lengths,
                                   int64_t n_docs, const int32_t* cand_ids, const int64_t* cand_offsets,
                                   int64_t n_cand, float* out_scores, cudaStream_t stream) {
    return tms::pq::score(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs, cand_ids,
                          cand_offsets, n_cand, out_scores, false, stream);
}

extern "C" tms_status tms_score_pq_f16(const float* lut, int n_queries, int nq, int m, int k, const uint8_t* codes,
                                       int64_t n_tokens, const int64_t* doc_offsets, const int32_t* doc_lengths,
                                       int64_t n_docs, const int32_t* cand_ids, const int64_t* cand_offsets,
                                       int64_t n_cand, float* out_scores, cudaStream_t stream) {
    return tms::pq::score(lut, n_queries, nq, m, k, codes, n_tokens, doc_offsets, doc_lengths, n_docs, cand_ids,
                          cand_offsets, n_cand, out_scores, true, stream);
}
