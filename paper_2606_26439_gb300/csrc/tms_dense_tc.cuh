// tms_dense_tc.cuh -- the tensor-core dense MaxSim kernel and its launcher.
//
// Computes Eq. 1 of the TileMaxSim paper, score = sum_i max_j q_i . d_j,
// for every candidate of every query, in one persistent launch, with the
// document and query rows stored as fp16 / bf16 or as FP8 E4M3 codes with
// one fp32 scale per row (F8).
//
//   * Producer warp: reads candidate metadata (id -> offset, length), and
//     streams each document's token rows from HBM into a ring of shared-
//     memory stages with TMA box loads (128-byte swizzle).  A stage holds
//     one or two 128-byte-wide dimension chunks (64 fp16/bf16 or 128 E4M3
//     elements) of up to 128 rows of ONE document, loaded as one box whose
//     height (8, 16, ..., 128) covers the tile's rows with at most 7 rows of
//     over-fetch.  Each token is read from HBM once (Theorem 1 with
//     BQ = Nq).
//   * MMA warp: one elected thread issues tcgen05.mma (M = 128 document
//     rows, N = Nq padded to 32, K = 32 bytes: 16 fp16/bf16 elements with
//     kind::f16, 32 E4M3 elements with kind::f8f6f4) over every dimension
//     chunk of a tile, accumulating the partial dot products in tensor
//     memory before any max is taken -- the paper's dimension tiling
//     (Section 3), with the K loop running through TMEM.
//   * Four epilogue warps: thread = document row (TMEM lane).  Each reads
//     its row's accumulators with tcgen05.ld, multiplies them by the row's
//     scale (F8), and takes per-query-token column maxima with redux.sync
//     over exactly the tile's valid rows.  At a document's end the four
//     warps' maxima meet in shared memory, one warp sums them over the Nq
//     query tokens (times each token's scale, F8) in a fixed order and
//     writes the score once.  The Nq x Nd similarity matrix never reaches
//     HBM and no atomics or memset are needed.
//
// Every wait is bounded (see tms_common.cuh); a timeout sets
// TMS_DEVERR_TIMEOUT and the CTA drains its in-flight copies and MMAs,
// frees its tensor memory and returns.
#pragma once

#include <algorithm>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {

namespace dense {

constexpr int kRows = 128;                    // document rows per tile (MMA M)
constexpr int kChunkBytes = kRows * 128;      // 16 KB: 128 rows x one 128-byte dimension chunk
// Elements per 128-byte dimension chunk (one 128-byte swizzle row).
__host__ __device__ constexpr int chunk_elems(bool f8) { return f8 ? 128 : 64; }
constexpr int kBoxKinds = kRows / 8;          // box heights 8, 16, ..., 128
constexpr int kInfoRing = 16;
// One epilogue group of 4 warps per CTA.  (The kernel keeps the general
// multi-group bookkeeping; two CTAs per SM -- each a full producer / MMA /
// epilogue pipeline -- replace a second group: the tensor core accepts one
// small MMA per ~84 cycles whatever its N, and the issuing thread blocks
// meanwhile, so a second CTA's MMA thread fills the tensor pipe while the
// first one waits or does its per-tile bookkeeping.)
__host__ __device__ constexpr int epi_groups(int NT) { return 1; }
__host__ __device__ constexpr int num_threads(int NT) { return 64 + 128 * epi_groups(NT); }
constexpr int kMaxStages = 16;
constexpr int kSmemLimit = 232448;            // 227 KB opt-in maximum per CTA

enum : int { kFirst = 1, kLast = 2, kEnd = 4 };

struct TileInfo {
    int f;      // flat candidate index
    int r;      // valid rows in this tile (1..128)
    int q;      // query index
    int flags;  // kFirst / kLast / kEnd
    int row0;   // token row of the tile's first row
    int pad;
};

struct Args {
    const int64_t* offsets;
    const int32_t* lengths;
    const int32_t* cand_ids;
    const int64_t* cand_offsets;
    float* out;
    const float* q_scales;  // F8: [n_queries * nq] per-query-token scales
    const float* t_scales;  // F8: [n_tokens] per-document-token scales
    unsigned int* err;
    int64_t n_docs;
    int64_t n_tokens;
    int64_t n_cand;    // entries of cand_ids
    int64_t n_flat;    // work items: n_cand, or n_groups * n_cand in shared mode
    int group;         // shared mode: queries per group (each a 32-column block); 0 otherwise
    int n_queries;
    int nq;
    int nchunks;   // ceil(d / chunk_elems)
    int cps;       // dimension chunks per stage: 2 with the 3-D tensor view (d % chunk_elems == 0), else 1
    int stages;
    int qslots;
    uint32_t idesc;
};

struct Layout {
    int stage_off, q_off, part_off, info_off, bar_off, misc_off, total;
};

// Shared-memory carve-up; the same arithmetic runs on host and device.
__host__ __device__ inline Layout make_layout(int stages, int cps, int qslots, int nchunks, int NT, int acc) {
    Layout L;
    L.stage_off = 0;
    L.q_off = stages * cps * kChunkBytes;
    L.part_off = L.q_off + qslots * nchunks * NT * 128;
    L.info_off = L.part_off + epi_groups(NT) * 2 * 4 * NT * 4;
    L.bar_off = L.info_off + kInfoRing * static_cast<int>(sizeof(TileInfo));
    const int nbar = 2 * stages + 2 * acc + 2 * qslots + 2 * kInfoRing + epi_groups(NT) * 4 + 1;
    L.misc_off = L.bar_off + nbar * 8;
    L.total = L.misc_off + 16;
    return L;
}

// A tile's K-steps are spread round-robin over `partials(NT)` accumulators
// so that consecutive MMAs never depend on each other (a chain of tiny
// M=128 x N=32 x K=16 MMAs into one accumulator is latency-bound); the
// epilogue adds the partials before the max.
//
// Each epilogue group owns its own ring of acc_buffers(NT) accumulators,
// used in the order of that group's tiles.  (With one shared ring a group
// that skips the other group's tiles could wait on the second use of an
// accumulator whose barrier has not finished its first phase -- and an
// mbarrier parity wait cannot tell those apart.)
__host__ __device__ constexpr int partials(int NT) { return NT <= 32 ? 4 : (NT <= 128 ? 2 : 1); }
__host__ __device__ constexpr int acc_buffers(int NT) { return 2; }

__host__ __device__ constexpr int acc_total(int NT) { return epi_groups(NT) * acc_buffers(NT); }

__host__ __device__ constexpr int tmem_cols(int NT) {
    return (acc_total(NT) * partials(NT) * NT <= 32) ? 32
         : (acc_total(NT) * partials(NT) * NT <= 64) ? 64
         : (acc_total(NT) * partials(NT) * NT <= 128) ? 128
         : (acc_total(NT) * partials(NT) * NT <= 256) ? 256 : 512;
}

// Candidate metadata for the producer: lane l of the warp holds the raw
// entry of candidate window position l.  Loads are only issued here; they
// are classified (meta_status) when the window becomes current, one window
// later, so the producer never waits on them.
struct Meta {
    int64_t off;
    int len;
    int id;
};

__device__ __forceinline__ int load_id(const Args& a, int64_t k) {
    const int64_t f = static_cast<int64_t>(blockIdx.x) + k * gridDim.x;
    if (f >= a.n_flat) return -1;
    return __ldg(a.cand_ids + (a.group ? f % a.n_cand : f));
}

__device__ __forceinline__ Meta load_meta(const Args& a, int id) {
    Meta m;
    m.id = id;
    m.off = 0;
    m.len = 0;
    if (id >= 0 && id < a.n_docs) {
        m.off = __ldg(a.offsets + id);
        m.len = __ldg(a.lengths + id);
    }
    return m;
}

// 0 ok, 1 bad id, 2 bad row range.
__device__ __forceinline__ int meta_status(const Args& a, int id, int64_t off, int len) {
    if (id < 0 || id >= a.n_docs) return 1;
    return (len < 0 || off < 0 || off + len > a.n_tokens) ? 2 : 0;
}

// Every lane waits (and so acquires the barrier's phase itself); the warp
// agrees on the outcome.  Returns false on timeout / abort.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* err) {
    const bool ok = mbar_wait(bar, parity, abort_flag, err);
    return __all_sync(0xffffffffu, ok) != 0;
}

// Drain wait: bounded, but ignores the abort flag (used to let in-flight
// asynchronous work land before the CTA exits).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitBudgetCycles) break;
    }
}

// Tensor maps of one launch.  doc[h] covers document rows with a box of
// 8 (h + 1) rows, so a tile of r rows is always ONE box (at most 7 rows of
// over-fetch).  With cps == 2 the document maps are the 3-D view
// {128 bytes of elements, rows, chunk} of the [n_tokens][d] array (chunk
// stride 128 bytes): one box brings two chunks of r rows, landing as
// [chunk][row][128 B] -- already the 128-byte-swizzle K-major layout.
struct Maps {
    CUtensorMap q;
    CUtensorMap doc[kBoxKinds];
};

// SH (shared mode): the launch's queries all score one candidate list; a
// "query" of the pipeline is then a group of up to NB queries stacked in
// the MMA's N dimension (32 columns each), so each document tile is read
// once per group, and the epilogue writes one score per query of the group.
// F8: rows are E4M3 codes; similarities are scaled by the document row's
// scale before the max and by the query token's scale before the sum.
template <int NB, int CTAS, bool SH, bool F8>
__global__ void __launch_bounds__(num_threads(NB * 32), CTAS)
    dense_tc_kernel(const __grid_constant__ Maps maps, const Args a) {
    constexpr int NT = NB * 32;
    constexpr int CE = chunk_elems(F8);
    constexpr int kEpiGroups = epi_groups(NT);
    constexpr int A = acc_buffers(NT);   // per epilogue group
    constexpr int P = partials(NT);
    constexpr uint32_t TCOLS = tmem_cols(NT);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    const int QS = a.qslots;
    const int NCH = a.nchunks;
    const int CPS = a.cps;
    const int stage_bytes = CPS * kChunkBytes;
    const int stages_per_tile = (NCH + CPS - 1) / CPS;
    const Layout L = make_layout(S, CPS, QS, NCH, NT, acc_total(NT));

    uint8_t* stage_base = smem + L.stage_off;
    uint8_t* q_base = smem + L.q_off;
    float* part = reinterpret_cast<float*>(smem + L.part_off);  // [group][2][4][NT]
    TileInfo* info = reinterpret_cast<TileInfo*>(smem + L.info_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* full = bars;
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + acc_total(NT);
    uint64_t* qfull = tempty + acc_total(NT);
    uint64_t* qempty = qfull + QS;
    uint64_t* ifull = qempty + QS;
    uint64_t* iempty = ifull + kInfoRing;
    uint64_t* pfull = iempty + kInfoRing;       // [group][2]
    uint64_t* pempty = pfull + 2 * kEpiGroups;  // [group][2]
    uint64_t* mdone = pempty + 2 * kEpiGroups;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < acc_total(NT); ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);
        }
        for (int i = 0; i < QS; ++i) {
            mbar_init(&qfull[i], 1);
            mbar_init(&qempty[i], 1);
        }
        for (int i = 0; i < kInfoRing; ++i) {
            mbar_init(&ifull[i], 1);
            mbar_init(&iempty[i], 1 + 4 * kEpiGroups);
        }
        for (int i = 0; i < 2 * kEpiGroups; ++i) {
            mbar_init(&pfull[i], 4);
            mbar_init(&pempty[i], 1);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        if (lane <= kBoxKinds) prefetch_tensormap(lane == 0 ? &maps.q : &maps.doc[lane - 1]);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------ producer
        const uint64_t pol_stream = policy_evict_first();
        const uint64_t pol_keep = policy_evict_last();
        int s = 0;
        uint32_t ph = 0;
        int64_t issued = 0;
        int t = 0;
        int qi = 0, cur_q = -1;
        int q = 0;
        int64_t q_end = 0;
        bool aborted = false;
        if (!SH) {
            const int64_t co_last = __ldg(a.cand_offsets + a.n_queries);
            if (co_last != a.n_cand && blockIdx.x == 0 && lane == 0) atomicOr(a.err, TMS_DEVERR_BAD_CSR);
            q_end = __ldg(a.cand_offsets + 1);
        }
        // three-window metadata pipeline: ids two windows ahead, offsets
        // and lengths one window ahead, the current window in registers.
        int id_next = load_id(a, 32 + lane);
        Meta cur = load_meta(a, load_id(a, lane));
        Meta nxt = load_meta(a, id_next);
        int id_next2 = load_id(a, 64 + lane);

        for (int64_t k = 0;; ++k) {
            const int kl = static_cast<int>(k & 31);
            const int64_t f = static_cast<int64_t>(blockIdx.x) + k * gridDim.x;
            if (f >= a.n_flat) break;
            const int cid = __shfl_sync(0xffffffffu, cur.id, kl);
            const int64_t off = __shfl_sync(0xffffffffu, cur.off, kl);
            const int len = __shfl_sync(0xffffffffu, cur.len, kl);
            const int status = meta_status(a, cid, off, len);
            if (SH) {
                q = static_cast<int>(f / a.n_cand);
            } else {
                while (f >= q_end && q < a.n_queries - 1) {
                    ++q;
                    q_end = __ldg(a.cand_offsets + q + 1);
                }
            }
            if (status != 0 || len == 0) {
                const float v = status != 0 ? __int_as_float(0x7fc00000) : -INFINITY;
                if (SH) {
                    const int64_t fc = f % a.n_cand;
                    if (lane < a.group && q * a.group + lane < a.n_queries)
                        a.out[static_cast<int64_t>(q * a.group + lane) * a.n_cand + fc] = v;
                } else if (lane == 0) {
                    a.out[f] = v;
                }
                if (status != 0 && lane == 0)
                    atomicOr(a.err, status == 1 ? TMS_DEVERR_BAD_ID : TMS_DEVERR_BAD_RANGE);
            } else {
                for (int r0 = 0; r0 < len; r0 += kRows) {
                    const int r = min(kRows, len - r0);
                    const int ii = t % kInfoRing;
                    if (!warp_wait(&iempty[ii], ((t / kInfoRing) & 1) ^ 1, abort_flag, a.err)) {
                        aborted = true;
                        break;
                    }
                    if (lane == 0) {
                        TileInfo ti;
                        ti.f = static_cast<int>(f);
                        ti.r = r;
                        ti.q = q;
                        ti.flags = (r0 == 0 ? kFirst : 0) | (r0 + kRows >= len ? kLast : 0);
                        ti.row0 = static_cast<int>(off) + r0;
                        ti.pad = 0;
                        info[ii] = ti;
                        mbar_arrive(&ifull[ii]);
                    }
                    ++t;
                    // A new query's rows go to the next query slot.  The
                    // tile info is published first: the MMA warp releases
                    // the old slot only once it sees the new query.
                    if (q != cur_q) {
                        const int slot = qi % QS;
                        if (!warp_wait(&qempty[slot], ((qi / QS) & 1) ^ 1, abort_flag, a.err)) {
                            aborted = true;
                            break;
                        }
                        if (lane == 0) {
                            mbar_arrive_expect_tx(&qfull[slot], static_cast<uint32_t>(NCH * NT * 128));
                            uint8_t* qdst = q_base + slot * NCH * NT * 128;
                            for (int kc = 0; kc < NCH; ++kc) {
                                if (SH) {  // one 32-row box per query of the group
                                    for (int g = 0; g < NB; ++g)
                                        tma_load_2d(qdst + kc * NT * 128 + g * 32 * 128, &maps.q, kc * CE,
                                                    (q * a.group + g) * a.nq, &qfull[slot], pol_keep);
                                } else {
                                    tma_load_2d(qdst + kc * NT * 128, &maps.q, kc * CE, q * a.nq,
                                                &qfull[slot], pol_keep);
                                }
                            }
                        }
                        ++qi;
                        cur_q = q;
                    }
                    const int n8 = (r + 7) & ~7;
                    const int y0 = static_cast<int>(off) + r0;
                    const CUtensorMap* dmap = &maps.doc[(n8 >> 3) - 1];
                    for (int st = 0; st < stages_per_tile; ++st) {
                        if (!warp_wait(&empty[s], ph ^ 1, abort_flag, a.err)) {
                            aborted = true;
                            break;
                        }
                        if (lane == 0) {
                            uint8_t* dst = stage_base + s * stage_bytes;
                            mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>(n8 * 128 * CPS));
                            if (CPS == 2)
                                tma_load_3d(dst, dmap, 0, y0, 2 * st, &full[s], pol_stream);
                            else
                                tma_load_2d(dst, dmap, st * CE, y0, &full[s], pol_stream);
                        }
                        ++issued;
                        if (++s == S) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    if (aborted) break;
                }
                if (aborted) break;
            }
            if (kl == 31) {
                cur = nxt;
                nxt = load_meta(a, id_next2);
                id_next2 = load_id(a, k + 65 + lane);
            }
        }
        if (!aborted) {
            const int ii = t % kInfoRing;
            if (warp_wait(&iempty[ii], ((t / kInfoRing) & 1) ^ 1, abort_flag, a.err)) {
                if (lane == 0) {
                    TileInfo ti;
                    ti.f = 0;
                    ti.r = 0;
                    ti.q = 0;
                    ti.flags = kEnd;
                    ti.row0 = 0;
                    ti.pad = 0;
                    info[ii] = ti;
                    mbar_arrive(&ifull[ii]);
                }
            }
        }
        // Let every copy still in flight land before the CTA can exit.
        if (lane == 0) {
            const int64_t n = issued < S ? issued : S;
            int ss = s;
            uint32_t pp = ph;
            for (int64_t i = 0; i < n; ++i) {
                if (--ss < 0) {
                    ss = S - 1;
                    pp ^= 1;
                }
                drain_wait(&full[ss], pp);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA
        // One thread runs this role: every wait is its own (no warp votes),
        // and descriptors advance by adding the 16-byte-unit offset of each
        // K-step to a per-stage base.
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int qi = 0, cur_q = -1, qslot = 0;
            int acc0 = 0, acc1 = 0;  // tiles issued for epilogue group 0 / 1
            uint32_t doc_ord = 0;
            int owner = 0;
            bool any = false;
            for (int t = 0;; ++t) {
                const int ii = t % kInfoRing;
                if (!mbar_wait(&ifull[ii], (t / kInfoRing) & 1, abort_flag, a.err)) break;
                const TileInfo ti = info[ii];
                mbar_arrive(&iempty[ii]);
                if (ti.flags & kEnd) break;
                if (ti.q != cur_q) {
                    if (cur_q >= 0) mma_commit(&qempty[qslot]);
                    qslot = qi % QS;
                    if (!mbar_wait(&qfull[qslot], (qi / QS) & 1, abort_flag, a.err)) break;
                    ++qi;
                    cur_q = ti.q;
                }
                if (ti.flags & kFirst) {
                    owner = static_cast<int>(doc_ord % kEpiGroups);
                    ++doc_ord;
                }
                const int k = owner == 0 ? acc0 : acc1;
                const int ab = owner * A + k % A;
                if (!mbar_wait(&tempty[ab], ((k / A) & 1) ^ 1, abort_flag, a.err)) break;
                tc_fence_after();
                bool ok = true;
                const uint32_t d_tmem = tbase + static_cast<uint32_t>(ab * P * NT);
                const uint64_t q_desc = desc_sw128(smem_u32(q_base + qslot * NCH * NT * 128));
                const int n8 = (ti.r + 7) & ~7;
                for (int st = 0; st < stages_per_tile; ++st) {
                    if (!mbar_wait(&full[s], ph, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // chunk c of the stage starts c * n8 rows in: its rows
                    // past n8 (and the tile's rows past r) are masked later.
                    const uint64_t s_desc = desc_sw128(smem_u32(stage_base + s * stage_bytes));
                    for (int c = 0; c < CPS; ++c) {
                        const int kc = st * CPS + c;
                        if (kc >= NCH) break;
                        const uint64_t a_desc = s_desc + static_cast<uint64_t>((c * n8 * 128) >> 4);
                        const uint64_t b_desc = q_desc + static_cast<uint64_t>((kc * NT * 128) >> 4);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const int ks = kc * 4 + kk;  // K-step of the tile
                            if (F8)
                                mma_f8(d_tmem + static_cast<uint32_t>((ks % P) * NT), a_desc + 2 * kk,
                                       b_desc + 2 * kk, a.idesc, ks >= P ? 1u : 0u);
                            else
                                mma_f16(d_tmem + static_cast<uint32_t>((ks % P) * NT), a_desc + 2 * kk,
                                        b_desc + 2 * kk, a.idesc, ks >= P ? 1u : 0u);
                        }
                    }
                    mma_commit(&empty[s]);
                    any = true;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&tfull[ab]);
                if (owner == 0)
                    ++acc0;
                else
                    ++acc1;
            }
            // Every MMA this thread issued must finish before TMEM is freed.
            if (any) {
                mma_commit(mdone);
                drain_wait(mdone, 0);
            }
        }
        __syncwarp();
    } else {
        // ----------------------------------------------------- epilogue
        // Thread = document row (TMEM lane), register c = query token c.
        // The column max over the tile's valid rows is one redux.sync.max
        // per column whose member mask is exactly those rows, so rows past
        // the document end never take part; the running maxima are held
        // warp-uniform (lane 0 always participates when any row is valid).
        // Group g (warps 2+4g .. 5+4g) takes the documents whose ordinal is
        // g mod kEpiGroups; both groups read every tile's info.
        const int qd = warp & 3;  // TMEM lane quadrant this warp may read
        const int grp = (warp - 2) >> 2;
        float* gpart = part + grp * 2 * 4 * NT;
        uint64_t* gpfull = pfull + 2 * grp;
        uint64_t* gpempty = pempty + 2 * grp;
        uint32_t doc_ord = 0;  // ordinal of the current document (all groups count all documents)
        bool mine = false;
        constexpr int RB = SH ? 1 : NB;  // blocks of warp-uniform maxima (normal mode)
        float rm[RB][32];
        float rmd[NB];                    // per-lane maxima (shared mode)
#pragma unroll
        for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int c = 0; c < 32; ++c) rm[b][c] = -INFINITY;
#pragma unroll
        for (int b = 0; b < NB; ++b) rmd[b] = -INFINITY;
        int acc = 0;
        uint32_t docs = 0;  // documents finished; buffer = docs & 1, its use count = docs >> 1
        for (int t = 0;; ++t) {
            const int ii = t % kInfoRing;
            if (!warp_wait(&ifull[ii], (t / kInfoRing) & 1, abort_flag, a.err)) break;
            const TileInfo ti = info[ii];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iempty[ii]);
            if (ti.flags & kEnd) break;
            if (ti.flags & kFirst) {
                mine = (doc_ord % kEpiGroups) == static_cast<uint32_t>(grp);
                ++doc_ord;
#pragma unroll
                for (int b = 0; b < RB; ++b)
#pragma unroll
                    for (int c = 0; c < 32; ++c) rm[b][c] = -INFINITY;
#pragma unroll
                for (int b = 0; b < NB; ++b) rmd[b] = -INFINITY;
            }
            if (!mine) continue;  // another group's tile
            // F8: this thread's document row scale, fetched before the
            // accumulator wait so the load overlaps it.
            float srow = 1.f;
            if (F8 && qd * 32 + lane < ti.r) srow = __ldg(a.t_scales + ti.row0 + qd * 32 + lane);
            const int ab = grp * A + acc % A;
            if (!warp_wait(&tfull[ab], (acc / A) & 1, abort_flag, a.err)) break;
            tc_fence_after();
            const int rows_here = ti.r - qd * 32;
            const int ksteps = NCH * 4;
            if (rows_here > 0) {
                const unsigned vmask = rows_here >= 32 ? 0xffffffffu : ((1u << rows_here) - 1u);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    // sum the partial accumulators that received any K-step
                    const uint32_t tl = tbase + (static_cast<uint32_t>(qd * 32) << 16) +
                                        static_cast<uint32_t>(ab * P * NT + b * 32);
                    float v[32];
                    tmem_ld32(tl, v);
#pragma unroll
                    for (int pp = 1; pp < P; ++pp) {
                        if (pp < ksteps) {
                            float w[32];
                            tmem_ld32(tl + static_cast<uint32_t>(pp * NT), w);
#pragma unroll
                            for (int c = 0; c < 32; ++c) v[c] += w[c];
                        }
                    }
                    if (F8) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) v[c] *= srow;
                    }
                    if (SH) {
                        // running max kept per lane: lane c owns column c of block b
                        if (rows_here < 32 && lane >= rows_here) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) v[c] = -INFINITY;
                        }
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float m = redux_max(v[c], 0xffffffffu);
                            if (lane == c) rmd[b] = fmaxf(rmd[b], m);
                        }
                    } else if (lane < rows_here) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) rm[b][c] = fmaxf(rm[b][c], redux_max(v[c], vmask));
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[ab]);
            ++acc;
            if (ti.flags & kLast) {
                const int pb = docs & 1;
                const uint32_t use = docs >> 1;
                if (!warp_wait(&gpempty[pb], (use & 1) ^ 1, abort_flag, a.err)) break;
                float* pp = gpart + pb * 4 * NT;
                if (SH) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) pp[qd * NT + b * 32 + lane] = rmd[b];
                } else if (lane == 0) {
#pragma unroll
                    for (int b = 0; b < RB; ++b)
#pragma unroll
                        for (int c = 0; c < 32; c += 4)
                            *reinterpret_cast<float4*>(pp + qd * NT + b * 32 + c) =
                                make_float4(rm[b][c], rm[b][c + 1], rm[b][c + 2], rm[b][c + 3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&gpfull[pb]);
                if (qd == 0) {
                    if (!warp_wait(&gpfull[pb], use & 1, abort_flag, a.err)) break;
                    if (SH) {
                        const int64_t fc = static_cast<int64_t>(ti.f) % a.n_cand;
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            const int col = b * 32 + lane;
                            const float m =
                                fmaxf(fmaxf(pp[col], pp[NT + col]), fmaxf(pp[2 * NT + col], pp[3 * NT + col]));
                            const int qq = ti.q * a.group + b;
                            float sq = 1.f;
                            if (F8 && lane < a.nq && b < a.group && qq < a.n_queries)
                                sq = __ldg(a.q_scales + static_cast<int64_t>(qq) * a.nq + lane);
                            const float sum = warp_sum(lane < a.nq ? (F8 ? m * sq : m) : 0.f);
                            if (lane == 0 && b < a.group && qq < a.n_queries)
                                a.out[static_cast<int64_t>(qq) * a.n_cand + fc] = sum;
                        }
                    } else {
                        float sum = 0.f;
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            const int col = b * 32 + lane;
                            const float m =
                                fmaxf(fmaxf(pp[col], pp[NT + col]), fmaxf(pp[2 * NT + col], pp[3 * NT + col]));
                            if (col < a.nq)
                                sum += F8 ? m * __ldg(a.q_scales + static_cast<int64_t>(ti.q) * a.nq + col) : m;
                        }
                        sum = warp_sum(sum);
                        if (lane == 0) a.out[ti.f] = sum;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&gpempty[pb]);
                }
                ++docs;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TCOLS);
    }
}

}  // namespace dense

namespace dense {

// Plan shared memory, encode the tensor maps and launch dense_tc_kernel.
// F8 ignores `dtype` (rows are E4M3 codes); a.nchunks must be
// ceil(d / chunk_elems(F8)).
template <int NB, bool SH, bool F8>
tms_status launch_tc(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                     const void* doc_tokens, int64_t n_tokens, Args a, cudaStream_t stream) {
    constexpr int NT = NB * 32;
    constexpr int A = acc_total(NT);   // all epilogue groups
    constexpr int CE = chunk_elems(F8);
    const CUtensorMapDataType tdt = F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                  : dtype == TMS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const uint64_t row_bytes = static_cast<uint64_t>(d) * (F8 ? 1 : 2);
    Maps maps;
    tms_status st = encode_tmap_2d(&maps.q, tdt, queries, d, static_cast<uint64_t>(n_queries) * nq, row_bytes,
                                   CE, SH ? 32 : NT);
    if (st != TMS_OK) return st;
    // Shared-memory plan.  Prefer two CTAs per SM (NT <= 64) when each
    // still gets a ring of at least 4 dimension chunks; within a plan take
    // the query-slot count (2, else 1) that gives the most stage chunks.
    const bool can3d = d % CE == 0 && a.nchunks >= 2;
    auto plan = [&](int per_cta_limit, int cps, int& stages, int& qslots) {
        int best = -1;
        for (int qs = 2; qs >= 1; --qs) {
            const Layout L0 = make_layout(0, cps, qs, a.nchunks, NT, A);
            const int sts = std::min(kMaxStages, (per_cta_limit - L0.total) / (cps * kChunkBytes + 16));
            if (sts * cps > best) {
                best = sts * cps;
                stages = sts;
                qslots = qs;
            }
        }
        return best;
    };
    int stages = 0, qslots = 1, ctas = 1;
    const int limit1 = std::min(kSmemLimit, dev.max_smem_optin) - 1024;
    const int limit2 = dev.smem_per_sm / 2 - dev.smem_reserved - 1024;
    a.cps = can3d ? 2 : 1;
    if (NT <= 64 && plan(limit2, a.cps, stages, qslots) >= 4 && stages >= 2) {
        ctas = 2;
    } else if (NT <= 64 && can3d && plan(limit2, 1, stages, qslots) >= 4) {
        ctas = 2;
        a.cps = 1;
    } else {
        a.cps = can3d ? 2 : 1;
        if (plan(limit1, a.cps, stages, qslots) < 2 || stages < 2) {
            a.cps = 1;
            if (plan(limit1, 1, stages, qslots) < 2) return TMS_ERR_UNSUPPORTED;
        }
    }
    for (int h = 0; h < kBoxKinds; ++h) {
        const uint32_t rows = static_cast<uint32_t>(8 * (h + 1));
        st = a.cps == 2
                 ? encode_tmap_rows_chunks(&maps.doc[h], tdt, doc_tokens, a.nchunks, n_tokens, row_bytes, rows, CE)
                 : encode_tmap_2d(&maps.doc[h], tdt, doc_tokens, d, n_tokens, row_bytes, CE, rows);
        if (st != TMS_OK) return st;
    }
    // format code 0 is f16 under kind::f16 and E4M3 under kind::f8f6f4
    a.idesc = make_idesc(kRows, NT, (!F8 && dtype == TMS_BF16) ? 1u : 0u);
    a.stages = stages;
    a.qslots = qslots;
    const Layout L = make_layout(stages, a.cps, qslots, a.nchunks, NT, A);
    const int smem = L.total + 1024;
    auto kern = ctas == 2 ? dense_tc_kernel<NB, (NB <= 2 ? 2 : 1), SH, F8> : dense_tc_kernel<NB, 1, SH, F8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return launch_status(cudaErrorInvalidValue);
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(dev.sm_count) * ctas, a.n_flat);
    kern<<<static_cast<unsigned>(grid), num_threads(NT), smem, stream>>>(maps, a);
    return launch_status(cudaGetLastError());
}

}  // namespace dense

}  // namespace tms
