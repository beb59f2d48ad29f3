// tms_dense_tc.cuh -- the tensor-core dense MaxSim kernel and its launcher.
//
// Computes Eq. 1 of the TileMaxSim paper, score = sum_i max_j q_i . d_j,
// for every candidate of every query, in one persistent launch, with the
// document and query rows stored as fp16 / bf16 or as FP8 E4M3 codes with
// one fp32 scale per row (F8).
//
// Orientation: the MMA computes S^T = Q D^T, query tokens along M (tensor-
// memory lanes, one per epilogue thread) and document rows along N
// (tensor-memory columns).  The max over a document's tokens (Eq. 1's
// inner max) is then a running max inside each thread's registers -- no
// cross-lane reduction per tile.  M is always 128: the query tile's 32-row
// blocks (token blocks of one query, or the queries of a shared group) are
// replicated down the 128 rows when they are fewer, and each copy scores
// its own slice of the tile's columns, so all four epilogue warps work on
// every tile.
//
//   * Producer warp: reads candidate metadata (id -> offset, length), and
//     streams each document's token rows from HBM into a ring of shared-
//     memory stages with TMA box loads (128-byte swizzle).  A stage holds
//     one or two 128-byte-wide dimension chunks (64 fp16/bf16 or 128 E4M3
//     elements) of up to 128 rows of ONE document, loaded as one box whose
//     height (8, 16, ..., 128) covers the tile's rows with at most 7 rows of
//     over-fetch.  Each token is read from HBM once (Theorem 1 with
//     BQ = Nq, or the whole group of queries in the shared schedule).  F8:
//     the tile's row scales follow through a small ring of TMA loads.
//   * MMA warp: one thread issues tcgen05.mma (M = 128 query rows,
//     N = the tile's rows rounded up to 16, K = 32 bytes: 16 fp16/bf16
//     elements with kind::f16, 32 E4M3 elements with kind::f8f6f4) over
//     every dimension chunk of a tile, accumulating the partial dot
//     products in tensor memory before any max is taken -- the paper's
//     dimension tiling (Section 3), with the K loop running through TMEM.
//   * Four epilogue warps: thread = query row (TMEM lane).  Each loads its
//     slice of the tile's columns with tcgen05.ld, multiplies column j by
//     document row j's scale (F8), drops columns past the tile's rows, and
//     folds the rest into its running max.  At a document's end the copies'
//     maxima meet in shared memory and one warp sums them over the query
//     tokens (times each token's scale, F8) in a fixed order and writes the
//     score once.  The Nq x Nd similarity matrix never reaches HBM and no
//     atomics or memset are needed.
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

constexpr int kRows = 128;                    // document rows per tile (MMA N at most)
constexpr int kChunkBytes = kRows * 128;      // 16 KB: 128 rows x one 128-byte dimension chunk
// Elements per 128-byte dimension chunk (one 128-byte swizzle row).
__host__ __device__ constexpr int chunk_elems(bool f8) { return f8 ? 128 : 64; }
constexpr int kBoxKinds = kRows / 8;          // box heights 8, 16, ..., 128
constexpr int kInfoRing = 16;
constexpr int kScaleRing = 8;                 // F8: tiles whose row scales are in flight or held
constexpr int kScaleBox = 136;                // floats per scale load: 128 rows + up to 3 of 16-byte alignment
constexpr int kScalePitch = 160;              // floats per scale slot (640 B, a multiple of 128 B)
constexpr int kEpiWarps = 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA, four epilogue warps
constexpr int kAcc = 2;                       // accumulator buffers (each H x 128 TMEM columns)
constexpr int kMaxStages = 16;
constexpr int kSmemLimit = 232448;            // 227 KB opt-in maximum per CTA

enum : int { kFirst = 1, kLast = 2, kEnd = 4 };

struct TileInfo {
    int f;      // flat candidate index
    int r;      // valid rows in this tile (1..128)
    int q;      // query index (shared mode: group index)
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
    int group;         // shared mode: queries per group; 0 otherwise
    int n_queries;
    int nq;
    int nchunks;   // ceil(d / chunk_elems)
    int cps;       // dimension chunks per stage: 2 with the 3-D tensor view (d % chunk_elems == 0), else 1
    int stages;
    int qslots;
    int bpc;         // 32-row query blocks per copy: ceil(nq / 32) token blocks, or the group's queries
    int reps;        // copies stacked in M; copy c scores tile columns [c * 128 / reps, (c + 1) * 128 / reps)
    int rows_alloc;  // query rows held per dimension chunk: 32 * bpc * reps
    int qbox;        // rows of one query TMA box: 32 * bpc (per-query), 32 (shared)
    uint32_t idesc;  // instruction descriptor, N field left 0 (set per tile)
};

struct Layout {
    int q_off, stage_off, part_off, sc_off, info_off, bar_off, misc_off, total;
};

// Shared-memory carve-up; the same arithmetic runs on host and device.
// The query region comes first: the MMA reads 128 (x H) rows from each
// query chunk, and rows past rows_alloc fall on the following chunk or on
// the stage ring -- always inside the allocation, and they only feed
// accumulator rows that nothing reads.  1 KB after the stage ring likewise
// absorbs the document operand's read of up to 8 rows past a chunk (N is
// the tile's rows rounded up to 16, the box up to 8).
__host__ __device__ inline Layout make_layout(int stages, int cps, int qslots, int nchunks, int rows_alloc, int H,
                                              bool f8) {
    Layout L;
    L.q_off = 0;
    L.stage_off = (qslots * nchunks * rows_alloc * 128 + 1023) & ~1023;
    L.part_off = L.stage_off + stages * cps * kChunkBytes + 1024;
    L.sc_off = L.part_off + 2 * 4 * H * 32 * 4;
    L.info_off = L.sc_off + (f8 ? kScaleRing * kScalePitch * 4 : 0);
    L.bar_off = L.info_off + kInfoRing * static_cast<int>(sizeof(TileInfo));
    const int nbar = 2 * stages + 2 * kAcc + 2 * qslots + 2 * kInfoRing + 4 + 2 * kScaleRing + 1;
    L.misc_off = L.bar_off + nbar * 8;
    L.total = L.misc_off + 16;
    return L;
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
// scales (F8): the [n_tokens] fp32 row scales, boxes of kScaleBox.
struct Maps {
    CUtensorMap q;
    CUtensorMap doc[kBoxKinds];
    CUtensorMap scales;
};

// H: 128-row halves of the query tile (2 for a shared group of 8 queries).
// SH (shared mode): the launch's queries all score one candidate list; a
// "query" of the pipeline is then a group of up to 4 H queries stacked in
// M, so each document tile is read once per group, and the epilogue
// writes one score per query of the group.
// F8: rows are E4M3 codes; similarities are scaled by the document row's
// scale before the max and by the query token's scale before the sum.
template <int H, int CTAS, bool SH, bool F8>
__global__ void __launch_bounds__(kThreads, CTAS)
    dense_tc_kernel(const __grid_constant__ Maps maps, const Args a) {
    constexpr int CE = chunk_elems(F8);
    constexpr uint32_t TCOLS = kAcc * H * 128;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    const int QS = a.qslots;
    const int NCH = a.nchunks;
    const int CPS = a.cps;
    const int stage_bytes = CPS * kChunkBytes;
    const int stages_per_tile = (NCH + CPS - 1) / CPS;
    const int qslot_bytes = NCH * a.rows_alloc * 128;
    const Layout L = make_layout(S, CPS, QS, NCH, a.rows_alloc, H, F8);

    uint8_t* q_base = smem + L.q_off;
    uint8_t* stage_base = smem + L.stage_off;
    float* part = reinterpret_cast<float*>(smem + L.part_off);  // [2][4 H][32]
    float* sc = reinterpret_cast<float*>(smem + L.sc_off);      // [kScaleRing][kScalePitch]
    TileInfo* info = reinterpret_cast<TileInfo*>(smem + L.info_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* full = bars;
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + kAcc;
    uint64_t* qfull = tempty + kAcc;
    uint64_t* qempty = qfull + QS;
    uint64_t* ifull = qempty + QS;
    uint64_t* iempty = ifull + kInfoRing;
    uint64_t* pfull = iempty + kInfoRing;  // [2]
    uint64_t* pempty = pfull + 2;          // [2]
    uint64_t* sfull = pempty + 2;          // [kScaleRing]
    uint64_t* sempty = sfull + kScaleRing; // [kScaleRing]
    uint64_t* mdone = sempty + kScaleRing;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < kAcc; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiWarps);
        }
        for (int i = 0; i < QS; ++i) {
            mbar_init(&qfull[i], 1);
            mbar_init(&qempty[i], 1);
        }
        for (int i = 0; i < kInfoRing; ++i) {
            mbar_init(&ifull[i], 1);
            mbar_init(&iempty[i], 1 + kEpiWarps);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&pfull[i], kEpiWarps);
            mbar_init(&pempty[i], 1);
        }
        for (int i = 0; i < kScaleRing; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], kEpiWarps);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        if (lane == 0) prefetch_tensormap(&maps.q);
        if (lane >= 1 && lane <= kBoxKinds) prefetch_tensormap(&maps.doc[lane - 1]);
        if (F8 && lane == kBoxKinds + 1) prefetch_tensormap(&maps.scales);
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
                    const int y0 = static_cast<int>(off) + r0;
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
                        ti.row0 = y0;
                        ti.pad = 0;
                        info[ii] = ti;
                        mbar_arrive(&ifull[ii]);
                    }
                    if (F8) {
                        // the tile's row scales, from the 16-byte boundary at or below its first row
                        const int j = t % kScaleRing;
                        if (!warp_wait(&sempty[j], ((t / kScaleRing) & 1) ^ 1, abort_flag, a.err)) {
                            aborted = true;
                            break;
                        }
                        if (lane == 0) {
                            mbar_arrive_expect_tx(&sfull[j], static_cast<uint32_t>(kScaleBox * 4));
                            tma_load_2d(sc + j * kScalePitch, &maps.scales, y0 & ~3, 0, &sfull[j], pol_stream);
                        }
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
                            mbar_arrive_expect_tx(&qfull[slot], static_cast<uint32_t>(qslot_bytes));
                            uint8_t* qdst = q_base + slot * qslot_bytes;
                            for (int kc = 0; kc < NCH; ++kc) {
                                uint8_t* cdst = qdst + kc * a.rows_alloc * 128;
                                for (int rp = 0; rp < a.reps; ++rp) {
                                    if (SH) {  // one 32-row box per query of the group
                                        for (int g = 0; g < a.bpc; ++g)
                                            tma_load_2d(cdst + (rp * a.bpc + g) * 32 * 128, &maps.q, kc * CE,
                                                        (q * a.group + g) * a.nq, &qfull[slot], pol_keep);
                                    } else {
                                        tma_load_2d(cdst + rp * a.qbox * 128, &maps.q, kc * CE, q * a.nq,
                                                    &qfull[slot], pol_keep);
                                    }
                                }
                            }
                        }
                        ++qi;
                        cur_q = q;
                    }
                    const int n8 = (r + 7) & ~7;
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
            if (F8) {
                const int ns = t < kScaleRing ? t : kScaleRing;
                for (int i = 1; i <= ns; ++i) drain_wait(&sfull[(t - i) % kScaleRing], ((t - i) / kScaleRing) & 1);
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
            int k = 0;  // tiles issued
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
                const int ab = k % kAcc;
                if (!mbar_wait(&tempty[ab], ((k / kAcc) & 1) ^ 1, abort_flag, a.err)) break;
                tc_fence_after();
                bool ok = true;
                const uint32_t d_tmem = tbase + static_cast<uint32_t>(ab * H * 128);
                const uint64_t q_desc = desc_sw128(smem_u32(q_base + qslot * qslot_bytes));
                const int n8 = (ti.r + 7) & ~7;
                const int n16 = (ti.r + 15) & ~15;
                const uint32_t idesc = a.idesc | (static_cast<uint32_t>(n16 >> 3) << 17);
                for (int st = 0; st < stages_per_tile; ++st) {
                    if (!mbar_wait(&full[s], ph, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // chunk c of the stage starts c * n8 rows in; the MMA
                    // reads n16 rows from there and the columns past the
                    // tile's r rows are dropped by the epilogue.
                    const uint64_t s_desc = desc_sw128(smem_u32(stage_base + s * stage_bytes));
                    for (int c = 0; c < CPS; ++c) {
                        const int kc = st * CPS + c;
                        if (kc >= NCH) break;
                        const uint64_t b_desc = s_desc + static_cast<uint64_t>((c * n8 * 128) >> 4);
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            const uint64_t a_desc =
                                q_desc + static_cast<uint64_t>(((kc * a.rows_alloc + h * 128) * 128) >> 4);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t accumulate = (kc > 0 || kk > 0) ? 1u : 0u;
                                if (F8)
                                    mma_f8(d_tmem + static_cast<uint32_t>(h * 128), a_desc + 2 * kk, b_desc + 2 * kk,
                                           idesc, accumulate);
                                else
                                    mma_f16(d_tmem + static_cast<uint32_t>(h * 128), a_desc + 2 * kk,
                                            b_desc + 2 * kk, idesc, accumulate);
                            }
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
                ++k;
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
        // Thread = query row 128 h + 32 qd + lane of half h (TMEM lane
        // 32 qd + lane).  Its 32-row block 4 h + qd is copy blk / bpc of
        // block blk % bpc; copy c owns tile columns [c W, c W + W) with
        // W = 128 / reps.  rmax[h] is the running max of that row over the
        // document's columns seen so far.
        const int qd = warp & 3;
        const int W = 128 / a.reps;
        float rmax[H];
#pragma unroll
        for (int h = 0; h < H; ++h) rmax[h] = -INFINITY;
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
#pragma unroll
                for (int h = 0; h < H; ++h) rmax[h] = -INFINITY;
            }
            const float* scl = nullptr;
            const int j = t % kScaleRing;
            if (F8) {
                if (!warp_wait(&sfull[j], (t / kScaleRing) & 1, abort_flag, a.err)) break;
                scl = sc + j * kScalePitch + (ti.row0 & 3);
            }
            const int ab = acc % kAcc;
            if (!warp_wait(&tfull[ab], (acc / kAcc) & 1, abort_flag, a.err)) break;
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int blk = 4 * h + qd;
                const int cp = blk / a.bpc;
                if (cp < a.reps) {
                    const int c_end = min(cp * W + W, ti.r);
                    for (int c0 = cp * W; c0 < c_end; c0 += 32) {
                        float v[32];
                        tmem_ld32(tbase + (static_cast<uint32_t>(qd * 32) << 16) +
                                      static_cast<uint32_t>((ab * H + h) * 128 + c0),
                                  v);
                        if (F8) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) v[c] *= scl[c0 + c];
                        }
                        if (c0 + 32 > ti.r) {
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                if (c0 + c >= ti.r) v[c] = -INFINITY;
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                            for (int c = 0; c < o; ++c) v[c] = fmaxf(v[c], v[c + o]);
                        rmax[h] = fmaxf(rmax[h], v[0]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&tempty[ab]);
                if (F8) mbar_arrive(&sempty[j]);
            }
            ++acc;
            if (ti.flags & kLast) {
                const int pb = docs & 1;
                const uint32_t use = docs >> 1;
                if (!warp_wait(&pempty[pb], (use & 1) ^ 1, abort_flag, a.err)) break;
                float* pp = part + pb * 4 * H * 32;
#pragma unroll
                for (int h = 0; h < H; ++h) pp[(4 * h + qd) * 32 + lane] = rmax[h];
                __syncwarp();
                if (lane == 0) mbar_arrive(&pfull[pb]);
                if (qd == 0) {
                    if (!warp_wait(&pfull[pb], use & 1, abort_flag, a.err)) break;
                    if (SH) {
                        const int64_t fc = static_cast<int64_t>(ti.f) % a.n_cand;
                        for (int b = 0; b < a.bpc; ++b) {
                            float m = pp[b * 32 + lane];
                            for (int rp = 1; rp < a.reps; ++rp) m = fmaxf(m, pp[(rp * a.bpc + b) * 32 + lane]);
                            const int qq = ti.q * a.group + b;
                            float sq = 1.f;
                            if (F8 && lane < a.nq && qq < a.n_queries)
                                sq = __ldg(a.q_scales + static_cast<int64_t>(qq) * a.nq + lane);
                            const float sum = warp_sum(lane < a.nq ? (F8 ? m * sq : m) : 0.f);
                            if (lane == 0 && qq < a.n_queries) a.out[static_cast<int64_t>(qq) * a.n_cand + fc] = sum;
                        }
                    } else {
                        float sum = 0.f;
                        for (int b = 0; b < a.bpc; ++b) {
                            float m = pp[b * 32 + lane];
                            for (int rp = 1; rp < a.reps; ++rp) m = fmaxf(m, pp[(rp * a.bpc + b) * 32 + lane]);
                            const int tok = b * 32 + lane;
                            if (tok < a.nq)
                                sum += F8 ? m * __ldg(a.q_scales + static_cast<int64_t>(ti.q) * a.nq + tok) : m;
                        }
                        sum = warp_sum(sum);
                        if (lane == 0) a.out[ti.f] = sum;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&pempty[pb]);
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

// Plan shared memory, encode the tensor maps and launch dense_tc_kernel.
// F8 ignores `dtype` (rows are E4M3 codes; t_scales in `a`).  The caller
// sets a.nchunks = ceil(d / chunk_elems(F8)), and a.bpc / a.qbox: per-query
// ceil(nq / 32) and 32 bpc, shared mode the group size and 32.
template <int H, bool SH, bool F8>
tms_status launch_tc(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                     const void* doc_tokens, int64_t n_tokens, Args a, cudaStream_t stream) {
    constexpr int CE = chunk_elems(F8);
    const CUtensorMapDataType tdt = F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                  : dtype == TMS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const uint64_t row_bytes = static_cast<uint64_t>(d) * (F8 ? 1 : 2);
    // With no document rows nothing is ever loaded through the document
    // maps; describe the query buffer so that they still encode.
    const void* dbase = n_tokens > 0 ? doc_tokens : queries;
    Maps maps;
    tms_status st = encode_tmap_2d(&maps.q, tdt, queries, d, static_cast<uint64_t>(n_queries) * nq, row_bytes,
                                   CE, static_cast<uint32_t>(a.qbox));
    if (st != TMS_OK) return st;
    // Shared-memory plan.  Prefer two CTAs per SM (H == 1: 256 TMEM columns
    // each) when each still gets a ring of at least 4 dimension chunks, with
    // as many copies of the query blocks as fit (fewer copies only narrow
    // the epilogue's share of each tile); else one CTA per SM.  Within a
    // plan take the query-slot count (2, else 1) that gives the most stage
    // chunks.
    const bool can3d = d % CE == 0 && a.nchunks >= 2;
    auto plan = [&](int per_cta_limit, int cps, int rows_alloc, int& stages, int& qslots) {
        int best = -1;
        for (int qs = 2; qs >= 1; --qs) {
            const Layout L0 = make_layout(0, cps, qs, a.nchunks, rows_alloc, H, F8);
            const int sts = std::min(kMaxStages, (per_cta_limit - L0.total) / (cps * kChunkBytes + 16));
            if (sts * cps > best) {
                best = sts * cps;
                stages = sts;
                qslots = qs;
            }
        }
        return best;
    };
    const int max_reps = SH ? (a.bpc == 2 ? 2 : 1) : (a.bpc == 3 ? 1 : 4 / a.bpc);
    const int limit1 = std::min(kSmemLimit, dev.max_smem_optin) - 1024;
    const int limit2 = dev.smem_per_sm / 2 - dev.smem_reserved - 1024;
    int stages = 0, qslots = 1, ctas = 0, reps = max_reps, cps = can3d ? 2 : 1;
    if (H == 1) {
        for (int rp = max_reps; rp >= 1 && ctas == 0; rp /= 2) {
            const int ra = 32 * a.bpc * rp;
            for (int c = can3d ? 2 : 1; c >= 1 && ctas == 0; --c) {
                if (plan(limit2, c, ra, stages, qslots) >= 4 && stages >= 2) {
                    ctas = 2;
                    reps = rp;
                    cps = c;
                }
            }
        }
    }
    for (int rp = max_reps; rp >= 1 && ctas == 0; rp /= 2) {
        const int ra = 32 * a.bpc * rp;
        for (int c = can3d ? 2 : 1; c >= 1 && ctas == 0; --c) {
            if (plan(limit1, c, ra, stages, qslots) >= 2 && stages >= 2) {
                ctas = 1;
                reps = rp;
                cps = c;
            }
        }
    }
    if (ctas == 0) return TMS_ERR_UNSUPPORTED;
    a.reps = reps;
    a.rows_alloc = 32 * a.bpc * reps;
    a.cps = cps;
    for (int h = 0; h < kBoxKinds; ++h) {
        const uint32_t rows = static_cast<uint32_t>(8 * (h + 1));
        st = a.cps == 2 ? encode_tmap_rows_chunks(&maps.doc[h], tdt, dbase, a.nchunks, n_tokens, row_bytes, rows, CE)
                        : encode_tmap_2d(&maps.doc[h], tdt, dbase, d, n_tokens, row_bytes, CE, rows);
        if (st != TMS_OK) return st;
    }
    if (F8) {
        st = encode_tmap_1d_f32(&maps.scales, n_tokens > 0 ? static_cast<const void*>(a.t_scales) : queries,
                                static_cast<uint64_t>(n_tokens), kScaleBox);
        if (st != TMS_OK) return st;
    } else {
        maps.scales = maps.q;  // never used
    }
    // format code 0 is f16 under kind::f16 and E4M3 under kind::f8f6f4
    a.idesc = make_idesc(128, 0, (!F8 && dtype == TMS_BF16) ? 1u : 0u);
    a.stages = stages;
    a.qslots = qslots;
    const Layout L = make_layout(stages, a.cps, qslots, a.nchunks, a.rows_alloc, H, F8);
    const int smem = L.total + 1024;
    auto kern = ctas == 2 ? dense_tc_kernel<H, (H == 1 ? 2 : 1), SH, F8> : dense_tc_kernel<H, 1, SH, F8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return launch_status(cudaErrorInvalidValue);
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(dev.sm_count) * ctas, a.n_flat);
    kern<<<static_cast<unsigned>(grid), kThreads, smem, stream>>>(maps, a);
    return launch_status(cudaGetLastError());
}

}  // namespace dense

}  // namespace tms
