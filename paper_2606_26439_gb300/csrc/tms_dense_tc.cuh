// tms_dense_tc.cuh -- the tensor-core dense MaxSim kernel and its launcher.
//
// Computes Eq. 1 of the TileMaxSim paper, score = sum_i max_j q_i . d_j,
// for every candidate of every query, in one persistent launch, with the
// document and query rows stored as fp16 / bf16, as FP8 E4M3 codes with one
// fp32 scale per row (F8), or as fp32 scored by split TF32 (TF: each
// operand x = hi + lo with hi = x with its 13 low mantissa bits cleared --
// the value a kind::tf32 MMA reads from an fp32 element -- and lo = x - hi
// exact; hi.hi + hi.lo + lo.hi on the tensor cores, the lo.lo term of
// relative size below 2^-20 dropped -- FP32-level accuracy).
//
// Orientation: the MMA computes S^T = Q D^T, query tokens along M (tensor-
// memory lanes, one per epilogue thread) and document rows along N
// (tensor-memory columns).  The max over a document's tokens (Eq. 1's
// inner max) is then a running max inside each thread's registers -- no
// cross-lane reduction.  M is always 128: the query tile's 32-row blocks
// (token blocks of one query, or the queries of a shared group) are
// replicated down the 128 rows when they are fewer.
//
// Super-tiles: consecutive document tiles (up to 128 rows each, padded to
// 8) are packed side by side into one super-tile of up to 256 rows (128
// with two query halves), and one run of MMAs (N = the packed rows rounded
// up to 16) scores them all.  The per-tile costs of the pipeline --
// barrier round trips, commits, MMA issue -- are paid once per super-tile,
// typically two to three documents.
//
//   * Planner warp: takes the candidates 32 at a time, one per lane
//     (metadata, validity, query, -inf / NaN for empty / bad documents),
//     packs their tiles into super-tiles and publishes each super-tile as
//     one record -- header plus tile list -- with a single barrier
//     arrival.  It also loads each query's tile (replicated, see above)
//     and, F8, every tile's row scales through a ring of small TMA loads.
//   * Loader warp: streams each super-tile from HBM into a ring of shared-
//     memory chunk stages (STR rows x 128 bytes: 64 fp16/bf16 or 128 E4M3
//     elements per row), one TMA box per tile and chunk, the tiles issued
//     by parallel lanes (128-byte swizzle).  Each token is read from HBM
//     once (Theorem 1 with BQ = Nq, or the whole group of queries in the
//     shared schedule).
//   * TF only -- four splitter warps: split every landed chunk stage (hi in
//     place, lo beside it) and every new query tile before the MMA reads
//     them.
//   * MMA warp: one thread issues tcgen05.mma (M = 128 query rows, K = 32
//     bytes: 16 fp16/bf16 elements with kind::f16, 32 E4M3 elements with
//     kind::f8f6f4, 8 TF32 elements -- three products -- with kind::tf32)
//     over every dimension chunk of a super-tile,
//     accumulating the partial dot products in tensor memory before any
//     max is taken -- the paper's dimension tiling (Section 3), with the K
//     loop running through TMEM.
//   * Four epilogue warps: thread = query row (TMEM lane).  Documents are
//     dealt round-robin to the copies of the query tile; the warps of a
//     copy load their document's columns with tcgen05.ld, multiply column
//     j by document row j's scale (F8), drop columns of other documents,
//     and fold the rest into a running max.  At the document's end each
//     warp sums its 32 query tokens (times their scales, F8); with one
//     token block per copy that sum is the score, else the copy's warps
//     add their sums in block order.  Each score is written once; the
//     Nq x Nd similarity matrix never reaches HBM and no atomics or memset
//     are needed.
//
// Every wait is bounded (see tms_common.cuh); a timeout sets
// TMS_DEVERR_TIMEOUT and the CTA drains its in-flight copies and MMAs,
// frees its tensor memory and returns.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>

#include "tms_common.cuh"
#include "tms_internal.h"

namespace tms {

namespace dense {

constexpr int kRows = 128;                    // document rows per tile
// Row types: fp16 / bf16, FP8 E4M3 codes + row scales, fp32 by split TF32,
// PQ codes decompressed into fp16 rows in shared memory (kPQ: M = 16
// subspaces of 8 dimensions, d = 128).
enum : int { kF16 = 0, kE4M3 = 1, kTF32 = 2, kPQ = 3 };
// Elements per 128-byte dimension chunk (one 128-byte swizzle row).
__host__ __device__ constexpr int chunk_elems(int kind) { return kind == kE4M3 ? 128 : (kind == kTF32 ? 32 : 64); }
constexpr int kPqM = 16;                      // kPQ: subspaces (16 code bytes per token)
constexpr int kPqCbBytes = 256 * kPqM * 16;   // kPQ: fp16 codebook, all 256 codes (64 KB)
constexpr int kCodeRing = 4;                  // kPQ: super-tiles whose code rows are in flight or held
constexpr int kBoxKinds = kRows / 8;          // box heights 8, 16, ..., 128
constexpr int kMaxSeg = 32;                   // tiles per super-tile (each >= 8 rows, one per planner lane)
// Super-tile records in flight.  A record slot is republished only after
// every role has passed it, so the ring also bounds how far the loader can
// run ahead of the epilogue: with HBM latencies of a few microseconds under
// load, the loads of many super-tiles must be in flight at once.
__host__ __device__ constexpr int st_ring(int) { return 16; }
constexpr int kEpiWarps = 4;
constexpr int kLoaderWarp = 2 + kEpiWarps;
constexpr int kThreads = 32 * (kLoaderWarp + 1);  // planner, MMA, four epilogue warps, loader
constexpr int kSplitWarps = 4;                    // TF: splitter warps after the loader; kPQ: decompressors
__host__ __device__ constexpr int kernel_threads(int kind) {
    return kThreads + ((kind == kTF32 || kind == kPQ) ? 32 * kSplitWarps : 0);
}
// Accumulator buffers (each H x STR tensor-memory columns): as many as the
// SM's 512 columns hold for the CTAs sharing it, at most one per epilogue
// warp.
__host__ __device__ constexpr int acc_count(int h, int str, int ctas) {
    return 512 / (h * str * ctas) < kEpiWarps ? 512 / (h * str * ctas) : kEpiWarps;
}
constexpr int kMaxAcc = kEpiWarps;
constexpr int kMaxStages = 16;
constexpr int kSmemLimit = 232448;            // 227 KB opt-in maximum per CTA

enum : int { kFirst = 1, kLast = 2, kEnd = 4, kStFirst = 8, kStLast = 16 };

// One document tile inside a super-tile (16 bytes).
struct SegInfo {
    int f;        // flat candidate index (shared mode: position in the candidate list)
    int row0;     // token row of the tile's first row
    short r;      // valid rows (1..128)
    short col;    // first column (row of the super-tile), a multiple of 8
    int flags;    // kFirst / kLast of the document
};

// One super-tile record (planner -> loader, MMA thread and epilogue).
struct StHdr {
    int q;      // query (group) whose tile it is scored against
    int n;      // MMA N: packed rows rounded up to 16
    int nseg;   // tiles
    int flags;  // kEnd
    int rows;   // packed rows (sum of the tiles' rows rounded up to 8)
    int pad[3];
};

struct StSlot {
    StHdr h;
    SegInfo seg[kMaxSeg];
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
    int nchunks;     // ceil(d / chunk_elems)
    int stages;      // chunk stages in the ring
    int qslots;      // resident query-tile slots; 0: the query is streamed with each chunk stage
    int bpc;         // 32-row query blocks per copy: ceil(nq / 32) token blocks, or the group's queries
    int reps;        // copies of the blocks stacked in M (1, 2 or 4); documents are dealt round-robin to them
    int rows_alloc;  // query rows held per dimension chunk: 32 * bpc * reps
    int qbox;        // rows of one query TMA box: 32 * bpc (per-query), 32 (shared)
    uint32_t idesc;  // instruction descriptor, N field left 0 (set per super-tile)
    const uint8_t* pq_codes;    // kPQ: [n_tokens][16] uint8
    const float* pq_codebook;   // kPQ: [16][pq_k][8] fp32
    int pq_k;                   // kPQ: centroids per subspace (codes >= pq_k read zeros)
    long long budget;           // SM cycles a pipeline wait may last (<= 0: kWaitBudgetCycles)
    int fault;                  // diagnostics: kFaultHoldAccumulator, else 0
};

// Diagnostics (tms_debug_set): the MMA thread of CTA 0 never signals its
// first accumulator, so that CTA's epilogue wait runs out of budget and the
// timeout path -- flag, abort, drain, tensor-memory release -- runs.
constexpr int kFaultHoldAccumulator = TMS_FAULT_HOLD_ACCUMULATOR;

struct Layout {
    int q_off, qlo_off, stage_off, stage_stride, part_off, fin_off, sc_off, cb_off, code_off, st_off, bar_off, misc_off,
        total;
};

// Finished documents waiting for their sum over query tokens, per epilogue
// warp: kFinRows rows of 32 row maxima (one row per document and query
// half), padded to 33 floats so that lane r reading row r walks distinct
// banks, then each document's (candidate, query) pair.
constexpr int kFinRows = 16;
constexpr int kFinWarpBytes = kFinRows * 33 * 4 + kFinRows * 8;

// Shared-memory carve-up; the same arithmetic runs on host and device.
// The query region comes first: the MMA reads 128 (x H) rows from each
// query chunk, and rows past rows_alloc fall on the following chunk or on
// the stage ring -- always inside the allocation, and they only feed
// accumulator rows that nothing reads.  A stage holds the full super-tile
// of str rows, so the document operand (N <= str) never reads past it.
// TF: the query region and every stage have a lo twin right after them.
// F8: per super-tile record slot, the row scale of every column.
// Streamed query (qslots = 0, qrows = 128 H): no resident query region;
// each chunk stage holds the str document rows, then the qrows query rows
// of the same dimension chunk.
__host__ __device__ inline Layout make_layout(int stages, int qslots, int nchunks, int rows_alloc, int str, int kind,
                                              int kacc, bool fin, int qrows) {
    const bool f8 = kind == kE4M3;
    const int twin = kind == kTF32 ? 2 : 1;
    Layout L;
    L.q_off = 0;
    L.qlo_off = qslots * nchunks * rows_alloc * 128;
    L.stage_off = (twin * L.qlo_off + 1023) & ~1023;
    L.stage_stride = twin * (str + qrows) * 128;
    L.part_off = L.stage_off + stages * L.stage_stride;
    L.fin_off = L.part_off + 128;  // after [2 copies][2 parities][4 blocks] partial sums
    L.sc_off = L.fin_off + (fin ? kEpiWarps * kFinWarpBytes : 0);  // 128-byte aligned
    L.cb_off = L.sc_off + (f8 ? st_ring(str) * str * 4 : 0);  // F8: [st_ring][str] column scales
    L.code_off = L.cb_off + (kind == kPQ ? kPqCbBytes : 0);                        // kPQ: fp16 codebook
    // kPQ: code-row ring, then per slot the valid rows of each 8-row group
    L.st_off = L.code_off + (kind == kPQ ? kCodeRing * (str * kPqM + kMaxSeg * 4) : 0);
    L.bar_off = L.st_off + st_ring(str) * static_cast<int>(sizeof(StSlot));
    const int nbar = 3 * stages + 2 * kacc + 3 * qslots + 3 * st_ring(str) + 8 + 1 + 2 * kCodeRing;
    L.misc_off = L.bar_off + nbar * 8;
    L.total = L.misc_off + 16;
    return L;
}

// Candidate metadata for the planner: lane l of the warp holds the raw
// entry of candidate window position l.  Loads are only issued here; they
// are classified (meta_status) when the window becomes current, one window
// later, so the planner never waits on them.
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

// Lane 0 polls the barrier and broadcasts the outcome; the warp barrier
// orders the other lanes after lane 0's acquire.  For barriers guarding
// data written by other threads or ordering tensor-core work.  Returns
// false on timeout / abort.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* err, long long budget) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, err, budget) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// Every lane waits (and so observes the phase itself): for barriers that
// complete the TMA bytes the lanes then read.
__device__ __forceinline__ bool warp_wait_all(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned int* err, long long budget) {
    const bool ok = mbar_wait(bar, parity, abort_flag, err, budget);
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

// x with its 13 low mantissa bits cleared: the TF32 value a kind::tf32 MMA
// reads from an fp32 element.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// Maxima of the four 8-column sub-blocks of 32 accumulator columns.
// Document tiles start on 8-column boundaries, so a tile covers whole
// sub-blocks except, at a document's end, a last partial one.
__device__ __forceinline__ void sub_maxima8(const float (&v)[32], float (&sb)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        sb[k] = fmax3(fmax3(v[8 * k], v[8 * k + 1], v[8 * k + 2]), fmax3(v[8 * k + 3], v[8 * k + 4], v[8 * k + 5]),
                      fmaxf(v[8 * k + 6], v[8 * k + 7]));
}

// max(m, v[lo..hi)) for 0 <= lo < hi <= 32 with lo a multiple of 8: the
// whole sub-blocks from their maxima sb, a partial last one (hi not a
// multiple of 8) from its hi % 8 leading columns.  A tile covering the
// whole group (the common case inside long documents) takes one branch
// and two maxima.
__device__ __forceinline__ float fold_cols(float m, const float (&v)[32], const float (&sb)[4], int lo, int hi) {
    if (lo == 0 && hi == 32) return fmax3(m, fmax3(sb[0], sb[1], sb[2]), sb[3]);
    const int kl = lo >> 3;
    const int kf = hi >> 3;
    // sub-blocks [kl, kf) as a 4-bit mask
    const uint32_t whole = (0xfu >> (4 - kf)) & ~((1u << kl) - 1u);
    float x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = (whole >> k) & 1u ? sb[k] : -INFINITY;
    m = fmax3(m, fmax3(x[0], x[1], x[2]), x[3]);
    const int rem = hi & 7;
    if (rem != 0) {  // sub-block kf < 4 holds rem columns of the tile
        // the sub-block's first 7 columns, picked by kf, then masked to rem
        float y[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const float lo2 = (kf & 1) ? v[8 + j] : v[j];
            const float hi2 = (kf & 1) ? v[24 + j] : v[16 + j];
            y[j] = j < rem ? ((kf & 2) ? hi2 : lo2) : -INFINITY;
        }
        m = fmax3(m, fmax3(y[0], y[1], y[2]), fmax3(y[3], y[4], fmaxf(y[5], y[6])));
    }
    return m;
}

// Tensor maps of one launch.  doc[h] covers document rows with a box of
// 8 (h + 1) rows x one 128-byte chunk, so a tile of r rows is always ONE
// box per chunk (at most 7 rows of over-fetch).
struct Maps {
    CUtensorMap q;
    CUtensorMap doc[kBoxKinds];
};

// H: 128-row halves of the query tile (2 for a shared group of 8 queries).
// STR: rows per super-tile (MMA N at most), 256 or 128.  CTAS: CTAs per SM
// (1 or 2); the CTA holds KACC = acc_count(H, STR, CTAS) accumulators of
// H x STR tensor-memory columns.
// SH (shared mode): the launch's queries all score one candidate list; a
// "query" of the pipeline is then a group of up to 4 H queries stacked in
// M, so each document tile is read once per group, and the epilogue
// writes one score per query of the group.
// F8: rows are E4M3 codes; similarities are scaled by the document row's
// scale before the max and by the query token's scale before the sum.
template <int H, int STR, int CTAS, bool SH, int KIND>
__global__ void __launch_bounds__(kernel_threads(KIND), CTAS)
    dense_tc_kernel(const __grid_constant__ Maps maps, const Args a) {
    constexpr bool F8 = KIND == kE4M3;
    constexpr bool TF = KIND == kTF32;
    constexpr bool PQ = KIND == kPQ;
    constexpr int CE = chunk_elems(KIND);
    constexpr int STAGE_BYTES = STR * 128;
    constexpr int KACC = acc_count(H, STR, CTAS);
    constexpr uint32_t TCOLS = KACC * H * STR;
    constexpr int kStRing = st_ring(STR);
    static_assert(KACC >= 2 && TCOLS * CTAS <= 512, "tensor memory of one SM");

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    const int QS = a.qslots;
    const int NCH = a.nchunks;
    const int qslot_bytes = NCH * a.rows_alloc * 128;
    const bool QSTREAM = QS == 0;  // the query rows come with every chunk stage
    const Layout L = make_layout(S, QS, NCH, a.rows_alloc, STR, KIND, KACC, SH || a.bpc == 1, QSTREAM ? 128 * H : 0);
    const int SSTRIDE = L.stage_stride;  // bytes between stages (TF: hi, then lo)

    uint8_t* q_base = smem + L.q_off;
    uint8_t* qlo_base = smem + L.qlo_off;  // TF: the lo twin of the query region
    uint8_t* stage_base = smem + L.stage_off;
    float* part = reinterpret_cast<float*>(smem + L.part_off);  // [copy][parity][block]
    uint8_t* fin_base = smem + L.fin_off;                       // [epilogue warp] finished-document rows
    float* sc = reinterpret_cast<float*>(smem + L.sc_off);      // F8: [kStRing][STR] scale of each column
    StSlot* slots = reinterpret_cast<StSlot*>(smem + L.st_off);
    uint8_t* cb = smem + L.cb_off;           // kPQ: fp16 codebook, entry (code, m) at (code * 16 + m) * 16
    uint8_t* code_ring = smem + L.code_off;  // kPQ: [kCodeRing][STR rows][16] code bytes
    uint8_t* gvalid = code_ring + kCodeRing * STR * kPqM;  // kPQ: [kCodeRing][STR / 8] valid rows per 8-row group
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* full = bars;
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;              // [KACC] accumulator ready
    uint64_t* tempty = tfull + KACC;          // [KACC] accumulator read by every active epilogue warp
    uint64_t* qfull = tempty + KACC;
    uint64_t* qempty = qfull + QS;
    uint64_t* xfull = qempty + QS;          // [kStRing]
    uint64_t* xempty = xfull + kStRing;     // [kStRing]
    uint64_t* pfull = xempty + kStRing;     // [copy][parity]
    uint64_t* pempty = pfull + 4;           // [copy][parity]
    uint64_t* scfull = pempty + 4;          // F8: [kStRing] a record slot's column scales landed
    uint64_t* mdone = scfull + kStRing;
    uint64_t* conv = mdone + 1;   // TF: [S] stage split
    uint64_t* qconv = conv + S;   // TF: [QS] query tile split
    uint64_t* codefull = qconv + QS;            // kPQ: [kCodeRing] code rows landed
    uint64_t* codeempty = codefull + kCodeRing;  // kPQ: [kCodeRing] code rows consumed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], PQ ? kSplitWarps : 1);  // kPQ: every decompressor warp wrote its rows
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < KACC; ++i) {
            mbar_init(&tfull[i], 1);
            // the active epilogue warps: those whose row block belongs to a copy
            mbar_init(&tempty[i], a.reps * a.bpc < kEpiWarps ? a.reps * a.bpc : kEpiWarps);
        }
        for (int i = 0; i < QS; ++i) {
            mbar_init(&qfull[i], 1);
            mbar_init(&qempty[i], 1);
        }
        for (int i = 0; i < kStRing; ++i) {
            mbar_init(&xfull[i], 1);
            mbar_init(&xempty[i], 2 + kEpiWarps + ((TF || PQ) ? kSplitWarps : 0));  // loader, MMA, epilogue, splitters
        }
        for (int i = 0; i < 4; ++i) {
            mbar_init(&pfull[i], a.bpc);
            mbar_init(&pempty[i], 1);
        }
        for (int i = 0; i < kStRing; ++i) mbar_init(&scfull[i], 32);  // one cp.async arrival per loader lane
        mbar_init(mdone, 1);
        for (int i = 0; i < S; ++i) mbar_init(&conv[i], kSplitWarps);
        for (int i = 0; i < QS; ++i) mbar_init(&qconv[i], kSplitWarps);
        for (int i = 0; i < kCodeRing; ++i) {
            mbar_init(&codefull[i], 1);
            mbar_init(&codeempty[i], kSplitWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kLoaderWarp) {
        if (lane < kBoxKinds) prefetch_tensormap(&maps.doc[lane]);
    }
    if (warp == 0 && lane == 0) prefetch_tensormap(&maps.q);
    if (warp == 1) {
        tmem_alloc(tmem_slot, TCOLS);
        tmem_relinquish();
    }
    // Nothing above reads global memory: the previous kernel of the stream
    // may still be running until here.
    griddep_wait();
    griddep_launch_dependents();
    if constexpr (PQ) {
        // the codebook, rounded to fp16 (nearest even), for all 256 codes:
        // codes >= pq_k get zeros
        for (int e = threadIdx.x; e < 256 * kPqM; e += blockDim.x) {
            const int code = e / kPqM;
            const int m = e - code * kPqM;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (code < a.pq_k) {
                const float4* src =
                    reinterpret_cast<const float4*>(a.pq_codebook + (static_cast<int64_t>(m) * a.pq_k + code) * 8);
                const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
                const __half2 h0 = __floats2half2_rn(x0.x, x0.y), h1 = __floats2half2_rn(x0.z, x0.w);
                const __half2 h2 = __floats2half2_rn(x1.x, x1.y), h3 = __floats2half2_rn(x1.z, x1.w);
                v = make_uint4(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1),
                               *reinterpret_cast<const uint32_t*>(&h2), *reinterpret_cast<const uint32_t*>(&h3));
            }
            *reinterpret_cast<uint4*>(cb + e * 16) = v;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------- planner
        const uint64_t pol_keep = policy_evict_last();
        int tst = 0;   // super-tiles published
        int qi = 0, cur_q = -1;
        bool aborted = false;
        // The open super-tile: its tile i lives in lane i's registers.
        int nseg = 0, rows_used = 0, st_q = 0;
        int my_f = 0, my_r = 0, my_flags = 0, my_row0 = 0, my_col = 0;

        // Publish the open super-tile: the record, and the query tile if the
        // query changed.
        auto close_st = [&]() -> bool {
            const bool has = lane < nseg;
            const int xs = tst % kStRing;
            if (!warp_wait(&xempty[xs], ((tst / kStRing) & 1) ^ 1, abort_flag, a.err, a.budget)) return false;
            StSlot* x = &slots[xs];
            if (has) {
                SegInfo si;
                si.f = my_f;
                si.row0 = my_row0;
                si.r = static_cast<short>(my_r);
                si.col = static_cast<short>(my_col);
                si.flags = my_flags;
                x->seg[lane] = si;
            }
            if (lane == 0) {
                StHdr h;
                h.q = st_q;
                h.n = (rows_used + 15) & ~15;
                h.nseg = nseg;
                h.flags = 0;
                h.rows = rows_used;
                h.pad[0] = h.pad[1] = h.pad[2] = 0;
                x->h = h;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&xfull[xs]);
            ++tst;
            // A new query's rows go to the next query slot.  The record is
            // published first: the MMA thread releases the old slot only
            // once it sees the new query.
            if (!QSTREAM && st_q != cur_q) {
                const int slot = qi % QS;
                if (!warp_wait(&qempty[slot], ((qi / QS) & 1) ^ 1, abort_flag, a.err, a.budget)) return false;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&qfull[slot], static_cast<uint32_t>(qslot_bytes));
                    uint8_t* qdst = q_base + slot * qslot_bytes;
                    for (int kc = 0; kc < NCH; ++kc) {
                        uint8_t* cdst = qdst + kc * a.rows_alloc * 128;
                        for (int rp = 0; rp < a.reps; ++rp) {
                            if (SH) {  // one 32-row box per query of the group
                                for (int g = 0; g < a.bpc; ++g)
                                    tma_load_2d(cdst + (rp * a.bpc + g) * 32 * 128, &maps.q, kc * CE,
                                                (st_q * a.group + g) * a.nq, &qfull[slot], pol_keep);
                            } else {
                                tma_load_2d(cdst + rp * a.qbox * 128, &maps.q, kc * CE, st_q * a.nq, &qfull[slot],
                                            pol_keep);
                            }
                        }
                    }
                }
                ++qi;
                cur_q = st_q;
            }
            nseg = 0;
            rows_used = 0;
            return true;
        };

        int qw = 0;            // query of the window's first candidate (per-query mode)
        int64_t qw_end = 0;    // its end in the flat list
        if (!SH) {
            const int64_t co_last = __ldg(a.cand_offsets + a.n_queries);
            if (co_last != a.n_cand && blockIdx.x == 0 && lane == 0) atomicOr(a.err, TMS_DEVERR_BAD_CSR);
            qw_end = __ldg(a.cand_offsets + 1);
        }
        // three-window metadata pipeline: ids two windows ahead, offsets
        // and lengths one window ahead, the current window in registers.
        int id_next = load_id(a, 32 + lane);
        Meta cur = load_meta(a, load_id(a, lane));
        Meta nxt = load_meta(a, id_next);
        int id_next2 = load_id(a, 64 + lane);

        for (int64_t k0 = 0;; k0 += 32) {
            if (static_cast<int64_t>(blockIdx.x) + k0 * gridDim.x >= a.n_flat) break;
            // lane = one candidate of the window
            const int64_t f = static_cast<int64_t>(blockIdx.x) + (k0 + lane) * gridDim.x;
            const bool valid = f < a.n_flat;
            const int status = valid ? meta_status(a, cur.id, cur.off, cur.len) : 3;
            int ql = 0;
            int64_t pos = f;  // shared mode: position in the candidate list
            if (SH) {
                if (valid) {
                    ql = static_cast<int>(f / a.n_cand);
                    pos = f - static_cast<int64_t>(ql) * a.n_cand;
                }
            } else {
                ql = qw;
                int64_t qe = qw_end;
                if (valid) {
                    while (f >= qe && ql < a.n_queries - 1) {
                        ++ql;
                        qe = __ldg(a.cand_offsets + ql + 1);
                    }
                }
                const int last = __popc(__ballot_sync(0xffffffffu, valid)) - 1;
                qw = __shfl_sync(0xffffffffu, ql, last);
                qw_end = __shfl_sync(0xffffffffu, qe, last);
            }
            if (valid && (status != 0 || cur.len == 0)) {
                const float v = status != 0 ? __int_as_float(0x7fc00000) : -INFINITY;
                if (SH) {
                    for (int g = 0; g < a.group; ++g)
                        if (ql * a.group + g < a.n_queries)
                            a.out[static_cast<int64_t>(ql * a.group + g) * a.n_cand + pos] = v;
                } else {
                    a.out[f] = v;
                }
                if (status != 0) atomicOr(a.err, status == 1 ? TMS_DEVERR_BAD_ID : TMS_DEVERR_BAD_RANGE);
            }
            // pack the window's documents, in order, into super-tiles
            unsigned docs = __ballot_sync(0xffffffffu, valid && status == 0 && cur.len > 0);
            while (docs != 0u) {
                const int i = __ffs(docs) - 1;
                docs &= docs - 1u;
                const int len = __shfl_sync(0xffffffffu, cur.len, i);
                const int off = static_cast<int>(__shfl_sync(0xffffffffu, cur.off, i));
                const int q = __shfl_sync(0xffffffffu, ql, i);
                const int fi = static_cast<int>(__shfl_sync(0xffffffffu, SH ? pos : f, i));
                // Tiles of at most kRows rows fill the open super-tile to its
                // last 8-row group: a document that does not fit is cut at
                // the super-tile's end and continues in the next one.
                for (int r0 = 0; r0 < len;) {
                    if (nseg > 0 && (q != st_q || rows_used == STR || nseg == STR / 8)) {
                        if (!close_st()) {
                            aborted = true;
                            break;
                        }
                    }
                    if (nseg == 0) st_q = q;
                    const int r = min(min(kRows, len - r0), STR - rows_used);
                    if (lane == nseg) {
                        my_f = fi;
                        my_r = r;
                        my_flags = (r0 == 0 ? kFirst : 0) | (r0 + r >= len ? kLast : 0);
                        my_row0 = off + r0;
                        my_col = rows_used;
                    }
                    rows_used += (r + 7) & ~7;
                    ++nseg;
                    r0 += r;
                }
                if (aborted) break;
            }
            if (aborted) break;
            cur = nxt;
            nxt = load_meta(a, id_next2);
            id_next2 = load_id(a, k0 + 96 + lane);
        }
        if (!aborted && nseg > 0 && !close_st()) aborted = true;
        if (!aborted) {
            const int xs = tst % kStRing;
            if (warp_wait(&xempty[xs], ((tst / kStRing) & 1) ^ 1, abort_flag, a.err, a.budget) && lane == 0) {
                StHdr h;
                h.q = 0;
                h.n = 0;
                h.nseg = 0;
                h.flags = kEnd;
                h.rows = 0;
                h.pad[0] = h.pad[1] = h.pad[2] = 0;
                slots[xs].h = h;
                mbar_arrive(&xfull[xs]);
            }
        }
        // Let every copy this warp issued land before the CTA can exit.
        if (lane == 0) {
            // every query slot whose load may still be in flight (QS of them)
            const int nqs = qi < QS ? qi : QS;
            for (int i = 1; i <= nqs; ++i) drain_wait(&qfull[(qi - i) % QS], ((qi - i) / QS) & 1);
        }
        __syncwarp();
    } else if (PQ && warp == kLoaderWarp) {
        // --------------------------------------------------- loader (kPQ)
        // Each super-tile's code rows (16 bytes per token, one bulk copy per
        // tile) go to a ring slot; the decompressors turn them into rows.
        int64_t issued = 0;
        for (int t = 0;; ++t) {
            const int xs = t % kStRing;
            if (!warp_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const StHdr h = slots[xs].h;
            if (h.flags & kEnd) break;
            const bool has = lane < h.nseg;
            int r = 0, row0 = 0, col = 0;
            if (has) {
                const SegInfo si = slots[xs].seg[lane];
                r = si.r;
                row0 = si.row0;
                col = si.col;
            }
            int bytes = r * kPqM;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            __syncwarp();
            if (lane == 0) mbar_arrive(&xempty[xs]);
            const int cs = t % kCodeRing;
            if (!warp_wait(&codeempty[cs], ((t / kCodeRing) & 1) ^ 1, abort_flag, a.err, a.budget)) break;
            if (has)  // valid rows of each 8-row group of this tile (a prefix of the group)
                for (int g8 = 0; g8 < (r + 7) >> 3; ++g8)
                    gvalid[cs * (STR / 8) + (col >> 3) + g8] = static_cast<uint8_t>(min(8, r - 8 * g8));
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&codefull[cs], static_cast<uint32_t>(bytes));
            __syncwarp();
            if (has)
                bulk_load(code_ring + (cs * STR + col) * kPqM, a.pq_codes + static_cast<int64_t>(row0) * kPqM,
                          static_cast<uint32_t>(r * kPqM), &codefull[cs]);
            ++issued;
        }
        // Let every copy still in flight land before the CTA can exit.
        if (lane == 0) {
            const int64_t n = issued < kCodeRing ? issued : kCodeRing;
            for (int64_t i = 1; i <= n; ++i)
                drain_wait(&codefull[(issued - i) % kCodeRing], static_cast<uint32_t>(((issued - i) / kCodeRing) & 1));
        }
        __syncwarp();
    } else if (warp == kLoaderWarp) {
        // -------------------------------------------------------- loader
        const uint64_t pol_stream = policy_evict_first();
        const uint64_t pol_keep = policy_evict_last();
        int s = 0;
        uint32_t ph = 0;
        int64_t issued = 0;
        int sc_sts = 0;  // F8: super-tiles whose column scales were issued
        for (int t = 0;; ++t) {
            const int xs = t % kStRing;
            if (!warp_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const StHdr h = slots[xs].h;
            if (h.flags & kEnd) break;
            const bool has = lane < h.nseg;
            int n8 = 8, row0 = 0, col = 0, rr = 0;
            if (has) {
                const SegInfo si = slots[xs].seg[lane];
                rr = si.r;
                n8 = (si.r + 7) & ~7;
                row0 = si.row0;
                col = si.col;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&xempty[xs]);
            if (F8) {
                // Each tile's row scales to its columns of the record slot's
                // scale array (4-byte copies: any row alignment; 32
                // consecutive rows per warp step), completing on scfull[xs].
                // The array is free: the slot was republished only after
                // every epilogue warp had finished with its previous use.
                float* dst = sc + xs * STR;
                for (int i = 0; i < h.nseg; ++i) {
                    const int ri = __shfl_sync(0xffffffffu, rr, i);
                    const int rowi = __shfl_sync(0xffffffffu, row0, i);
                    const int coli = __shfl_sync(0xffffffffu, col, i);
                    for (int j = lane; j < ri; j += 32) cp_async4(dst + coli + j, a.t_scales + rowi + j);
                }
                cp_async_mbar_arrive(&scfull[xs]);
                ++sc_sts;
            }
            const CUtensorMap* dmap = &maps.doc[(n8 >> 3) - 1];
            bool ok = true;
            for (int kc = 0; kc < NCH; ++kc) {
                if (!warp_wait(&empty[s], ph ^ 1, abort_flag, a.err, a.budget)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>((h.rows + (QSTREAM ? a.rows_alloc : 0)) * 128));
                    if (QSTREAM) {
                        // the query (group) rows of this chunk, laid out as one
                        // chunk of the resident query region
                        uint8_t* qdst = stage_base + s * SSTRIDE + STR * 128;
                        for (int rp = 0; rp < a.reps; ++rp) {
                            if (SH) {
                                for (int g = 0; g < a.bpc; ++g)
                                    tma_load_2d(qdst + (rp * a.bpc + g) * 32 * 128, &maps.q, kc * CE,
                                                (h.q * a.group + g) * a.nq, &full[s], pol_keep);
                            } else {
                                tma_load_2d(qdst + rp * a.qbox * 128, &maps.q, kc * CE, h.q * a.nq, &full[s], pol_keep);
                            }
                        }
                    }
                }
                __syncwarp();
                if (has) tma_load_2d(stage_base + s * SSTRIDE + col * 128, dmap, kc * CE, row0, &full[s], pol_stream);
                ++issued;
                if (++s == S) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
        }
        // Let every copy still in flight land before the CTA can exit.
        if (F8) {
            cp_async_wait_all();
            __syncwarp();
            if (lane == 0) {
                const int n = sc_sts < kStRing ? sc_sts : kStRing;
                for (int i = 1; i <= n; ++i) drain_wait(&scfull[(sc_sts - i) % kStRing], ((sc_sts - i) / kStRing) & 1);
            }
        }
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
    } else if (PQ && warp > kLoaderWarp) {
        // ------------------------------------------------- decompressors
        // Thread = (row, 16-byte unit) pairs of every chunk stage: the unit
        // u of row R in chunk kc is the fp16 centroid of subspace 8 kc + u
        // for that row's code, written at unit u ^ (R % 8) -- the 128-byte
        // swizzle TMA would have produced -- so the MMA reads decompressed
        // rows exactly as it reads loaded ones.  Padding rows of a tile are
        // zero.  A quarter-warp covers one row: eight subspaces, eight
        // distinct codebook bank groups, one 128-byte store.
        const int tid = (warp - kLoaderWarp - 1) * 32 + lane;
        constexpr int kDecThreads = 32 * kSplitWarps;
        int s = 0;
        uint32_t ph = 0;
        for (int t = 0;; ++t) {
            const int xs = t % kStRing;
            if (!warp_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const StHdr h = slots[xs].h;
            if (h.flags & kEnd) break;
            const int cs = t % kCodeRing;
            if (!warp_wait_all(&codefull[cs], (t / kCodeRing) & 1, abort_flag, a.err, a.budget)) break;
            const uint8_t* crow = code_ring + cs * STR * kPqM;
            bool ok = true;
            for (int kc = 0; kc < NCH; ++kc) {
                if (!warp_wait(&empty[s], ph ^ 1, abort_flag, a.err, a.budget)) {
                    ok = false;
                    break;
                }
                uint8_t* stg = stage_base + s * SSTRIDE;
                const uint8_t* gv = gvalid + cs * (STR / 8);
                const int u = tid & 7;              // unit (subspace 8 kc + u) of every row this thread writes
                const int m = kc * 8 + u;
                // Rows tid / 8 + kRowStep j, eight per batch.  Every load of a
                // batch is unconditional (a stale code byte of a padding row
                // still indexes inside the codebook and the ring slot) and
                // issued before the batch's stores, so the three dependent
                // shared-memory loads of the eight rows overlap; padding rows
                // are then written as zeros.
                constexpr int kBatch = 8;
                constexpr int kRowStep = kDecThreads / 8;
                for (int r0 = tid >> 3; r0 < h.rows; r0 += kRowStep * kBatch) {
                    uint4 v[kBatch];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int R = min(r0 + kRowStep * j, STR - 1);
                        const uint32_t code = crow[R * kPqM + m];
                        const uint4 e = *reinterpret_cast<const uint4*>(cb + (code * kPqM + m) * 16);
                        const bool ok = (R & 7) < gv[R >> 3];
                        v[j] = ok ? e : make_uint4(0u, 0u, 0u, 0u);
                    }
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int R = r0 + kRowStep * j;
                        if (R < h.rows) *reinterpret_cast<uint4*>(stg + R * 128 + ((u ^ (R & 7)) << 4)) = v[j];
                    }
                }
                fence_proxy_async_smem();  // generic-proxy writes, read next by the tensor cores
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
                if (++s == S) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&codeempty[cs]);
                mbar_arrive(&xempty[xs]);
            }
        }
    } else if (TF && warp > kLoaderWarp) {
        // ------------------------------------------------------ splitters
        // Split each new query tile and every landed chunk stage: the MMA
        // reads an fp32 element as hi = tf32_trunc(x), so x stays in place
        // as its own hi part and lo = x - hi (exact, |lo| < 2^-10 |x|) goes
        // to the twin region; then publish the split to the MMA thread.
        // Elements are independent, so the 128-byte swizzle needs no
        // decoding: x and lo keep the same byte positions.
        const int tid = (warp - kLoaderWarp - 1) * 32 + lane;
        constexpr int kSplitThreads = 32 * kSplitWarps;
        auto split = [&](uint8_t* hi_p, uint8_t* lo_p, int bytes) {
            float4* hv = reinterpret_cast<float4*>(hi_p);
            float4* lv = reinterpret_cast<float4*>(lo_p);
            for (int v = tid; v < bytes / 16; v += kSplitThreads) {
                const float4 x = hv[v];
                lv[v] = make_float4(x.x - tf32_trunc(x.x), x.y - tf32_trunc(x.y), x.z - tf32_trunc(x.z),
                                    x.w - tf32_trunc(x.w));
            }
            fence_proxy_async_smem();  // generic-proxy writes, read next by the tensor cores
            __syncwarp();
        };
        int s = 0;
        uint32_t ph = 0;
        int qi = 0, cur_q = -1;
        for (int t = 0;; ++t) {
            const int xs = t % kStRing;
            if (!warp_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const StHdr h = slots[xs].h;
            if (h.flags & kEnd) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&xempty[xs]);
            bool ok = true;
            if (h.q != cur_q) {
                const int slot = qi % QS;
                if (!warp_wait_all(&qfull[slot], (qi / QS) & 1, abort_flag, a.err, a.budget)) break;
                split(q_base + slot * qslot_bytes, qlo_base + slot * qslot_bytes, qslot_bytes);
                if (lane == 0) mbar_arrive(&qconv[slot]);
                ++qi;
                cur_q = h.q;
            }
            for (int kc = 0; kc < NCH; ++kc) {
                if (!warp_wait_all(&full[s], ph, abort_flag, a.err, a.budget)) {
                    ok = false;
                    break;
                }
                split(stage_base + s * SSTRIDE, stage_base + s * SSTRIDE + STAGE_BYTES, h.rows * 128);
                if (lane == 0) mbar_arrive(&conv[s]);
                if (++s == S) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA
        // One thread runs this role: every wait is its own (no warp votes),
        // and descriptors advance by adding the 16-byte-unit offset of each
        // K-step to a per-stage base.
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int qi = 0, cur_q = -1, qslot = 0;
            bool any = false;
            for (int t = 0;; ++t) {
                const int xs = t % kStRing;
                if (!mbar_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
                const StHdr x = slots[xs].h;
                if (x.flags & kEnd) break;
                mbar_arrive(&xempty[xs]);
                if (!QSTREAM && x.q != cur_q) {
                    if (cur_q >= 0) mma_commit(&qempty[qslot]);
                    qslot = qi % QS;
                    if (!mbar_wait(TF ? &qconv[qslot] : &qfull[qslot], (qi / QS) & 1, abort_flag, a.err, a.budget)) break;
                    ++qi;
                    cur_q = x.q;
                }
                const int ab = t % KACC;
                if (!mbar_wait(&tempty[ab], ((t / KACC) & 1) ^ 1, abort_flag, a.err, a.budget)) break;
                tc_fence_after();
                bool ok = true;
                const uint32_t d_tmem = tbase + static_cast<uint32_t>(ab * H * STR);
                const uint64_t q_desc = desc_sw128(smem_u32(q_base + qslot * qslot_bytes));
                const uint64_t qlo_desc = desc_sw128(smem_u32(qlo_base + qslot * qslot_bytes));
                const uint32_t idesc = a.idesc | (static_cast<uint32_t>(x.n >> 3) << 17);
                for (int kc = 0; kc < NCH; ++kc) {
                    if (!mbar_wait(TF ? &conv[s] : &full[s], ph, abort_flag, a.err, a.budget)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t b_desc = desc_sw128(smem_u32(stage_base + s * SSTRIDE));
                    const uint64_t blo_desc = desc_sw128(smem_u32(stage_base + s * SSTRIDE + STAGE_BYTES));
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        const uint64_t qoff =
                            QSTREAM ? 0 : static_cast<uint64_t>(((kc * a.rows_alloc + h * 128) * 128) >> 4);
                        const uint64_t a_desc =
                            QSTREAM ? desc_sw128(smem_u32(stage_base + s * SSTRIDE + (STR + h * 128) * 128))
                                    : q_desc + qoff;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t accumulate = (kc > 0 || kk > 0) ? 1u : 0u;
                            if (TF) {  // hi.hi + hi.lo + lo.hi
                                const uint32_t dt = d_tmem + static_cast<uint32_t>(h * STR);
                                mma_tf32(dt, a_desc + 2 * kk, b_desc + 2 * kk, idesc, accumulate);
                                mma_tf32(dt, a_desc + 2 * kk, blo_desc + 2 * kk, idesc, 1u);
                                mma_tf32(dt, qlo_desc + qoff + 2 * kk, b_desc + 2 * kk, idesc, 1u);
                            } else if (F8)
                                mma_f8(d_tmem + static_cast<uint32_t>(h * STR), a_desc + 2 * kk, b_desc + 2 * kk, idesc,
                                       accumulate);
                            else
                                mma_f16(d_tmem + static_cast<uint32_t>(h * STR), a_desc + 2 * kk, b_desc + 2 * kk,
                                        idesc, accumulate);
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
                if (a.fault != kFaultHoldAccumulator || blockIdx.x != 0 || t != 0)
                    mma_commit(&tfull[ab]);
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
        // 32 qd + lane).  Row block 4 h + qd is copy (4 h + qd) / bpc of
        // block (4 h + qd) % bpc; the copies hold the same sums.  Documents
        // are dealt round-robin to the copies (by their order in the
        // records), so each warp owns whole documents: rmax[h] is the
        // running max of its row over the current document's columns, kept
        // in registers from one super-tile to the next when a document is
        // cut at a super-tile's end.  Every active warp passes every
        // super-tile and loads only the column groups of its documents.
        const int qd = warp & 3;
        const int copy = qd / a.bpc;
        const int blk = qd - copy * a.bpc;
        const bool active = copy < a.reps;
        float rmax[H];
#pragma unroll
        for (int h = 0; h < H; ++h) rmax[h] = -INFINITY;
        uint32_t ord = 0;     // documents begun (all copies)
        uint32_t mydocs = 0;  // documents this warp finished
        bool mine = false;
        bool aborted = false;
        // F8: this thread's query-token scale(s), reloaded when the query changes
        float qsc[H];
        int qsc_q = -1;
#pragma unroll
        for (int h = 0; h < H; ++h) qsc[h] = 1.f;

        // A document's score(s) from its row maxima m.  False on abort.
        auto finish_now = [&](int64_t f, int q, const float (&m)[H]) -> bool {
            if (SH) {
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const int b = (4 * h + qd) % a.bpc;
                    const int qq = q * a.group + b;
                    const float sum = warp_sum(lane < a.nq ? (F8 ? m[h] * qsc[h] : m[h]) : 0.f);
                    if (lane == 0 && qq < a.n_queries) a.out[static_cast<int64_t>(qq) * a.n_cand + f] = sum;
                }
            } else {
                const int tok = blk * 32 + lane;
                float v = 0.f;
                if (tok < a.nq) v = F8 ? m[0] * qsc[0] : m[0];
                const float sum = warp_sum(v);
                if (a.bpc == 1) {
                    if (lane == 0) a.out[f] = sum;
                } else {
                    // the copy's warps add their block sums in block order
                    const int pb = copy * 2 + (mydocs & 1);
                    const uint32_t use = mydocs >> 1;
                    if (!warp_wait(&pempty[pb], (use & 1) ^ 1, abort_flag, a.err, a.budget)) return false;
                    if (lane == 0) {
                        part[pb * 4 + blk] = sum;
                        mbar_arrive(&pfull[pb]);
                    }
                    if (blk == 0) {
                        if (!warp_wait(&pfull[pb], use & 1, abort_flag, a.err, a.budget)) return false;
                        if (lane == 0) {
                            float tot = part[pb * 4];
                            for (int bb = 1; bb < a.bpc; ++bb) tot += part[pb * 4 + bb];
                            a.out[f] = tot;
                            mbar_arrive(&pempty[pb]);
                        }
                    }
                }
            }
            ++mydocs;
            return true;
        };
        // Documents are finished in batches, off the path that releases the
        // accumulator: their 32 row maxima (times the query-token scales,
        // F8; 0 past nq) go to this warp's rows in shared memory, and every
        // kFinRows / 2 rows lane r sums row r in token order and stores the
        // score -- the same fixed order for every document, wherever it
        // sits in a batch.  With several 32-token blocks per query (nq > 32)
        // the copy's warps combine block sums at once instead (finish_now).
        const bool batched = SH || a.bpc == 1;
        float* fin_rows = reinterpret_cast<float*>(fin_base + qd * kFinWarpBytes);
        int* fin_ids = reinterpret_cast<int*>(fin_base + qd * kFinWarpBytes + kFinRows * 33 * 4);
        int nfin = 0;  // rows in use
        auto flush = [&]() {
            __syncwarp();
            if (lane < nfin) {
                float sum = 0.f;
#pragma unroll 8
                for (int i = 0; i < 32; ++i) sum += fin_rows[lane * 33 + i];
                const int doc = lane / H;
                const int f = fin_ids[2 * doc];
                const int q = fin_ids[2 * doc + 1];
                if (SH) {
                    const int b = (4 * (lane % H) + qd) % a.bpc;
                    const int qq = q * a.group + b;
                    if (qq < a.n_queries) a.out[static_cast<int64_t>(qq) * a.n_cand + f] = sum;
                } else {
                    a.out[f] = sum;
                }
            }
            __syncwarp();
            nfin = 0;
        };
        auto finish = [&](int64_t f, int q, const float (&m)[H]) -> bool {
            if (!batched) return finish_now(f, q, m);
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int tok = SH ? lane : blk * 32 + lane;
                fin_rows[(nfin + h) * 33 + lane] = tok < a.nq ? (F8 ? m[h] * qsc[h] : m[h]) : 0.f;
            }
            if (lane == 0) {
                fin_ids[2 * (nfin / H)] = static_cast<int>(f);
                fin_ids[2 * (nfin / H) + 1] = q;
            }
            nfin += H;
            if (nfin == kFinRows) flush();
            return true;
        };
        // 32 accumulator columns of this warp's lanes in each half, and
        // their 8-column sub-block maxima.  F8: each column times its
        // document row's scale; the scales, the same for every half, are
        // read from shared memory once, before the tensor-memory loads,
        // and every half's load is in flight before one wait (for bf16 /
        // fp16 the half-by-half order measured faster).
        auto load_group = [&](uint32_t taddr, const float* scales, float (&v)[H][32], float (&sb)[H][4]) {
            if constexpr (F8) {
                float4 s4[8];
                const float4* p4 = reinterpret_cast<const float4*>(scales);
#pragma unroll
                for (int i = 0; i < 8; ++i) s4[i] = p4[i];
                uint32_t r[H][32];
#pragma unroll
                for (int h = 0; h < H; ++h) tmem_ld32_issue(taddr + static_cast<uint32_t>(h * STR), r[h]);
#pragma unroll
                for (int h = 0; h < H; ++h) tmem_ld_wait32(r[h]);
#pragma unroll
                for (int h = 0; h < H; ++h) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[h][i] = __uint_as_float(r[h][i]);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        mul_f32x2(v[h][4 * i], v[h][4 * i + 1], s4[i].x, s4[i].y);
                        mul_f32x2(v[h][4 * i + 2], v[h][4 * i + 3], s4[i].z, s4[i].w);
                    }
                    sub_maxima8(v[h], sb[h]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    tmem_ld32(taddr + static_cast<uint32_t>(h * STR), v[h]);
                    sub_maxima8(v[h], sb[h]);
                }
            }
        };

        for (int t = 0; !aborted; ++t) {
            const int xs = t % kStRing;
            if (!warp_wait(&xfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const StHdr xh = slots[xs].h;
            if (xh.flags & kEnd) break;
            if (!active) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&xempty[xs]);
                continue;
            }
            const int ab = t % KACC;
            if (!warp_wait(&tfull[ab], (t / KACC) & 1, abort_flag, a.err, a.budget)) break;
            tc_fence_after();
            if (F8 && xh.q != qsc_q) {
                qsc_q = xh.q;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const int b = (4 * h + qd) % a.bpc;
                    const int qq = SH ? xh.q * a.group + b : xh.q;
                    const int tok = SH ? lane : b * 32 + lane;
                    qsc[h] = (tok < a.nq && qq < a.n_queries)
                                 ? __ldg(a.q_scales + static_cast<int64_t>(qq) * a.nq + tok)
                                 : 0.f;
                }
            }
            if (F8 && !warp_wait_all(&scfull[xs], (t / kStRing) & 1, abort_flag, a.err, a.budget)) break;
            const float* scol = sc + xs * STR;  // F8: scale of each column's document row
            float v[H][32], sb[H][4];
            int held = -1;  // the column group in v
            for (int i = 0; i < xh.nseg; ++i) {
                const SegInfo si = slots[xs].seg[i];
                if (si.flags & kFirst) {
                    mine = static_cast<int>(ord & static_cast<uint32_t>(a.reps - 1)) == copy;
                    ++ord;
                    if (mine) {
#pragma unroll
                        for (int h = 0; h < H; ++h) rmax[h] = -INFINITY;
                    }
                }
                if (!mine) continue;
                const int c_hi = si.col + si.r;
                for (int g0 = si.col & ~31; g0 < c_hi; g0 += 32) {
                    if (g0 != held) {
                        load_group(tbase + (static_cast<uint32_t>(qd * 32) << 16) +
                                       static_cast<uint32_t>(ab * H * STR + g0),
                                   scol + g0, v, sb);
                        held = g0;
                    }
                    const int lo = max(si.col - g0, 0);
                    const int hi = min(c_hi - g0, 32);
#pragma unroll
                    for (int h = 0; h < H; ++h) rmax[h] = fold_cols(rmax[h], v[h], sb[h], lo, hi);
                }
                if ((si.flags & kLast) && !finish(si.f, xh.q, rmax)) {
                    aborted = true;
                    break;
                }
            }
            if (aborted) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&tempty[ab]);
                mbar_arrive(&xempty[xs]);
            }
            if (nfin >= kFinRows / 2) flush();
        }
        if (!aborted && nfin > 0) flush();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TCOLS);
    }
}

// A launch configuration -- the kernel's counterpart of the paper's tile
// shape (Section 6.9, Table tile_ablation): rows per super-tile (documents
// per MMA run) and CTAs per SM, copies of the query blocks stacked in M
// (query tokens per epilogue warp), at most `stages` chunk stages (0: as
// many as fit), `qslots` resident query-tile slots (0: whichever gives
// more stages), or (qstream) the query streamed with each chunk stage
// instead of held resident -- the paper's dimension tiling applied to the
// query tile too.
struct Config {
    int str;
    int ctas;
    int reps;
    int stages;
    int qslots;
    int qstream;
};

// Configurations chosen by the autotuner, per device and launch shape.
struct TuneKey {
    int device, kind, h, sh, nchunks, bpc;
    bool operator<(const TuneKey& o) const {
        const int x[6] = {device, kind, h, sh, nchunks, bpc};
        const int y[6] = {o.device, o.kind, o.h, o.sh, o.nchunks, o.bpc};
        for (int i = 0; i < 6; ++i)
            if (x[i] != y[i]) return x[i] < y[i];
        return false;
    }
};
inline std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}
inline std::map<TuneKey, Config>& tune_table() {
    static std::map<TuneKey, Config> t;
    return t;
}
// Shared candidate lists: the query group size the autotuner chose, per
// device, row type, dimension chunks and queries per launch (capped at 8).
inline std::map<TuneKey, int>& group_table() {
    static std::map<TuneKey, int> t;
    return t;
}
inline TuneKey group_key(int device, int kind, int nchunks, int n_queries) {
    return TuneKey{device, kind, 0, 1, nchunks, n_queries < 8 ? n_queries : 8};
}

// The configurations an instantiation has kernels for.
template <int H, bool SH, int KIND>
inline int config_shapes(Config* out) {
    if (H == 2 || KIND == kTF32) {
        out[0] = {128, 1, 0, 0, 0, 0};
        return 1;
    }
    if (KIND == kPQ) {  // one query half
        out[0] = {256, 1, 0, 0, 0, 0};
        return 1;
    }
    out[0] = {256, 1, 0, 0, 0, 0};
    out[1] = {128, 1, 0, 0, 0, 0};
    out[2] = {128, 2, 0, 0, 0, 0};
    return 3;
}

// Plan shared memory, encode the tensor maps and launch dense_tc_kernel.
// Without a tuned or forced configuration: one CTA per SM with 256-row
// super-tiles (about two documents per MMA run) by default; per-query lists
// on the FP8 store prefer two CTAs per SM with 128-row super-tiles (two of
// every pipeline role per SM; measured faster for its 128-byte rows, slower
// for fp16/bf16); a shared group of 8 (H = 2) and split TF32 (fp32 rows,
// stages twice the size) take one CTA with 128-row super-tiles.  KIND
// selects the row type; kE4M3 ignores `dtype` (rows are E4M3 codes;
// t_scales in `a`).  The caller sets a.nchunks = ceil(d / chunk_elems(KIND)),
// and a.bpc / a.qbox: per-query ceil(nq / 32) and 32 bpc, shared mode the
// group size and 32.  `force` (the autotuner's) overrides the choice;
// TMS_ERR_UNSUPPORTED when it does not fit.
// The resolved launch configuration: every field of Config set (qslots 0:
// the query is streamed).
struct Plan {
    int str, ctas, reps, stages, qslots;
    bool operator==(const Plan& o) const {
        return str == o.str && ctas == o.ctas && reps == o.reps && stages == o.stages && qslots == o.qslots;
    }
};

// The configuration a launch of this instantiation takes: `force` if it
// fits (else TMS_ERR_UNSUPPORTED), else the autotuner's for this shape if
// one fits, else the default below.
template <int H, bool SH, int KIND>
tms_status plan_tc(const DeviceInfo& dev, const Args& a, const Config* force, Plan* out) {
    constexpr bool F8 = KIND == kE4M3;
    constexpr bool TF = KIND == kTF32;
    constexpr bool PQ = KIND == kPQ;
    (void)F8;
    // Shared-memory plan for (rows per super-tile, CTAs per SM, copies):
    // the query-slot count (2, else 1) that gives the most stages; the
    // plan fits with at least 4 chunk stages (2 with one CTA per SM).
    const int max_reps = H == 2 ? 1 : (a.bpc == 3 ? 1 : 4 / a.bpc);
    auto fits = [&](int str, int ctas, int rp, int need, int& stages, int& qslots, int cap = 0, int want_qs = 0,
                    bool stream = false) {
        if (rp < 1 || rp > max_reps) return false;
        if (stream && (TF || PQ)) return false;  // their query tiles are split / decompressed in place
        const int limit = ctas == 2 ? dev.smem_per_sm / 2 - dev.smem_reserved - 1024
                                    : std::min(kSmemLimit, dev.max_smem_optin) - 1024;
        int best = -1;
        for (int qs = stream ? 0 : 2; qs >= (stream ? 0 : 1); --qs) {
            if (!stream && want_qs && qs != want_qs) continue;
            const Layout L0 = make_layout(0, qs, a.nchunks, 32 * a.bpc * rp, str, KIND, acc_count(H, str, ctas),
                                          SH || a.bpc == 1, stream ? 128 * H : 0);
            int sts = std::min(kMaxStages, (limit - L0.total) / (L0.stage_stride + 24));
            if (cap > 0 && sts > cap) sts = cap;
            if (sts > best) {
                best = sts;
                stages = sts;
                qslots = qs;
            }
        }
        return best >= std::max(need, ctas == 2 ? 4 : 2);
    };
    // default: as many copies as fit with 4 stages, else (one CTA) with 2
    auto plan = [&](int str, int ctas, int& stages, int& qslots, int& reps) {
        for (int need = 4; need >= (ctas == 2 ? 4 : 2); need -= 2)
            for (int rp = max_reps; rp >= 1; rp /= 2)
                if (fits(str, ctas, rp, need, stages, qslots)) {
                    reps = rp;
                    return true;
                }
        return false;
    };
    int stages = 0, qslots = 1, reps = 0, str = 0, ctas = 0;
    Config tuned{0, 0, 0, 0, 0, 0};
    if (!force) {
        std::lock_guard<std::mutex> lk(tune_mutex());
        const auto it = tune_table().find(TuneKey{dev.ordinal, KIND, H, SH ? 1 : 0, a.nchunks, a.bpc});
        if (it != tune_table().end()) tuned = it->second;
    }
    const Config* want = force ? force : (tuned.ctas ? &tuned : nullptr);
    if (want) {
        if (fits(want->str, want->ctas, want->reps, 2, stages, qslots, want->stages, want->qslots, want->qstream != 0)) {
            str = want->str;
            ctas = want->ctas;
            reps = want->reps;
        } else if (force) {
            return TMS_ERR_UNSUPPORTED;
        }
    }
    if (ctas == 0) {
        if (PQ && H == 1) {
            if (plan(256, 1, stages, qslots, reps)) str = 256, ctas = 1;
        } else if (H == 2 || TF) {
            if (plan(128, 1, stages, qslots, reps)) str = 128, ctas = 1;
        } else if (!SH && a.nchunks == 1) {
            // 128-byte rows (FP8 at d <= 128, fp16 / bf16 at d <= 64): a
            // super-tile carries few bytes for its fixed pipeline costs, so
            // two CTAs per SM run two pipelines side by side
            if (plan(128, 2, stages, qslots, reps)) str = 128, ctas = 2;
            else if (plan(256, 1, stages, qslots, reps)) str = 256, ctas = 1;
            else if (plan(128, 1, stages, qslots, reps)) str = 128, ctas = 1;
        } else {
            // 256-row super-tiles unless the query tile leaves no room for
            // their stages; then 128-row ones
            if (plan(256, 1, stages, qslots, reps)) str = 256, ctas = 1;
            else if (plan(128, 1, stages, qslots, reps)) str = 128, ctas = 1;
        }
    }
    if (ctas == 0 && !TF && !PQ) {
        // the resident query tile leaves no room: stream it with every chunk
        // stage (the copies a 128-row half needs, at least two stages)
        const int sh[2][2] = {{H == 2 ? 128 : 256, 1}, {128, 1}};
        for (int i = 0; i < 2 && ctas == 0; ++i)
            for (int rp = max_reps; rp >= 1 && ctas == 0; rp /= 2)
                if (fits(sh[i][0], sh[i][1], rp, 2, stages, qslots, 0, 0, true)) {
                    str = sh[i][0];
                    ctas = sh[i][1];
                    reps = rp;
                }
    }
    if (ctas == 0) return TMS_ERR_UNSUPPORTED;
    *out = Plan{str, ctas, reps, stages, qslots};
    return TMS_OK;
}

template <int H, bool SH, int KIND>
tms_status launch_tc(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                     const void* doc_tokens, int64_t n_tokens, Args a, cudaStream_t stream,
                     const Config* force = nullptr) {
    constexpr bool F8 = KIND == kE4M3;
    constexpr bool TF = KIND == kTF32;
    constexpr bool PQ = KIND == kPQ;
    constexpr int CE = chunk_elems(KIND);
    Plan p;
    tms_status st = plan_tc<H, SH, KIND>(dev, a, force, &p);
    if (st != TMS_OK) return st;
    const int str = p.str, ctas = p.ctas, reps = p.reps, stages = p.stages, qslots = p.qslots;
    const CUtensorMapDataType tdt = F8   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                  : TF ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : dtype == TMS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const uint64_t row_bytes = static_cast<uint64_t>(d) * (F8 ? 1 : (TF ? 4 : 2));
    // With no document rows nothing is ever loaded through the document
    // maps; describe the query buffer so that they still encode.
    const void* dbase = n_tokens > 0 ? doc_tokens : queries;
    Maps maps;
    st = encode_tmap_2d(&maps.q, tdt, queries, d, static_cast<uint64_t>(n_queries) * nq, row_bytes, CE,
                        static_cast<uint32_t>(a.qbox));
    if (st != TMS_OK) return st;
    a.reps = reps;
    a.rows_alloc = 32 * a.bpc * reps;
    for (int h = 0; h < kBoxKinds; ++h) {
        if (PQ) {  // rows are decompressed in shared memory, never loaded by TMA
            maps.doc[h] = maps.q;
            continue;
        }
        st = encode_tmap_2d(&maps.doc[h], tdt, dbase, d, n_tokens, row_bytes, CE, static_cast<uint32_t>(8 * (h + 1)));
        if (st != TMS_OK) return st;
    }
    // format code 0 is f16 under kind::f16 and E4M3 under kind::f8f6f4; 2 is TF32
    a.idesc = make_idesc(128, 0, TF ? 2u : ((!F8 && dtype == TMS_BF16) ? 1u : 0u));
    a.stages = stages;
    a.qslots = qslots;
    const Layout L = make_layout(stages, qslots, a.nchunks, a.rows_alloc, str, KIND, acc_count(H, str, ctas),
                                 SH || a.bpc == 1, qslots == 0 ? 128 * H : 0);
    const int smem = L.total + 1024;
    void (*kern)(const Maps, const Args);
    if constexpr (H == 2) {
        kern = dense_tc_kernel<2, 128, 1, SH, KIND>;
    } else if constexpr (PQ) {
        kern = dense_tc_kernel<1, 256, 1, true, kPQ>;  // H == 2 took the first branch
    } else if constexpr (TF) {
        kern = dense_tc_kernel<1, 128, 1, false, kTF32>;
    } else {
        kern = str == 256 ? dense_tc_kernel<1, 256, 1, SH, KIND>
                          : (ctas == 2 ? dense_tc_kernel<1, 128, 2, SH, KIND> : dense_tc_kernel<1, 128, 1, SH, KIND>);
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return launch_status(cudaErrorInvalidValue);
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(dev.sm_count) * ctas, a.n_flat);
    return launch_status(launch_dependent(kern, dim3(static_cast<unsigned>(grid)), dim3(kernel_threads(KIND)),
                                          static_cast<size_t>(smem), stream, maps, a));
}

// Autotuner: time every configuration this instantiation has kernels for
// that fits the launch -- super-tile shape x copies x query tile (resident
// in 1 or 2 slots, or streamed) x stage cap (all that fit / 4), skipping
// plans already timed -- with 3
// timed launches after one warm-up each (CUDA events on `stream`), remember
// the fastest for the launch shape, and report how many were timed and the
// best mean time per launch.  Each launch writes the scores, so the last
// (the chosen configuration, launched again) leaves them in place.
template <int H, bool SH, int KIND>
tms_status tune_tc(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                   const void* doc_tokens, int64_t n_tokens, const Args& a, cudaStream_t stream, int* n_timed,
                   float* best_ms_out = nullptr, bool relaunch = true) {
    Config shapes[3];
    const int ns = config_shapes<H, SH, KIND>(shapes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return TMS_ERR_CUDA;
    }
    float best_ms = 0.f;
    Config best{0, 0, 0, 0, 0, 0};
    int timed = 0;
    tms_status st = TMS_OK;
    Plan seen[64];
    int nseen = 0;
    for (int i = 0; i < ns && st == TMS_OK; ++i) {
        for (int rp = 4; rp >= 1 && st == TMS_OK; rp /= 2) {
            for (int qs = 0; qs <= 2 && st == TMS_OK; ++qs) {  // 0: the query streamed
                for (int cap = 0; cap <= 4 && st == TMS_OK; cap += 4) {
                    const Config c{shapes[i].str, shapes[i].ctas, rp, cap, qs, qs == 0 ? 1 : 0};
                    Plan pl;
                    if (plan_tc<H, SH, KIND>(dev, a, &c, &pl) != TMS_OK) continue;
                    bool dup = false;
                    for (int j = 0; j < nseen; ++j) dup = dup || seen[j] == pl;
                    if (dup || nseen == 64) continue;
                    seen[nseen++] = pl;
                    tms_status r = launch_tc<H, SH, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens,
                                                          a, stream, &c);
                    if (r == TMS_ERR_UNSUPPORTED) continue;
                    if (r != TMS_OK) {
                        st = r;
                        break;
                    }
                    cudaEventRecord(e0, stream);
                    for (int k = 0; k < 3 && r == TMS_OK; ++k)
                        r = launch_tc<H, SH, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a,
                                                   stream, &c);
                    cudaEventRecord(e1, stream);
                    float ms = 0.f;
                    if (r != TMS_OK || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        st = r != TMS_OK ? r : TMS_ERR_CUDA;
                        break;
                    }
                    ++timed;
                    if (best.ctas == 0 || ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    if (st != TMS_OK) return st;
    if (best.ctas == 0) return TMS_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        tune_table()[TuneKey{dev.ordinal, KIND, H, SH ? 1 : 0, a.nchunks, a.bpc}] = best;
    }
    if (n_timed) *n_timed = timed;
    if (best_ms_out) *best_ms_out = best_ms / 3.f;
    // leave the scores of the chosen configuration in place
    return relaunch ? launch_tc<H, SH, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a, stream,
                                             &best)
                    : TMS_OK;
}

// Shared candidate lists in groups of `group` queries stacked in M (group
// 8: two 128-row halves): launch, or (tune) time the configurations of
// that group size first.  a.nchunks and the list fields are set by the
// caller.
template <int KIND>
inline tms_status shared_group_launch(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq,
                               int d, const void* doc_tokens, int64_t n_tokens, Args a, int group,
                               cudaStream_t stream, bool tune, int* n_timed, float* ms) {
    const int64_t n_groups = (n_queries + group - 1) / group;
    if (n_groups * a.n_cand >= (int64_t(1) << 31)) return TMS_ERR_UNSUPPORTED;
    a.n_flat = n_groups * a.n_cand;
    a.group = group;
    a.bpc = group;
    a.qbox = 32;
    if (tune)
        return group == 8 ? tune_tc<2, true, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a,
                                                    stream, n_timed, ms, false)
                          : tune_tc<1, true, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a,
                                                    stream, n_timed, ms, false);
    return group == 8 ? launch_tc<2, true, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a, stream)
                      : launch_tc<1, true, KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a, stream);
}

// Group sizes tried, largest first: up to 8 queries, no more than the
// launch has (rounded up to a power of two), at least 2.
inline int first_group(int n_queries) { return n_queries >= 5 ? 8 : (n_queries >= 3 ? 4 : 2); }

// Score (or tune, then score) shared candidate lists: the autotuner's group
// size for this shape if it has one and it fits, else the largest group
// whose stacked query tile fits shared memory.  Tuning times every group
// size's configurations and keeps the fastest group and configuration.
template <int KIND>
inline tms_status shared_run(const DeviceInfo& dev, const void* queries, tms_dtype dtype, int n_queries, int nq, int d,
                      const void* doc_tokens, int64_t n_tokens, const Args& a, cudaStream_t stream, bool tune,
                      int* n_configs) {
    const TuneKey gk = group_key(dev.ordinal, KIND, a.nchunks, n_queries);
    if (tune) {
        int best_group = 0, total = 0;
        float best_ms = 0.f;
        for (int group = first_group(n_queries); group >= 2; group /= 2) {
            int n = 0;
            float ms = 0.f;
            const tms_status st =
                shared_group_launch<KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a, group, stream,
                                          true, &n, &ms);
            if (st == TMS_ERR_UNSUPPORTED) continue;
            if (st != TMS_OK) return st;
            total += n;
            if (best_group == 0 || ms < best_ms) {
                best_group = group;
                best_ms = ms;
            }
        }
        if (best_group == 0) return TMS_ERR_UNSUPPORTED;
        {
            std::lock_guard<std::mutex> lk(tune_mutex());
            group_table()[gk] = best_group;
        }
        if (n_configs) *n_configs = total;
    }
    int tuned_group = 0;
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        const auto it = group_table().find(gk);
        if (it != group_table().end()) tuned_group = it->second;
    }
    if (tuned_group) {
        const tms_status st = shared_group_launch<KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens,
                                                        a, tuned_group, stream, false, nullptr, nullptr);
        if (st != TMS_ERR_UNSUPPORTED) return st;
    }
    for (int group = first_group(n_queries); group >= 2; group /= 2) {
        const tms_status st = shared_group_launch<KIND>(dev, queries, dtype, n_queries, nq, d, doc_tokens, n_tokens, a,
                                                        group, stream, false, nullptr, nullptr);
        if (st != TMS_ERR_UNSUPPORTED) return st;
    }
    return TMS_ERR_UNSUPPORTED;
}

}  // namespace dense

}  // namespace tms
