/*
 * tms.h -- C ABI of libtms, GB300 (sm_103a) late-interaction MaxSim scoring.
 *
 * The operations are those of the TileMaxSim paper (arxiv 2606.26439):
 *   - MaxSim (Section 2.1, Eq. 1):  score(Q, D) = sum_i max_j q_i . d_j,
 *     computed without materialising the Nq x Nd similarity matrix
 *     (Section 3, Algorithm 3 "V2-MQ"), with the embedding dimension
 *     tiled into chunks whose partial dot products are summed before the
 *     max (Section 3, dimension tiling; Section 6.8, Table dim_scaling);
 *   - the PQ distance table (Section 4.2, Phase 1) and fused PQ scoring
 *     through it without decompression (Section 4.2, Phase 2);
 *   - top-k selection after scoring (Section 6.8, end-to-end retrieval latency).
 *
 * Conventions shared by every entry point:
 *   - All array arguments are DEVICE pointers on the current CUDA device,
 *     unless stated otherwise.  The caller owns every buffer; the library
 *     allocates no per-call memory.
 *   - Work is enqueued on `stream` and returns without synchronising
 *     (tms_get_device_error is the one call that synchronises).
 *   - Errors are returned, never thrown.  Host-side argument checks return
 *     TMS_ERR_INVALID_ARG or TMS_ERR_UNSUPPORTED before anything is
 *     enqueued; a failed launch returns TMS_ERR_CUDA.
 *   - Data errors found on the device never fault: the affected score is
 *     written as NaN and a bit is set in the per-device error word that
 *     tms_get_device_error reads and clears.
 *   - Documents are packed: document `id` owns rows
 *     [doc_offsets[id], doc_offsets[id] + doc_lengths[id]) of a row-major
 *     [n_tokens][d] token array.  A document of length 0 scores -inf.
 *   - Candidate lists of n_queries queries are given in CSR form:
 *     query q scores cand_ids[cand_offsets[q] .. cand_offsets[q+1]),
 *     cand_offsets is non-decreasing with cand_offsets[0] = 0 and
 *     cand_offsets[n_queries] = n_cand, and the score of the candidate at
 *     flat position c is written to out_scores[c].
 *   - Scores are fp32, accumulated in fp32.  Each score is written exactly
 *     once, by one owner, in a fixed summation order: results are bitwise
 *     reproducible run to run.
 */
#ifndef TMS_H
#define TMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef enum {
    TMS_OK = 0,
    TMS_ERR_INVALID_ARG = -1, /* a size, pointer or alignment check failed  */
    TMS_ERR_UNSUPPORTED = -2, /* valid, but outside this build's limits     */
    TMS_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed        */
    TMS_ERR_DEVICE_FLAG = -5, /* tms_get_device_error found flags set       */
    TMS_ERR_TIMEOUT = -6,     /* a bounded wait ran out                      */
    TMS_ERR_BUSY = -7         /* admission refused: too many pending requests */
} tms_status;

typedef enum { TMS_F16 = 0, TMS_BF16 = 1, TMS_F32 = 2 } tms_dtype;

/* Bits of the per-device error word (see tms_get_device_error). */
#define TMS_DEVERR_BAD_ID 1u      /* candidate id outside [0, n_docs)          */
#define TMS_DEVERR_BAD_RANGE 2u   /* negative length/offset or rows past n_tokens */
#define TMS_DEVERR_TIMEOUT 4u     /* a pipeline wait exceeded its budget       */
#define TMS_DEVERR_BAD_CSR 8u     /* cand_offsets[n_queries] != n_cand, or a list
                                     with a negative start or a decreasing end */

/*
 * Dense MaxSim (Eq. 1) of n_queries queries over their candidate lists.
 *
 *   queries      [n_queries][nq][d] of `dtype`, row-major.
 *   doc_tokens   [n_tokens][d] of `dtype`, row-major, packed documents.
 *   doc_offsets  [n_docs] int64 first row;  doc_lengths [n_docs] int32.
 *   cand_ids     [n_cand] int32 document ids;  cand_offsets [n_queries+1].
 *   out_scores   [n_cand] fp32.
 *
 * Limits: 1 <= nq <= 128; 8 <= d <= 1024 with d % 8 == 0 (16-byte rows);
 * 1 <= n_queries <= 4096; n_tokens < 2^31; queries, doc_tokens and every
 * index array 16-byte aligned.  For fp16/bf16 the query tile stays in
 * shared memory when it fits beside the document stages (nq * d * 2 bytes,
 * nq rounded up to 32 and d to 64, up to 188,416) and is otherwise streamed
 * from L2 with each 128-byte dimension chunk of the documents (Section 3's
 * dimension tiling applied to the query as well), so every nq and d above
 * is supported.  fp16/bf16 run on the tensor cores
 * (tcgen05, fp32 accumulation in tensor memory); fp32 runs split TF32 on
 * the tensor cores (x = hi + lo, hi = x with its 13 low mantissa bits
 * cleared, lo the exact rest; hi.hi + hi.lo + lo.hi, FP32-level accuracy)
 * when its doubled query tile fits, else an
 * exact fp32 CUDA-core kernel (any supported nq, d).  A candidate with a bad id or row range scores NaN and sets
 * TMS_DEVERR_BAD_ID / TMS_DEVERR_BAD_RANGE.
 */
tms_status tms_score_dense(const void *queries, tms_dtype dtype, int n_queries, int nq, int d,
                           const void *doc_tokens, int64_t n_tokens,
                           const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                           const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                           float *out_scores, cudaStream_t stream);

/*
 * Autotuner for tms_score_dense (the tile-shape search of Section 6.9,
 * Table tile_ablation, over this kernel's own tile parameters): the same
 * arguments and effect (out_scores holds the scores when it returns), but
 * first every distinct tensor-core launch configuration that fits this
 * shape is timed on these inputs -- rows per super-tile (256 / 128: the
 * documents of one MMA run), CTAs per SM (1 / 2), copies of the query tile
 * (4 / 2 / 1: query tokens per epilogue warp), query-tile slots (1 / 2)
 * and chunk stages (all that fit / at most 4) -- and the fastest is
 * remembered for every later tms_score_dense call on this device with the
 * same dtype class (fp16/bf16 or fp32), ceil(nq / 32) and number of
 * dimension chunks.  Scores do not depend on the configuration (bitwise).
 * This call synchronises `stream`.  *n_configs (HOST, may be NULL)
 * receives the number of configurations timed (0 when fp32 falls back to
 * the CUDA-core kernel, which has none).
 */
tms_status tms_tune_dense(const void *queries, tms_dtype dtype, int n_queries, int nq, int d,
                          const void *doc_tokens, int64_t n_tokens,
                          const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                          const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                          float *out_scores, cudaStream_t stream, int *n_configs);

/*
 * Dense MaxSim of n_queries queries that all score ONE candidate list
 * (e.g. every query over the whole corpus, the dimension-scaling workload
 * of Section 6.8).  Same arithmetic as tms_score_dense, but queries are
 * processed in groups of up to 8 stacked in the tensor-core N dimension,
 * so each document tile is read from HBM once per group instead of once
 * per query (Theorem 1 with BQ = 32 x group).
 *
 *   cand_ids     [n_cand] int32, shared by all queries.
 *   out_scores   [n_queries][n_cand] fp32: score of query q for cand_ids[c]
 *                at out_scores[q * n_cand + c].
 *   other arguments as for tms_score_dense.
 *
 * Limits: fp16 / bf16 only, 1 <= nq <= 32, n_queries / group * n_cand
 * < 2^31.  The stacked query tile of a group stays in shared memory when
 * it fits and is otherwise streamed with each dimension chunk (groups of 8
 * at every d); tms_tune_dense_shared may choose a smaller resident group
 * instead.  fp32 or nq > 32 return TMS_ERR_UNSUPPORTED.
 */
tms_status tms_score_dense_shared(const void *queries, tms_dtype dtype, int n_queries, int nq, int d,
                                  const void *doc_tokens, int64_t n_tokens,
                                  const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                                  const int32_t *cand_ids, int64_t n_cand, float *out_scores,
                                  cudaStream_t stream);

/*
 * Autotuner for tms_score_dense_shared: as tms_tune_dense, and the query
 * group size (8 / 4 / 2 queries stacked in M, those the launch allows and
 * shared memory holds) is searched too; the fastest group and its
 * configuration are remembered for later tms_score_dense_shared calls on
 * this device with the same dimension chunks and min(n_queries, 8).
 * Scores are bitwise those of tms_score_dense_shared with any group.
 */
tms_status tms_tune_dense_shared(const void *queries, tms_dtype dtype, int n_queries, int nq, int d,
                                 const void *doc_tokens, int64_t n_tokens,
                                 const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                                 const int32_t *cand_ids, int64_t n_cand, float *out_scores,
                                 cudaStream_t stream, int *n_configs);

/*
 * FP8 E4M3 token store (an extension of the paper's fp16/bf16 scoring;
 * E4M3 = 1 sign, 4 exponent (bias 7) and 3 fraction bits, max 448, no
 * infinities).  A stored row of d codes with scale s stands for the vector
 * s * decode(codes).
 *
 * Quantize `rows` rows of x [rows][d] (dtype fp16 / bf16 / fp32, finite
 * values), one warp per row: amax = max |x[r][t]| and
 * scales[r] = amax / 448, codes[r][t] = E4M3(x[r][t] / scales[r]) rounded
 * to nearest even with saturation to +-448; both divisions are IEEE fp32.
 * A row with scale 0 gets zero codes.  Used for document rows (the store)
 * and query rows alike.
 *
 *   codes   [rows][d] uint8 (output), 16-byte aligned.
 *   scales  [rows] fp32 (output), 4-byte aligned.
 *
 * Limits: 16 <= d <= 1024, d % 16 == 0; x 16-byte aligned.
 */
tms_status tms_quantize_e4m3(const void *x, tms_dtype dtype, int64_t rows, int d, uint8_t *codes, float *scales,
                             cudaStream_t stream);

/*
 * Dense MaxSim (Eq. 1) on the FP8 store: with q_i = q_scales[q][i] *
 * decode(q_codes[q][i]) and x_j = doc_scales[row] * decode(doc_codes[row]),
 *   score = sum_i max_j q_i . x_j
 *         = sum_i q_scales[q][i] * max_j (doc_scales[row_j] * (codes_i . codes_j))
 * with the E4M3 x E4M3 products summed in fp32 on the tensor cores
 * (tcgen05 kind::f8f6f4): the row scale is applied before the max.
 *
 *   q_codes     [n_queries][nq][d] uint8;  q_scales [n_queries][nq] fp32.
 *   doc_codes   [n_tokens][d] uint8, packed like doc_tokens;
 *   doc_scales  [n_tokens] fp32.
 *   other arguments and the error behaviour as for tms_score_dense.
 *
 * Limits: 1 <= nq <= 128; 16 <= d <= 1024 with d % 16 == 0; codes,
 * doc_scales and index arrays 16-byte aligned, q_scales 4-byte aligned
 * (every supported nq and d fits shared memory).  Scales must be finite
 * and >= 0.
 */
tms_status tms_score_fp8(const uint8_t *q_codes, const float *q_scales, int n_queries, int nq, int d,
                         const uint8_t *doc_codes, const float *doc_scales, int64_t n_tokens,
                         const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                         const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                         float *out_scores, cudaStream_t stream);

/*
 * tms_score_fp8 for queries that all score ONE candidate list, stacked in
 * groups of up to 8 in the MMA N dimension (as tms_score_dense_shared):
 * out_scores [n_queries][n_cand].  Limits as tms_score_fp8 with nq <= 32
 * (nq > 32 returns TMS_ERR_UNSUPPORTED) and n_queries / group * n_cand < 2^31.
 */
tms_status tms_score_fp8_shared(const uint8_t *q_codes, const float *q_scales, int n_queries, int nq, int d,
                                const uint8_t *doc_codes, const float *doc_scales, int64_t n_tokens,
                                const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                                const int32_t *cand_ids, int64_t n_cand, float *out_scores, cudaStream_t stream);

/*
 * Autotuners for the FP8 store, as tms_tune_dense / tms_tune_dense_shared:
 * same arguments and effect as tms_score_fp8 / tms_score_fp8_shared, the
 * configurations (and, shared lists, the group size) timed first and the
 * fastest remembered for later calls of the same shape on this device.
 * These calls synchronise `stream`; *n_configs (HOST, may be NULL)
 * receives the number of configurations timed.
 */
tms_status tms_tune_fp8(const uint8_t *q_codes, const float *q_scales, int n_queries, int nq, int d,
                        const uint8_t *doc_codes, const float *doc_scales, int64_t n_tokens,
                        const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                        const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                        float *out_scores, cudaStream_t stream, int *n_configs);
tms_status tms_tune_fp8_shared(const uint8_t *q_codes, const float *q_scales, int n_queries, int nq, int d,
                               const uint8_t *doc_codes, const float *doc_scales, int64_t n_tokens,
                               const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                               const int32_t *cand_ids, int64_t n_cand, float *out_scores, cudaStream_t stream,
                               int *n_configs);

/*
 * PQ distance table (Section 4.2, Phase 1):
 *   lut[q][i][mm][kk] = sum_{t < d/m} queries[q][i][mm*(d/m) + t] * codebook[mm][kk][t]
 * computed in fp32 with fused multiply-adds in ascending t.
 *
 *   queries  [n_queries][nq][d] of qdtype;  codebook [m][k][d/m] fp32.
 *   lut      [n_queries][nq][m][k] fp32 (output).
 *
 * Limits: d % m == 0, 1 <= m <= 64, 1 <= k <= 256, 1 <= nq <= 128.
 */
tms_status tms_build_pq_lut(const void *queries, tms_dtype qdtype, int n_queries, int nq, int d,
                            const float *codebook, int m, int k, float *lut, cudaStream_t stream);

/*
 * Fused PQ MaxSim (Section 4.2, Phase 2):
 *   score = sum_i max_j sum_mm lut[q][i][mm][codes[j][mm]]
 * read straight from the uint8 codes through the table held in shared
 * memory -- no token is decompressed.
 *
 *   lut        [n_queries][nq][m][k] fp32 (from tms_build_pq_lut or any
 *              caller-built table).
 *   codes      [n_tokens][m] uint8, packed like doc_tokens.
 *   other arguments as for tms_score_dense.
 *
 * Limits: m in {4, 8, 16, 32}; 1 <= k <= 256 with m*k <= 4096; 1 <= nq <= 128;
 * codes must be < k (a larger code reads an unspecified table entry but
 * never faults).  The table is processed in chunks of 8 query tokens; the
 * chunk partial sums are added in ascending chunk order through out_scores.
 */
tms_status tms_score_pq(const float *lut, int n_queries, int nq, int m, int k,
                        const uint8_t *codes, int64_t n_tokens,
                        const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                        const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                        float *out_scores, cudaStream_t stream);

/*
 * Fused PQ MaxSim through an fp16 table: tms_score_pq with every table
 * entry rounded to the nearest fp16 (ties to even) when it is staged into
 * shared memory.  Same arguments, layouts and error behaviour as
 * tms_score_pq; the entries of one token are added in fp32 (each fp16
 * entry widened exactly), so the only departure from the fp32 table is the
 * rounding of each entry to 11 significant bits (Section 4.2 keeps the
 * table in fp32; this is a precision variant of it).  Entries beyond the
 * fp16 range (|x| > 65504) round to +-inf: use tms_score_pq for such tables.
 * The table is processed in chunks of 16 query tokens, so a 128 KB chunk
 * serves twice the query tokens of tms_score_pq and each gather returns
 * twice the entries.
 *
 * Limits: m in {16, 32} (TMS_ERR_UNSUPPORTED otherwise); the rest as for
 * tms_score_pq.
 */
tms_status tms_score_pq_f16(const float *lut, int n_queries, int nq, int m, int k,
                            const uint8_t *codes, int64_t n_tokens,
                            const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                            const int32_t *cand_ids, const int64_t *cand_offsets, int64_t n_cand,
                            float *out_scores, cudaStream_t stream);

/*
 * PQ MaxSim on the tensor cores for queries that share one candidate list
 * (e.g. every query over the whole corpus): each document tile's codes are
 * decompressed into shared memory -- token j's row is the concatenation of
 * its centroids codebook[mm][codes[j][mm]] (Section 4.1's explicit
 * decompression), each centroid rounded to the nearest fp16 -- and scored
 * by Eq. 1 with the dense pipeline (fp32 accumulation), in groups of up to
 * 8 queries per decompressed tile.  Unlike tms_score_pq nothing here
 * depends on a per-query table, so the decompression is shared by the
 * group.
 *
 *   queries      [n_queries][nq][d] fp16.
 *   codebook     [m][k][d/m] fp32;  codes [n_tokens][m] uint8, packed like
 *                doc_tokens.
 *   cand_ids     [n_cand] int32, shared by all queries;  out_scores
 *                [n_queries][n_cand], as for tms_score_dense_shared.
 *
 * Error bound against Eq. 1 on the fp32 centroids: each centroid element
 * carries a relative rounding error <= 2^-11, plus the fp32 sums.
 * Limits: qdtype TMS_F16, m = 16, d = 128 (dsub = 8), 1 <= k <= 256,
 * 1 <= nq <= 32 (TMS_ERR_UNSUPPORTED otherwise); codes must be < k (a
 * larger code reads a zero centroid); n_tokens < 2^31.
 */
tms_status tms_score_pq_tc_shared(const void *queries, tms_dtype qdtype, int n_queries, int nq, int d,
                                  const float *codebook, int m, int k, const uint8_t *codes, int64_t n_tokens,
                                  const int64_t *doc_offsets, const int32_t *doc_lengths, int64_t n_docs,
                                  const int32_t *cand_ids, int64_t n_cand, float *out_scores,
                                  cudaStream_t stream);

/*
 * Top-k per query over scores laid out like out_scores above (Section 6.8).
 *
 *   scores        [n_cand] fp32, query q's list at cand_offsets[q]..[q+1].
 *   out_scores    [n_queries][topk] fp32;  out_pos [n_queries][topk] int32:
 *                 the r-th best score and its position within the query's
 *                 candidate list (the caller maps positions to ids).
 *
 * Order: score descending; equal scores by ascending position; NaN after
 * every number (-inf included).  Lists shorter than topk are padded with
 * (-inf, -1).  Limits: 1 <= topk <= 1024, list length < 2^31.
 *
 * cand_offsets must be a valid CSR over the scores buffer: 0 <= [q] <=
 * [q+1] and every list inside it (the library cannot see the buffer's
 * length).  A negative start or a decreasing pair sets TMS_DEVERR_BAD_CSR
 * and never reads below the start of `scores`: a negative start reads the
 * list as empty, a decreasing end is clamped to its start.  An end past the
 * buffer is not detectable here.
 */
tms_status tms_topk(const float *scores, const int64_t *cand_offsets, int n_queries, int topk,
                    float *out_scores, int32_t *out_pos, cudaStream_t stream);

/*
 * tms_topk on the whole GPU: each query's list is cut into S contiguous
 * slices, one CTA selects each slice's top-k into `workspace`, and one CTA
 * per query selects the final top-k from its S x topk entries.  The result
 * is bit-identical to tms_topk (same order, same ties, same padding); only
 * the work is spread over S times more CTAs, which matters when there are
 * few queries with long lists (e.g. 16 lists of 100,000 scores).
 *
 *   n_cand         cand_offsets[n_queries] (HOST value): fixes S with
 *                  n_queries, topk and the device's SM count.
 *   workspace      DEVICE scratch of workspace_bytes bytes, 16-byte
 *                  aligned, owned by the caller; its contents on entry do
 *                  not matter and are overwritten.  Calls that may run at
 *                  the same time need separate workspaces.
 *
 * tms_topk_workspace_size gives the bytes needed on the current device
 * (n_queries * S * topk * 8; 0 when S = 1, then workspace may be NULL and
 * the call is tms_topk).  A smaller workspace returns TMS_ERR_INVALID_ARG
 * before anything is enqueued.  Other arguments and limits as tms_topk.
 */
tms_status tms_topk_workspace_size(int n_queries, int topk, int64_t n_cand, int64_t *bytes);

tms_status tms_topk_split(const float *scores, const int64_t *cand_offsets, int n_queries, int topk,
                          int64_t n_cand, float *out_scores, int32_t *out_pos, void *workspace,
                          int64_t workspace_bytes, cudaStream_t stream);

/*
 * tms_topk_split without a workspace argument, for callers that cannot
 * allocate device memory: a plugin whose host application owns every
 * device allocation through its own pool, or a serving path that must
 * make no cudaMalloc after start-up because the call can synchronise the
 * device and has no bounded latency.  The paper has no counterpart; this
 * is an interface variant of the top-k step (Section 6.8), not a new
 * operation.  Same arguments, order, ties, padding and limits as
 * tms_topk_split, and bit-identical results.
 *
 * The slice entries live in one 4 MiB array of device memory inside the
 * library (a file-scope __device__ array): every GPU that loads libtms
 * holds those 4 MiB until the process exits, and the call itself
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and remembers it;
 *     make that first call before any stream capture on the device.
 *   - Every call on a device shares the one array and it keeps the last
 *     call's contents.  Nothing in it needs clearing (each call writes
 *     every entry it reads), but calls whose work may overlap on the GPU
 *     (different streams with no ordering between them) race on it: order
 *     them on one stream, or use tms_topk_split with separate workspaces.
 *   - The entries needed are tms_topk_workspace_size's bytes
 *     (n_queries * S * topk * 8); above 4,194,304 bytes the call returns
 *     TMS_ERR_UNSUPPORTED before anything is enqueued.
 */
tms_status tms_topk_split_noalloc(const float *scores, const int64_t *cand_offsets, int n_queries, int topk,
                                  int64_t n_cand, float *out_scores, int32_t *out_pos, cudaStream_t stream);

/*
 * Serving loop: a device-resident corpus (a dense store and optionally a PQ
 * store and an FP8 copy of the dense store) and a worker thread that scores
 * requests -- one query of nq tokens
 * against its own candidate list, top-k back to the host -- with continuous
 * batching: every launch takes all pending requests that fit the batch
 * buffers, requests arriving meanwhile go into the next launch, and the
 * host side of one batch (staging, completion) overlaps the GPU work of the
 * next.  Scores come from tms_score_dense / tms_score_pq / tms_score_fp8
 * and tms_topk, whose results do not depend on the batch they run in: a
 * request's result is bitwise the same alone and in any mix.
 *
 * The config's device pointers are owned by the caller and must stay valid
 * until tms_server_destroy; the server owns its own batch buffers (device
 * and pinned host memory, allocated in tms_server_create).  Host pointers
 * passed to submit are copied before it returns.
 */
typedef struct tms_server tms_server;

typedef enum { TMS_STORE_DENSE = 0, TMS_STORE_PQ = 1, TMS_STORE_FP8 = 2 } tms_store;

typedef struct {
    /* dense store (required), as for tms_score_dense */
    const void *doc_tokens;
    tms_dtype dtype;            /* TMS_F16 or TMS_BF16 */
    int d;
    int64_t n_tokens;
    const int64_t *doc_offsets;
    const int32_t *doc_lengths;
    int64_t n_docs;
    /* PQ store (optional: pq_codes == NULL for none), as for tms_score_pq;
     * queries of PQ requests have the dense store's dtype and d */
    const uint8_t *pq_codes;
    const float *pq_codebook;   /* [pq_m][pq_k][d / pq_m] fp32 */
    int pq_m;
    int pq_k;
    int64_t pq_n_tokens;
    const int64_t *pq_offsets;
    const int32_t *pq_lengths;
    int64_t pq_n_docs;
    /* FP8 store (optional: fp8_codes == NULL for none): the dense store's
     * documents as E4M3 codes with one fp32 scale per token (as written by
     * tms_quantize_e4m3 from doc_tokens), with the dense store's ids,
     * offsets and lengths; needs d % 16 == 0.  A request to it has its
     * query quantized on the device and every candidate scored by
     * tms_score_fp8; with rescore_k > 0 its rescore_k best candidates are
     * scored again on the dense store (tms_score_dense) and the top-k is
     * taken from those fp16 scores, so the returned scores are the dense
     * store's; with rescore_k == 0 they are the FP8 scores. */
    const uint8_t *fp8_codes;   /* [n_tokens][d] */
    const float *fp8_scales;    /* [n_tokens], 16-byte aligned */
    int rescore_k;              /* 0, or topk..1024 */
    /* requests */
    int nq;                        /* query tokens per request, 1..128 */
    int topk;                      /* results per request, 1..1024 */
    int max_batch_requests;        /* requests per launch, 1..4096 (1 = no batching) */
    int64_t max_batch_candidates;  /* candidates per launch (all requests), >= 1 */
    int max_pending;               /* admitted but unfinished requests, >= 1 */
    int64_t max_pending_bytes;     /* device bytes admitted but unfinished requests may claim in the
                                      batch buffers -- query + 8 per candidate (id and score) --
                                      0 = no byte limit */
    int inject_error_batch;        /* test hook: > 0 fails that batch (1-based) on the host, 0 = off */
} tms_server_config;

typedef struct {
    uint64_t requests;     /* completed */
    uint64_t batches;      /* launches */
    uint64_t candidates;   /* scored */
    uint64_t rejected;     /* refused by admission */
    double enqueue_s;      /* host time spent staging and enqueueing batches (seconds) */
} tms_server_stats;

/* Create the server and start its worker on the current device.  Returns
 * TMS_ERR_INVALID_ARG for a bad config, TMS_ERR_CUDA if the buffers cannot
 * be allocated. */
tms_status tms_server_create(const tms_server_config *cfg, tms_server **out);

/*
 * Submit one request (HOST pointers, copied): query [nq][d] of the dense
 * store's dtype, cand_ids [n_cand] document ids of `store` (the FP8 store
 * shares the dense store's ids).  *ticket receives its handle.  Every id
 * is checked on the host against the store's document count (pq_n_docs for
 * the PQ store, n_docs otherwise): an id outside [0, count) returns
 * TMS_ERR_INVALID_ARG and nothing is admitted.  Admission:
 * TMS_ERR_BUSY when max_pending requests are unfinished or their device
 * bytes plus this one's would pass max_pending_bytes; TMS_ERR_UNSUPPORTED
 * when n_cand exceeds max_batch_candidates, the request alone exceeds
 * max_pending_bytes, or the store is absent.  Safe to call from several
 * threads, also while others wait.
 */
tms_status tms_server_submit(tms_server *s, tms_store store, const void *query, const int32_t *cand_ids,
                             int64_t n_cand, uint64_t *ticket);

/*
 * Wait (at most timeout_s seconds) for a request and take its result (HOST
 * pointers): out_scores [topk] fp32 and out_ids [topk] int32 document ids,
 * ordered as tms_topk orders them (ids -1 past the list's end);
 * *latency_s (may be NULL) receives submit-to-completion time.  Returns the
 * request's status (TMS_ERR_CUDA if its batch failed), TMS_ERR_TIMEOUT if
 * it is not done in time (it stays waitable), TMS_ERR_INVALID_ARG for an
 * unknown ticket or one whose result another waiter already took (a
 * result is handed out once).  Safe to call from several threads.
 */
tms_status tms_server_wait(tms_server *s, uint64_t ticket, double timeout_s, float *out_scores, int32_t *out_ids,
                           double *latency_s);

tms_status tms_server_get_stats(tms_server *s, tms_server_stats *out);

/* Finish every admitted request, stop the worker and free the server. */
tms_status tms_server_destroy(tms_server *s);

/*
 * Read and clear the current device's error word after `stream` drains.
 * *flags (HOST pointer) receives the TMS_DEVERR_* bits.  Returns
 * TMS_ERR_DEVICE_FLAG when any bit was set, TMS_OK otherwise.  This call
 * synchronises `stream`.
 */
tms_status tms_get_device_error(cudaStream_t stream, int *flags);

/*
 * Diagnostics: exercises the timeout path of the pipelined kernels; not
 * needed in normal use.  Every wait between the roles of those kernels
 * (tms_score_dense on the tensor cores, the FP8 and shared-list calls,
 * tms_score_pq_tc_shared, and the staged fused-PQ kernel) is bounded by a
 * budget of SM clock cycles (default 2e9, about one second at 2 GHz); when
 * it runs out the kernel sets TMS_DEVERR_TIMEOUT, lets every copy and MMA
 * it issued land, frees its tensor memory and returns, so the context stays
 * usable.  tms_debug_set changes, for launches prepared after it returns
 * (process-wide):
 *   wait_budget_cycles  the budget (0 restores the default; drain waits at
 *                       exit always keep the default);
 *   fault               0, or TMS_FAULT_HOLD_ACCUMULATOR: in the tensor-core
 *                       dense kernels, CTA 0 never signals its first
 *                       accumulator as ready, so that CTA's epilogue wait
 *                       runs out of budget (a flag nothing sets).
 * Returns TMS_ERR_INVALID_ARG for a negative budget or an unknown fault.
 */
#define TMS_FAULT_HOLD_ACCUMULATOR 1
tms_status tms_debug_set(int64_t wait_budget_cycles, int fault);

/* Static English text for a status code. */
const char *tms_status_string(tms_status s);

/* Library ABI version (major * 100 + minor). */
int tms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TMS_H */
