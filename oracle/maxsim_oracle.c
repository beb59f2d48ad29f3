/*
 * maxsim_oracle.c -- FP64 CPU oracle for late-interaction MaxSim scoring.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may link, load or call this file.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * It is a plain, slow, obviously correct restatement of the definitions in
 * the TileMaxSim paper (arxiv 2606.26439).  Every floating-point value is
 * read exactly as stored (fp16 / bf16 / fp32 / fp64 decoded bit-exactly to
 * double) and every sum, product and max is taken in IEEE double precision,
 * in the plain loop order of the definition.  There is no blocking, fusion
 * or reordering.  OpenMP only spreads independent candidates over threads;
 * each candidate's arithmetic is sequential and therefore the result does
 * not depend on the thread count.
 *
 * Definitions restated here:
 *   - MaxSim (Section 2.1, Eq. 1):
 *         score(Q, D) = sum_{i<Nq} max_{j<Nd} q_i . d_j
 *   - PQ reconstruction (Section 4.1): d^_j is the concatenation over the
 *     M subspaces of the centroid C[m][code_{j,m}] (dsub = d / M values each).
 *   - PQ distance table (Section 4.2):
 *         T[i][m][k] = q_i[m*dsub : (m+1)*dsub] . C[m][k]
 *     and the approximate similarity  q_i . d^_j = sum_m T[i][m][code_{j,m}].
 *   - Top-k after scoring (Section 6.8, end-to-end retrieval latency): the k largest
 *     scores of a query's candidate list.
 *   - A per-token scaled FP8 store (not part of the paper, which scores
 *     fp16 inputs with fp32 accumulation, Section 6.1): each stored row is
 *     E4M3 codes with one fp32 scale, the vector it stands for is
 *     scale * decode(codes), and MaxSim is Eq. 1 on those vectors -- the
 *     row scale multiplies each similarity before the max.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Inner product, not cosine: Eq. 1 is a raw dot product; normalisation is
 *     the input generator's job.
 *   - Variable-length documents are stored packed: document id has tokens
 *     rows [offsets[id], offsets[id] + lengths[id]) of a [n_tokens][d] array.
 *   - An empty document (length 0) scores -inf: the max over the empty set
 *     is -inf, and -inf survives the sum.
 *   - A candidate whose id is outside [0, n_docs), or whose row range is
 *     negative or runs past n_tokens, is a data error and scores NaN.
 *   - NaN inside a similarity is skipped by the max (the comparison
 *     "dot > running max" is false for NaN), matching IEEE maxNum.
 *   - Top-k order: score descending, ties broken by the lower candidate
 *     position; NaN sorts after every number; when the list is shorter than
 *     k the tail is padded with (-inf, -1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { TMSO_F16 = 0, TMSO_BF16 = 1, TMSO_F32 = 2, TMSO_F64 = 3, TMSO_E4M3 = 4 };

/* ---- exact decoding of stored element types ------------------------- */

/* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction
 * bits.  Exponent 0 encodes zero and subnormals (fraction * 2^-24);
 * exponent 31 encodes infinities and NaNs. */
double tmso_f16_to_f64(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int expo = (h >> 10) & 0x1f;
    int frac = h & 0x3ff;
    double v;
    if (expo == 0)
        v = ldexp((double)frac, -24);
    else if (expo == 31)
        v = frac ? NAN : INFINITY;
    else
        v = ldexp((double)(frac | 0x400), expo - 25);
    return sign ? -v : v;
}

/* bfloat16 is by definition the upper 16 bits of an IEEE binary32. */
double tmso_bf16_to_f64(uint16_t h)
{
    uint32_t bits = (uint32_t)h << 16;
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

/* OCP FP8 E4M3 ("e4m3fn"): 1 sign bit, 4 exponent bits (bias 7), 3 fraction
 * bits.  Exponent 0 encodes zero and subnormals (fraction * 2^-9); there
 * are no infinities, and S.1111.111 is NaN (max finite 448). */
double tmso_e4m3_to_f64(uint8_t b)
{
    int sign = (b >> 7) & 1;
    int expo = (b >> 3) & 0xf;
    int frac = b & 0x7;
    double v;
    if (expo == 15 && frac == 7)
        v = NAN;
    else if (expo == 0)
        v = ldexp((double)frac, -9);
    else
        v = ldexp((double)(frac | 0x8), expo - 10);
    return sign ? -v : v;
}

static double load_elem(const void *base, int dtype, int64_t idx)
{
    switch (dtype) {
    case TMSO_E4M3:
        return tmso_e4m3_to_f64(((const uint8_t *)base)[idx]);
    case TMSO_F16:
        return tmso_f16_to_f64(((const uint16_t *)base)[idx]);
    case TMSO_BF16:
        return tmso_bf16_to_f64(((const uint16_t *)base)[idx]);
    case TMSO_F32:
        return (double)((const float *)base)[idx];
    default:
        return ((const double *)base)[idx];
    }
}

/* Decode n consecutive stored elements starting at element idx. */
static void load_row(const void *base, int dtype, int64_t idx, int n, double *dst)
{
    for (int t = 0; t < n; ++t)
        dst[t] = load_elem(base, dtype, idx + t);
}

static int dtype_ok(int dt) { return dt >= TMSO_F16 && dt <= TMSO_E4M3; }

/* ---- FP8 E4M3 quantization ------------------------------------------ */

/* Magnitude code (0..126) of the finite E4M3 value nearest to a >= 0: the
 * nearest of the 127 finite non-negative values by exhaustive search, an
 * exact tie going to the even code (round to nearest, ties to even).
 * Anything above 448 is nearest to 448 -- the saturating conversion. */
static int e4m3_nearest_code(double a)
{
    int best = 0;
    double best_err = fabs(a);
    for (int c = 1; c <= 126; ++c) {
        double err = fabs(tmso_e4m3_to_f64((uint8_t)c) - a);
        if (err < best_err || (err == best_err && (c & 1) == 0)) {
            best = c;
            best_err = err;
        }
    }
    return best;
}

/* E4M3 code of the fp32 value v: sign bit of v, magnitude by nearest-even. */
uint8_t tmso_e4m3_encode(float v)
{
    int sign = signbit(v) ? 1 : 0;
    return (uint8_t)((sign << 7) | e4m3_nearest_code(fabs((double)v)));
}

/*
 * Per-row FP8 E4M3 quantization with one fp32 scale per row.  For row r,
 * in fp32 arithmetic: amax = max_t |x[r][t]|, s = amax / 448 (the largest
 * finite E4M3 magnitude) and code[r][t] = encode(x[r][t] / s), both
 * divisions IEEE fp32.  A row whose s is 0 gets all-zero codes.  Inputs are
 * finite fp16 / bf16 / fp32 values.
 */
int tmso_quantize_e4m3(const void *x, int dtype, int64_t rows, int d, uint8_t *codes, float *scales)
{
    if (rows < 0 || d <= 0 || (dtype != TMSO_F16 && dtype != TMSO_BF16 && dtype != TMSO_F32))
        return -1;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        float amax = 0.0f;
        for (int t = 0; t < d; ++t) {
            float v = (float)load_elem(x, dtype, r * d + t);
            if (fabsf(v) > amax)
                amax = fabsf(v);
        }
        float s = amax / 448.0f;
        scales[r] = s;
        for (int t = 0; t < d; ++t) {
            if (s == 0.0f) {
                codes[r * d + t] = 0;
            } else {
                float v = (float)load_elem(x, dtype, r * d + t) / s;
                codes[r * d + t] = tmso_e4m3_encode(v);
            }
        }
    }
    return 0;
}

int tmso_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void tmso_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Row range of document `id`, or -1 when the candidate is a data error. */
static int doc_range(int64_t id, const int64_t *offsets, const int32_t *lengths,
                     int64_t n_docs, int64_t n_tokens, int64_t *off, int64_t *len)
{
    if (id < 0 || id >= n_docs)
        return -1;
    *off = offsets[id];
    *len = lengths[id];
    if (*len < 0 || *off < 0 || *off + *len > n_tokens)
        return -1;
    return 0;
}

/* MaxSim of one query Q[nq][d] against one document X[len][d] (Eq. 1),
 * both already decoded to double. */
static double maxsim_one(const double *Q, int nq, int d, const double *X, int64_t len)
{
    double score = 0.0;
    for (int i = 0; i < nq; ++i) {
        double best = -INFINITY;
        for (int64_t j = 0; j < len; ++j) {
            double dot = 0.0;
            for (int t = 0; t < d; ++t)
                dot += Q[(int64_t)i * d + t] * X[j * d + t];
            if (dot > best)
                best = dot;
        }
        score += best;
    }
    return score;
}

/*
 * Dense MaxSim of one query over a candidate list (Eq. 1).
 *   queries  [nq][d] of qdtype
 *   tokens   [n_tokens][d] of tdtype, packed documents
 *   offsets  [n_docs] first row of each document, lengths [n_docs]
 *   cand_ids [n_cand] document ids to score
 *   out      [n_cand] scores in double
 * Returns 0, or -1 on invalid arguments.
 */
int tmso_dense_scores(const void *queries, int qdtype, int nq, int d,
                      const void *tokens, int tdtype, int64_t n_tokens,
                      const int64_t *offsets, const int32_t *lengths, int64_t n_docs,
                      const int32_t *cand_ids, int64_t n_cand, double *out)
{
    if (nq <= 0 || d <= 0 || n_cand < 0 || !dtype_ok(qdtype) || !dtype_ok(tdtype))
        return -1;
    double *Q = (double *)malloc(sizeof(double) * (size_t)nq * (size_t)d);
    if (!Q)
        return -1;
    for (int i = 0; i < nq; ++i)
        load_row(queries, qdtype, (int64_t)i * d, d, Q + (int64_t)i * d);

    int failed = 0;
#pragma omp parallel
    {
        double *X = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < n_cand; ++c) {
            int64_t off, len;
            if (doc_range(cand_ids[c], offsets, lengths, n_docs, n_tokens, &off, &len)) {
                out[c] = NAN;
                continue;
            }
            if (len > cap) {
                free(X);
                cap = len;
                X = (double *)malloc(sizeof(double) * (size_t)len * (size_t)d);
                if (!X) {
#pragma omp atomic write
                    failed = 1;
                    cap = 0;
                    out[c] = NAN;
                    continue;
                }
            }
            for (int64_t j = 0; j < len; ++j)
                load_row(tokens, tdtype, (off + j) * d, d, X + j * d);
            out[c] = maxsim_one(Q, nq, d, X, len);
        }
        free(X);
    }
    free(Q);
    return failed ? -1 : 0;
}

/*
 * Dense MaxSim (Eq. 1) on row-scaled stored values: the vectors scored are
 * q_i = q_scales[i] * Q[i][:] and d_j = t_scales[row] * X[row][:] (a NULL
 * scale array means 1).  This is the definition of a per-token scaled
 * store (e.g. FP8 E4M3 codes with an fp32 scale per token): dequantize,
 * then Eq. 1.
 */
int tmso_dense_scores_scaled(const void *queries, int qdtype, const float *q_scales, int nq, int d,
                             const void *tokens, int tdtype, const float *t_scales, int64_t n_tokens,
                             const int64_t *offsets, const int32_t *lengths, int64_t n_docs,
                             const int32_t *cand_ids, int64_t n_cand, double *out)
{
    if (nq <= 0 || d <= 0 || n_cand < 0 || !dtype_ok(qdtype) || !dtype_ok(tdtype))
        return -1;
    double *Q = (double *)malloc(sizeof(double) * (size_t)nq * (size_t)d);
    if (!Q)
        return -1;
    for (int i = 0; i < nq; ++i) {
        load_row(queries, qdtype, (int64_t)i * d, d, Q + (int64_t)i * d);
        double sc = q_scales ? (double)q_scales[i] : 1.0;
        for (int t = 0; t < d; ++t)
            Q[(int64_t)i * d + t] *= sc;
    }
    int failed = 0;
#pragma omp parallel
    {
        double *X = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < n_cand; ++c) {
            int64_t off, len;
            if (doc_range(cand_ids[c], offsets, lengths, n_docs, n_tokens, &off, &len)) {
                out[c] = NAN;
                continue;
            }
            if (len > cap) {
                free(X);
                cap = len;
                X = (double *)malloc(sizeof(double) * (size_t)len * (size_t)d);
                if (!X) {
#pragma omp atomic write
                    failed = 1;
                    cap = 0;
                    out[c] = NAN;
                    continue;
                }
            }
            for (int64_t j = 0; j < len; ++j) {
                load_row(tokens, tdtype, (off + j) * d, d, X + j * d);
                double sc = t_scales ? (double)t_scales[off + j] : 1.0;
                for (int t = 0; t < d; ++t)
                    X[j * d + t] *= sc;
            }
            out[c] = maxsim_one(Q, nq, d, X, len);
        }
        free(X);
    }
    free(Q);
    return failed ? -1 : 0;
}

/*
 * PQ MaxSim by explicit decompress-then-dot (Section 4.1): every document
 * token is rebuilt as the concatenation of its M centroids (fp32 codebook
 * values read exactly), then scored with Eq. 1.
 *   codebook [M][K][dsub] fp32, dsub = d / M;  codes [n_tokens][M] uint8.
 * A code >= K is a data error and makes the candidate's score NaN.
 */
int tmso_pq_decompress_scores(const void *queries, int qdtype, int nq, int d,
                              const float *codebook, int M, int K,
                              const uint8_t *codes, int64_t n_tokens,
                              const int64_t *offsets, const int32_t *lengths, int64_t n_docs,
                              const int32_t *cand_ids, int64_t n_cand, double *out)
{
    if (nq <= 0 || d <= 0 || M <= 0 || K <= 0 || d % M != 0 || n_cand < 0 || !dtype_ok(qdtype))
        return -1;
    const int dsub = d / M;
    double *Q = (double *)malloc(sizeof(double) * (size_t)nq * (size_t)d);
    if (!Q)
        return -1;
    for (int i = 0; i < nq; ++i)
        load_row(queries, qdtype, (int64_t)i * d, d, Q + (int64_t)i * d);

    int failed = 0;
#pragma omp parallel
    {
        double *X = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < n_cand; ++c) {
            int64_t off, len;
            if (doc_range(cand_ids[c], offsets, lengths, n_docs, n_tokens, &off, &len)) {
                out[c] = NAN;
                continue;
            }
            if (len > cap) {
                free(X);
                cap = len;
                X = (double *)malloc(sizeof(double) * (size_t)len * (size_t)d);
                if (!X) {
#pragma omp atomic write
                    failed = 1;
                    cap = 0;
                    out[c] = NAN;
                    continue;
                }
            }
            int bad = 0;
            for (int64_t j = 0; j < len && !bad; ++j) {
                for (int m = 0; m < M; ++m) {
                    int code = codes[(off + j) * M + m];
                    if (code >= K) {
                        bad = 1;
                        break;
                    }
                    const float *cent = codebook + ((int64_t)m * K + code) * dsub;
                    for (int t = 0; t < dsub; ++t)
                        X[j * d + m * dsub + t] = (double)cent[t];
                }
            }
            out[c] = bad ? NAN : maxsim_one(Q, nq, d, X, len);
        }
        free(X);
    }
    free(Q);
    return failed ? -1 : 0;
}

/*
 * PQ distance table in double (Section 4.2):
 *   lut[i][m][k] = sum_{t<dsub} q_i[m*dsub + t] * C[m][k][t].
 */
int tmso_pq_lut(const void *queries, int qdtype, int nq, int d,
                const float *codebook, int M, int K, double *lut)
{
    if (nq <= 0 || d <= 0 || M <= 0 || K <= 0 || d % M != 0 || !dtype_ok(qdtype))
        return -1;
    const int dsub = d / M;
    for (int i = 0; i < nq; ++i)
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < K; ++k) {
                double acc = 0.0;
                for (int t = 0; t < dsub; ++t)
                    acc += load_elem(queries, qdtype, (int64_t)i * d + m * dsub + t) *
                           (double)codebook[((int64_t)m * K + k) * dsub + t];
                lut[((int64_t)i * M + m) * K + k] = acc;
            }
    return 0;
}

/*
 * PQ MaxSim through a distance table (Section 4.2, Phase 2):
 *   score = sum_i max_j sum_m lut[i][m][code_{j,m}]
 * with lut given as [nq][M][K] of ltype (fp16, fp32 or fp64), read exactly
 * (an fp16 table is the fp32 table of Section 4.2 rounded entry by entry;
 * the sums stay in double).
 */
int tmso_pq_lut_scores(const void *lut, int ltype, int nq, int M, int K,
                       const uint8_t *codes, int64_t n_tokens,
                       const int64_t *offsets, const int32_t *lengths, int64_t n_docs,
                       const int32_t *cand_ids, int64_t n_cand, double *out)
{
    if (nq <= 0 || M <= 0 || K <= 0 || n_cand < 0 ||
        (ltype != TMSO_F16 && ltype != TMSO_F32 && ltype != TMSO_F64))
        return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < n_cand; ++c) {
        int64_t off, len;
        if (doc_range(cand_ids[c], offsets, lengths, n_docs, n_tokens, &off, &len)) {
            out[c] = NAN;
            continue;
        }
        int bad = 0;
        for (int64_t j = 0; j < len && !bad; ++j)
            for (int m = 0; m < M; ++m)
                if (codes[(off + j) * M + m] >= K)
                    bad = 1;
        if (bad) {
            out[c] = NAN;
            continue;
        }
        double score = 0.0;
        for (int i = 0; i < nq; ++i) {
            double best = -INFINITY;
            for (int64_t j = 0; j < len; ++j) {
                double s = 0.0;
                for (int m = 0; m < M; ++m)
                    s += load_elem(lut, ltype,
                                   ((int64_t)i * M + m) * K + codes[(off + j) * M + m]);
                if (s > best)
                    best = s;
            }
            score += best;
        }
        out[c] = score;
    }
    return 0;
}

/* ---- top-k ------------------------------------------------------------ */

typedef struct {
    double score;
    int64_t pos;
} tmso_entry;

/* Order: larger score first; NaN after every number; equal scores (and
 * NaN vs NaN) by ascending position. */
static int entry_cmp(const void *pa, const void *pb)
{
    const tmso_entry *a = (const tmso_entry *)pa, *b = (const tmso_entry *)pb;
    int an = isnan(a->score), bn = isnan(b->score);
    if (an != bn)
        return an ? 1 : -1;
    if (!an && a->score != b->score)
        return a->score > b->score ? -1 : 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

/*
 * Top-k of one score list: out_scores[r], out_pos[r] for r < k hold the
 * r-th entry in the order above; entries past n are (-inf, -1).
 */
int tmso_topk(const double *scores, int64_t n, int k, double *out_scores, int64_t *out_pos)
{
    if (n < 0 || k < 0)
        return -1;
    tmso_entry *e = (tmso_entry *)malloc(sizeof(tmso_entry) * (size_t)(n > 0 ? n : 1));
    if (!e)
        return -1;
    for (int64_t c = 0; c < n; ++c) {
        e[c].score = scores[c];
        e[c].pos = c;
    }
    qsort(e, (size_t)n, sizeof(tmso_entry), entry_cmp);
    for (int r = 0; r < k; ++r) {
        if (r < n) {
            out_scores[r] = e[r].score;
            out_pos[r] = e[r].pos;
        } else {
            out_scores[r] = -INFINITY;
            out_pos[r] = -1;
        }
    }
    free(e);
    return 0;
}
