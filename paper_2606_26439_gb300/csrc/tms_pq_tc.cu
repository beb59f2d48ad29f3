// tms_pq_tc.cu -- PQ MaxSim scored on the tensor cores: the uint8 codes are
// decompressed in shared memory and the dense kernel's MMA pipeline scores
// the rebuilt rows.
//
// Section 4.1 scores PQ documents by decompressing every token and taking
// Eq. 1 on the result; Section 4.2 avoids the decompression with a distance
// table per query.  Here the decompression is done where it costs no HBM
// traffic -- into the shared-memory stages the MMA reads -- and it is
// query-independent, so in the shared-list schedule one decompressed tile
// serves a whole group of queries stacked in the MMA's M dimension.  Rows
// are fp16: each centroid is rounded to the nearest fp16 (ties to even)
// once, when the codebook is copied into shared memory; products and sums
// are fp32 as in the dense path.
#include "tms_dense_tc.cuh"

extern "C" tms_status tms_score_pq_tc_shared(const void* queries, tms_dtype qdtype, int n_queries, int nq, int d,
                                             const float* codebook, int m, int k, const uint8_t* codes,
                                             int64_t n_tokens, const int64_t* doc_offsets,
                                             const int32_t* doc_lengths, int64_t n_docs, const int32_t* cand_ids,
                                             int64_t n_cand, float* out_scores, cudaStream_t stream) {
    using namespace tms;
    if (qdtype != TMS_F16 && qdtype != TMS_BF16 && qdtype != TMS_F32) return TMS_ERR_INVALID_ARG;
    if (n_queries < 1 || n_queries > 4096 || nq < 1 || nq > 128 || d < 1 || m < 1 || m > 64 || k < 1 || k > 256 ||
        d % m != 0)
        return TMS_ERR_INVALID_ARG;
    if (qdtype != TMS_F16 || nq > 32 || m != dense::kPqM || d != 8 * dense::kPqM) return TMS_ERR_UNSUPPORTED;
    if (n_tokens < 0 || n_tokens >= (int64_t(1) << 31) || n_docs < 0 || n_cand < 0) return TMS_ERR_INVALID_ARG;
    if (!queries || !codebook || !aligned16(queries) || !aligned16(codebook)) return TMS_ERR_INVALID_ARG;
    if (n_cand > 0 && (!cand_ids || !out_scores || !aligned16(cand_ids) || !aligned16(out_scores)))
        return TMS_ERR_INVALID_ARG;
    if (n_docs > 0 && (!doc_offsets || !doc_lengths || !aligned16(doc_offsets) || !aligned16(doc_lengths)))
        return TMS_ERR_INVALID_ARG;
    if (n_tokens > 0 && (!codes || !aligned16(codes))) return TMS_ERR_INVALID_ARG;
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
    a.nchunks = d / dense::chunk_elems(dense::kPQ);
    a.pq_codes = codes;
    a.pq_codebook = codebook;
    a.pq_k = k;
    // Queries per group (32 MMA rows each): 8 (two 128-row halves of the
    // tile, one decompressed super-tile serving both), 4 or 2; a smaller
    // group when the larger one does not fit shared memory.
    for (int group = n_queries >= 5 ? 8 : (n_queries >= 3 ? 4 : 2); group >= 2; group /= 2) {
        const int64_t n_groups = (n_queries + group - 1) / group;
        if (n_groups * n_cand >= (int64_t(1) << 31)) return TMS_ERR_UNSUPPORTED;
        a.n_flat = n_groups * n_cand;
        a.group = group;
        a.bpc = group;
        a.qbox = 32;
        st = group == 8
                 ? dense::launch_tc<2, true, dense::kPQ>(dev, queries, TMS_F16, n_queries, nq, d, codes, n_tokens, a,
                                                         stream)
                 : dense::launch_tc<1, true, dense::kPQ>(dev, queries, TMS_F16, n_queries, nq, d, codes, n_tokens, a,
                                                         stream);
        if (st != TMS_ERR_UNSUPPORTED) return st;
    }
    return TMS_ERR_UNSUPPORTED;
}
