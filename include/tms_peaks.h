/*
 * tms_peaks.h -- measured ceilings for the roofline figures of libtms.
 *
 * The scoring kernels are bound by a memory stream, not by arithmetic: the
 * dense and FP8 kernels by HBM reads (Section 3.4, Theorem 1: every
 * embedding is read once), the fused PQ kernels by shared-memory loads of
 * the distance table (Section 4.2, Phase 2: one table entry per subspace,
 * query token and document token).  These two calls measure those ceilings
 * on the current device with plain streams of the same access, so the
 * kernels' achieved bandwidth can be stated as a fraction of a measured
 * peak.  Both synchronise `stream` and return TMS_ERR_INVALID_ARG for bad
 * arguments, TMS_ERR_CUDA when a launch or an event fails.
 */
#ifndef TMS_PEAKS_H
#define TMS_PEAKS_H

#include <stdint.h>

#include "tms.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Shared-memory load bandwidth: one 1024-thread CTA per SM, each thread
 * issuing iters x 8 conflict-free 128-bit ld.shared (a warp instruction
 * reads 512 consecutive bytes: four wavefronts), timed with events over
 * three launches after a warm-up.  *gbs (HOST) receives bytes loaded per
 * second, in GB/s, summed over all SMs.  Limits: 1 <= iters <= 2^24.
 */
tms_status tms_peak_shared_load(int iters, cudaStream_t stream, double *gbs);

/*
 * HBM read bandwidth: a grid-stride stream of 128-bit loads that bypass L1
 * over the caller's device buffer `buf` of `bytes` bytes (16-byte aligned,
 * a multiple of 16; pass more than the L2 size, e.g. >= 1 GB), timed with
 * events over `reps` passes after one warm-up pass.  *gbs (HOST) receives
 * bytes read per second in GB/s.  Limits: 1 <= reps <= 1000.
 */
tms_status tms_peak_hbm_read(const void *buf, int64_t bytes, int reps, cudaStream_t stream, double *gbs);

#ifdef __cplusplus
}
#endif

#endif /* TMS_PEAKS_H */
