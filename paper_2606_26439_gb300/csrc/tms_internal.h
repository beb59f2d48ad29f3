// tms_internal.h -- host-side helpers shared by the libtms translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tms.h"

namespace tms {

// Per-device facts and state, created lazily on first use of a device.
struct DeviceInfo {
    int ordinal;
    int sm_count;
    int max_smem_optin;       // largest dynamic shared memory a CTA may request
    int smem_per_sm;          // shared memory of one SM
    int smem_reserved;        // shared memory the system reserves per CTA
    unsigned int* err;        // device address of the error word (file-scope __device__)
};

// Info for the current device (cached per ordinal).  Returns TMS_ERR_CUDA
// when the runtime cannot report it.
tms_status current_device(DeviceInfo* out);

// Encode a 2-D row-major tensor map: `rows` rows of `cols` elements of
// `elem_bytes` each, row pitch `row_bytes`, box of box_cols x box_rows,
// 128-byte swizzle, zero fill outside the tensor.
tms_status encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t cols,
                          uint64_t rows, uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows);


// Diagnostics set by tms_debug_set, read when a launch is prepared: the
// bound of every pipeline wait in SM cycles (0 = the kernels' default) and
// the fault to inject (0 = none).
long long debug_wait_budget();
int debug_fault();

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline tms_status launch_status(cudaError_t e) {
    if (e == cudaSuccess) return TMS_OK;
    (void)cudaGetLastError();  // clear the sticky-free launch error
    return TMS_ERR_CUDA;
}

}  // namespace tms
