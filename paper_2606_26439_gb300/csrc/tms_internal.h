// tms_internal.h -- host-side helpers shared by the libtms translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

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

// Launch with programmatic stream serialization: the kernel may be
// scheduled while the previous kernel of the stream is finishing (once all
// of its CTAs have issued griddepcontrol.launch_dependents or exited), and
// runs only its own set-up (barriers, tensor memory, descriptor prefetch)
// before griddepcontrol.wait, which returns when that kernel has completed
// and its memory is visible.  Every kernel launched this way waits before
// its first global-memory access.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                             Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace tms
