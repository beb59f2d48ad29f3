// tms_api.cu -- status strings, the device error word and per-device state.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "tms_internal.h"

// One error word per device (each device that loads the library gets its
// own copy of this module).  Kernels receive its address as a plain
// pointer and OR TMS_DEVERR_* bits into it; tms_get_device_error reads
// and clears it.
__device__ unsigned int g_tms_error_word = 0;

namespace tms {

namespace {
std::atomic<long long> g_debug_budget{0};
std::atomic<int> g_debug_fault{0};
}  // namespace

long long debug_wait_budget() { return g_debug_budget.load(std::memory_order_relaxed); }
int debug_fault() { return g_debug_fault.load(std::memory_order_relaxed); }

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
bool g_have[kMaxDevices] = {};
DeviceInfo g_info[kMaxDevices];
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};
}  // namespace

tms_status current_device(DeviceInfo* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TMS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_have[dev]) {
        DeviceInfo d{};
        d.ordinal = dev;
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return TMS_ERR_CUDA;
        }
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tms_error_word) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return TMS_ERR_CUDA;
        }
        d.err = static_cast<unsigned int*>(p);
        g_info[dev] = d;
        g_have[dev] = true;
    }
    *out = g_info[dev];
    return TMS_OK;
}

namespace {
bool load_encoder() {
    if (g_encode.load(std::memory_order_acquire) != nullptr) return true;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_encode.load(std::memory_order_relaxed) == nullptr) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || fn == nullptr) {
            (void)cudaGetLastError();
            return false;
        }
        g_encode.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn), std::memory_order_release);
    }
    return true;
}

// A tensor map holds only an address, a shape, strides and a box, so equal
// arguments always encode to the same map: each host thread remembers its
// last kTmapCache encodings (round-robin replacement).
struct TmapKey {
    CUtensorMapDataType dtype;
    const void* base;
    uint64_t cols, rows, row_bytes;
    uint32_t box_cols, box_rows;
    bool operator==(const TmapKey& o) const {
        return dtype == o.dtype && base == o.base && cols == o.cols && rows == o.rows && row_bytes == o.row_bytes &&
               box_cols == o.box_cols && box_rows == o.box_rows;
    }
};
constexpr int kTmapCache = 32;
struct TmapCache {
    TmapKey key[kTmapCache];
    CUtensorMap map[kTmapCache];
    int used = 0, next = 0;
};
thread_local TmapCache t_tmaps;
}  // namespace

tms_status encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t cols,
                          uint64_t rows, uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows) {
    if (!load_encoder()) return TMS_ERR_CUDA;
    const TmapKey key{dtype, base, cols, rows, row_bytes, box_cols, box_rows};
    TmapCache& c = t_tmaps;
    for (int i = 0; i < c.used; ++i)
        if (c.key[i] == key) {
            std::memcpy(map, &c.map[i], sizeof(CUtensorMap));
            return TMS_OK;
        }
    // A zero-row tensor is not encodable; callers never load from it then,
    // so describe one row (the box reads zero fill beyond it).
    const cuuint64_t dims[2] = {cols, rows > 0 ? rows : 1};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode.load(std::memory_order_relaxed)(
        map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return TMS_ERR_INVALID_ARG;
    const int slot = c.used < kTmapCache ? c.used++ : (c.next++ % kTmapCache);
    c.key[slot] = key;
    std::memcpy(&c.map[slot], map, sizeof(CUtensorMap));
    return TMS_OK;
}

}  // namespace tms

extern "C" {

tms_status tms_get_device_error(cudaStream_t stream, int* flags) {
    if (flags == nullptr) return TMS_ERR_INVALID_ARG;
    tms::DeviceInfo dev;
    tms_status st = tms::current_device(&dev);
    if (st != TMS_OK) return st;
    unsigned int v = 0;
    if (cudaStreamSynchronize(stream) != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, g_tms_error_word, sizeof v) != cudaSuccess) {
        (void)cudaGetLastError();
        return TMS_ERR_CUDA;
    }
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_tms_error_word, &zero, sizeof zero) != cudaSuccess) {
        (void)cudaGetLastError();
        return TMS_ERR_CUDA;
    }
    *flags = static_cast<int>(v);
    return v ? TMS_ERR_DEVICE_FLAG : TMS_OK;
}

tms_status tms_debug_set(int64_t wait_budget_cycles, int fault) {
    if (wait_budget_cycles < 0 || (fault != 0 && fault != TMS_FAULT_HOLD_ACCUMULATOR)) return TMS_ERR_INVALID_ARG;
    tms::g_debug_budget.store(wait_budget_cycles, std::memory_order_relaxed);
    tms::g_debug_fault.store(fault, std::memory_order_relaxed);
    return TMS_OK;
}

const char* tms_status_string(tms_status s) {
    switch (s) {
        case TMS_OK: return "ok";
        case TMS_ERR_INVALID_ARG: return "invalid argument";
        case TMS_ERR_UNSUPPORTED: return "unsupported shape for this build";
        case TMS_ERR_CUDA: return "CUDA runtime or launch error";
        case TMS_ERR_DEVICE_FLAG: return "device-side data error flagged";
        case TMS_ERR_TIMEOUT: return "bounded wait timed out";
        case TMS_ERR_BUSY: return "admission refused: too many pending requests";
    }
    return "unknown status";
}

int tms_version(void) { return 100; }

}  // extern "C"
