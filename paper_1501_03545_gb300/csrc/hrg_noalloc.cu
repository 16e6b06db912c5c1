// hrg_noalloc.cu -- row offsets from degrees without any device allocation.
//
// hrg_row_offsets_noalloc runs the same exclusive scan that turns degrees
// into CSR row offsets inside hrg_generate_begin, but its scratch (the
// per-tile partial sums of the scan) lives in the file-scope device array
// below instead of in context-owned memory obtained with cudaMalloc.  It is
// meant for callers that may not allocate device memory themselves.
#include <mutex>

#include "../../include/hrg.h"
#include "hrg_internal.h"

namespace {

// 1 MiB of scratch (int64 words), enough for the scan of up to 2^28 degrees.
// Every device that loads the library holds this array until the process
// exits.  All calls share it; its contents after a call are the partial sums
// of that call.
constexpr int64_t kScratchWords = 131072 + 512;
constexpr int64_t kMaxN = (int64_t)1 << 28;
static __device__ __align__(256) int64_t g_scan_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// `g_scan_scratch` only names a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scan_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int hrg_row_offsets_noalloc(const int32_t *deg, int64_t n, int64_t *row_off, void *stream)
{
    if (n < 0 || n > kMaxN) return HRG_EINVAL;
    if (!row_off || (n > 0 && !deg)) return HRG_EINVAL;
    if (hrg::scan_workspace_bytes(n) > sizeof(int64_t) * (size_t)kScratchWords) return HRG_EINVAL;
    void *ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) {
        cudaGetLastError();
        return HRG_ECUDA;
    }
    // The scan overwrites every scratch word it reads (tile sums first, then
    // their prefix sums), so nothing needs clearing between calls.
    if (hrg::scan_i32_to_i64(deg, row_off, n, ws, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HRG_ECUDA;
    }
    return HRG_OK;
}
