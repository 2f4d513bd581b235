// os_sort_noalloc: the sort for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs inside a host
// framework which owns every byte of device memory (a fixed pool handed out at
// start-up), or a path that must never allocate after initialisation because an
// allocation can block, fail under fragmentation or synchronise the device.
// os_sort needs a caller-provided workspace of os_workspace_size bytes; this
// entry point instead uses one scratch array compiled into the library.
//
// The scratch is a file-scope __device__ array of OS_NOALLOC_SCRATCH_BYTES.  Host
// code cannot use its name as a device address, so the first call on each
// device (with that device current) asks the runtime for the array's address
// with cudaGetSymbolAddress and remembers it; later calls on that device reuse
// it (a cudaDeviceReset invalidates the remembered address: calls after one are
// not supported).  The array is shared by every call on a device and keeps the
// last call's contents; os_sort clears everything that must start at zero,
// including the status word the kernels flag errors in, which a call with
// statistics reads back.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ossort.h"
#include "api_util.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[OS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
}  // namespace

extern "C" int os_sort_noalloc(int key_type, const void* d_keys_in, void* d_keys_out,
                               const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                               const os_params* prm, void* stream, os_stats* stats) {
    size_t need = 0;
    int rc = os_workspace_size(key_type, n, d_vals_in != nullptr, prm, &need);
    if (rc != OS_OK) return rc;
    if (need > (size_t)OS_NOALLOC_SCRATCH_BYTES) return OS_ERR_UNSUPPORTED;   // beyond the scratch
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ossort::cuda_fail(e);
    }
    if (dev < 0 || dev >= kMaxDevices) return OS_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        scratch = g_noalloc_ptr[dev];
        if (scratch == nullptr) {
            e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
            if (e != cudaSuccess || scratch == nullptr) {
                cudaGetLastError();
                return ossort::cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            }
            g_noalloc_ptr[dev] = scratch;
        }
    }
    return os_sort(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, prm, scratch,
                   (size_t)OS_NOALLOC_SCRATCH_BYTES, stream, stats);
}
