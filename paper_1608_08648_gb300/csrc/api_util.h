// Helpers shared by the C-ABI translation units (defined in api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ossort {
// Record a failed CUDA call for os_last_cuda_error; returns OS_ERR_CUDA.
int cuda_fail(cudaError_t e);
// Multiprocessor count of the current device (152 if it cannot be queried).
int num_sms_of_current_device();
// Add kernels launched outside the OS_LAUNCH path (graph launches) to the count.
void add_launches(uint64_t k);
}  // namespace ossort
