// Launch accounting of the library: every kernel launch is counted, and while
// profiling is on (os_profile_start / os_profile_stop) a CUDA event pair is
// recorded around it on its own stream, giving per-kernel device times.
#pragma once

#include <cuda_runtime.h>

namespace ossort {
void prof_before(cudaStream_t st, const char* name);
void prof_after(cudaStream_t st);
}  // namespace ossort

#define OS_LAUNCH(st, name, ...)              \
    do {                                      \
        ::ossort::prof_before((st), (name));  \
        __VA_ARGS__;                          \
        ::ossort::prof_after((st));           \
    } while (0)
