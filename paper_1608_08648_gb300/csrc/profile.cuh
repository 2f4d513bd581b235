// Launch accounting of the library: every kernel launch is counted, and while
// profiling is on (os_profile_start / os_profile_stop) a CUDA event pair is
// recorded around it on its own stream, giving per-kernel device times.
// With the environment variable OSSORT_DEBUG_SYNC=1 every launch is followed
// by a stream synchronization and a check, naming the first kernel that fails.
#pragma once

#include <cuda_runtime.h>

namespace ossort {
void prof_before(cudaStream_t st, const char* name);
void prof_after(cudaStream_t st, const char* name);
}  // namespace ossort

#ifndef OSSORT_NO_LAUNCH
#define OS_LAUNCH(st, name, ...)              \
    do {                                      \
        ::ossort::prof_before((st), (name));  \
        __VA_ARGS__;                          \
        ::ossort::prof_after((st), (name));   \
    } while (0)
#define os_memset_async(ptr, v, bytes, st) cudaMemsetAsync((ptr), (v), (bytes), (st))
#else
// Planning-only builds (the workspace-plan test) never touch the device.
#define OS_LAUNCH(st, name, ...) do { } while (0)
#define os_memset_async(ptr, v, bytes, st) ((void)0)
#endif
