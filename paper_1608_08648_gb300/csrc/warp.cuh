// Warp-level grouping of lanes by bucket without __match_any_sync (which costs
// tens of cycles per call): runs of equal neighbours, found with one shuffle
// and one ballot, and exact peer masks built from one ballot per bit.
#pragma once

#include "common.cuh"

namespace ossort {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

// Runs of consecutive lanes holding the same value v (all 32 lanes active).
// head: the first lane of my run; len: the run's length (meaningful on heads).
struct WarpRun {
    int head;
    int len;
    bool is_head;
};

__device__ __forceinline__ WarpRun warp_run(uint32_t v) {
    const int lane = threadIdx.x & 31;
    const uint32_t left = __shfl_up_sync(0xffffffffu, v, 1);
    const bool is_head = lane == 0 || left != v;
    const unsigned heads = __ballot_sync(0xffffffffu, is_head);
    WarpRun r;
    r.is_head = is_head;
    r.head = 31 - __clz(heads & lanemask_le());
    const unsigned later = heads & ~lanemask_le();
    r.len = (later ? __ffs(later) - 1 : 32) - lane;
    return r;
}

// Add the number of lanes in each bucket to cnt[v] (one atomic per run).
__device__ __forceinline__ void warp_count(uint32_t v, uint32_t* cnt) {
    const WarpRun r = warp_run(v);
    if (r.is_head) atomicAdd(&cnt[v], (uint32_t)r.len);
}

// A distinct slot for every lane among the lanes of its bucket, taken from
// cnt[v] (slot order inside a bucket is not defined across runs).
__device__ __forceinline__ uint32_t warp_slot(uint32_t v, uint32_t* cnt) {
    const WarpRun r = warp_run(v);
    uint32_t base = 0;
    if (r.is_head) base = atomicAdd(&cnt[v], (uint32_t)r.len);
    base = __shfl_sync(0xffffffffu, base, r.head);
    return base + (uint32_t)((threadIdx.x & 31) - r.head);
}

// Mask of the lanes whose v equals mine, v < 2^nbits (all 32 lanes active).
__device__ __forceinline__ unsigned warp_peers(uint32_t v, int nbits) {
    unsigned m = 0xffffffffu;
    for (int bit = 0; bit < nbits; ++bit) {
        const bool on = (v >> bit) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, on);
        m &= on ? bb : ~bb;
    }
    return m;
}

}  // namespace ossort
