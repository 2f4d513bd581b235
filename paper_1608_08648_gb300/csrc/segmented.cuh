// Batched segmented sort (os_sort_segmented): many independent arrays held
// back to back in one buffer, every one sorted exactly as SqRan (Algorithm 2,
// sample on original positions) sorts it alone with the parameters of its
// length class and the seed u(seed, 2, g), by the fixed kernel sequence of
// seg_core (driver.cuh):
//
//   k_seg_plan       per segment: class, p_g, s_g, tiles; exclusive scans of
//                    tiles, buckets and histogram entries (one CTA)
//   k_seg_splitters  steps 2-3 per segment: p_g s_g - 1 random positions, the
//                    tagged sample sorted in shared memory, p_g - 1 splitters
//   k_seg_classify   step 4: bucket of every key of every partitioned segment,
//                    per-tile bucket counts
//   k_seg_scan       per segment: bucket-major scan of its tile counts, bucket
//                    sizes, and the work items of step 5
//   k_seg_scatter    step 4: keys (and payloads) into contiguous buckets
//   k_repart/k_leaf  step 5: every bucket, and every segment too small to
//                    sample, sorted through the shared work lists
//
// The host only knows n, the number of segments and the class table, so the
// launch sequence does not depend on the segment lengths: it can be captured
// once in a CUDA graph and replayed for new keys and new offsets of the same
// totals.
#pragma once

#include "driver.cuh"

namespace ossort {

// Everything one os_sort_segmented call needs, independent of the key type.
struct SegArgs {
    const void* kin;
    void* kout;
    const uint32_t* vin;
    uint32_t* vout;
    bool has_vals;
    uint64_t n;
    const uint64_t* off;     // device [nseg + 1]
    uint32_t nseg;
    SegClasses cls;
    uint64_t seed;
    void* ws;                // nullptr: measure only
    size_t ws_bytes;
    cudaStream_t st;
    int num_sms;
    const os_seg_stats* stats;
    // outputs
    size_t used;
    uint32_t* status;
};

template <class KT>
int run_segmented(SegArgs& a) {
    using T = typename KT::T;
    Ctx c;
    c.st = a.st;
    c.num_sms = a.num_sms;
    c.ar.base = static_cast<char*>(a.ws);
    c.ar.cap = a.ws_bytes;
    c.status = c.ar.take<uint32_t>(8);
    if (c.live()) os_memset_async(c.status, 0, 8 * sizeof(uint32_t), c.st);
    T* alt = c.ar.take<T>(a.n);
    uint32_t* valt = a.has_vals ? c.ar.take<uint32_t>(a.n) : nullptr;
    const SegSource src{a.off, nullptr, a.nseg, a.n};
    const T* kin = static_cast<const T*>(a.kin);
    T* kout = static_cast<T*>(a.kout);
    if (a.has_vals) seg_core<KT, true>(c, src, a.cls, kin, a.vin, kout, a.vout, alt, valt, a.seed, a.stats);
    else seg_core<KT, false>(c, src, a.cls, kin, nullptr, kout, nullptr, alt, nullptr, a.seed, a.stats);
    a.used = c.ar.used;
    a.status = c.status;
    return c.ar.failed ? OS_ERR_WS : OS_OK;
}

int run_seg_i32(SegArgs& a);
int run_seg_u64(SegArgs& a);
int run_seg_f64(SegArgs& a);

}  // namespace ossort
