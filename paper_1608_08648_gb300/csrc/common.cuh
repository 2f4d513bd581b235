// Shared device definitions of the GB300 sample sort: key traits, tagged keys,
// the counter-based SplitMix64, launch constants and the workspace arena.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ossort {

// ---------------------------------------------------------------------------
// Key traits.  Every kernel works on an unsigned "ordered" image of the key
// whose unsigned order is the key order, and converts back on store.
//   int32  : flip the sign bit.
//   uint64 : identity.
//   float64: IEEE 754 totalOrder map -- negative numbers have every bit
//            inverted, non-negative ones get the sign bit set.
//   uint32 : identity (internal: sorting sample positions).
// ---------------------------------------------------------------------------
struct KeyI32 {
    using T = int32_t;
    using O = uint32_t;
    static __host__ __device__ __forceinline__ O ord(T x) { return (uint32_t)x ^ 0x80000000u; }
    static __host__ __device__ __forceinline__ T key(O o) { return (int32_t)(o ^ 0x80000000u); }
};
struct KeyU32 {
    using T = uint32_t;
    using O = uint32_t;
    static __host__ __device__ __forceinline__ O ord(T x) { return x; }
    static __host__ __device__ __forceinline__ T key(O o) { return o; }
};
struct KeyU64 {
    using T = uint64_t;
    using O = uint64_t;
    static __host__ __device__ __forceinline__ O ord(T x) { return x; }
    static __host__ __device__ __forceinline__ T key(O o) { return o; }
};
struct KeyF64 {  // T holds the raw bits of the double
    using T = uint64_t;
    using O = uint64_t;
    static __host__ __device__ __forceinline__ O ord(T b) {
        return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    }
    static __host__ __device__ __forceinline__ T key(O o) {
        return (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
    }
};

template <class O> struct OMax;
template <> struct OMax<uint32_t> { static constexpr uint32_t v = 0xFFFFFFFFu; };
template <> struct OMax<uint64_t> { static constexpr uint64_t v = 0xFFFFFFFFFFFFFFFFull; };

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), counter form: output i of
// the generator whose state starts at `state` is mix(state + (i + 1) GAMMA);
// stream `st` of `seed` starts at mix(seed + (st + 1) GAMMA).
// ---------------------------------------------------------------------------
constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm_stream(uint64_t seed, uint64_t st) {
    return sm_mix(seed + (st + 1) * SM_GAMMA);
}
__host__ __device__ __forceinline__ uint64_t sm_at(uint64_t state, uint64_t i) {
    return sm_mix(state + (i + 1) * SM_GAMMA);
}

// ---------------------------------------------------------------------------
// Launch constants.
// ---------------------------------------------------------------------------
constexpr int MAX_P = 4096;          // largest p (bucket ids fit 16 bits)
constexpr int TOP_NT = 256;          // threads of the grid-wide classify / scatter
constexpr int TOP_IT = 16;           // keys per thread per tile
constexpr int TOP_TILE = TOP_NT * TOP_IT;
constexpr int TOP_WARPS = TOP_NT / 32;
// Top-level classify and scatter.  SUPER is the unit both passes walk (a CTA
// owns a contiguous run of units).  Keys alone are staged a whole unit at a
// time by 512 threads (8192 keys: runs of twice as many keys per bucket as
// halves, fewer partly written 32-byte sectors).  Payload sorts (whose per-warp
// stable-ranking counters must fit shared memory for p up to MAX_P) use 256
// threads and 8192-key units in two halves.  Classify uses the same thread
// count, since both passes split the array among the same number of CTAs.
// WIDE (payload sorts with p <= hv_wide_max_p, where the per-warp counters
// still fit): 4-byte keys 1024 threads and 16384-key tiles, 8-byte keys 768
// threads and 12288-key tiles, so that each bucket's run in a tile spans whole
// 32-byte sectors more often, and the payloads are loaded with the keys instead
// of after the ranking (measured on GB300, int32 + payload at p = 512: 3.69 ->
// 3.00 ms).
template <class T> constexpr int hv_wide_max_p() { return sizeof(T) == 4 ? 768 : 1024; }
template <class T, bool HV, bool WIDE = false> struct ScatterCfg {
    static constexpr int NT = WIDE ? (sizeof(T) == 4 ? 4 * TOP_NT : 3 * TOP_NT) : (HV ? TOP_NT : 2 * TOP_NT);
    static constexpr int WARPS = NT / 32;
    static constexpr int SUB = NT * TOP_IT;
    static constexpr int SUPER = SUB > 2 * TOP_TILE ? SUB : 2 * TOP_TILE;
    static constexpr bool PREFETCH = WIDE;   // payloads loaded with the keys
};

constexpr int BK_NT = 512;           // threads of the bucket kernel
constexpr int BK_WARPS = BK_NT / 32;
constexpr int MAXP2 = 256;           // largest fan-out of an in-bucket repartition
constexpr int MAXP2_LBITS = 9;       // bins of its splitter table: 2 * MAXP2
constexpr int MAX_DEPTH = 4;         // repartition levels below a segment
constexpr int SAMPLE2 = 4096;        // sample size of an in-bucket repartition

// Largest segment the shared-memory bucket sort takes: 8192 keys of 4 bytes,
// 4096 of 8 bytes.
template <class O> struct Cap { static constexpr int v = sizeof(O) == 4 ? 8192 : 4096; };
// Threads and keys per thread of the leaf sort: 4-byte keys alone use 128
// threads with 64 keys each (one shared-memory merge round fewer; 80 registers,
// six CTAs per SM), 8-byte keys alone 256 threads with 16; (key, position) pairs
// use 512 threads with half the 256-thread count, to stay within 64 registers.
template <class O, bool HV> struct LeafCfg {
    static constexpr int NT = HV ? 512 : (sizeof(O) == 4 ? 128 : 256);
    static constexpr int IT = Cap<O>::v / NT;
};

// Error bits of the device status word.
constexpr uint32_t ERR_DEPTH = 1u;         // a bucket still too large at MAX_DEPTH
constexpr uint32_t ERR_SIZES = 2u;         // a work list overflowed
constexpr uint32_t ERR_SAMPLE = 4u;        // sample larger than its buffer
constexpr uint32_t ERR_BOUNDS = 8u;        // an index failed its range check (access skipped)
constexpr uint32_t ERR_TIMEOUT = 32u;      // a bounded wait for a bulk copy gave up (the kernel stopped early)

// Record a failed range check in the status word: the error bit, the first
// failing site in status[6] and its index in status[7].  The access is skipped
// by the caller, so a wrong index never touches memory outside its buffer.
__device__ __forceinline__ void flag_bounds(uint32_t* status, uint32_t site, uint64_t idx) {
    atomicOr(status, ERR_BOUNDS);
    if (atomicCAS(status + 6, 0u, site) == 0u) status[7] = (uint32_t)idx;
}

// ---------------------------------------------------------------------------
// Workspace arena: a bump allocator over the caller's workspace.  In measure
// mode (base == nullptr) it only adds up sizes, so os_workspace_size runs the
// same planning code as os_sort.  Measure mode hands out distinct non-null
// placeholder addresses (never dereferenced: no kernel is launched while
// measuring), so a decision that looks at a pointer takes the same branch in
// both modes.  A live request beyond the capacity sets `failed`, after which
// nothing more is launched and the sort reports a workspace error.
// ---------------------------------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    bool failed = false;
    bool measure() const { return base == nullptr; }
    template <class X> X* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(X);
        if (measure()) return reinterpret_cast<X*>(static_cast<uintptr_t>(0x10000) + off);
        if (used > cap) {
            failed = true;
            return nullptr;
        }
        return reinterpret_cast<X*>(base + off);
    }
};

}  // namespace ossort
