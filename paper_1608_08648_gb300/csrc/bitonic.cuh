// Block-wide bitonic sort held in registers (the shared-memory bucket sort of
// step 5).  NT threads each own IT consecutive elements (element e sits in
// register e % IT of thread e / IT).  Batcher's bitonic network is run stage by
// stage: a compare-exchange partner at distance j < IT lies in the same thread
// (plain register min / max), at IT <= j < 32 IT in another lane of the warp
// (__shfl_xor_sync), and at j >= 32 IT in another warp (one exchange through
// shared memory).  Every stage is data independent, so the IT compare-exchanges
// of a thread overlap instead of forming a dependence chain.
//
// Stability: the network is not stable, so where equal keys must keep their
// order (a payload travels with the key) the element compared is the pair
// (ordered key, position inside the leaf), which is unique; keys alone need no
// tie-break because equal keys are identical bit patterns.
#pragma once

#include "blocksort.cuh"
#include "common.cuh"

namespace ossort {

// One sortable element.  E32: 32-bit key; E64: 64-bit key, or a 32-bit key
// packed above its 32-bit position; E96: 64-bit key and a 32-bit position.
struct E32 {
    uint32_t k;
    __device__ __forceinline__ static bool lt(const E32& a, const E32& b) { return a.k < b.k; }
    __device__ __forceinline__ static E32 shfl(const E32& a, int m) {
        return E32{__shfl_xor_sync(0xffffffffu, a.k, m)};
    }
};
struct E64 {
    uint64_t k;
    __device__ __forceinline__ static bool lt(const E64& a, const E64& b) { return a.k < b.k; }
    __device__ __forceinline__ static E64 shfl(const E64& a, int m) {
        return E64{__shfl_xor_sync(0xffffffffu, a.k, m)};
    }
};
struct E96 {
    uint64_t k;
    uint32_t p;
    __device__ __forceinline__ static bool lt(const E96& a, const E96& b) {
        return (a.k < b.k) | ((a.k == b.k) & (a.p < b.p));
    }
    __device__ __forceinline__ static E96 shfl(const E96& a, int m) {
        return E96{__shfl_xor_sync(0xffffffffu, a.k, m), __shfl_xor_sync(0xffffffffu, a.p, m)};
    }
};

// Element type of a leaf sort and how keys, positions and elements convert.
template <class O, bool HV> struct LeafElem;
template <> struct LeafElem<uint32_t, false> {
    using E = E32;
    static __device__ __forceinline__ E make(uint32_t o, uint32_t) { return E{o}; }
    static __device__ __forceinline__ uint32_t key(const E& e) { return e.k; }
    static __device__ __forceinline__ uint32_t pos(const E&) { return 0; }
};
template <> struct LeafElem<uint32_t, true> {
    using E = E64;
    static __device__ __forceinline__ E make(uint32_t o, uint32_t p) { return E{((uint64_t)o << 32) | p}; }
    static __device__ __forceinline__ uint32_t key(const E& e) { return (uint32_t)(e.k >> 32); }
    static __device__ __forceinline__ uint32_t pos(const E& e) { return (uint32_t)e.k; }
};
template <> struct LeafElem<uint64_t, false> {
    using E = E64;
    static __device__ __forceinline__ E make(uint64_t o, uint32_t) { return E{o}; }
    static __device__ __forceinline__ uint64_t key(const E& e) { return e.k; }
    static __device__ __forceinline__ uint32_t pos(const E&) { return 0; }
};
template <> struct LeafElem<uint64_t, true> {
    using E = E96;
    static __device__ __forceinline__ E make(uint64_t o, uint32_t p) { return E{o, p}; }
    static __device__ __forceinline__ uint64_t key(const E& e) { return e.k; }
    static __device__ __forceinline__ uint32_t pos(const E& e) { return e.p; }
};

template <class E>
__device__ __forceinline__ void cas_dir(E& a, E& b, bool up) {
    const bool sw = E::lt(b, a) == up;   // up: a <- min, b <- max
    const E lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

template <class E>
__device__ __forceinline__ E keep(const E& mine, const E& other, bool keep_min) {
    const bool o_less = E::lt(other, mine);
    return (o_less == keep_min) ? other : mine;
}

// Sorts the elements x[0..IT) of every thread as one sequence of `total`
// elements in blocked order (total: a power of two, a multiple of 32*IT, at
// most NT*IT).  Warps whose elements all lie at or beyond `total` take no part
// in the exchanges but still reach every __syncthreads.  ex: shared memory for
// NT*IT elements in padded layout.
template <class E, int NT, int IT>
__device__ void bitonic_block(E (&x)[IT], E* ex, int total) {
    constexpr int LOG_IT = IT == 4 ? 2 : IT == 8 ? 3 : IT == 16 ? 4 : 5;
    constexpr int LOG_NT = NT == 128 ? 7 : NT == 256 ? 8 : NT == 512 ? 9 : 10;
    constexpr int LOG_N = LOG_IT + LOG_NT;
    static_assert((1 << LOG_IT) == IT && (1 << LOG_NT) == NT, "IT and NT must be powers of two");
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool active = tid * IT < total;
    const int base = tid * IT;
#pragma unroll
    for (int lk = 1; lk <= LOG_N; ++lk) {
        const int kk = 1 << lk;
        if (kk > total) continue;   // uniform across the block
#pragma unroll
        for (int lj = lk - 1; lj >= 0; --lj) {
            const int jj = 1 << lj;
            if (jj < IT) {
                if (active) {
#pragma unroll
                    for (int i = 0; i < IT; ++i) {
                        if ((i & jj) == 0) {
                            const bool up = ((base + i) & kk) == 0;
                            cas_dir(x[i], x[i + jj], up);
                        }
                    }
                }
            } else if (jj < 32 * IT) {
                if (active) {
                    const int lm = jj / IT;
                    const bool keep_min = ((base & jj) == 0) == ((base & kk) == 0);
#pragma unroll
                    for (int i = 0; i < IT; ++i) x[i] = keep(x[i], E::shfl(x[i], lm), keep_min);
                }
            } else {
                __syncthreads();
                if (active) {
#pragma unroll
                    for (int i = 0; i < IT; ++i) ex[pad_idx<E>(base + i)] = x[i];
                }
                __syncthreads();
                if (active) {
                    const bool keep_min = ((base & jj) == 0) == ((base & kk) == 0);
#pragma unroll
                    for (int i = 0; i < IT; ++i) x[i] = keep(x[i], ex[pad_idx<E>((base + i) ^ jj)], keep_min);
                }
            }
        }
    }
}

// Bitonic sort of G = 16 * GIT elements held by a 16-lane group (lane l of the
// group owns elements l*GIT .. l*GIT+GIT-1 in registers).  Only the stages of a
// network over `ext` elements run (ext: a power of two, warp-uniform, at most
// G; elements at or beyond ext must be the maximum).  Both 16-lane groups of a
// warp execute the same stages.  Keys only (E32 / E64): ascending.
template <class E, int GIT>
__device__ __forceinline__ void bitonic_group16(E (&x)[GIT], int ext) {
    constexpr int LOG_GIT = GIT == 8 ? 3 : GIT == 16 ? 4 : 5;
    static_assert((1 << LOG_GIT) == GIT, "GIT must be 8, 16 or 32");
    constexpr int LOG_G = LOG_GIT + 4;
    const int gl = threadIdx.x & 15;          // lane inside the group
    const int base = gl * GIT;
#pragma unroll
    for (int lk = 1; lk <= LOG_G; ++lk) {
        const int kk = 1 << lk;
        if (kk > ext) continue;
#pragma unroll
        for (int lj = lk - 1; lj >= 0; --lj) {
            const int jj = 1 << lj;
            if (jj < GIT) {
#pragma unroll
                for (int i = 0; i < GIT; ++i) {
                    if ((i & jj) == 0) {
                        const bool up = ((base + i) & kk) == 0;
                        cas_dir(x[i], x[i + jj], up);
                    }
                }
            } else {
                const int lm = jj / GIT;      // < 16: the partner stays inside the group
                const bool keep_min = ((base & jj) == 0) == ((base & kk) == 0);
#pragma unroll
                for (int i = 0; i < GIT; ++i) x[i] = keep(x[i], E::shfl(x[i], lm), keep_min);
            }
        }
    }
}

}  // namespace ossort
