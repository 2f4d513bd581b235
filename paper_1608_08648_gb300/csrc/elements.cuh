// Sortable elements of the shared-memory bucket sort.  Keys are compared as
// their ordered unsigned images; where equal keys must keep their input order
// (a payload travels with the key) the element is the pair (ordered key,
// position inside the segment), which is unique, so any correct sort of the
// pairs is stable for the keys.
#pragma once

#include "common.cuh"

namespace ossort {

// One sortable element.  E32: 32-bit key; E64: 64-bit key, or a 32-bit key
// packed above its 32-bit position; E96: 64-bit key and a 32-bit position.
struct E32 {
    static constexpr bool kSingleWord = true;
    uint32_t k;
    __device__ __forceinline__ static bool lt(const E32& a, const E32& b) { return a.k < b.k; }
    __device__ __forceinline__ static E32 shfl(const E32& a, int m) {
        return E32{__shfl_xor_sync(0xffffffffu, a.k, m)};
    }
};
struct E64 {
    static constexpr bool kSingleWord = true;
    uint64_t k;
    __device__ __forceinline__ static bool lt(const E64& a, const E64& b) { return a.k < b.k; }
    __device__ __forceinline__ static E64 shfl(const E64& a, int m) {
        return E64{__shfl_xor_sync(0xffffffffu, a.k, m)};
    }
};
struct E96 {
    static constexpr bool kSingleWord = false;
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

template <class E> struct EMax;
template <> struct EMax<E32> { static __device__ __forceinline__ E32 v() { return E32{0xFFFFFFFFu}; } };
template <> struct EMax<E64> { static __device__ __forceinline__ E64 v() { return E64{~0ull}; } };
template <> struct EMax<E96> { static __device__ __forceinline__ E96 v() { return E96{~0ull, ~0u}; } };

}  // namespace ossort
