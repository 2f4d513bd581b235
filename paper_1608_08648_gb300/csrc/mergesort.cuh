// Block-wide merge sort of up to NT*IT elements held in registers (the
// shared-memory bucket sort of step 5).
//
//  1. Every thread sorts its IT consecutive elements in registers with
//     Batcher's odd-even merge network (compile-time compare-exchanges).
//  2. log2(len / IT) rounds merge pairs of sorted runs through shared memory.
//     In a round a thread owns IT consecutive outputs of its pair: a merge-path
//     binary search finds where they start in the left run (ai) and the right
//     run (bi); the thread then merges serially, keeping the two run heads in
//     registers and refilling the consumed side with one shared load per output
//     ((key, position) triples instead take the IT candidates of each run and
//     sort their elementwise minimum, a bitonic sequence, in registers).
//
// Runs are padded: every thread stores all IT of its elements, and positions at
// or beyond len hold +infinity, so a ragged last run needs no special case.  The
// shared buffer therefore spans NT*IT positions.  The elements are compared whole
// (E::lt); equal elements are interchangeable (keys alone, or unique
// (key, position) pairs), so no stability rule is needed in the merge itself.
#pragma once

#include "blocksort.cuh"
#include "common.cuh"
#include "elements.cuh"

namespace ossort {

template <class E>
__device__ __forceinline__ void cas_up(E& a, E& b) {   // a <- min, b <- max
    const bool sw = E::lt(b, a);
    const E lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

template <class E>
__device__ __forceinline__ E emin(const E& a, const E& b) { return E::lt(b, a) ? b : a; }

// Single-word elements order as plain unsigned integers: min / max.
template <>
__device__ __forceinline__ void cas_up<E32>(E32& a, E32& b) {
    const uint32_t lo = min(a.k, b.k), hi = max(a.k, b.k);
    a.k = lo;
    b.k = hi;
}
template <>
__device__ __forceinline__ void cas_up<E64>(E64& a, E64& b) {
    const uint64_t lo = min(a.k, b.k), hi = max(a.k, b.k);
    a.k = lo;
    b.k = hi;
}
template <>
__device__ __forceinline__ E32 emin<E32>(const E32& a, const E32& b) { return E32{min(a.k, b.k)}; }
template <>
__device__ __forceinline__ E64 emin<E64>(const E64& a, const E64& b) { return E64{min(a.k, b.k)}; }

// Batcher's odd-even merge sort of x[0..IT) ascending (IT a power of two): 191
// compare-exchanges for 32 elements against 240 for the bitonic network.  The
// network is unrolled by template recursion so that every index is a
// compile-time constant (the elements stay in registers).
template <class E, int IT, int PP, int KK, int J, int I>
__device__ __forceinline__ void oe_pairs(E (&x)[IT]) {
    if constexpr (I < KK && I + J + KK < IT) {
        if constexpr ((I + J) / (2 * PP) == (I + J + KK) / (2 * PP)) cas_up(x[I + J], x[I + J + KK]);
        oe_pairs<E, IT, PP, KK, J, I + 1>(x);
    }
}
template <class E, int IT, int PP, int KK, int J>
__device__ __forceinline__ void oe_blocks(E (&x)[IT]) {
    if constexpr (J + KK < IT) {
        oe_pairs<E, IT, PP, KK, J, 0>(x);
        oe_blocks<E, IT, PP, KK, J + 2 * KK>(x);
    }
}
template <class E, int IT, int PP, int KK>
__device__ __forceinline__ void oe_stages(E (&x)[IT]) {
    if constexpr (KK >= 1) {
        oe_blocks<E, IT, PP, KK, KK % PP>(x);
        oe_stages<E, IT, PP, KK / 2>(x);
    }
}
template <class E, int IT, int PP>
__device__ __forceinline__ void oe_merges(E (&x)[IT]) {
    if constexpr (PP < IT) {
        oe_stages<E, IT, PP, PP>(x);
        oe_merges<E, IT, 2 * PP>(x);
    }
}
template <class E, int IT>
__device__ __forceinline__ void oddeven_sort_regs(E (&x)[IT]) {
    oe_merges<E, IT, 1>(x);
}

// Bitonic sort of x[0..IT) ascending (IT a power of two); every compare-exchange
// and its direction are fixed at compile time.
template <class E, int IT>
__device__ __forceinline__ void bitonic_sort_regs(E (&x)[IT]) {
#pragma unroll
    for (int kk = 2; kk <= IT; kk <<= 1)
#pragma unroll
        for (int jj = kk >> 1; jj >= 1; jj >>= 1)
#pragma unroll
            for (int i = 0; i < IT; ++i)
                if ((i & jj) == 0) {
                    if ((i & kk) == 0) cas_up(x[i], x[i + jj]);
                    else cas_up(x[i + jj], x[i]);
                }
}

// Sort a bitonic sequence x[0..IT) ascending.
template <class E, int IT>
__device__ __forceinline__ void bitonic_merge_regs(E (&x)[IT]) {
#pragma unroll
    for (int jj = IT / 2; jj >= 1; jj >>= 1)
#pragma unroll
        for (int i = 0; i < IT; ++i)
            if ((i & jj) == 0) cas_up(x[i], x[i + jj]);
}

// x: the thread's IT elements at positions tid*IT + i (blocked; positions >= len
// must hold EMax).  sk: shared memory for padded_len<E>(NT*IT) elements; the
// whole block must hold NT*IT >= len.  On
// return x holds the thread's IT outputs of the sorted sequence.  All NT threads
// must call; starts and ends with __syncthreads.
template <class E, int NT, int IT>
__device__ __forceinline__ void merge_sort_block(E (&x)[IT], E* sk, int len) {
    const int base = threadIdx.x * IT;
    const bool active = base < len;
    if (active) {
        // (key, position) triples keep the bitonic network: its shorter live
        // ranges fit the 64-register budget of the 512-thread leaf.
        if constexpr (sizeof(E) <= 8) oddeven_sort_regs<E, IT>(x);
        else bitonic_sort_regs<E, IT>(x);
    }
    for (int run = IT; run < len; run *= 2) {
        // A pair of runs that fits in one warp's elements is merged by that warp
        // alone, so only the larger rounds need the whole block.
        const bool block_wide = 2 * run > 32 * IT;
        if (block_wide) __syncthreads();
        else __syncwarp();
#pragma unroll
        for (int i = 0; i < IT; ++i) sk[pad_idx<E>(base + i)] = x[i];   // beyond len: +infinity
        if (block_wide) __syncthreads();
        else __syncwarp();
        if (active) {
            const int pb = base & ~(2 * run - 1);      // first position of the pair
            const int d = base - pb;                   // output diagonal inside the pair
            const E* A = sk;                           // A[j] = sk[pb + j]
            int lo = max(0, d - run), hi = min(d, run);
            while (lo < hi) {                          // left-run outputs among the first d
                const int mid = (lo + hi) >> 1;
                const E av = A[pad_idx<E>(pb + mid)];
                const E bv = A[pad_idx<E>(pb + run + d - 1 - mid)];
                if (E::lt(bv, av)) hi = mid;
                else lo = mid + 1;
            }
            if constexpr (sizeof(E) <= 8) {
                // Serial merge of the thread's IT outputs: the heads of both runs in
                // registers, one shared load per output to refill the consumed side
                // (ties go to the left run).
                int ia = lo, ib = d - lo;
                E av = ia < run ? A[pad_idx<E>(pb + ia)] : EMax<E>::v();
                E bv = ib < run ? A[pad_idx<E>(pb + run + ib)] : EMax<E>::v();
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const bool take_b = E::lt(bv, av);
                    x[i] = take_b ? bv : av;
                    if (i + 1 < IT) {
                        const int nx = take_b ? ib + 1 : ia + 1;
                        const int nidx = take_b ? pb + run + nx : pb + nx;
                        const E nv = nx < run ? A[pad_idx<E>(nidx)] : EMax<E>::v();
                        ia += take_b ? 0 : 1;
                        ib += take_b ? 1 : 0;
                        av = take_b ? av : nv;
                        bv = take_b ? nv : bv;
                    }
                }
            } else {
                // (key, position) triples: the IT smallest of A[ai, ai+IT) and
                // B[bi, bi+IT) as min(A[ai+i], B[bi+IT-1-i]) (a bitonic sequence,
                // the half-cleaner of a bitonic merge), sorted by log2(IT) register
                // stages; fewer live registers than the serial merge of triples.
                const int ai = lo, bi = d - lo;
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const int ia = ai + i, ib = bi + IT - 1 - i;
                    const E av = ia < run ? A[pad_idx<E>(pb + ia)] : EMax<E>::v();
                    const E bv = ib < run ? A[pad_idx<E>(pb + run + ib)] : EMax<E>::v();
                    x[i] = emin(av, bv);
                }
                bitonic_merge_regs<E, IT>(x);
            }
        }
    }
    __syncthreads();
}

}  // namespace ossort
