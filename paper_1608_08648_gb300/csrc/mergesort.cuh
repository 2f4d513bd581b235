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
template <class E>
__device__ __forceinline__ E emax(const E& a, const E& b) { return E::lt(b, a) ? a : b; }

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
template <>
__device__ __forceinline__ E32 emax<E32>(const E32& a, const E32& b) { return E32{max(a.k, b.k)}; }
template <>
__device__ __forceinline__ E64 emax<E64>(const E64& a, const E64& b) { return E64{max(a.k, b.k)}; }

// Two 16-bit keys in one word: the low halves of a thread's words form one set,
// the high halves another, and one network sorts both sets at once with the
// SIMD minimum / maximum of unsigned 16-bit halves.
struct P16 {
    uint32_t k;
};
template <>
__device__ __forceinline__ void cas_up<P16>(P16& a, P16& b) {
    uint32_t lo, hi;
    asm("min.u16x2 %0, %2, %3;\n\tmax.u16x2 %1, %2, %3;" : "=r"(lo), "=r"(hi) : "r"(a.k), "r"(b.k));
    a.k = lo;
    b.k = hi;
}

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

// Bitonic merging of a warp's 32 * IT elements held blocked (lane l has elements
// l IT .. l IT + IT - 1 in x), from runs of IT that every lane has sorted
// ascending.  Level v (v = 0 .. levels - 1) merges pairs of ascending 2^v-lane
// runs into ascending 2^(v+1)-lane runs with Batcher's bitonic merge, the second
// run taken in reverse: the first stage compares every element with its mirror
// image in the block (lane l ^ (2^(v+1) - 1), register IT - 1 - i), the lower
// half keeping the minima -- which leaves two bitonic halves, all of the lower
// one below all of the upper one -- and the half-cleaners that follow run
// ascending: across lanes by shuffles for distances of IT elements and more,
// inside the lane for the last log2(IT).
//
// Each inline-PTX block handles four elements with one predicate, and takes all
// its shuffled values before it changes any of them (the mirror stage sends the
// registers it later updates), so the shuffles stay next to their compares
// instead of being hoisted ahead of them, which would hold every shuffled copy
// of the 32 IT elements live at once.
#define OSS_XLANE4(TY, S0, S1, S2, S3)                                            \
    "{\n\t.reg .b32 t0, t1, t2, t3;\n\t.reg .pred pl;\n\t"                       \
    "setp.ne.u32 pl, %5, 0;\n\t"                                                 \
    "shfl.sync.bfly.b32 t0, " S0 ", %4, 0x1f, 0xffffffff;\n\t"                    \
    "shfl.sync.bfly.b32 t1, " S1 ", %4, 0x1f, 0xffffffff;\n\t"                    \
    "shfl.sync.bfly.b32 t2, " S2 ", %4, 0x1f, 0xffffffff;\n\t"                    \
    "shfl.sync.bfly.b32 t3, " S3 ", %4, 0x1f, 0xffffffff;\n\t"                    \
    "@pl min." TY " %0, %0, t0;\n\t"                                             \
    "@!pl max." TY " %0, %0, t0;\n\t"                                            \
    "@pl min." TY " %1, %1, t1;\n\t"                                             \
    "@!pl max." TY " %1, %1, t1;\n\t"                                            \
    "@pl min." TY " %2, %2, t2;\n\t"                                             \
    "@!pl max." TY " %2, %2, t2;\n\t"                                            \
    "@pl min." TY " %3, %3, t3;\n\t"                                             \
    "@!pl max." TY " %3, %3, t3;\n\t}"

__device__ __forceinline__ void xlane_cas4(E32& a, E32& b, E32& c, E32& d, int dl, uint32_t lower) {
    asm volatile(OSS_XLANE4("u32", "%0", "%1", "%2", "%3")
                 : "+r"(a.k), "+r"(b.k), "+r"(c.k), "+r"(d.k)
                 : "r"(dl), "r"(lower));
}
__device__ __forceinline__ void xlane_cas4(P16& a, P16& b, P16& c, P16& d, int dl, uint32_t lower) {
    asm volatile(OSS_XLANE4("u16x2", "%0", "%1", "%2", "%3")
                 : "+r"(a.k), "+r"(b.k), "+r"(c.k), "+r"(d.k)
                 : "r"(dl), "r"(lower));
}

// The mirror stage for two pairs of registers (a, b) = (x[k], x[IT-1-k]) and
// (c, d) = (x[k+1], x[IT-2-k]): a meets the partner's b, b the partner's a, and
// so on, partner = lane ^ m.
__device__ __forceinline__ void xlane_mirror4(E32& a, E32& b, E32& c, E32& d, int m, uint32_t lower) {
    asm volatile(OSS_XLANE4("u32", "%1", "%0", "%3", "%2")
                 : "+r"(a.k), "+r"(b.k), "+r"(c.k), "+r"(d.k)
                 : "r"(m), "r"(lower));
}
__device__ __forceinline__ void xlane_mirror4(P16& a, P16& b, P16& c, P16& d, int m, uint32_t lower) {
    asm volatile(OSS_XLANE4("u16x2", "%1", "%0", "%3", "%2")
                 : "+r"(a.k), "+r"(b.k), "+r"(c.k), "+r"(d.k)
                 : "r"(m), "r"(lower));
}
#undef OSS_XLANE4

template <class E, int IT>
__device__ __forceinline__ void warp_bitonic_level(E (&x)[IT], int v) {
    static_assert(IT % 4 == 0, "elements go four at a time across lanes");
    const int lane = threadIdx.x & 31;
    const uint32_t lower = (lane & (1 << v)) == 0;             // lower half of the 2^(v+1)-lane block
    const int m = (2 << v) - 1;
#pragma unroll
    for (int k = 0; k < IT / 2; k += 2) xlane_mirror4(x[k], x[IT - 1 - k], x[k + 1], x[IT - 2 - k], m, lower);
#pragma unroll 1
    for (int dl = 1 << v >> 1; dl >= 1; dl >>= 1) {
        const uint32_t lo = (lane & dl) == 0;
#pragma unroll
        for (int i = 0; i < IT; i += 4) xlane_cas4(x[i], x[i + 1], x[i + 2], x[i + 3], dl, lo);
    }
    bitonic_merge_regs<E, IT>(x);
}

template <class E, int IT>
__device__ __forceinline__ void warp_bitonic_levels(E (&x)[IT], int levels) {
#pragma unroll 1
    for (int v = 0; v < levels; ++v) warp_bitonic_level<E, IT>(x, v);
}

// Layout of the runs in sk during the merge rounds.  4-byte elements (IT a
// multiple of the 32-element padding group) keep the second run of every pair
// descending, so that a pair is one bitonic sequence (up, then down): the
// smallest element not yet output always sits at one of the two ends of the
// part not yet output, and the serial merge takes the smaller end with no
// end-of-run test.  Other elements keep both runs ascending (measured: 8-byte
// elements, 16 a thread, lose more to the half-warp branch of the reversed
// stores in the warp-level rounds than the merge saves).
template <class E, int IT> struct MergeRev {
    static constexpr bool v = sizeof(E) == 4 && IT % 32 == 0;
};

// Store the thread's IT sorted elements (positions base .. base+IT-1 of the
// block's sequence) as the runs of length `run` that the next round merges.
template <class E, int IT>
__device__ __forceinline__ void store_run(const E (&x)[IT], E* sk, int base, int run) {
    if constexpr (MergeRev<E, IT>::v) {
        const int pb = base & ~(2 * run - 1);
        if (base - pb >= run) {
            // second run of its pair, descending: position q goes to 2 pb + 3 run - 1 - q;
            // mb is a multiple of the padding group, so pad_idx splits into a
            // register part and a constant part
            const int mb = 2 * pb + 3 * run - base - IT;
            E* s0 = sk + pad_idx<E>(mb);
#pragma unroll
            for (int i = 0; i < IT; ++i) s0[pad_idx<E>(IT - 1 - i)] = x[i];
            return;
        }
        E* s0 = sk + pad_idx<E>(base);
#pragma unroll
        for (int i = 0; i < IT; ++i) s0[pad_idx<E>(i)] = x[i];
    } else {
#pragma unroll
        for (int i = 0; i < IT; ++i) sk[pad_idx<E>(base + i)] = x[i];
    }
}

// One merge round: the thread's IT outputs (diagonal d of its pair, the pair of
// runs of length `run` starting at pb) from the runs in sk, laid out as
// store_run leaves them.  sk spans padded_len<E>(NT IT) elements, 2 run <= NT IT.
template <class E, int IT>
__device__ __forceinline__ void merge_pair(E (&x)[IT], const E* sk, int base, int run) {
    const int pb = base & ~(2 * run - 1);      // first position of the pair
    const int d = base - pb;                   // output diagonal inside the pair
    const E* A = sk;                           // A[j] = sk[pb + j]
    constexpr bool REV = MergeRev<E, IT>::v;
    // ascending element k of the second run sits at pb + run + k, or (descending
    // layout) at pb + 2 run - 1 - k
    int lo = max(0, d - run), hi = min(d, run);
    while (lo < hi) {                          // left-run outputs among the first d
        const int mid = (lo + hi) >> 1;
        const E av = A[pad_idx<E>(pb + mid)];
        const E bv = A[pad_idx<E>(REV ? pb + 2 * run - d + mid : pb + run + d - 1 - mid)];
        if (E::lt(bv, av)) hi = mid;
        else lo = mid + 1;
    }
    if constexpr (REV) {
        // Serial merge over the bitonic pair: the part not yet output is
        // [i, j]; its smallest element is sk[i] or sk[j]; one shared load per
        // output refills the consumed end.  While outputs remain, some element
        // remains, so i <= j and every load stays inside the pair.
        int i = pb + lo, j = pb + 2 * run - 1 - (d - lo);
        E si = A[pad_idx<E>(i)], sj = A[pad_idx<E>(j)];
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const bool tj = E::lt(sj, si);
            x[k] = tj ? sj : si;
            if (k + 1 < IT) {
                i += tj ? 0 : 1;
                j -= tj ? 1 : 0;
                const E nl = A[pad_idx<E>(tj ? j : i)];
                si = tj ? si : nl;
                sj = tj ? nl : sj;
            }
        }
    } else if constexpr (sizeof(E) <= 8) {
        // Serial merge of the thread's IT outputs: the heads of both runs in
        // registers, one shared load per output to refill the consumed side
        // (ties go to the left run).  The loads are unconditional: a run's end
        // reads at most position pb + 2 run <= NT IT, inside the padded buffer,
        // and the value read there is replaced by +infinity (no branch).
        int ia = lo, ib = d - lo;
        const E a0 = A[pad_idx<E>(pb + ia)], b0 = A[pad_idx<E>(pb + run + ib)];
        E av = ia < run ? a0 : EMax<E>::v();
        E bv = ib < run ? b0 : EMax<E>::v();
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const bool take_b = E::lt(bv, av);
            x[k] = take_b ? bv : av;
            if (k + 1 < IT) {
                const int nx = take_b ? ib + 1 : ia + 1;
                const int nidx = take_b ? pb + run + nx : pb + nx;
                const E nl = A[pad_idx<E>(nidx)];
                const E nv = nx < run ? nl : EMax<E>::v();
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
        for (int k = 0; k < IT; ++k) {
            const int ia = ai + k, ib = bi + IT - 1 - k;
            const E av = ia < run ? A[pad_idx<E>(pb + ia)] : EMax<E>::v();
            const E bv = ib < run ? A[pad_idx<E>(pb + run + ib)] : EMax<E>::v();
            x[k] = emin(av, bv);
        }
        bitonic_merge_regs<E, IT>(x);
    }
}

// The merge rounds from sorted runs of `run` (thread-blocked in x, or already
// in sk as store_run leaves them when in_smem) up to len; a round whose runs are
// in sk runs even when run >= len.  Ends with __syncthreads.  Callers share
// this one copy of the unrolled merge (its code is large; copies of it cost
// instruction fetches).
template <class E, int NT, int IT>
__device__ __forceinline__ void merge_rounds(E (&x)[IT], E* sk, int len, int run, bool in_smem) {
    const int base = threadIdx.x * IT;
    const bool active = base < len;
    for (; run < len || in_smem; run *= 2) {
        // A pair of runs that fits in one warp's elements is merged by that warp
        // alone, so only the larger rounds need the whole block.
        const bool block_wide = 2 * run > 32 * IT;
        if (!in_smem) {
            if (block_wide) __syncthreads();
            else __syncwarp();
            store_run<E, IT>(x, sk, base, run);     // beyond len: +infinity
        }
        in_smem = false;
        if (block_wide) __syncthreads();
        else __syncwarp();
        if (active) merge_pair<E, IT>(x, sk, base, run);
    }
    __syncthreads();
}

// Sorts each warp's 32 IT single-word elements in registers: every lane its IT
// (Batcher), then the warp's lanes together (bitonic levels), as far as the
// first min(len, 32 IT) elements need.  Padding lanes take part (the shuffles
// need the whole warp).
template <class E, int IT>
__device__ __forceinline__ void warp_register_sort(E (&x)[IT], int len) {
    oddeven_sort_regs<E, IT>(x);
    const int wlen = min(len, 32 * IT);     // elements the warps must order among themselves
    int levels = 0;
    while ((IT << levels) < wlen) ++levels;
    warp_bitonic_levels<E, IT>(x, levels);
}

// x: the thread's IT elements at positions tid*IT + i (blocked; positions >= len
// must hold EMax).  sk: shared memory for padded_len<E>(NT*IT) elements; the
// whole block must hold NT*IT >= len.  On
// return x holds the thread's IT outputs of the sorted sequence.  All NT threads
// must call; starts and ends with __syncthreads.
// 32-bit elements (4-byte keys alone) sort each warp's 32 IT elements in
// registers (warp_bitonic_levels) and merge through shared memory only the
// runs of whole warps; wider elements merge every round through shared memory
// (their shuffles and compares take two instructions each, measured slower).
template <class E, int NT, int IT>
__device__ __forceinline__ void merge_sort_block(E (&x)[IT], E* sk, int len) {
    const int base = threadIdx.x * IT;
    const bool active = base < len;
    int run0 = IT;
    if constexpr (sizeof(E) == 4) {
        warp_register_sort<E, IT>(x, len);
        run0 = 32 * IT;
    } else if (active) {
        // (key, position) triples keep the bitonic network: its shorter live
        // ranges fit the 64-register budget of the 512-thread leaf.
        if constexpr (sizeof(E) <= 8) oddeven_sort_regs<E, IT>(x);
        else bitonic_sort_regs<E, IT>(x);
    }
    merge_rounds<E, NT, IT>(x, sk, len, run0, false);
}

// The register phase for single-word elements sk[pad_idx(j)], j < len, all
// within 0xFFFF of kmin (kmin <= 0xFFFF0000): a leaf whose keys span at most
// 2^16 values.  Each thread packs its IT elements as IT/2 words of two 16-bit
// offsets from kmin (padding: 0xFFFF, which unpacks to kmin + 0xFFFF, no
// smaller than any element); one register network sorts the low-half set and
// the high-half set of every warp (IT/2 a lane, then across the warp), half the
// instructions per element of the 32-bit network.  The two sets of each warp go
// back to sk, unpacked, as the two runs of 16 IT of one pair (the second
// descending, as store_run lays it out): merge_rounds with run = 16 IT and
// in_smem merges them and carries on.  A warp reads and writes
// only its own 32 IT positions; ends with __syncwarp.
template <int IT>
__device__ __forceinline__ void narrow_register_sort(E32* sk, int len, uint32_t kmin) {
    constexpr int H = IT / 2;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = threadIdx.x * IT;
    P16 y[H];
#pragma unroll
    for (int r = 0; r < H; ++r) {
        const int j0 = base + 2 * r, j1 = j0 + 1;
        const uint32_t o0 = j0 < len ? sk[pad_idx<E32>(j0)].k - kmin : 0xFFFFu;
        const uint32_t o1 = j1 < len ? sk[pad_idx<E32>(j1)].k - kmin : 0xFFFFu;
        y[r].k = o0 | (o1 << 16);
    }
    warp_register_sort<P16, H>(y, (len + 1) / 2);   // lanes of 2 H positions: as for IT positions
    __syncwarp();                               // the warp's lanes have read their input
    // low set ascending at w 32 IT + 32 lane + r, high set descending (the
    // layout store_run gives the second run of a pair) from the warp's end
    static_assert(H % 32 == 0, "lane blocks of whole padding groups");
    E32* lo0 = sk + pad_idx<E32>(w * 32 * IT + lane * H);
    E32* hi0 = sk + pad_idx<E32>(w * 32 * IT + 32 * IT - H - lane * H);
#pragma unroll
    for (int r = 0; r < H; ++r) {
        lo0[pad_idx<E32>(r)] = E32{kmin + (y[r].k & 0xFFFFu)};
        hi0[pad_idx<E32>(H - 1 - r)] = E32{kmin + (y[r].k >> 16)};
    }
    __syncwarp();
}

}  // namespace ossort
