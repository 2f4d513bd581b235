// Bucket lookup of step 4: the bucket of a key x is the number of splitters
// strictly below x in the tagged order of Section 2.2 -- (ordered key, tag)
// compared lexicographically -- so a key equal to a splitter closes the lower
// bucket.
//
// The splitters sit sorted in shared memory.  A table over the high bits of
// (key - smallest splitter key) gives, for every bin of keys, how many
// splitters lie below the bin; only splitters whose key falls into the key's
// own bin (usually none or one) are compared one by one, and a bin crowded
// with splitters (equal keys told apart by their tags) is binary searched.
// The count is exact: it never depends on the bin layout.
#pragma once

#include "common.cuh"

namespace ossort {

template <class O> struct SplitTable;

// Shared-memory footprint of a table of up to m splitters and 2^lbits bins.
template <class O>
__host__ __device__ constexpr size_t split_table_bytes(int m, int lbits) {
    return (((size_t)(sizeof(O) == 4 ? 8 : 12) * (m + 1) + 15) & ~size_t(15)) +
           (((size_t)4 * ((1 << lbits) + 1) + 15) & ~size_t(15));
}

template <class O>
struct SplitTableBase {
    uint32_t* lut;   // [L + 1]: splitters with key < lo + (i << shift)
    int m;           // number of splitters
    O lo, hi;        // smallest and largest splitter key
    int shift;
};

// 32-bit keys: a splitter is one u64, key << 32 | tag.
template <>
struct SplitTable<uint32_t> : SplitTableBase<uint32_t> {
    uint64_t* sc;
    __device__ __forceinline__ void bind(char* p, int mmax, int lbits) {
        sc = reinterpret_cast<uint64_t*>(p);
        lut = reinterpret_cast<uint32_t*>(p + ((8 * (size_t)(mmax + 1) + 15) & ~size_t(15)));
        (void)lbits;
    }
    __device__ __forceinline__ void set(int i, uint32_t o, uint32_t t) { sc[i] = ((uint64_t)o << 32) | t; }
    __device__ __forceinline__ uint32_t key(int i) const { return (uint32_t)(sc[i] >> 32); }
    // splitter i < (o, t)
    template <bool LAZY = false>
    __device__ __forceinline__ bool below(int i, uint32_t o, uint32_t t) const {
        return sc[i] < (((uint64_t)o << 32) | t);
    }
};

// 64-bit keys: key and tag in two arrays.
template <>
struct SplitTable<uint64_t> : SplitTableBase<uint64_t> {
    uint64_t* so;
    uint32_t* st;
    __device__ __forceinline__ void bind(char* p, int mmax, int lbits) {
        so = reinterpret_cast<uint64_t*>(p);
        st = reinterpret_cast<uint32_t*>(p + 8 * (size_t)(mmax + 1));
        lut = reinterpret_cast<uint32_t*>(p + ((12 * (size_t)(mmax + 1) + 15) & ~size_t(15)));
        (void)lbits;
    }
    __device__ __forceinline__ void set(int i, uint64_t o, uint32_t t) { so[i] = o; st[i] = t; }
    __device__ __forceinline__ uint64_t key(int i) const { return so[i]; }
    // LAZY: read the tag only when the keys are equal -- fewer shared loads
    // where a bin holds about one splitter (the bucket phase), more divergent
    // where bins hold several (measured slower for the top-level classify).
    template <bool LAZY = false>
    __device__ __forceinline__ bool below(int i, uint64_t o, uint32_t t) const {
        const uint64_t k = so[i];
        if (LAZY) {
            if (k != o) return k < o;
            return st[i] < t;
        }
        return (k < o) | ((k == o) & (st[i] < t));
    }
};

template <class O> __device__ __forceinline__ int bit_width(O x);
template <> __device__ __forceinline__ int bit_width<uint32_t>(uint32_t x) { return 32 - __clz(x); }
template <> __device__ __forceinline__ int bit_width<uint64_t>(uint64_t x) { return 64 - __clzll(x); }

// After the m sorted splitters have been set (and a __syncthreads), build the
// bin table with 2^lbits bins.  Called by the whole block; ends with a barrier.
template <class O>
__device__ void split_table_finish(SplitTable<O>& tb, int m, int lbits) {
    tb.m = m;
    if (m == 0) {
        tb.lo = tb.hi = O(0);
        tb.shift = 0;
        __syncthreads();
        return;
    }
    tb.lo = tb.key(0);
    tb.hi = tb.key(m - 1);
    const int w = bit_width<O>(tb.hi - tb.lo);
    tb.shift = w > lbits ? w - lbits : 0;
    const int L = 1 << lbits;
    const O top = (tb.hi - tb.lo) >> tb.shift;   // largest bin index in use (< L)
    for (int i = threadIdx.x; i <= L; i += blockDim.x) {
        uint32_t c;
        if ((O)i > top) {
            c = (uint32_t)m;
        } else {
            const O bound = tb.lo + ((O)i << tb.shift);
            int a = 0, b = m;                    // splitters with key < bound
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (tb.key(mid) < bound) a = mid + 1;
                else b = mid;
            }
            c = (uint32_t)a;
        }
        tb.lut[i] = c;
    }
    __syncthreads();
}

// Number of splitters strictly below (o, t).
template <class O, bool LAZY = false>
__device__ __forceinline__ int split_find(const SplitTable<O>& tb, O o, uint32_t t) {
    if (tb.m == 0 || o < tb.lo) return 0;
    if (o > tb.hi) return tb.m;
    const uint32_t idx = (uint32_t)((o - tb.lo) >> tb.shift);
    int j = (int)tb.lut[idx];
    int k = (int)tb.lut[idx + 1];
    if (k - j > 4) {
        while (j < k) {
            const int mid = (j + k) >> 1;
            if (tb.template below<LAZY>(mid, o, t)) j = mid + 1;
            else k = mid;
        }
        return j;
    }
    int c = j;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (j + u < k && tb.template below<LAZY>(j + u, o, t)) ++c;   // the splitters below form a prefix
    return c;
}

}  // namespace ossort
