// 32-byte string keys in memcmp order (the paper's workload, Section 3).
//
// A key is 32 bytes compared as unsigned bytes, lexicographically; word k of a
// key is its bytes 8k..8k+7 read big-endian, so memcmp order is the
// lexicographic order of its four words.  The sort runs the method on the
// first word: SqRan / SqDet sort the pairs (word 0, original index), the index
// riding along as the payload, so the partition is in the tagged order
// (word 0, index) of Section 2.2.  Keys that tie on word 0 are then contiguous
// and in index order; each run of such keys is sorted by word 1 with the
// segmented sort (stable, so full ties stay in index order), runs tying on
// words 0-1 by word 2, and on words 0-2 by word 3.  A final gather moves the
// 32-byte records (and payloads) into the order of the indices.  Only 12 bytes
// per key (a word and an index) travel through the sort.
#pragma once

#include "driver.cuh"

namespace ossort {

struct Str32 {
    uint64_t w[4];   // the 32 bytes as four machine words
};

// Byte reversal: the big-endian reading of a word stored little-endian.
__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
}

constexpr int STR_NT = 256;
constexpr int STR_IT = 8;
constexpr int STR_BLK = STR_NT * STR_IT;   // elements per block of the flag / compaction passes

// Word 0 of every key and the identity permutation.
static __global__ void k_str_init(const Str32* __restrict__ in, uint32_t n, uint64_t* __restrict__ P,
                                  uint32_t* __restrict__ I) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        P[i] = bswap64(in[i].w[0]);
        I[i] = i;
    }
}

// e_out[j] = 1 when positions j-1 and j hold keys equal on words 0..w-1 (the
// sorted word-0 array Ps decides w = 1; deeper levels extend e_in with word
// w-1 of the two keys, whose positions stay in the same run at every level).
static __global__ void k_str_eq(int w, const Str32* __restrict__ in, const uint64_t* __restrict__ Ps,
                                const uint32_t* __restrict__ Is, const uint8_t* __restrict__ e_in, uint32_t n,
                                uint8_t* __restrict__ e_out) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        uint8_t e = 0;
        if (j > 0) {
            if (w == 1) {
                e = Ps[j] == Ps[j - 1];
            } else if (e_in[j]) {
                e = in[Is[j]].w[w - 1] == in[Is[j - 1]].w[w - 1];
            }
        }
        e_out[j] = e;
    }
}

// Per block of STR_BLK positions: elements inside a run of two or more equal
// keys (m) and the first element of each such run (h).
__device__ __forceinline__ void str_flags(const uint8_t* e, uint32_t n, uint32_t j, uint32_t& m, uint32_t& h) {
    const uint32_t ej = j < n ? e[j] : 0u;
    const uint32_t en = j + 1 < n ? e[j + 1] : 0u;
    m = (j < n) && (ej | en);
    h = m && !ej;
}

static __global__ void __launch_bounds__(STR_NT)
k_str_count(const uint8_t* __restrict__ e, uint32_t n, uint32_t* __restrict__ blk) {
    __shared__ uint32_t sm[2][STR_NT / 32];
    const uint32_t base = blockIdx.x * STR_BLK + threadIdx.x * STR_IT;
    uint32_t cm = 0, ch = 0;
#pragma unroll
    for (int i = 0; i < STR_IT; ++i) {
        uint32_t m, h;
        str_flags(e, n, base + i, m, h);
        cm += m;
        ch += h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm += __shfl_xor_sync(0xffffffffu, cm, o);
        ch += __shfl_xor_sync(0xffffffffu, ch, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = cm;
        sm[1][threadIdx.x >> 5] = ch;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int w = 0; w < STR_NT / 32; ++w) {
            a += sm[0][w];
            b += sm[1][w];
        }
        blk[2 * blockIdx.x] = a;
        blk[2 * blockIdx.x + 1] = b;
    }
}

// Exclusive scan of the per-block pairs (one CTA); tot = {elements, runs}.
static __global__ void __launch_bounds__(1024)
k_str_scan(uint32_t* blk, uint32_t nblk, uint32_t* __restrict__ tot) {
    __shared__ uint32_t buf[2][1024];
    __shared__ uint32_t scratch[32];
    uint32_t carry[2] = {0, 0};
    for (uint32_t b0 = 0; b0 < nblk; b0 += 1024) {
        const int len = (int)min(1024u, nblk - b0);
        for (int q = 0; q < 2; ++q) {
            for (int i = threadIdx.x; i < len; i += blockDim.x) buf[q][i] = blk[2 * (b0 + i) + q];
            const uint32_t t = block_exclusive_scan(buf[q], len, scratch);
            for (int i = threadIdx.x; i < len; i += blockDim.x) blk[2 * (b0 + i) + q] = buf[q][i] + carry[q];
            carry[q] += t;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        tot[0] = carry[0];
        tot[1] = carry[1];
    }
}

// Compaction of the run elements: W = word w of each (the next sort key), Iw =
// its index, pos = its position; seg[r] = compacted start of run r, seg[runs] =
// the element count.
static __global__ void __launch_bounds__(STR_NT)
k_str_compact(int w, const Str32* __restrict__ in, const uint32_t* __restrict__ Is, const uint8_t* __restrict__ e,
              uint32_t n, const uint32_t* __restrict__ blk, const uint32_t* __restrict__ tot,
              uint64_t* __restrict__ W, uint32_t* __restrict__ Iw, uint32_t* __restrict__ pos,
              uint32_t* __restrict__ seg) {
    __shared__ uint32_t sm[2][STR_NT];
    __shared__ uint32_t scratch[32];
    const uint32_t base = blockIdx.x * STR_BLK + threadIdx.x * STR_IT;
    uint32_t mf = 0, hf = 0;   // bit i: element base + i is in a run / starts one
    uint32_t cm = 0, ch = 0;
#pragma unroll
    for (int i = 0; i < STR_IT; ++i) {
        uint32_t m, h;
        str_flags(e, n, base + i, m, h);
        mf |= m << i;
        hf |= h << i;
        cm += m;
        ch += h;
    }
    sm[0][threadIdx.x] = cm;
    sm[1][threadIdx.x] = ch;
    block_exclusive_scan(sm[0], STR_NT, scratch);
    block_exclusive_scan(sm[1], STR_NT, scratch);
    uint32_t om = blk[2 * blockIdx.x] + sm[0][threadIdx.x];
    uint32_t oh = blk[2 * blockIdx.x + 1] + sm[1][threadIdx.x];
#pragma unroll
    for (int i = 0; i < STR_IT; ++i) {
        if ((mf >> i) & 1u) {
            const uint32_t j = base + i;
            const uint32_t idx = Is[j];
            W[om] = bswap64(in[idx].w[w]);
            Iw[om] = idx;
            pos[om] = j;
            if ((hf >> i) & 1u) seg[oh++] = om;
            ++om;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) seg[tot[1]] = tot[0];
}

// Sorted run elements back to their positions.
static __global__ void k_str_put(const uint32_t* __restrict__ Iw, const uint32_t* __restrict__ pos,
                                 const uint32_t* __restrict__ tot, uint32_t* __restrict__ Is) {
    const uint32_t cnt = tot[0];
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x)
        Is[pos[k]] = Iw[k];
}

// out[j] = in[Is[j]] (and the payloads alike).
static __global__ void k_str_gather(const Str32* __restrict__ in, const uint32_t* __restrict__ vin,
                                    const uint32_t* __restrict__ Is, uint32_t n, Str32* __restrict__ out,
                                    uint32_t* __restrict__ vout) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t i = Is[j];
        out[j] = in[i];
        if (vin) vout[j] = vin[i];
    }
}

// The 32-byte keys of the p - 1 splitters: the splitter's tag names a position
// of the word-0 array the splitters were drawn from; map (SqDet: the indices in
// the order of the sorted sequences) or the identity (SqRan) gives its key.
static __global__ void k_str_splitters(const Str32* __restrict__ in, const uint32_t* __restrict__ spl_t,
                                       const uint32_t* __restrict__ map, uint32_t m, Str32* __restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[i] = in[map ? map[spl_t[i]] : spl_t[i]];
}

// Bytes seg_core takes for a refinement of up to n keys in up to n/2 runs.
inline size_t str_refine_bytes(uint64_t n) {
    Ctx m;
    SegSource src{nullptr, nullptr, (uint32_t)std::max<uint64_t>(1, n / 2), n};
    seg_core<KeyU64, true>(m, src, bucket_classes<uint64_t>(), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                           0, nullptr);
    return m.ar.used + 256;
}

}  // namespace ossort
