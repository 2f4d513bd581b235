// Kernels of the GB300 oversampling sample sort.
//
// Paper step -> kernel (the k_seg_* kernels are in segkernels.cuh):
//   step 1 (SqDet BaselineSorting)      the segmented sort over p uniform sequences
//   step 2 (SqDet regular sample)       k_det_sample
//   step 2 (SqRan random sample)        k_ran_positions + k_gather_tagged
//   steps 2-3 (sample sort, splitters)  k_leaf (or a nested sort) + k_pick_splitters
//   step 4 (split)                      k_classify + k_column_scan + k_bucket_offsets
//                                       + k_scatter (keys land in contiguous buckets)
//   step 5 (sort every bucket)          the segmented sort over the p buckets: an
//                                       oversized bucket is split again by SqRan
//                                       (k_seg_*), a rare oversized child by
//                                       k_repart, every leaf by k_leaf
#pragma once

#include "blocksort.cuh"
#include "classify.cuh"
#include "warp.cuh"
#include "mergesort.cuh"
#include "common.cuh"

#include <type_traits>

namespace ossort {

// In-place exclusive scan of a[0, len) in shared memory by the whole block;
// returns the total.  scratch: 32 words.  Starts and ends with __syncthreads.
static __device__ uint32_t block_exclusive_scan(uint32_t* a, int len, uint32_t* scratch) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (len + nt - 1) / nt;
    const int lo = min(len, tid * per), hi = min(len, lo + per);
    __syncthreads();
    uint32_t sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    const int lane = tid & 31, w = tid >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = nt >> 5;
        uint32_t z = lane < nw ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) scratch[lane] = z;   // inclusive warp totals
    }
    __syncthreads();
    uint32_t run = x - sum + (w > 0 ? scratch[w - 1] : 0);
    const uint32_t total = scratch[(nt >> 5) - 1];
    for (int i = lo; i < hi; ++i) {
        uint32_t c = a[i];
        a[i] = run;
        run += c;
    }
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// Step 2 of SqRan: sample positions floor(u_j n / 2^64), u_j = output j of
// stream 1 of SplitMix64 keyed by seed.
// ---------------------------------------------------------------------------
static __global__ void k_ran_positions(uint32_t* pos, uint32_t m, uint64_t n, uint64_t seed) {
    const uint64_t state = sm_stream(seed, 1);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
        pos[j] = (uint32_t)__umul64hi(sm_at(state, j), n);
}

// T_j = (keys[pos_j], tag pos_j)
template <class KT>
__global__ void k_gather_tagged(const typename KT::T* __restrict__ keys, uint32_t n, const uint32_t* __restrict__ pos,
                                uint32_t m, typename KT::T* tk, uint32_t* tt, uint32_t* status) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint32_t q = pos[j];
        if (q >= n) {
            flag_bounds(status, 1, q);
            continue;
        }
        tk[j] = keys[q];
        tt[j] = q;
    }
}

// Step 2 of SqDet: sequence k = [floor(kn/p), floor((k+1)n/p)) of the sorted
// sequences A gives mm = r p samples; sample j (1..mm) is its key of local rank
// ceil(j c / mm) - 1 (the ends of mm near-equal segments; j = mm is the max).
// The tag is the position in A, i.e. start_k + local rank.
template <class KT>
__global__ void k_det_sample(const typename KT::T* __restrict__ A, uint64_t n, uint32_t p, uint32_t mm,
                             typename KT::T* tk, uint32_t* tt, uint32_t* status) {
    const uint64_t total = (uint64_t)p * mm;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = q / mm, j = q % mm + 1;
        const uint64_t cs = k * n / p, c = (k + 1) * n / p - cs;
        const uint64_t l = (j * c + mm - 1) / mm - 1;
        if (c == 0 || cs + l >= n) {
            flag_bounds(status, 2, cs + l);
            continue;
        }
        tk[q] = A[cs + l];
        tt[q] = (uint32_t)(cs + l);
    }
}

// Step 3: S_i = the (i * stride)-th smallest of the sorted sample, i = 1..p-1.
template <class KT>
__global__ void k_pick_splitters(const typename KT::T* __restrict__ tk, const uint32_t* __restrict__ tt,
                                 uint32_t p, uint64_t stride, typename KT::O* spl_o, uint32_t* spl_t) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x + 1; i < p; i += gridDim.x * blockDim.x) {
        const uint64_t q = (uint64_t)i * stride - 1;
        spl_o[i - 1] = KT::ord(tk[q]);
        spl_t[i - 1] = tt[q];
    }
}

// ---------------------------------------------------------------------------
// Step 4: every CTA of the grid-wide passes owns a contiguous run of units of
// SUPER keys: CTA g of G owns units [tile_lo(g, G), tile_lo(g + 1, G)).  Pass 1
// (k_classify_v of distribute.cuh, with or without a payload) finds the bucket
// of each key (tag = its position in the array), stores it in bid (two bytes a
// key, read back by the scatter) and counts keys per bucket, bucket-major.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint32_t tile_lo(uint32_t g, uint32_t G, uint32_t ntiles) {
    return (uint32_t)(((uint64_t)g * ntiles) / G);
}

// Exclusive scan of every bucket's column of CTA counts (one warp per bucket),
// and the bucket sizes.
static __global__ void k_column_scan(const uint32_t* __restrict__ hist, uint32_t p, uint32_t G,
                              uint32_t* __restrict__ col, uint32_t* __restrict__ bsize) {
    const int lane = threadIdx.x & 31;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= p) return;
    const uint32_t* h = hist + (size_t)b * G;
    uint32_t* c = col + (size_t)b * G;
    uint32_t carry = 0;
    for (uint32_t g0 = 0; g0 < G; g0 += 32) {
        const uint32_t g = g0 + lane;
        const uint32_t x = g < G ? h[g] : 0;
        uint32_t y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (g < G) c[g] = carry + y - x;
        carry += __shfl_sync(0xffffffffu, y, 31);
    }
    if (lane == 0) bsize[b] = carry;
}

// Bucket start offsets: exclusive scan of the sizes; boff[p] = n.  One block.
static __global__ void k_bucket_offsets(const uint32_t* __restrict__ bsize, uint32_t p,
                                        uint32_t* __restrict__ boff) {
    __shared__ uint32_t buf[MAX_P + 1];
    __shared__ uint32_t scratch[32];
    for (uint32_t b = threadIdx.x; b < p; b += blockDim.x) buf[b] = bsize[b];
    const uint32_t total = block_exclusive_scan(buf, (int)p, scratch);
    for (uint32_t b = threadIdx.x; b < p; b += blockDim.x) boff[b] = buf[b];
    if (threadIdx.x == 0) boff[p] = total;
}

// ---------------------------------------------------------------------------
// Step 4, pass 2 (payload sorts; keys alone take k_scatter_v): each scatter
// CTA walks its units (those of cstep classify CTAs) in tiles of SUB keys and
// moves the keys and payloads into their buckets, using the bucket ids of
// pass 1 (a classify CTA count per bucket every cstep columns).  Keys are
// staged in shared memory grouped by bucket and written out as contiguous runs.
// With a payload the scatter is stable: a key's rank among the tile's keys of
// its bucket comes from per-warp counters (peer masks from ballots) plus a
// cross-warp prefix, so every bucket receives its keys in input order.  Keys
// alone need no order inside a bucket (equal keys are identical), so
// shared-memory atomics, one per run of equal neighbours, hand out the slots.
// ---------------------------------------------------------------------------
template <class KT, bool HV, bool WIDE = false>
__global__ void __launch_bounds__(ScatterCfg<typename KT::T, HV, WIDE>::NT,
                                  ScatterCfg<typename KT::T, HV, WIDE>::NT >= 768 ? 1
                                  : ScatterCfg<typename KT::T, HV, WIDE>::NT == 512 ? 2
                                  : (sizeof(typename KT::T) == 4 ? 4 : 3))
k_scatter(const typename KT::T* __restrict__ keys, const uint32_t* __restrict__ vals,
          const uint16_t* __restrict__ bid, uint32_t n, int p, const uint32_t* __restrict__ col, uint32_t cstep,
          const uint32_t* __restrict__ boff, typename KT::T* __restrict__ out, uint32_t* __restrict__ vout,
          uint32_t ntiles, uint32_t* status) {
    using T = typename KT::T;
    using SC = ScatterCfg<typename KT::T, HV, WIDE>;
    constexpr bool PF = HV && SC::PREFETCH;
    constexpr int SNT = SC::NT, SWARPS = SC::WARPS, SUB = SC::SUB, SUPER = SC::SUPER;
    extern __shared__ __align__(16) char smem[];
    char* q = smem;
    T* sk = reinterpret_cast<T*>(q);                 q += sizeof(T) * SUB;
    uint32_t* sv = reinterpret_cast<uint32_t*>(q);    q += HV ? sizeof(uint32_t) * SUB : 0;
    uint32_t* tile_off = reinterpret_cast<uint32_t*>(q); q += sizeof(uint32_t) * (p + 1);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(q);   q += sizeof(uint32_t) * p;
    uint32_t* scratch = reinterpret_cast<uint32_t*>(q);  q += sizeof(uint32_t) * 32;
    uint16_t* sb = reinterpret_cast<uint16_t*>(q);       q += sizeof(uint16_t) * SUB;
    uint16_t* cnt = reinterpret_cast<uint16_t*>(q);      // HV: [SWARPS][p + 1]
    const int cstride = p + 1;

    const uint32_t G = gridDim.x, g = blockIdx.x;
    // the classify ran with cstep CTAs per scatter CTA covering its units: this
    // CTA's keys of bucket b start at column g * cstep
    for (int b = threadIdx.x; b < p; b += SNT) cursor[b] = boff[b] + col[((size_t)b * G + g) * cstep];

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint16_t* mycnt = cnt + w * cstride;
    const uint32_t t0 = tile_lo(g, G, ntiles), t1 = tile_lo(g + 1, G, ntiles);
    for (uint32_t t = t0 * (SUPER / SUB); t < t1 * (SUPER / SUB); ++t) {   // tiles of SUB keys
        const uint32_t tbase = t * SUB;
        const uint32_t base = tbase + w * (TOP_IT * 32) + lane;
        T kv[TOP_IT];
        uint32_t br[TOP_IT];   // bucket << 16 | rank inside the tile's part of the bucket
        uint32_t vv[PF ? TOP_IT : 1];
#pragma unroll
        for (int i = 0; i < TOP_IT; ++i) {
            const uint32_t e = base + i * 32;
            kv[i] = e < n ? keys[e] : T(0);
            br[i] = e < n ? (uint32_t)bid[e] : (uint32_t)p;
            if constexpr (PF) vv[i] = e < n ? vals[e] : 0u;
        }
        if (HV) {
            for (int b = lane; b <= p; b += 32) mycnt[b] = 0;
        } else {
            for (int b = threadIdx.x; b <= p; b += SNT) tile_off[b] = 0;
        }
        __syncthreads();   // counters cleared; previous tile fully written out
        if (HV) {
            const int nbits = 32 - __clz(p);     // bucket ids 0..p fit
#pragma unroll
            for (int i = 0; i < TOP_IT; ++i) {
                const int b = (int)br[i];
                const unsigned m = warp_peers((uint32_t)b, nbits);
                const uint32_t c0 = mycnt[b];
                br[i] = ((uint32_t)b << 16) | (c0 + __popc(m & lanemask_lt()));
                __syncwarp();
                if (lane == __ffs(m) - 1) mycnt[b] = (uint16_t)(c0 + __popc(m));
                __syncwarp();
            }
            __syncthreads();
            // Cross-warp exclusive prefix per bucket; tile totals into tile_off.
            for (int b = threadIdx.x; b < p; b += SNT) {
                uint32_t run = 0;
#pragma unroll
                for (int ww = 0; ww < SWARPS; ++ww) {
                    const uint32_t c = cnt[ww * cstride + b];
                    cnt[ww * cstride + b] = (uint16_t)run;
                    run += c;
                }
                tile_off[b] = run;
            }
        } else {
#pragma unroll
            for (int i = 0; i < TOP_IT; ++i) {
                const uint32_t b = br[i];
                br[i] = (b << 16) | warp_slot(b, tile_off);
            }
        }
        const uint32_t tvalid = block_exclusive_scan(tile_off, p, scratch);
        if (threadIdx.x == 0) tile_off[p] = tvalid;
        // Stage keys grouped by bucket.
#pragma unroll
        for (int i = 0; i < TOP_IT; ++i) {
            const int b = (int)(br[i] >> 16);
            if (b < p) {
                const uint32_t loc = tile_off[b] + (HV ? mycnt[b] : 0u) + (br[i] & 0xFFFFu);
                if (loc >= (uint32_t)SUB) {
                    flag_bounds(status, 8, loc);
                    continue;
                }
                sk[loc] = kv[i];
                if constexpr (PF) sv[loc] = vv[i];
                else if (HV) sv[loc] = vals[base + i * 32];
                sb[loc] = (uint16_t)b;
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < tvalid; j += SNT) {
            const int b = sb[j];
            const uint32_t dst = cursor[b] + (j - tile_off[b]);
            if (dst >= n) {
                flag_bounds(status, 3, dst);
                continue;
            }
            out[dst] = sk[j];
            if (HV) vout[dst] = sv[j];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < p; b += SNT) cursor[b] += tile_off[b + 1] - tile_off[b];
        __syncthreads();   // tile_off is cleared at the top of the next tile
    }
}

// ---------------------------------------------------------------------------
// Step 5 (and step 1 of SqDet), after the segmented split: every leaf of at
// most CAP keys is sorted in shared memory by one CTA (k_leaf).  A child still
// larger than CAP is repartitioned by one CTA (k_repart) -- the introduction of
// the paper lets split keys be sorted again with the same partitioning scheme:
// a stratified random sample of SAMPLE2 tagged keys gives p2 - 1 splitters
// (tag = position inside the segment), a counting pass and a stable scatter
// move the keys into p2 child segments in another buffer, and the children go
// to the leaf list or to the next level's list.
// Buffers: id 0 = the segmented sort's input, 1 = its output, 2 = scratch.
// Children of a level-d repartition are written to buffer 1 (d even) or 2
// (d odd); leaves always write the sorted keys to `out`.
// ---------------------------------------------------------------------------
struct SegSpec {
    const uint32_t* off;   // segment offsets [nseg + 1] (unless uniform)
    uint32_t nseg;
    uint32_t uniform;      // 1: segment k = [floor(kn/nseg), floor((k+1)n/nseg)); off unused
    uint64_t n;            // length of the array the segments tile
    uint64_t base = 0;     // off[k] - base is the offset (off[0] == base); the bucket phase only
    static SegSpec offsets(const uint32_t* o, uint32_t nseg, uint64_t n) { return SegSpec{o, nseg, 0u, n}; }
    static SegSpec offsets_at(const uint32_t* o, uint32_t nseg, uint64_t n, uint64_t base) {
        return SegSpec{o, nseg, 0u, n, base};
    }
    static SegSpec even(uint32_t nseg, uint64_t n) { return SegSpec{nullptr, nseg, 1u, n}; }
};

__device__ __forceinline__ void seg_bounds(const SegSpec& ss, uint32_t k, uint32_t& beg, uint32_t& len) {
    if (!ss.uniform) {
        beg = ss.off[k];
        len = ss.off[k + 1] - beg;
    } else {
        const uint64_t a = (uint64_t)k * ss.n / ss.nseg, b = (uint64_t)(k + 1) * ss.n / ss.nseg;
        beg = (uint32_t)a;
        len = (uint32_t)(b - a);
    }
}

template <class KT, bool HV>
struct BucketSmem {
    using O = typename KT::O;
    static constexpr int CAP = Cap<O>::v;
    static constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }
    static constexpr size_t sk_bytes = al16(sizeof(O) * padded_len<O>(CAP));
    static constexpr size_t sv_bytes = al16(sizeof(uint32_t) * padded_len<uint32_t>(CAP));
    static constexpr size_t sb_bytes = al16(sizeof(uint16_t) * CAP);
    static constexpr size_t tree_bytes = al16(split_table_bytes<O>(MAXP2 - 1, MAXP2_LBITS));
    static constexpr size_t cnt_bytes = al16(sizeof(uint16_t) * BK_WARPS * (MAXP2 + 1));
    static constexpr size_t small_bytes = sizeof(uint32_t) * (4 * (MAXP2 + 1) + 32);
    static constexpr size_t bytes = sk_bytes + sv_bytes + sb_bytes + tree_bytes + cnt_bytes + small_bytes + 64;
};

// Shared memory of one leaf sort: the exchange area of the merge sort (which
// also stages the keys) and, with a payload, the payloads in input order.
template <class KT, bool HV>
struct LeafSmem {
    using O = typename KT::O;
    using E = typename LeafElem<O, HV>::E;
    static constexpr int NT = LeafCfg<O, HV>::NT;
    static constexpr int IT = LeafCfg<O, HV>::IT;
    static constexpr int CAP = Cap<O>::v;
    static constexpr size_t ex_bytes = (sizeof(E) * padded_len<E>(CAP) + 15) & ~size_t(15);
    // 4-byte keys alone: the per-warp key minima and maxima of the narrow test
    static constexpr bool NARROW = sizeof(O) == 4 && !HV;
    // keys with a payload: the same for the packed (offset, position) test
    static constexpr bool PACK = HV;
    static constexpr size_t red_bytes = NARROW ? sizeof(uint32_t) * 2 * (NT / 32)
                                               : (PACK ? sizeof(uint64_t) * 2 * (NT / 32) : 0);
    static constexpr size_t bytes = ex_bytes + (HV ? sizeof(uint32_t) * CAP : 0) + red_bytes;
};

// Sort [beg, beg+len) of `in` (len <= CAP) into the same range of `out`.
template <class KT, bool HV>
__device__ __forceinline__ void leaf_sort(const typename KT::T* in, const uint32_t* vin, typename KT::T* out, uint32_t* vout,
                          uint32_t beg, uint32_t len, char* smem) {
    using O = typename KT::O;
    using LE = LeafElem<O, HV>;
    using E = typename LE::E;
    using LS = LeafSmem<KT, HV>;
    constexpr int IT = LS::IT, NT = LS::NT;
    E* ex = reinterpret_cast<E*>(smem);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem + LS::ex_bytes);
    E x[IT];
    const int base = threadIdx.x * IT;
    if constexpr (LS::NARROW) {
        // A leaf whose keys span at most 2^16 values sorts 16-bit offsets, two a
        // register (merge_sort_block_narrow); the test needs the key range.
        uint32_t* red = reinterpret_cast<uint32_t*>(smem + LS::ex_bytes);   // [NT/32] minima, [NT/32] maxima
        uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
        for (int j = threadIdx.x; j < (int)len; j += NT) {
            const E e = LE::make(KT::ord(in[beg + j]), (uint32_t)j);
            ex[pad_idx<E>(j)] = e;
            kmin = min(kmin, e.k);
            kmax = max(kmax, e.k);
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = kmin;
            red[NT / 32 + (threadIdx.x >> 5)] = kmax;
        }
        __syncthreads();
#pragma unroll
        for (int ww = 0; ww < NT / 32; ++ww) {
            kmin = min(kmin, red[ww]);
            kmax = max(kmax, red[NT / 32 + ww]);
        }
        const bool narrow = kmax - kmin <= 0xFFFFu && kmin <= 0xFFFF0000u;
        if (narrow) {
            narrow_register_sort<IT>(ex, (int)len, kmin);
#pragma unroll
            for (int i = 0; i < IT; ++i) x[i] = EMax<E>::v();
        } else {
#pragma unroll
            for (int i = 0; i < IT; ++i) x[i] = base + i < (int)len ? ex[pad_idx<E>(base + i)] : EMax<E>::v();
            warp_register_sort<E, IT>(x, (int)len);
        }
        merge_rounds<E, NT, IT>(x, ex, (int)len, narrow ? 16 * IT : 32 * IT, narrow);
    } else if constexpr (LS::PACK) {
        // Keys with a payload: (key, position) pairs, unique.  In a leaf whose
        // key range is narrow enough (the usual case: the keys of one leaf
        // share their high bits) the pair packs into one word,
        // (key - kmin) << PB | position, PB = log2(CAP) bits for positions,
        // which orders as the pair does: 8-byte keys spanning less than
        // 2^(64-PB) - 1 values sort 64-bit words instead of (key, position)
        // triples, 4-byte keys spanning less than 2^(32-PB) - 1 sort 32-bit
        // words on the register network instead of 64-bit pairs.  Other leaves
        // sort the pairs.
        using W = std::conditional_t<sizeof(O) == 8, uint64_t, uint32_t>;
        using EP = std::conditional_t<sizeof(O) == 8, E64, E32>;
        constexpr int PB = LS::CAP == 4096 ? 12 : 13;
        static_assert((1 << PB) == LS::CAP, "positions fill PB bits");
        constexpr W LIMIT = (W(1) << (8 * sizeof(W) - PB)) - 1;
        uint64_t* red = reinterpret_cast<uint64_t*>(smem + LS::ex_bytes + sizeof(uint32_t) * LS::CAP);
        constexpr int LD = (LS::CAP + NT - 1) / NT;       // keys a thread loads
        O kk[LD];
        uint64_t kmin = ~0ull, kmax = 0;
#pragma unroll
        for (int i = 0; i < LD; ++i) {
            const int j = threadIdx.x + i * NT;
            kk[i] = j < (int)len ? KT::ord(in[beg + j]) : O(0);
            if (j < (int)len) {
                sv[j] = vin[beg + j];
                kmin = min(kmin, (uint64_t)kk[i]);
                kmax = max(kmax, (uint64_t)kk[i]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = kmin;
            red[NT / 32 + (threadIdx.x >> 5)] = kmax;
        }
        __syncthreads();
#pragma unroll
        for (int ww = 0; ww < NT / 32; ++ww) {
            kmin = min(kmin, red[ww]);
            kmax = max(kmax, red[NT / 32 + ww]);
        }
        if (kmax - kmin < (uint64_t)LIMIT) {
            EP* exp = reinterpret_cast<EP*>(smem);
            const O omin = (O)kmin;
#pragma unroll
            for (int i = 0; i < LD; ++i) {
                const int j = threadIdx.x + i * NT;
                if (j < (int)len) exp[pad_idx<EP>(j)] = EP{(W)(((W)(kk[i] - omin) << PB) | (W)j)};
            }
            __syncthreads();
            EP y[IT];
#pragma unroll
            for (int i = 0; i < IT; ++i) y[i] = base + i < (int)len ? exp[pad_idx<EP>(base + i)] : EMax<EP>::v();
            merge_sort_block<EP, NT, IT>(y, exp, (int)len);
#pragma unroll
            for (int i = 0; i < IT; ++i)
                if (base + i < (int)len) exp[pad_idx<EP>(base + i)] = y[i];
            __syncthreads();
            for (int j = threadIdx.x; j < (int)len; j += NT) {
                const W e = exp[pad_idx<EP>(j)].k;
                out[beg + j] = KT::key((O)(omin + (O)(e >> PB)));
                vout[beg + j] = sv[(uint32_t)e & (uint32_t)(LS::CAP - 1)];
            }
            __syncthreads();
            return;
        }
#pragma unroll
        for (int i = 0; i < LD; ++i) {
            const int j = threadIdx.x + i * NT;
            if (j < (int)len) ex[pad_idx<E>(j)] = LE::make(kk[i], (uint32_t)j);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) x[i] = base + i < (int)len ? ex[pad_idx<E>(base + i)] : EMax<E>::v();
        merge_sort_block<E, NT, IT>(x, ex, (int)len);
    } else {
        for (int j = threadIdx.x; j < (int)len; j += NT) {
            ex[pad_idx<E>(j)] = LE::make(KT::ord(in[beg + j]), (uint32_t)j);
            if (HV) sv[j] = vin[beg + j];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) x[i] = base + i < (int)len ? ex[pad_idx<E>(base + i)] : EMax<E>::v();
        merge_sort_block<E, NT, IT>(x, ex, (int)len);
    }
#pragma unroll
    for (int i = 0; i < IT; ++i)
        if (base + i < (int)len) ex[pad_idx<E>(base + i)] = x[i];
    __syncthreads();
    for (int j = threadIdx.x; j < (int)len; j += NT) {
        const E y = ex[pad_idx<E>(j)];
        out[beg + j] = KT::key(LE::key(y));
        if (HV) vout[beg + j] = sv[LE::pos(y)];
    }
    __syncthreads();
}

// Repartition [beg, beg+len) of `in` into p2 children written to `outb`; child
// offsets (relative to beg) go to off[0..p2].  Returns p2.
template <class KT, bool HV>
__device__ int cta_partition(const typename KT::T* in, const uint32_t* vin, typename KT::T* outb, uint32_t* voutb,
                             uint32_t beg, uint32_t len, int level, uint64_t seed, char* smem_base,
                             uint32_t* off, uint32_t* status) {
    using O = typename KT::O;
    using T = typename KT::T;
    using L = BucketSmem<KT, HV>;
    constexpr int IT = 8;                 // keys per thread in the two passes (lower register use)
    constexpr int TILE = BK_NT * IT;
    constexpr int CAP = L::CAP;
    char* q = smem_base;
    O* sk = reinterpret_cast<O*>(q);               q += L::sk_bytes;
    uint32_t* sv = reinterpret_cast<uint32_t*>(q); q += L::sv_bytes;
    uint16_t* sb = reinterpret_cast<uint16_t*>(q); q += L::sb_bytes;
    SplitTable<O> stab;
    stab.bind(q, MAXP2 - 1, MAXP2_LBITS);             q += L::tree_bytes;
    uint16_t* cnt = reinterpret_cast<uint16_t*>(q); q += L::cnt_bytes;
    uint32_t* part = reinterpret_cast<uint32_t*>(q);     q += sizeof(uint32_t) * (MAXP2 + 1);
    uint32_t* tile_off = reinterpret_cast<uint32_t*>(q); q += sizeof(uint32_t) * (MAXP2 + 1);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(q);   q += sizeof(uint32_t) * (MAXP2 + 1);
    uint32_t* scratch = reinterpret_cast<uint32_t*>(q);

    // Fan-out: children of about 0.72 CAP on average (so that nearly all of a
    // leaf sort's threads have keys and few children overflow), at most MAXP2.
    const uint64_t want = ((uint64_t)len * 25 + 18 * (uint64_t)CAP - 1) / (18 * (uint64_t)CAP);
    const int p2 = want < 2 ? 2 : (want > (uint64_t)MAXP2 ? MAXP2 : (int)want);
    const int lbits2 = 32 - __clz(2 * p2 - 1);      // bins: the power of two >= 2 p2
    const int s2 = SAMPLE2 / p2;
    const int m2 = p2 * s2;

    // 1. Stratified random sample: one key from each of m2 near-equal strata,
    //    tagged with its position (strata are in position order, so a stable
    //    sort by key leaves the sample in tagged order).
    const uint64_t state = sm_stream(seed ^ ((uint64_t)beg * SM_GAMMA), 2 + level);
    for (int j = threadIdx.x; j < m2; j += BK_NT) {
        const uint32_t lo = (uint32_t)((uint64_t)j * len / m2);
        const uint32_t hi = (uint32_t)((uint64_t)(j + 1) * len / m2);
        uint32_t pos = lo + (uint32_t)(sm_at(state, j) % (uint64_t)max(hi - lo, 1u));
        if (pos >= len) {
            flag_bounds(status, 5, pos);
            pos = 0;
        }
        sk[pad_idx<O>(j)] = KT::ord(in[beg + pos]);
        sv[pad_idx<uint32_t>(j)] = pos;
    }
    for (int j = m2 + threadIdx.x; j < SAMPLE2; j += BK_NT) {   // pad to a full block: sorts last
        sk[pad_idx<O>(j)] = OMax<O>::v;
        sv[pad_idx<uint32_t>(j)] = 0xFFFFFFFFu;
    }
    static_assert(SAMPLE2 == BK_NT * IT, "the sample is sorted as one block of BK_NT x IT keys");
    block_merge_sort<O, true, BK_NT, IT>(sk, sv, SAMPLE2);
    for (int i = threadIdx.x + 1; i < p2; i += BK_NT)
        stab.set(i - 1, sk[pad_idx<O>(i * s2 - 1)], sv[pad_idx<uint32_t>(i * s2 - 1)]);
    for (int b = threadIdx.x; b <= p2; b += BK_NT) part[b] = 0;
    __syncthreads();
    split_table_finish<O>(stab, p2 - 1, lbits2);

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // 2. Counting pass.
    for (uint32_t tb = 0; tb < len; tb += TILE) {
        const uint32_t base = tb + w * (IT * 32) + lane;
        O o[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t e = base + i * 32;
            o[i] = e < len ? KT::ord(in[beg + e]) : O(0);
        }
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t e = base + i * 32;
            const int b = e < len ? split_find<O>(stab, o[i], e) : p2;
            warp_count((uint32_t)b, part);
        }
    }
    const uint32_t total = block_exclusive_scan(part, p2, scratch);
    for (int b = threadIdx.x; b < p2; b += BK_NT) {
        off[b] = part[b];
        cursor[b] = beg + part[b];
    }
    if (threadIdx.x == 0) off[p2] = total;
    // 3. Scatter pass (ranking as in k_scatter: stable with a payload, atomic
    //    slots for keys alone).
    const int cstride = MAXP2 + 1;
    uint16_t* mycnt = cnt + w * cstride;
    for (uint32_t tb = 0; tb < len; tb += TILE) {
        const uint32_t base = tb + w * (IT * 32) + lane;
        T kv[IT];
        uint32_t br[IT];   // bucket << 16 | rank inside the tile's part of the child
        int bk[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t e = base + i * 32;
            kv[i] = e < len ? in[beg + e] : T(0);
        }
        if (HV) {
            for (int b = lane; b <= p2; b += 32) mycnt[b] = 0;
        } else {
            for (int b = threadIdx.x; b <= p2; b += BK_NT) tile_off[b] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) bk[i] = split_find<O>(stab, KT::ord(kv[i]), base + i * 32);
        if (HV) {
            const int nbits = 32 - __clz(p2);
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const uint32_t e = base + i * 32;
                const bool valid = e < len;
                const int b = valid ? bk[i] : p2;
                const unsigned m = warp_peers((uint32_t)b, nbits);
                const uint32_t c0 = mycnt[b];
                br[i] = ((uint32_t)b << 16) | (c0 + __popc(m & lanemask_lt()));
                __syncwarp();
                if (lane == __ffs(m) - 1) mycnt[b] = (uint16_t)(c0 + __popc(m));
                __syncwarp();
            }
            __syncthreads();
            for (int b = threadIdx.x; b < p2; b += BK_NT) {
                uint32_t run = 0;
#pragma unroll
                for (int ww = 0; ww < BK_WARPS; ++ww) {
                    const uint32_t c = cnt[ww * cstride + b];
                    cnt[ww * cstride + b] = (uint16_t)run;
                    run += c;
                }
                tile_off[b] = run;
            }
        } else {
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const uint32_t e = base + i * 32;
                const uint32_t b = e < len ? (uint32_t)bk[i] : (uint32_t)p2;
                br[i] = (b << 16) | warp_slot(b, tile_off);
            }
        }
        const uint32_t tvalid = block_exclusive_scan(tile_off, p2, scratch);
        if (threadIdx.x == 0) tile_off[p2] = tvalid;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int b = (int)(br[i] >> 16);
            if (b < p2) {
                const uint32_t loc = tile_off[b] + (HV ? mycnt[b] : 0u) + (br[i] & 0xFFFFu);
                if (loc >= (uint32_t)TILE) {
                    flag_bounds(status, 9, loc);
                    continue;
                }
                sk[loc] = KT::ord(kv[i]);
                if (HV) sv[loc] = vin[beg + base + i * 32];
                sb[loc] = (uint16_t)b;
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < tvalid; j += BK_NT) {
            const int b = sb[j];
            const uint32_t dst = cursor[b] + (j - tile_off[b]);
            if (dst < beg || dst - beg >= len) {
                flag_bounds(status, 4, dst);
                continue;
            }
            outb[dst] = KT::key(sk[j]);
            if (HV) voutb[dst] = sv[j];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < p2; b += BK_NT) cursor[b] += tile_off[b + 1] - tile_off[b];
        __syncthreads();   // tile_off is cleared at the top of the next tile
    }
    return p2;
}

struct WorkItem {
    uint32_t beg, len, buf, pad;
};

template <class KT>
struct SortBufs {
    typename KT::T* k[3];
    uint32_t* v[3];
    typename KT::T* out;
    uint32_t* vout;
    // constant-index selection keeps the pointers in parameter space
    __device__ __forceinline__ typename KT::T* key_buf(uint32_t id) const { return id == 0 ? k[0] : (id == 1 ? k[1] : k[2]); }
    __device__ __forceinline__ uint32_t* val_buf(uint32_t id) const { return id == 0 ? v[0] : (id == 1 ? v[1] : v[2]); }
};

struct WorkLists {
    WorkItem* leaf;       // leaves of every level
    uint32_t leaf_cap;
    WorkItem* part[2];    // segments to repartition, alternating by level parity
    uint32_t part_cap;
    uint32_t* counts;     // [0] leaves, [1 + d] segments of level d
};

__device__ __forceinline__ void push_item(WorkItem* list, uint32_t* count, uint32_t cap, uint32_t beg, uint32_t len,
                                          uint32_t buf, uint32_t* status) {
    const uint32_t i = atomicAdd(count, 1u);
    if (i < cap) list[i] = WorkItem{beg, len, buf, 0u};
    else atomicOr(status, ERR_SIZES);
}

// Leaves of at most SMALL_CAP keys are sorted by one warp each (k_leaf_small)
// instead of a whole CTA.  They share the leaf array with the larger leaves,
// filled from its far end (count in wl.counts[SMALL_COUNT]): both kinds come
// from the same buckets and children, so together they stay within leaf_cap.
constexpr uint32_t SMALL_CAP = 256;
constexpr int SMALL_COUNT = MAX_DEPTH + 1;
constexpr int WL_COUNTS = MAX_DEPTH + 2;   // entries of wl.counts

__device__ __forceinline__ void push_leaf(const WorkLists& wl, uint32_t beg, uint32_t len, uint32_t buf,
                                          uint32_t* status) {
    if (len <= SMALL_CAP) {
        const uint32_t i = atomicAdd(&wl.counts[SMALL_COUNT], 1u);
        if (i < wl.leaf_cap) wl.leaf[wl.leaf_cap - 1 - i] = WorkItem{beg, len, buf, 0u};
        else atomicOr(status, ERR_SIZES);
    } else {
        push_item(wl.leaf, &wl.counts[0], wl.leaf_cap, beg, len, buf, status);
    }
}

// One repartition level d >= 1: walks the list filled by level d - 1 (level 1:
// by the segmented split).  Persistent: CTAs stride over the work.
template <class KT, bool HV>
__global__ void __launch_bounds__(BK_NT, 2)
k_repart(int level, SegSpec ss, SortBufs<KT> bufs, WorkLists wl, uint64_t seed, uint32_t* status,
         uint32_t* depth_max, unsigned long long* moved) {
    using O = typename KT::O;
    using L = BucketSmem<KT, HV>;
    extern __shared__ __align__(16) char smem[];
    uint32_t* off = reinterpret_cast<uint32_t*>(smem + L::bytes - sizeof(uint32_t) * (MAXP2 + 1) - 16);
    if (level < 1) return;
    const uint32_t nwork = min(wl.counts[level], wl.part_cap);
    const WorkItem* in_list = wl.part[(level - 1) & 1];
    WorkItem* next_list = wl.part[level & 1];
    const uint32_t outbuf = (level & 1) ? 2u : 1u;
    for (uint32_t it = blockIdx.x; it < nwork; it += gridDim.x) {
        const WorkItem w = in_list[it];
        const uint32_t beg = w.beg, len = w.len, inbuf = w.buf;
        if (len == 0) continue;
        if (len <= (uint32_t)L::CAP) {
            if (threadIdx.x == 0) push_leaf(wl, beg, len, inbuf, status);
            continue;
        }
        if ((uint64_t)beg + len > ss.n) {
            if (threadIdx.x == 0) flag_bounds(status, 7, (uint64_t)beg + len);
            continue;
        }
        const int p2 = cta_partition<KT, HV>(bufs.key_buf(inbuf), bufs.val_buf(inbuf), bufs.key_buf(outbuf),
                                             bufs.val_buf(outbuf), beg, len, level, seed, smem, off, status);
        if (threadIdx.x == 0) {
            atomicMax(depth_max, (uint32_t)(level + 1));
            atomicAdd(moved, (unsigned long long)len);
        }
        for (int b = threadIdx.x; b < p2; b += BK_NT) {
            const uint32_t cb = beg + off[b], cl = off[b + 1] - off[b];
            if (cl == 0) continue;
            if (cl <= (uint32_t)L::CAP) push_leaf(wl, cb, cl, outbuf, status);
            else if (level + 1 < MAX_DEPTH)
                push_item(next_list, &wl.counts[level + 1], wl.part_cap, cb, cl, outbuf, status);
            else atomicOr(status, ERR_DEPTH);
        }
        __syncthreads();
    }
}

// Shared-memory sort of every leaf: the segments of ss directly (direct = true)
// or the leaf list.  Persistent: CTAs stride over the work.
// Resident leaf CTAs per SM the register budget is sized for: 64 registers a
// thread, except 4-byte keys alone (six 128-thread CTAs, up to 85 registers).
template <class KT, bool HV> struct LeafOcc {
    static constexpr int v = (sizeof(typename KT::O) == 4 && !HV) ? 6 : 65536 / (64 * LeafCfg<typename KT::O, HV>::NT);
};

template <class KT, bool HV>
__global__ void __launch_bounds__(LeafCfg<typename KT::O, HV>::NT, LeafOcc<KT, HV>::v)
k_leaf(bool direct, SegSpec ss, SortBufs<KT> bufs, WorkLists wl, uint64_t seed, uint32_t* status) {
    using L = BucketSmem<KT, HV>;
    extern __shared__ __align__(16) char smem[];
    const uint32_t nwork = direct ? ss.nseg : min(wl.counts[0], wl.leaf_cap);
    for (uint32_t it = blockIdx.x; it < nwork; it += gridDim.x) {
        uint32_t beg, len, buf;
        if (direct) {
            seg_bounds(ss, it, beg, len);
            buf = 0;
        } else {
            const WorkItem w = wl.leaf[it];
            beg = w.beg;
            len = w.len;
            buf = w.buf;
        }
        if (len == 0) continue;
        if (len > (uint32_t)L::CAP || (uint64_t)beg + len > ss.n) {
            if (threadIdx.x == 0) flag_bounds(status, 6, (uint64_t)beg + len);
            continue;
        }
        leaf_sort<KT, HV>(bufs.key_buf(buf), bufs.val_buf(buf), bufs.out, bufs.vout, beg, len, smem);
    }
}

// Bitonic sort of a warp's 32 M elements, element m * 32 + lane in x[m] of that
// lane: exchanges across lanes by shuffles (distance below 32), within a lane
// in registers (distance 32 and above).  Ascending.
template <class E, int M>
__device__ __forceinline__ void warp_bitonic(E (&x)[M]) {
    const int lane = threadIdx.x & 31;
    constexpr int N = 32 * M;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int d = k >> 1; d > 0; d >>= 1) {
            if (d >= 32) {
                const int dm = d >> 5;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    if ((m & dm) == 0) {
                        if (((m * 32) & k) == 0) cas_up(x[m], x[m + dm]);   // k >= 64: the lane bits do not count
                        else cas_up(x[m + dm], x[m]);
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const E y = E::shfl(x[m], d);
                    const bool up = ((m * 32 + lane) & k) == 0;
                    const bool lower = (lane & d) == 0;          // the smaller index of the pair
                    const bool take_min = lower == up;
                    const bool y_less = E::lt(y, x[m]);
                    x[m] = (take_min == y_less) ? y : x[m];
                }
            }
        }
    }
}

// One leaf of at most 32 M keys sorted by the calling warp (elements made and
// read back as in leaf_sort; padding is +infinity).
template <class KT, bool HV, int M>
__device__ __forceinline__ void warp_leaf_sort(const typename KT::T* in, const uint32_t* vin, typename KT::T* out,
                                               uint32_t* vout, uint32_t beg, uint32_t len) {
    using LE = LeafElem<typename KT::O, HV>;
    using E = typename LE::E;
    const uint32_t lane = threadIdx.x & 31;
    E x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const uint32_t i = m * 32 + lane;
        x[m] = i < len ? LE::make(KT::ord(in[beg + i]), i) : EMax<E>::v();
    }
    warp_bitonic<E, M>(x);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const uint32_t i = m * 32 + lane;
        if (i < len) {
            out[beg + i] = KT::key(LE::key(x[m]));
            if (HV) vout[beg + i] = vin[beg + LE::pos(x[m])];
        }
    }
}

// The small leaves (at most SMALL_CAP keys), one warp each, from the far end
// of the leaf array.  Persistent: warps stride over the items.
constexpr int SMALL_NT = 256;
template <class KT, bool HV>
__global__ void __launch_bounds__(SMALL_NT)
k_leaf_small(SortBufs<KT> bufs, WorkLists wl, uint64_t n, uint32_t* status) {
    const uint32_t nfront = min(wl.counts[0], wl.leaf_cap);
    const uint32_t nsmall = min(wl.counts[SMALL_COUNT], wl.leaf_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (uint64_t)nfront + nsmall > wl.leaf_cap) atomicOr(status, ERR_SIZES);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (SMALL_NT / 32);
    for (uint32_t it = blockIdx.x * (SMALL_NT / 32) + (threadIdx.x >> 5); it < nsmall; it += warps) {
        const WorkItem w = wl.leaf[wl.leaf_cap - 1 - it];
        if (w.len == 0) continue;
        if (w.len > SMALL_CAP || (uint64_t)w.beg + w.len > n) {
            if (lane == 0) flag_bounds(status, 14, (uint64_t)w.beg + w.len);
            continue;
        }
        const typename KT::T* in = bufs.key_buf(w.buf);
        const uint32_t* vin = bufs.val_buf(w.buf);
        if (w.len <= 32) warp_leaf_sort<KT, HV, 1>(in, vin, bufs.out, bufs.vout, w.beg, w.len);
        else if (w.len <= 64) warp_leaf_sort<KT, HV, 2>(in, vin, bufs.out, bufs.vout, w.beg, w.len);
        else if (w.len <= 128) warp_leaf_sort<KT, HV, 4>(in, vin, bufs.out, bufs.vout, w.beg, w.len);
        else warp_leaf_sort<KT, HV, 8>(in, vin, bufs.out, bufs.vout, w.beg, w.len);
    }
}

}  // namespace ossort
