// Kernels of the segmented sort: many independent arrays (segments of one
// buffer) sorted by one fixed sequence of persistent kernels, each of which
// walks the whole segment table.  Used by the batched entry point and by the
// bucket phase of every sort (the buckets are the segments).  Every segment g is sorted exactly as SqRan (Algorithm 2,
// sample on original positions) sorts it alone with the parameters of its length
// class and the seed u(seed, 2, g):
//
//   k_seg_plan       per segment: class, p_g, s_g, tiles; exclusive scans of
//                    tiles, buckets and histogram entries (one CTA)
//   k_seg_splitters  step 2-3 per segment: p_g s_g - 1 random positions, the
//                    tagged sample sorted in shared memory, p_g - 1 splitters
//   k_seg_classify   step 4: bucket of every key of every partitioned segment,
//                    per-tile bucket counts
//   k_seg_scan       per segment: bucket-major scan of its tile counts, bucket
//                    sizes, and the work items of step 5
//   k_seg_scatter    step 4: keys (and payloads) into contiguous buckets
//   k_repart/k_leaf  step 5 (kernels.cuh): every bucket, and every segment too
//                    small to sample, sorted through the shared work lists
//
// A segment whose class has p = 1, or that is shorter than 2 p s (the small-n
// rule of the plain sort), is one unit of step 5.  The host only knows n, the
// number of segments and the class table, so the launch sequence does not
// depend on the segment lengths: it can be captured once in a CUDA graph and
// replayed for new keys and new offsets of the same totals.
#pragma once

#include "kernels.cuh"

namespace ossort {

constexpr int SEG_NT = 256;                 // threads of classify / scatter
constexpr int SEG_WARPS = SEG_NT / 32;
constexpr int SEG_IT = 8;                   // keys per thread per sub-tile
constexpr int SEG_SUB = SEG_NT * SEG_IT;    // 2048 keys: tiles are multiples of this
constexpr int SEG_SPL_NT = 512;             // threads of the per-segment sample sort
constexpr int SEG_SPL_IT = 8;
constexpr int SEG_SAMPLE = SEG_SPL_NT * SEG_SPL_IT;   // largest p s (the sample is p s - 1)
constexpr int SEG_MAX_CLASSES = 32;
constexpr int SEG_SCAN_NT = 256;
constexpr int SEG_SCAN_CHUNK = 4096;
constexpr uint32_t ERR_SEGS = 16u;          // segment offsets not non-decreasing from 0 to n

struct SegClass {
    uint64_t max_len;
    uint32_t p, s, tile, pad;
};
// Length classes.  With auto_child > 0 every segment longer than c[0].max_len
// instead gets p = clamp(ceil(len / auto_child), 2, auto_pmax) and the largest
// s <= auto_s with p s <= SEG_SAMPLE and 2 p s <= len (the bucket phase of a
// sort: children of about auto_child keys, and every segment above the cutoff
// partitioned, as auto_child >= 2 makes 2 p s <= len reachable with s = 1).
struct SegClasses {
    SegClass c[SEG_MAX_CLASSES];
    uint32_t n;
    uint32_t auto_child, auto_pmax, auto_s;
};

constexpr uint32_t SEG_MAX_TILES = 256;     // tiles of one segment at most (larger tiles beyond)

// Per-segment plan written by k_seg_plan.
struct SegRec {
    uint32_t beg, len;
    uint32_t p, s;       // p == 1: not partitioned (one unit of step 5)
    uint32_t tile;       // keys per tile
    uint32_t ntile;      // tiles (0 when p == 1)
    uint32_t bkt0;       // first bucket of the segment in the bucket arrays
    uint32_t hist0;      // first entry of its bucket-major tile-count matrix
    uint64_t seed;       // seed of its sample
};

struct SegTotals {
    uint32_t tiles, buckets, hist, ok;
    uint32_t nparts;     // segments with p > 1, listed (in no particular order) in the plan's pseg array
};

constexpr uint32_t SEG_PLAN_MAXB = 1024;    // most CTAs of the plan (one thread each in its block scan)

// Where segment g starts: a 64-bit or 32-bit offset array of nseg + 1 entries,
// or (neither given) the even split floor(g n / nseg).
struct SegSource {
    const uint64_t* off64;
    const uint32_t* off32;
    uint32_t nseg;
    uint64_t n;
    uint64_t base = 0;   // subtracted from the given offsets (a range of a larger table)
    __device__ __forceinline__ uint64_t at(uint32_t g) const {
        if (off64) return off64[g] - base;
        if (off32) return off32[g] - base;
        return (uint64_t)g * n / nseg;
    }
};

__device__ __forceinline__ int seg_lbits(int p) {
    int b = 1;
    while ((1 << b) < 2 * p && b < 13) ++b;
    return b;
}

// Segment owning global tile t: the last g with tile0[g] <= t (tile0 has nseg+1
// non-decreasing entries, tile0[0] = 0 <= t < tile0[nseg]).
__device__ __forceinline__ uint32_t seg_of_tile(const uint32_t* tile0, uint32_t nseg, uint32_t t) {
    uint32_t lo = 0, hi = nseg;          // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tile0[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Inclusive warp scan of a 64-bit value.
__device__ __forceinline__ uint64_t warp_incl_u64(uint64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// ---------------------------------------------------------------------------
// Plan: every CTA of 1024 threads walks its range of `chunk` segments 1024 at a
// time, with offsets relative to the range, and lists the partitioned segments
// in pseg.  One CTA (blk == nullptr) writes the totals itself; with more, each
// CTA leaves its three sums in blk for k_seg_plan_scan and k_seg_plan_apply.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024)
k_seg_plan(SegSource src, SegClasses cls, uint64_t seed, SegRec* __restrict__ rec, uint32_t* __restrict__ tile0,
           SegTotals* __restrict__ tot, uint64_t tile_cap, uint64_t bkt_cap, uint64_t hist_cap, uint32_t chunk,
           uint64_t* __restrict__ blk, uint32_t* __restrict__ pseg, uint32_t* status) {
    const uint32_t nseg = src.nseg;
    const uint64_t n = src.n;
    __shared__ uint64_t wsum[3][32];
    __shared__ uint64_t carry[3];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid < 3) carry[tid] = 0;
    const uint64_t state = sm_stream(seed, 2);
    if (blockIdx.x == 0 && tid == 0 && nseg > 0 && (src.at(0) != 0 || src.at(nseg) != n)) atomicOr(status, ERR_SEGS);
    const uint32_t g0 = blockIdx.x * chunk;
    const uint32_t g1 = (uint64_t)g0 + chunk < nseg ? g0 + chunk : nseg;
    __syncthreads();
    for (uint32_t base = g0; base < g1; base += 1024) {
        const uint32_t g = base + tid;
        uint64_t v[3] = {0, 0, 0};
        SegRec r{};
        if (g < g1) {
            uint64_t a = src.at(g), b = src.at(g + 1);
            if (a > b || b > n) {
                atomicOr(status, ERR_SEGS);
                a = a > n ? n : a;
                b = a;
            }
            r.beg = (uint32_t)a;
            r.len = (uint32_t)(b - a);
            uint32_t k = 0;
            while (k + 1 < cls.n && (uint64_t)r.len > cls.c[k].max_len) ++k;
            r.p = cls.c[k].p;
            r.s = cls.c[k].s;
            r.tile = cls.c[k].tile;
            if (cls.auto_child && (uint64_t)r.len > cls.c[0].max_len) {
                const uint32_t want = (r.len + cls.auto_child - 1) / cls.auto_child;
                r.p = want < 2 ? 2 : (want > cls.auto_pmax ? cls.auto_pmax : want);
                r.s = cls.auto_s;
                while (r.s > 1 && ((uint64_t)r.p * r.s > (uint64_t)SEG_SAMPLE || 2ull * r.p * r.s > r.len)) --r.s;
                r.tile = cls.c[0].tile;
            }
            if (r.p > 1 && (uint64_t)r.len < 2ull * r.p * r.s) r.p = 1;   // too small to sample
            if (r.p > 1 && (r.len + r.tile - 1) / r.tile > SEG_MAX_TILES)   // long segment: larger tiles
                r.tile = ((r.len + SEG_MAX_TILES - 1) / SEG_MAX_TILES + SEG_SUB - 1) / SEG_SUB * SEG_SUB;
            r.ntile = r.p > 1 ? (r.len + r.tile - 1) / r.tile : 0;
            r.seed = sm_at(state, g);
            v[0] = r.ntile;
            v[1] = r.p;
            v[2] = (uint64_t)r.p * r.ntile;
        }
        uint64_t incl[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            incl[q] = warp_incl_u64(v[q]);
            if (lane == 31) wsum[q][w] = incl[q];
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const uint64_t x = warp_incl_u64(wsum[q][lane]);
                wsum[q][lane] = x;
            }
        }
        __syncthreads();
        uint64_t ex[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) ex[q] = carry[q] + incl[q] - v[q] + (w > 0 ? wsum[q][w - 1] : 0);
        if (g < g1) {
            r.bkt0 = (uint32_t)ex[1];
            r.hist0 = (uint32_t)ex[2];
            rec[g] = r;
            tile0[g] = (uint32_t)ex[0];
        }
        // the partitioned segments into pseg (one atomic per warp)
        const bool part = g < g1 && r.p > 1;
        const unsigned pm = __ballot_sync(0xffffffffu, part);
        if (pm) {
            uint32_t at = 0;
            if (lane == __ffs(pm) - 1) at = atomicAdd(&tot->nparts, (uint32_t)__popc(pm));
            at = __shfl_sync(0xffffffffu, at, __ffs(pm) - 1);
            if (part) pseg[at + __popc(pm & lanemask_lt())] = g;
        }
        __syncthreads();
        if (tid < 3) carry[tid] += wsum[tid][31];
        __syncthreads();
    }
    if (blk) {
        if (tid < 3) blk[3 * (size_t)blockIdx.x + tid] = carry[tid];
        return;
    }
    if (tid == 0) {
        const bool ok = carry[0] <= tile_cap && carry[1] <= bkt_cap && carry[2] <= hist_cap;
        if (!ok) atomicOr(status, ERR_SIZES);
        tile0[nseg] = ok ? (uint32_t)carry[0] : 0u;
        tot->tiles = ok ? (uint32_t)carry[0] : 0u;
        tot->buckets = ok ? (uint32_t)carry[1] : 0u;
        tot->hist = ok ? (uint32_t)carry[2] : 0u;
        tot->ok = ok ? 1u : 0u;
    }
}

// Plan with several CTAs: exclusive scan of the CTAs' sums (in place in blk)
// and the totals.  One CTA of SEG_PLAN_MAXB threads.
static __global__ void __launch_bounds__(SEG_PLAN_MAXB)
k_seg_plan_scan(uint64_t* __restrict__ blk, uint32_t nblk, uint32_t nseg, uint32_t* __restrict__ tile0,
                SegTotals* __restrict__ tot, uint64_t tile_cap, uint64_t bkt_cap, uint64_t hist_cap, uint32_t* status) {
    __shared__ uint64_t wsum[3][32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint64_t v[3], incl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        v[q] = (uint32_t)tid < nblk ? blk[3 * (size_t)tid + q] : 0;
        incl[q] = warp_incl_u64(v[q]);
        if (lane == 31) wsum[q][w] = incl[q];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) wsum[q][lane] = warp_incl_u64(lane < (SEG_PLAN_MAXB / 32) ? wsum[q][lane] : 0);
    }
    __syncthreads();
    if ((uint32_t)tid < nblk) {
#pragma unroll
        for (int q = 0; q < 3; ++q) blk[3 * (size_t)tid + q] = incl[q] - v[q] + (w > 0 ? wsum[q][w - 1] : 0);
    }
    if (tid == 0) {
        const uint64_t t0 = wsum[0][31], t1 = wsum[1][31], t2 = wsum[2][31];
        const bool ok = t0 <= tile_cap && t1 <= bkt_cap && t2 <= hist_cap;
        if (!ok) atomicOr(status, ERR_SIZES);
        tile0[nseg] = ok ? (uint32_t)t0 : 0u;
        tot->tiles = ok ? (uint32_t)t0 : 0u;
        tot->buckets = ok ? (uint32_t)t1 : 0u;
        tot->hist = ok ? (uint32_t)t2 : 0u;
        tot->ok = ok ? 1u : 0u;
    }
}

// Plan with several CTAs: every CTA adds its range's scanned offsets.
static __global__ void __launch_bounds__(1024)
k_seg_plan_apply(SegRec* __restrict__ rec, uint32_t* __restrict__ tile0, uint32_t nseg, uint32_t chunk,
                 const uint64_t* __restrict__ blk, const SegTotals* __restrict__ tot) {
    if (!tot->ok) return;
    const uint32_t g0 = blockIdx.x * chunk;
    const uint32_t g1 = (uint64_t)g0 + chunk < nseg ? g0 + chunk : nseg;
    const uint32_t o_t = (uint32_t)blk[3 * (size_t)blockIdx.x], o_b = (uint32_t)blk[3 * (size_t)blockIdx.x + 1],
                   o_h = (uint32_t)blk[3 * (size_t)blockIdx.x + 2];
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        rec[g].bkt0 += o_b;
        rec[g].hist0 += o_h;
        tile0[g] += o_t;
    }
}

// ---------------------------------------------------------------------------
// Steps 2-3 per segment: positions floor(u_j len / 2^64) for j < p s - 1 from
// stream 1 of the segment's seed, the tagged sample (key, position) sorted in
// shared memory, splitter i at rank i s - 1.  One CTA per segment.
// ---------------------------------------------------------------------------
template <class KT>
__global__ void __launch_bounds__(SEG_SPL_NT)
k_seg_splitters(const typename KT::T* __restrict__ keys, const SegRec* __restrict__ rec, const uint32_t* __restrict__ pseg,
                const SegTotals* __restrict__ tot, typename KT::O* __restrict__ spl_o,
                uint32_t* __restrict__ spl_t, uint32_t* status) {
    using O = typename KT::O;
    using LE = LeafElem<O, true>;
    using E = typename LE::E;
    extern __shared__ __align__(16) char smem[];
    E* ex = reinterpret_cast<E*>(smem);
    if (!tot->ok) return;
    const uint32_t nparts = tot->nparts;
    for (uint32_t i = blockIdx.x; i < nparts; i += gridDim.x) {
        const uint32_t g = pseg[i];
        const SegRec r = rec[g];
        if (r.p < 2) continue;
        const uint32_t m = r.p * r.s - 1;
        if (m > (uint32_t)SEG_SAMPLE) {
            if (threadIdx.x == 0) atomicOr(status, ERR_SAMPLE);
            continue;
        }
        const uint64_t state = sm_stream(r.seed, 1);
        E x[SEG_SPL_IT];
        const int base = threadIdx.x * SEG_SPL_IT;
#pragma unroll
        for (int i = 0; i < SEG_SPL_IT; ++i) {
            const uint32_t j = base + i;
            if (j < m) {
                const uint32_t pos = (uint32_t)__umul64hi(sm_at(state, j), (uint64_t)r.len);
                x[i] = LE::make(KT::ord(keys[r.beg + pos]), pos);
            } else {
                x[i] = EMax<E>::v();
            }
        }
        merge_sort_block<E, SEG_SPL_NT, SEG_SPL_IT>(x, ex, (int)m);
#pragma unroll
        for (int i = 0; i < SEG_SPL_IT; ++i) {
            const uint32_t q = base + i + 1;          // rank + 1
            if (q <= m && q % r.s == 0) {
                const uint32_t k = q / r.s;           // splitter k (1 .. p-1)
                spl_o[r.bkt0 + k - 1] = LE::key(x[i]);
                spl_t[r.bkt0 + k - 1] = LE::pos(x[i]);
            }
        }
    }
}

template <class KT>
size_t seg_classify_smem(int maxp) {
    int lb = 1;
    while ((1 << lb) < 2 * maxp && lb < 13) ++lb;
    return split_table_bytes<typename KT::O>(maxp, lb) + sizeof(uint32_t) * (maxp + 1);
}

// ---------------------------------------------------------------------------
// Step 4, pass 1: every CTA owns a contiguous run of the global tiles; a tile
// lies inside one segment.  The splitter table is rebuilt when the segment
// changes.  Counts go to hist[hist0 + b * ntile + tile-in-segment].
// ---------------------------------------------------------------------------
template <class KT>
__global__ void __launch_bounds__(SEG_NT, 3)
k_seg_classify(const typename KT::T* __restrict__ keys, const SegRec* __restrict__ rec,
               const uint32_t* __restrict__ tile0, uint32_t nseg, const SegTotals* __restrict__ tot,
               const typename KT::O* __restrict__ spl_o, const uint32_t* __restrict__ spl_t, int maxp,
               uint32_t* __restrict__ hist, uint16_t* __restrict__ bid) {
    using O = typename KT::O;
    extern __shared__ __align__(16) char smem[];
    int maxlb = 1;
    while ((1 << maxlb) < 2 * maxp && maxlb < 13) ++maxlb;
    SplitTable<O> tb;
    tb.bind(smem, maxp, maxlb);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + split_table_bytes<O>(maxp, maxlb));   // [maxp + 1]
    const uint32_t T = tot->tiles;
    const uint32_t t0 = tile_lo(blockIdx.x, gridDim.x, T), t1 = tile_lo(blockIdx.x + 1, gridDim.x, T);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SegRec r{};
    uint32_t seg_t0 = 0, seg_t1 = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        if (t >= seg_t1 || t < seg_t0) {
            const uint32_t g = seg_of_tile(tile0, nseg, t);
            r = rec[g];
            seg_t0 = tile0[g];
            seg_t1 = tile0[g + 1];
            __syncthreads();                              // the previous table is no longer read
            for (int i = threadIdx.x; i < (int)r.p - 1; i += SEG_NT)
                tb.set(i, spl_o[r.bkt0 + i], spl_t[r.bkt0 + i]);
            __syncthreads();
            split_table_finish<O>(tb, (int)r.p - 1, seg_lbits((int)r.p));
        }
        const int p = (int)r.p;
        const uint32_t tl = t - seg_t0;
        for (int b = threadIdx.x; b <= p; b += SEG_NT) cnt[b] = 0;
        __syncthreads();
        constexpr int CIT = SEG_IT;                        // (16 a thread measured slower: registers)
        const uint32_t tend = min(r.len, (tl + 1) * r.tile);
        for (uint32_t sub = 0; sub < r.tile; sub += SEG_NT * CIT) {
            const uint32_t lbase = tl * r.tile + sub;
            if (lbase >= tend) break;
            const uint32_t base = lbase + w * (CIT * 32) + lane;
            O o[CIT];
#pragma unroll
            for (int i = 0; i < CIT; ++i) {
                const uint32_t e = base + i * 32;
                o[i] = e < tend ? KT::ord(keys[r.beg + e]) : O(0);
            }
#pragma unroll
            for (int i = 0; i < CIT; ++i) {
                const uint32_t e = base + i * 32;
                int b = p;                                  // past the end: a spare counter
                if (e < tend) {
                    b = split_find<O, true>(tb, o[i], e);
                    bid[r.beg + e] = (uint16_t)b;
                }
                warp_count((uint32_t)b, cnt);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < p; b += SEG_NT) hist[r.hist0 + (size_t)b * r.ntile + tl] = cnt[b];
        __syncthreads();
    }
}

__device__ __forceinline__ void seg_push(const WorkLists& wl, uint32_t beg, uint32_t len, uint32_t buf, uint32_t cap,
                                         uint32_t* status) {
    if (len <= cap) push_leaf(wl, beg, len, buf, status);
    else push_item(wl.part[0], &wl.counts[1], wl.part_cap, beg, len, buf, status);
}

// seg_push for a whole warp (every lane calls; lanes with act push one item):
// one atomic per list per warp.
__device__ __forceinline__ void seg_push_warp(const WorkLists& wl, bool act, uint32_t beg, uint32_t len, uint32_t buf,
                                              uint32_t cap, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int kind = !act ? 0 : (len <= SMALL_CAP ? 1 : (len <= cap ? 2 : 3));
#pragma unroll
    for (int kk = 1; kk <= 3; ++kk) {
        const unsigned m = __ballot_sync(0xffffffffu, kind == kk);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        uint32_t* cnt = kk == 1 ? &wl.counts[SMALL_COUNT] : (kk == 2 ? &wl.counts[0] : &wl.counts[1]);
        uint32_t at = 0;
        if (lane == leader) at = atomicAdd(cnt, (uint32_t)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (kind == kk) {
            const uint32_t i = at + __popc(m & lanemask_lt());
            const WorkItem it{beg, len, buf, 0u};
            if (kk == 3) {
                if (i < wl.part_cap) wl.part[0][i] = it;
                else atomicOr(status, ERR_SIZES);
            } else if (i < wl.leaf_cap) {
                wl.leaf[kk == 1 ? wl.leaf_cap - 1 - i : i] = it;
            } else {
                atomicOr(status, ERR_SIZES);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Per segment: exclusive bucket-major scan of its tile counts (in place: entry
// (b, t) becomes the offset of tile t's keys of bucket b inside the segment),
// bucket sizes, and the step-5 work items: every non-empty bucket (in buffer
// 1, where the scatter puts it), or the whole segment (buffer 0, the input)
// when it is not partitioned.  cap: the leaf capacity.  src_is_alt: buffer 0
// is also the scratch of the deeper repartition levels, so an unpartitioned
// segment must fit a leaf (the class tables of the bucket phase guarantee it).
// moved / depth_max: keys partitioned here and the repartition depth reached.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(SEG_SCAN_NT)
k_seg_scan(const SegRec* __restrict__ rec, uint32_t nseg, const uint32_t* __restrict__ pseg,
           const SegTotals* __restrict__ tot, uint32_t* hist, uint32_t* __restrict__ bsize, WorkLists wl, uint32_t cap,
           uint32_t src_is_alt, uint32_t* status, uint32_t* depth_max, unsigned long long* moved) {
    __shared__ uint32_t buf[SEG_SCAN_CHUNK];
    __shared__ uint32_t scratch[32];
    if (!tot->ok) return;
    // segments kept whole: one a thread
    const uint32_t nthreads = gridDim.x * SEG_SCAN_NT;
    for (uint32_t g0 = blockIdx.x * SEG_SCAN_NT; g0 < nseg; g0 += nthreads) {
        const uint32_t g = g0 + threadIdx.x;
        bool act = false;
        uint32_t beg = 0, len = 0;
        if (g < nseg) {
            const SegRec r = rec[g];
            if (r.p < 2) {
                bsize[r.bkt0] = r.len;
                if (src_is_alt && r.len > cap) atomicOr(status, ERR_SIZES);
                else if (r.len > 0) {
                    act = true;
                    beg = r.beg;
                    len = r.len;
                }
            }
        }
        seg_push_warp(wl, act, beg, len, 0u, cap, status);
    }
    // partitioned segments: one a CTA
    const uint32_t nparts = tot->nparts;
    for (uint32_t i = blockIdx.x; i < nparts; i += gridDim.x) {
        const uint32_t g = pseg[i];
        const SegRec r = rec[g];
        if (r.p < 2) continue;
        if (threadIdx.x == 0) {
            atomicMax(depth_max, 1u);
            atomicAdd(moved, (unsigned long long)r.len);
        }
        const uint32_t M = r.p * r.ntile;
        uint32_t* h = hist + r.hist0;
        uint32_t carry = 0;
        for (uint32_t c0 = 0; c0 < M; c0 += SEG_SCAN_CHUNK) {
            const int len = (int)min((uint32_t)SEG_SCAN_CHUNK, M - c0);
            for (int i = threadIdx.x; i < len; i += SEG_SCAN_NT) buf[i] = h[c0 + i];
            const uint32_t t = block_exclusive_scan(buf, len, scratch);
            for (int i = threadIdx.x; i < len; i += SEG_SCAN_NT) h[c0 + i] = buf[i] + carry;
            carry += t;
            __syncthreads();
        }
        if (carry != r.len) {
            if (threadIdx.x == 0) atomicOr(status, ERR_SIZES);
            continue;
        }
        for (uint32_t b = threadIdx.x; b < r.p; b += SEG_SCAN_NT) {
            const uint32_t a = h[(size_t)b * r.ntile];
            const uint32_t z = b + 1 < r.p ? h[(size_t)(b + 1) * r.ntile] : r.len;
            bsize[r.bkt0 + b] = z - a;
            if (z > a) seg_push(wl, r.beg + a, z - a, 1u, cap, status);
        }
        __syncthreads();
    }
}

// Scatter staging: 256 threads stage 16 4-byte keys or 8 8-byte keys each at a
// time (measured on GB300 against 512 threads and the other key counts).
template <class T, bool HV> struct SegScatterCfg {
    static constexpr int NT = SEG_NT;
    static constexpr int IT = sizeof(T) == 4 ? 2 * SEG_IT : SEG_IT;
    static constexpr int WARPS = NT / 32;
    static constexpr int SUB = NT * IT;
};

template <class KT, bool HV>
size_t seg_scatter_smem(int maxp) {
    using T = typename KT::T;
    using SC = SegScatterCfg<T, HV>;
    size_t b = sizeof(T) * SC::SUB + (HV ? sizeof(uint32_t) * SC::SUB : 0);
    b += sizeof(uint32_t) * (maxp + 1) + sizeof(uint32_t) * maxp + sizeof(uint32_t) * 32;
    b += sizeof(uint16_t) * SC::SUB + (HV ? sizeof(uint16_t) * SC::WARPS * (maxp + 1) : 0);
    return b;
}

// ---------------------------------------------------------------------------
// Step 4, pass 2: the tiles again; each tile starts its buckets' cursors at the
// scanned offsets and moves its keys sub-tile by sub-tile, ranked as in
// k_scatter (stable with a payload).  Output buffer: out.
// ---------------------------------------------------------------------------
template <class KT, bool HV>
__global__ void __launch_bounds__(SegScatterCfg<typename KT::T, HV>::NT, 4)
k_seg_scatter(const typename KT::T* __restrict__ keys, const uint32_t* __restrict__ vals,
              const uint16_t* __restrict__ bid, const SegRec* __restrict__ rec, const uint32_t* __restrict__ tile0,
              uint32_t nseg, const SegTotals* __restrict__ tot, const uint32_t* __restrict__ col, int maxp,
              typename KT::T* __restrict__ out, uint32_t* __restrict__ vout, uint32_t* status) {
    using T = typename KT::T;
    using SC = SegScatterCfg<T, HV>;
    constexpr int SNT = SC::NT, SWARPS = SC::WARPS, SUB = SC::SUB, IT = SC::IT;
    extern __shared__ __align__(16) char smem[];
    char* q = smem;
    T* sk = reinterpret_cast<T*>(q);                     q += sizeof(T) * SUB;
    uint32_t* sv = reinterpret_cast<uint32_t*>(q);       q += HV ? sizeof(uint32_t) * SUB : 0;
    uint32_t* tile_off = reinterpret_cast<uint32_t*>(q); q += sizeof(uint32_t) * (maxp + 1);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(q);   q += sizeof(uint32_t) * maxp;
    uint32_t* scratch = reinterpret_cast<uint32_t*>(q);  q += sizeof(uint32_t) * 32;
    uint16_t* sb = reinterpret_cast<uint16_t*>(q);       q += sizeof(uint16_t) * SUB;
    uint16_t* cnt = reinterpret_cast<uint16_t*>(q);      // HV: [SWARPS][p + 1]

    const uint32_t T_ = tot->tiles;
    const uint32_t t0 = tile_lo(blockIdx.x, gridDim.x, T_), t1 = tile_lo(blockIdx.x + 1, gridDim.x, T_);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SegRec r{};
    uint32_t seg_t0 = 0, seg_t1 = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        if (t >= seg_t1 || t < seg_t0) {
            const uint32_t g = seg_of_tile(tile0, nseg, t);
            r = rec[g];
            seg_t0 = tile0[g];
            seg_t1 = tile0[g + 1];
        }
        const int p = (int)r.p;
        const int cstride = p + 1;
        uint16_t* mycnt = cnt + w * cstride;
        const uint32_t tl = t - seg_t0;
        const uint32_t seg_end = r.beg + r.len;
        __syncthreads();                                  // previous tile's cursors are no longer read
        for (int b = threadIdx.x; b < p; b += SNT) cursor[b] = r.beg + col[r.hist0 + (size_t)b * r.ntile + tl];
        const uint32_t tend = min(r.len, (tl + 1) * r.tile);   // end of this tile inside the segment
        for (uint32_t sub = 0; sub < r.tile; sub += SUB) {
            const uint32_t lbase = tl * r.tile + sub;
            if (lbase >= tend) break;
            const uint32_t base = lbase + w * (IT * 32) + lane;
            T kv[IT];
            uint32_t br[IT];   // bucket << 16 | rank inside the sub-tile's part of the bucket
            uint32_t vv[HV ? IT : 1];   // payloads loaded with the keys (their latency overlaps the ranking)
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const uint32_t e = base + i * 32;
                kv[i] = e < tend ? keys[r.beg + e] : T(0);
                br[i] = e < tend ? (uint32_t)bid[r.beg + e] : (uint32_t)p;
                if constexpr (HV) vv[i] = e < tend ? vals[r.beg + e] : 0u;
            }
            if (HV) {
                for (int b = lane; b <= p; b += 32) mycnt[b] = 0;
            } else {
                for (int b = threadIdx.x; b <= p; b += SNT) tile_off[b] = 0;
            }
            __syncthreads();
            if (HV) {
                const int nbits = 32 - __clz(p);
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const int b = (int)br[i];
                    const unsigned m = warp_peers((uint32_t)b, nbits);
                    const uint32_t c0 = mycnt[b];
                    br[i] = ((uint32_t)b << 16) | (c0 + __popc(m & lanemask_lt()));
                    __syncwarp();
                    if (lane == __ffs(m) - 1) mycnt[b] = (uint16_t)(c0 + __popc(m));
                    __syncwarp();
                }
                __syncthreads();
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
                // Slots from shared-memory atomics, one per key; a warp whose lanes
                // each see one bucket from their first key to their last (sorted or
                // duplicate-heavy input, where one counter would take up to 32
                // atomics at once) takes one atomic per run of lanes with the same
                // bucket instead.  Either form is exact; the test only picks the
                // faster (measured: uniform int32 0.97 -> 0.79 ms, all-equal and
                // 32-value inputs unchanged).
                if (__all_sync(0xffffffffu, br[0] == br[IT - 1])) {
#pragma unroll
                    for (int i = 0; i < IT; ++i) {
                        const uint32_t b = br[i];
                        br[i] = (b << 16) | warp_slot(b, tile_off);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < IT; ++i) {
                        const uint32_t b = br[i];
                        br[i] = (b << 16) | atomicAdd(&tile_off[b], 1u);
                    }
                }
            }
            const uint32_t tvalid = block_exclusive_scan(tile_off, p, scratch);
            if (threadIdx.x == 0) tile_off[p] = tvalid;
            // cursor[b] becomes the offset of staged index j's destination: dst =
            // cursor[b] + j (restored below, by the thread that owns b)
            for (int b = threadIdx.x; b < p; b += SNT) cursor[b] -= tile_off[b];
            // range checks predicate the accesses; a failed one is reported once
            // per thread after the write-out (no branch per key)
            uint32_t bad_site = 0, bad_at = 0;
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int b = (int)(br[i] >> 16);
                if (HV) {
                    if (b < p) {
                        const uint32_t loc = tile_off[b] + mycnt[b] + (br[i] & 0xFFFFu);
                        if (loc >= (uint32_t)SUB) {
                            flag_bounds(status, 10, loc);
                            continue;
                        }
                        sk[loc] = kv[i];
                        sv[loc] = vv[i];
                        sb[loc] = (uint16_t)b;
                    }
                } else {
                    const uint32_t loc = tile_off[min(b, p)] + (br[i] & 0xFFFFu);
                    const bool real = b < p, ok = real && loc < (uint32_t)SUB;
                    if (ok) {
                        sk[loc] = kv[i];
                        sb[loc] = (uint16_t)b;
                    }
                    if (real && !ok) bad_site = 10, bad_at = loc;
                }
            }
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < tvalid; j += SNT) {
                const int b = sb[j];                       // >= p: a slot no key was staged to
                const int bc = min(b, p - 1);              // cursor holds p entries
                const uint32_t dst = cursor[bc] + j;
                const bool ok = b < p && dst >= r.beg && dst < seg_end;
                if (ok) {
                    out[dst] = sk[j];
                    if (HV) vout[dst] = sv[j];
                }
                if (!ok) bad_site = 11, bad_at = dst;
            }
            if (bad_site) flag_bounds(status, bad_site, bad_at);
            __syncthreads();
            for (int b = threadIdx.x; b < p; b += SNT) cursor[b] += tile_off[b + 1];
            __syncthreads();
        }
    }
}

// Statistics: first bucket of every segment, and the splitters as keys.
template <class KT>
__global__ void k_seg_export(const SegRec* __restrict__ rec, uint32_t nseg, const SegTotals* __restrict__ tot,
                             const typename KT::O* __restrict__ spl_o, const uint32_t* __restrict__ spl_t,
                             const uint32_t* __restrict__ bsize, uint64_t cap, uint32_t* bucket_base,
                             uint32_t* bucket_sizes, typename KT::T* spl_keys, uint32_t* spl_tags) {
    const uint32_t nb = tot->buckets;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (bucket_base) {
        for (uint64_t g = i0; g <= nseg; g += stride) bucket_base[g] = g < nseg ? rec[g].bkt0 : nb;
    }
    for (uint64_t b = i0; b < nb && b < cap; b += stride) {
        if (bucket_sizes) bucket_sizes[b] = bsize[b];
    }
    // splitters: segment g's p - 1 splitters sit at [bkt0, bkt0 + p - 1)
    for (uint64_t g = i0; g < nseg; g += stride) {
        const SegRec r = rec[g];
        for (uint32_t k = 0; k + 1 < r.p && r.bkt0 + k < cap; ++k) {
            if (spl_keys) spl_keys[r.bkt0 + k] = KT::key(spl_o[r.bkt0 + k]);
            if (spl_tags) spl_tags[r.bkt0 + k] = spl_t[r.bkt0 + k];
        }
    }
}

}  // namespace ossort
