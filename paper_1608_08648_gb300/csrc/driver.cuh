// Host-side orchestration of one sort: plans the workspace, launches the
// kernels of kernels.cuh on the caller's stream, never synchronizes.
//
// SqRan (Algorithm 2, with the sample on original positions):
//   sample p s - 1 positions, sort them, gather the tagged keys, sort the sample,
//   pick p - 1 splitters, classify + scatter every key into its bucket, sort
//   every bucket.
// SqDet (Algorithm 1):
//   sort the p sequences (step 1), take r p regular samples from each (step 2),
//   sort the r p^2 samples and pick the splitters (step 3), classify + scatter
//   the sorted sequences into buckets (step 4), sort every bucket (step 5).
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/ossort.h"
#include "kernels.cuh"
#include "profile.cuh"
#include "segkernels.cuh"
#include "distribute.cuh"

namespace ossort {

struct Ctx {
    cudaStream_t st = nullptr;
    Arena ar;
    int num_sms = 152;
    uint32_t* status = nullptr;   // [0] error bits, [1] depth, [2..3] u64 keys split by the bucket phase's SqRan,
                                  // [4..5] u64 keys repartitioned by k_repart, [6..7] range check
    bool nested = false;          // inside the sort of a sample (launch names get a ".sample" suffix)
    bool live() const { return !ar.measure() && !ar.failed; }
};

inline uint32_t pow2_ceil(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
inline int log2_exact(uint32_t x) {
    int h = 0;
    while ((1u << h) < x) ++h;
    return h;
}
inline unsigned grid_for(uint64_t work, int threads, unsigned cap = 4096) {
    uint64_t g = (work + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, cap));
}

constexpr uint32_t G_CAP = 2048;   // most CTAs of the grid-wide classify / scatter

// A kernel's dynamic shared-memory limit (cudaFuncAttributeMaxDynamicSharedMemorySize)
// is process-wide state of the kernel, shared by every host thread.  It is
// written exactly once per (device, kernel), to the most the device allows that
// kernel (the opt-in maximum less its static shared memory), by the first call
// that needs the kernel, under a lock, and before that call launches it.  Every
// launch of the kernel, on any thread, comes after its own call here, so no
// attribute write can overlap a launch of the same kernel on another thread and
// no later call ever changes a limit a queued launch was checked against.  The
// limit is only a ceiling: the shared memory a launch gets is the size it asks
// for, so occupancy and grid sizes are unchanged by it.
inline void smem_at_least(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> cur;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cur.find({dev, fn});
    if (it != cur.end()) return;   // set once; a launch above the limit fails with a launch error
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
        return;
    const size_t most = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    (void)bytes;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) == cudaSuccess)
        cur[{dev, fn}] = most;
}

template <class K>
int occupancy(K kernel, int threads, size_t smem) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    return occ > 0 ? occ : 1;
}

// ---------------------------------------------------------------------------
// Segmented sort core (kernels of segkernels.cuh), shared by the bucket phase
// of every sort and by the batched entry point.
// ---------------------------------------------------------------------------

// Upper bounds, from n, the number of segments and the class table alone, of
// the planned totals (the workspace is sized by them).  A segment g that is
// partitioned by a class has len_g >= 2 p_g s_g, so p_g <= len_g / (2 s_min);
// with automatic p, p_g <= len_g / auto_child + 1.  A segment has at most
// SEG_MAX_TILES tiles and at most len_g / tile_min + 1.
struct SegBounds {
    uint64_t tiles = 0, buckets = 0, hist = 0;
    int maxp = 1;
    bool any_part = false;
};

inline SegBounds seg_bounds_of(uint64_t n, uint32_t nseg, const SegClasses& cls) {
    SegBounds b;
    uint64_t smin = ~0ull, tmin = ~0ull;
    for (uint32_t k = 0; k < cls.n; ++k) {
        if (cls.c[k].p < 2 && !(cls.auto_child && k > 0)) continue;
        b.any_part = true;
        b.maxp = std::max<int>(b.maxp, (int)cls.c[k].p);
        smin = std::min<uint64_t>(smin, cls.c[k].s);
        tmin = std::min<uint64_t>(tmin, cls.c[k].tile);
    }
    uint64_t extra = 0;      // buckets beyond one per segment
    if (b.any_part) extra += n / (2 * smin) + 1;
    if (cls.auto_child) {
        b.any_part = true;
        b.maxp = std::max<int>(b.maxp, (int)cls.auto_pmax);
        tmin = std::min<uint64_t>(tmin, cls.c[0].tile);
        extra += n / cls.auto_child + 1;
    }
    if (!b.any_part) {
        b.buckets = nseg;
        return b;
    }
    b.tiles = std::min<uint64_t>(n / tmin + 1 + nseg, (uint64_t)SEG_MAX_TILES * nseg);
    b.buckets = std::min<uint64_t>((uint64_t)nseg * b.maxp, nseg + extra);
    b.hist = std::min<uint64_t>((uint64_t)b.maxp * (n / tmin + 1) + b.buckets, (uint64_t)SEG_MAX_TILES * b.buckets);
    return b;
}

// Class table of the bucket phase: buckets up to a CTA's capacity are sorted
// whole; a larger one is split by SqRan into children of about 0.72 of the
// capacity (p from its length, s up to 64).
template <class O>
SegClasses bucket_classes() {
    constexpr uint32_t CAP = (uint32_t)Cap<O>::v;
    SegClasses t{};
    t.n = 1;
    t.c[0] = SegClass{CAP, 1u, 1u, 16384u, 0u};   // histogram tiles of the split (measured best of 4K..64K)
    t.auto_child = (CAP * 18u) / 25u;
    t.auto_pmax = 1024;                 // s >= 4 with p s <= SEG_SAMPLE
    t.auto_s = 64;
    return t;
}

// Sort every segment of `src` into the same range of kout: segments above
// their class's cutoff are partitioned by SqRan (k_seg_*), then every bucket
// and every segment kept whole is sorted by the repartition levels (k_repart)
// and the shared-memory sorts (k_leaf).  Buffers: 0 = kin (read only, unless it
// is also alt), 1 = kout, 2 = alt (n keys of scratch; may be kin when every
// segment longer than a leaf is partitioned, which bucket_classes guarantees).
template <class KT, bool HV>
void seg_core(Ctx& c, const SegSource& src, const SegClasses& cls, const typename KT::T* kin, const uint32_t* vin,
              typename KT::T* kout, uint32_t* vout, typename KT::T* alt, uint32_t* valt, uint64_t seed,
              const os_seg_stats* stats) {
    using T = typename KT::T;
    using O = typename KT::O;
    using LE = LeafElem<O, true>;
    using E = typename LE::E;
    constexpr uint32_t CAP = (uint32_t)Cap<O>::v;
    const uint64_t n = src.n;
    const uint32_t nseg = src.nseg;
    const SegBounds B = seg_bounds_of(n, nseg, cls);
    SegRec* rec = c.ar.take<SegRec>(nseg);
    uint32_t* tile0 = c.ar.take<uint32_t>((size_t)nseg + 1);
    SegTotals* tot = c.ar.take<SegTotals>(1);
    uint32_t* pseg = c.ar.take<uint32_t>(std::max<uint32_t>(nseg, 1u));
    uint64_t* pblk = c.ar.take<uint64_t>(3 * (size_t)SEG_PLAN_MAXB);
    O* spl_o = c.ar.take<O>(B.buckets);
    uint32_t* spl_t = c.ar.take<uint32_t>(B.buckets);
    uint32_t* bsize = c.ar.take<uint32_t>(B.buckets);
    uint32_t* hist = B.any_part ? c.ar.take<uint32_t>(B.hist) : nullptr;
    uint16_t* bid = B.any_part ? c.ar.take<uint16_t>(n) : nullptr;
    WorkLists wl{};
    wl.counts = c.ar.take<uint32_t>(WL_COUNTS);
    wl.part_cap = (uint32_t)(n / CAP + 1);
    wl.leaf_cap = (uint32_t)(B.buckets + (uint64_t)MAX_DEPTH * 6 * wl.part_cap);
    wl.leaf = c.ar.take<WorkItem>(wl.leaf_cap);
    wl.part[0] = c.ar.take<WorkItem>(wl.part_cap);
    wl.part[1] = c.ar.take<WorkItem>(wl.part_cap);
    if (!c.live()) return;

    const bool nest = c.nested;
    os_memset_async(wl.counts, 0, sizeof(uint32_t) * WL_COUNTS, c.st);
    os_memset_async(tot, 0, sizeof(SegTotals), c.st);
    // the plan: CTAs of 1024 threads over ranges of `chunk` segments (one CTA for
    // up to 1024 segments; more, up to two per SM, for long segment tables)
    const uint32_t want = std::max<uint32_t>(
        1u, std::min<uint32_t>((nseg + 1023) / 1024, std::min<uint32_t>(SEG_PLAN_MAXB, 2u * (uint32_t)c.num_sms)));
    const uint32_t chunk = std::max<uint32_t>(1024u, (uint32_t)((((uint64_t)nseg + want - 1) / want + 1023) / 1024 * 1024));
    const uint32_t nblk = std::max<uint32_t>(1u, (uint32_t)(((uint64_t)nseg + chunk - 1) / chunk));
    OS_LAUNCH(c.st, nest ? "k_seg_plan.sample" : "k_seg_plan",
              k_seg_plan<<<nblk, 1024, 0, c.st>>>(src, cls, seed, rec, tile0, tot, B.tiles, B.buckets, B.hist, chunk,
                                                  nblk > 1 ? pblk : nullptr, pseg, c.status));
    if (nblk > 1) {
        OS_LAUNCH(c.st, nest ? "k_seg_plan.sample" : "k_seg_plan",
                  k_seg_plan_scan<<<1, SEG_PLAN_MAXB, 0, c.st>>>(pblk, nblk, nseg, tile0, tot, B.tiles, B.buckets,
                                                                 B.hist, c.status));
        OS_LAUNCH(c.st, nest ? "k_seg_plan.sample" : "k_seg_plan",
                  k_seg_plan_apply<<<nblk, 1024, 0, c.st>>>(rec, tile0, nseg, chunk, pblk, tot));
    }
    const uint32_t gseg = std::max<uint32_t>(1, std::min<uint32_t>(nseg, (uint32_t)c.num_sms * 8));
    if (B.any_part) {
        const size_t sm_spl = sizeof(E) * padded_len<E>(SEG_SAMPLE);
        smem_at_least(reinterpret_cast<const void*>(k_seg_splitters<KT>), sm_spl);
        const uint32_t g_spl = std::min<uint32_t>(
            nseg, (uint32_t)(c.num_sms * occupancy(k_seg_splitters<KT>, SEG_SPL_NT, sm_spl)));
        OS_LAUNCH(c.st, nest ? "k_seg_splitters.sample" : "k_seg_splitters",
                  k_seg_splitters<KT><<<std::max<uint32_t>(g_spl, 1), SEG_SPL_NT, sm_spl, c.st>>>(
                      kin, rec, pseg, tot, spl_o, spl_t, c.status));
        const size_t sm_c = seg_classify_v_smem<KT>(B.maxp);
        smem_at_least(reinterpret_cast<const void*>(k_seg_classify_v<KT>), sm_c);
        const uint32_t g_c = (uint32_t)(c.num_sms * occupancy(k_seg_classify_v<KT>, SEG_NT, sm_c));
        OS_LAUNCH(c.st, nest ? "k_seg_classify.sample" : "k_seg_classify",
                  k_seg_classify_v<KT><<<g_c, SEG_NT, sm_c, c.st>>>(kin, rec, tile0, nseg, tot, spl_o, spl_t,
                                                                     B.maxp, hist, bid));
    }
    OS_LAUNCH(c.st, nest ? "k_seg_scan.sample" : "k_seg_scan",
              k_seg_scan<<<gseg, SEG_SCAN_NT, 0, c.st>>>(rec, nseg, pseg, tot, hist, bsize, wl, CAP,
                                                         (uint32_t)(static_cast<const void*>(alt) ==
                                                                    static_cast<const void*>(kin)),
                                                         c.status, c.status + 1,
                                                         reinterpret_cast<unsigned long long*>(c.status + 2)));
    if (B.any_part) {
        const size_t sm_s = seg_scatter_smem<KT, HV>(B.maxp);
        smem_at_least(reinterpret_cast<const void*>(k_seg_scatter<KT, HV>), sm_s);
        constexpr int SNT = SegScatterCfg<T, HV>::NT;
        const uint32_t g_s = (uint32_t)(c.num_sms * occupancy(k_seg_scatter<KT, HV>, SNT, sm_s));
        OS_LAUNCH(c.st, nest ? "k_seg_scatter.sample" : "k_seg_scatter",
                  k_seg_scatter<KT, HV><<<g_s, SNT, sm_s, c.st>>>(kin, vin, bid, rec, tile0, nseg, tot, hist,
                                                                     B.maxp, kout, vout, c.status));
    }
    SortBufs<KT> bufs;
    bufs.k[0] = const_cast<T*>(kin);
    bufs.v[0] = const_cast<uint32_t*>(vin);
    bufs.k[1] = kout;
    bufs.v[1] = vout;
    bufs.k[2] = alt;
    bufs.v[2] = valt;
    bufs.out = kout;
    bufs.vout = vout;
    const SegSpec ss{nullptr, 0u, 0u, n};
    using L = BucketSmem<KT, HV>;
    smem_at_least(reinterpret_cast<const void*>(k_repart<KT, HV>), L::bytes);
    const uint32_t grid_r = (uint32_t)(c.num_sms * occupancy(k_repart<KT, HV>, BK_NT, L::bytes));
    const uint64_t inner_seed = sm_mix(seed ^ 0x5E6D5E6Dull);
    for (int level = 1; level < MAX_DEPTH; ++level)
        OS_LAUNCH(c.st, nest ? "k_repart.sample" : "k_repart",
                  k_repart<KT, HV><<<grid_r, BK_NT, L::bytes, c.st>>>(level, ss, bufs, wl, inner_seed, c.status,
                                                                      c.status + 1,
                                                                      reinterpret_cast<unsigned long long*>(c.status + 4)));
    const size_t leaf_smem = LeafSmem<KT, HV>::bytes;
    smem_at_least(reinterpret_cast<const void*>(k_leaf<KT, HV>), leaf_smem);
    constexpr int LNT = LeafCfg<O, HV>::NT;
    const uint32_t grid_l = (uint32_t)(c.num_sms * occupancy(k_leaf<KT, HV>, LNT, leaf_smem));
    OS_LAUNCH(c.st, nest ? "k_leaf.sample" : "k_leaf",
              k_leaf<KT, HV><<<grid_l, LNT, leaf_smem, c.st>>>(false, ss, bufs, wl, inner_seed, c.status));
    const uint32_t grid_small = (uint32_t)(c.num_sms * occupancy(k_leaf_small<KT, HV>, SMALL_NT, 0));
    OS_LAUNCH(c.st, nest ? "k_leaf_small.sample" : "k_leaf_small",
              k_leaf_small<KT, HV><<<grid_small, SMALL_NT, 0, c.st>>>(bufs, wl, n, c.status));
    if (stats) {
        OS_LAUNCH(c.st, "k_seg_export",
                  k_seg_export<KT><<<gseg, 256, 0, c.st>>>(rec, nseg, tot, spl_o, spl_t, bsize, stats->bucket_cap,
                                                           stats->bucket_base, stats->bucket_sizes,
                                                           static_cast<T*>(stats->splitter_keys),
                                                           stats->splitter_tags));
    }
}

// Sort every segment of ss (stably, in the tagged order of positions inside
// the segment) from src into the same range of out.  alt: scratch of n keys
// (may be src when src may be overwritten).  Segments of at most a CTA's
// capacity given as an even split are sorted directly in shared memory.
template <class KT, bool HV>
void segment_sort(Ctx& c, SegSpec ss, const typename KT::T* src, const uint32_t* vsrc, typename KT::T* out,
                  uint32_t* vout, typename KT::T* alt, uint32_t* valt, uint64_t seed) {
    using O = typename KT::O;
    using L = BucketSmem<KT, HV>;
    constexpr uint64_t CAP = (uint64_t)L::CAP;
    if (ss.nseg == 0 || ss.n == 0) return;
    const bool direct = ss.uniform && (ss.n + ss.nseg - 1) / ss.nseg <= CAP;
    if (!direct) {
        const SegSource s{nullptr, ss.uniform ? nullptr : ss.off, ss.nseg, ss.n, ss.base};
        seg_core<KT, HV>(c, s, bucket_classes<O>(), src, vsrc, out, vout, alt, valt, seed, nullptr);
        return;
    }
    if (!c.live()) return;
    SortBufs<KT> bufs{};
    bufs.k[0] = const_cast<typename KT::T*>(src);
    bufs.v[0] = const_cast<uint32_t*>(vsrc);
    bufs.out = out;
    bufs.vout = vout;
    const WorkLists wl{};
    const size_t leaf_smem = LeafSmem<KT, HV>::bytes;
    smem_at_least(reinterpret_cast<const void*>(k_leaf<KT, HV>), leaf_smem);
    constexpr int LNT = LeafCfg<O, HV>::NT;
    const uint32_t grid_l = (uint32_t)(c.num_sms * occupancy(k_leaf<KT, HV>, LNT, leaf_smem));
    OS_LAUNCH(c.st, c.nested ? "k_leaf.sample" : "k_leaf",
              k_leaf<KT, HV><<<std::min(ss.nseg, grid_l), LNT, leaf_smem, c.st>>>(true, ss, bufs, wl, seed, c.status));
}

// Bins of the top-level splitter table: the power of two >= 2p (at most 2^13).
inline int table_lbits(uint32_t p) {
    int b = 1;
    while ((1u << b) < 2 * p && b < 13) ++b;
    return b;
}

template <class KT>
size_t classify_smem(int p, int lbits) {
    return split_table_bytes<typename KT::O>(p - 1, lbits) + sizeof(uint32_t) * (p + 1);
}

template <class KT, bool HV, bool WIDE = false>
size_t scatter_smem(int p) {
    using T = typename KT::T;
    using SC = ScatterCfg<T, HV, WIDE>;
    constexpr int SUB = SC::SUB;
    size_t b = sizeof(T) * SUB + (HV ? sizeof(uint32_t) * SUB : 0);
    b += sizeof(uint32_t) * (p + 1) + sizeof(uint32_t) * p + sizeof(uint32_t) * 32;
    b += sizeof(uint16_t) * SUB + (HV ? sizeof(uint16_t) * SC::WARPS * (p + 1) : 0);
    return b;
}

// Step 4: classify every key of src (tag = position) against the p-1 sorted
// splitters and scatter keys (and payloads) into contiguous buckets of dst.
// Bucket b occupies [boff[b], boff[b+1]); bsize[b] = its size.
// Keys without a payload take the vector passes of distribute.cuh: units of
// SUPER keys, classify with NTC threads, scatter with NTS threads holding
// SUPER / NTS keys each.  Measured best on GB300 (units of 4096-16384 keys):
// 4-byte keys 16384-key units with 1024 threads (the scatter's two unit buffers
// then fill most of an SM's shared memory, one CTA per SM), as long as p <= 2048
// leaves room for its counters, else 8192-key units with 512 threads; 8-byte keys
// 8192-key units with 1024 threads.  The choice depends on p alone, so the
// workspace plan and the launches agree.
template <int SUPER_, int NTS_> struct TopVCfg {
    static constexpr int SUPER = SUPER_;
    static constexpr int NTC = 512;
    static constexpr int NTS = NTS_;
};

// Bins of the vector classify's splitter table: the power of two >= 4p (at most
// 2^13), so that few bins hold two splitters and need a search.
inline int table_lbits_v(uint32_t p) {
    int b = 1;
    while ((1u << b) < 4 * p && b < 13) ++b;
    return b;
}

// copy: NULL, or a device buffer of n keys that the classify fills with the keys
// it reads (src then lies in host memory the device reads over the host link,
// once); the scatter reads the copy.
template <class KT, class CF>
void partition_top_v_cfg(Ctx& c, const typename KT::T* src, uint32_t n, const typename KT::O* spl_o,
                         const uint32_t* spl_t, uint32_t p, typename KT::T* dst, uint32_t* boff, uint32_t* bsize,
                         typename KT::T* copy) {
    using T = typename KT::T;
    constexpr uint32_t SUPER = CF::SUPER;
    const int lb = table_lbits_v(p);
    const uint32_t ntiles = (n + SUPER - 1) / SUPER;
    const uint32_t gmax = std::min<uint32_t>(std::max<uint32_t>(ntiles, 1), G_CAP);
    uint32_t* hist = c.ar.take<uint32_t>((size_t)p * gmax);
    uint32_t* col = c.ar.take<uint32_t>((size_t)p * gmax);
    uint16_t* bid = c.ar.take<uint16_t>(n);
    if (!c.live()) return;
    auto ks = k_scatter_v<KT, CF::NTS, CF::SUPER>;
    const size_t sm_s = scatter_v_smem<T>((int)p, CF::SUPER);
    smem_at_least(reinterpret_cast<const void*>(ks), sm_s);
    const int occ = occupancy(ks, CF::NTS, sm_s);
    const uint32_t G = std::max<uint32_t>(1, std::min<uint32_t>(gmax, (uint32_t)(c.num_sms * occ)));
    // The classify may run more CTAs than the scatter: cstep of its CTAs cover
    // exactly one scatter CTA's units (tile_lo(g cstep, G cstep) = tile_lo(g, G)),
    // so the scatter reads its starting counts every cstep columns.
    auto grid_c = [&](int occ_c) {
        const uint32_t m = std::max<uint32_t>(1, (uint32_t)(c.num_sms * occ_c) / G);
        return (uint64_t)G * m <= gmax ? m : 1u;
    };
    auto kc = k_classify_v<KT, CF::NTC, CF::SUPER>;
    const size_t sm_c = classify_smem<KT>(p, lb);
    smem_at_least(reinterpret_cast<const void*>(kc), sm_c);
    const uint32_t cstep = grid_c(occupancy(kc, CF::NTC, sm_c));
    OS_LAUNCH(c.st, c.nested ? "k_classify.sample" : "k_classify",
              kc<<<G * cstep, CF::NTC, sm_c, c.st>>>(src, n, spl_o, spl_t, (int)p, lb, hist, bid, ntiles, copy));
    OS_LAUNCH(c.st, c.nested ? "k_column_scan.sample" : "k_column_scan",
              k_column_scan<<<grid_for((uint64_t)p * 32, 256), 256, 0, c.st>>>(hist, p, G * cstep, col, bsize));
    OS_LAUNCH(c.st, c.nested ? "k_bucket_offsets.sample" : "k_bucket_offsets",
              k_bucket_offsets<<<1, 1024, 0, c.st>>>(bsize, p, boff));
    OS_LAUNCH(c.st, c.nested ? "k_scatter.sample" : "k_scatter",
              ks<<<G, CF::NTS, sm_s, c.st>>>(copy ? copy : src, bid, n, (int)p, col, cstep, boff, dst, ntiles,
                                             c.status));
}

template <class KT>
void partition_top_v(Ctx& c, const typename KT::T* src, uint32_t n, const typename KT::O* spl_o,
                     const uint32_t* spl_t, uint32_t p, typename KT::T* dst, uint32_t* boff, uint32_t* bsize,
                     typename KT::T* copy = nullptr) {
    if constexpr (sizeof(typename KT::T) == 4) {
        if (p <= 2048)
            partition_top_v_cfg<KT, TopVCfg<16384, 1024>>(c, src, n, spl_o, spl_t, p, dst, boff, bsize, copy);
        else
            partition_top_v_cfg<KT, TopVCfg<8192, 512>>(c, src, n, spl_o, spl_t, p, dst, boff, bsize, copy);
    } else {
        partition_top_v_cfg<KT, TopVCfg<8192, 1024>>(c, src, n, spl_o, spl_t, p, dst, boff, bsize, copy);
    }
}

template <class KT, bool HV, bool WIDE>
void partition_top_cfg(Ctx& c, const typename KT::T* src, const uint32_t* vsrc, uint32_t n,
                       const typename KT::O* spl_o, const uint32_t* spl_t, uint32_t p, typename KT::T* dst,
                       uint32_t* vdst, uint32_t* boff, uint32_t* bsize) {
    using SC = ScatterCfg<typename KT::T, HV, WIDE>;
    const int lb = table_lbits_v(p);
    constexpr uint32_t SUPER = SC::SUPER;
    const uint32_t ntiles = (n + SUPER - 1) / SUPER;
    const uint32_t gmax = std::min<uint32_t>(std::max<uint32_t>(ntiles, 1), G_CAP);
    uint32_t* hist = c.ar.take<uint32_t>((size_t)p * gmax);
    uint32_t* col = c.ar.take<uint32_t>((size_t)p * gmax);
    uint16_t* bid = c.ar.take<uint16_t>(n);
    if (!c.live()) return;
    constexpr int NTS = SC::NT;
    constexpr int NTC = 512;
    // the vector classify over the same units (the payload takes no part in it)
    auto kc = k_classify_v<KT, NTC, (int)SUPER>;
    auto ks = k_scatter<KT, HV, WIDE>;
    const size_t sm_c = classify_smem<KT>(p, lb), sm_s = scatter_smem<KT, HV, WIDE>(p);
    smem_at_least(reinterpret_cast<const void*>(kc), sm_c);
    smem_at_least(reinterpret_cast<const void*>(ks), sm_s);
    const int occ = occupancy(ks, NTS, sm_s);
    const uint32_t G = std::max<uint32_t>(1, std::min<uint32_t>(gmax, (uint32_t)(c.num_sms * occ)));
    // cstep classify CTAs cover one scatter CTA's units (as in partition_top_v_cfg)
    const uint32_t mc = std::max<uint32_t>(1, (uint32_t)(c.num_sms * occupancy(kc, NTC, sm_c)) / G);
    const uint32_t cstep = (uint64_t)G * mc <= gmax ? mc : 1u;
    OS_LAUNCH(c.st, c.nested ? "k_classify.sample" : "k_classify",
              kc<<<G * cstep, NTC, sm_c, c.st>>>(src, n, spl_o, spl_t, (int)p, lb, hist, bid, ntiles, nullptr));
    OS_LAUNCH(c.st, c.nested ? "k_column_scan.sample" : "k_column_scan",
              k_column_scan<<<grid_for((uint64_t)p * 32, 256), 256, 0, c.st>>>(hist, p, G * cstep, col, bsize));
    OS_LAUNCH(c.st, c.nested ? "k_bucket_offsets.sample" : "k_bucket_offsets", k_bucket_offsets<<<1, 1024, 0, c.st>>>(bsize, p, boff));
    OS_LAUNCH(c.st, c.nested ? "k_scatter.sample" : "k_scatter",
              ks<<<G, NTS, sm_s, c.st>>>(src, vsrc, bid, n, (int)p, col, cstep, boff, dst, vdst, ntiles, c.status));
}

// Keys alone take the vector passes; payload sorts the stable pair above, with
// the WIDE configuration while p <= hv_wide_max_p (a choice on p alone, so that
// the workspace plan and the launches agree).
template <class KT, bool HV>
void partition_top(Ctx& c, const typename KT::T* src, const uint32_t* vsrc, uint32_t n,
                   const typename KT::O* spl_o, const uint32_t* spl_t, uint32_t p, typename KT::T* dst,
                   uint32_t* vdst, uint32_t* boff, uint32_t* bsize) {
    if constexpr (!HV) {
        partition_top_v<KT>(c, src, n, spl_o, spl_t, p, dst, boff, bsize);
    } else {
        if (p <= (uint32_t)hv_wide_max_p<typename KT::T>())
            partition_top_cfg<KT, HV, true>(c, src, vsrc, n, spl_o, spl_t, p, dst, vdst, boff, bsize);
        else
            partition_top_cfg<KT, HV, false>(c, src, vsrc, n, spl_o, spl_t, p, dst, vdst, boff, bsize);
    }
}

template <class KT, bool HV>
void sort_array(Ctx& c, const typename KT::T* src, const uint32_t* vsrc, typename KT::T* out, uint32_t* vout,
                uint32_t n, uint64_t seed);

// Step 2 (SqRan) and step 3: p s - 1 tagged random keys, sorted; splitters at
// ranks i s - 1.
template <class KT>
void splitters_ran(Ctx& c, const typename KT::T* keys, uint32_t n, uint32_t p, uint32_t s, uint64_t seed,
                   typename KT::O* spl_o, uint32_t* spl_t) {
    using T = typename KT::T;
    const uint32_t m = p * s - 1;
    uint32_t* pos = c.ar.take<uint32_t>(m);
    uint32_t* pos_s = c.ar.take<uint32_t>(m);
    T* tk = c.ar.take<T>(m);
    uint32_t* tt = c.ar.take<uint32_t>(m);
    T* tks = c.ar.take<T>(m);
    uint32_t* tts = c.ar.take<uint32_t>(m);
    if (c.live())
        OS_LAUNCH(c.st, "k_ran_positions",
                  k_ran_positions<<<grid_for(m, 256, 1024), 256, 0, c.st>>>(pos, m, n, seed));
    // Positions in increasing order, so that a stable sort by key leaves equal
    // keys in tag order.
    const bool was_nested = c.nested;
    c.nested = true;
    sort_array<KeyU32, false>(c, pos, nullptr, pos_s, nullptr, m, sm_mix(seed ^ 0x51ull));
    if (c.live())
        OS_LAUNCH(c.st, "k_gather_tagged",
                  k_gather_tagged<KT><<<grid_for(m, 256, 1024), 256, 0, c.st>>>(keys, n, pos_s, m, tk, tt, c.status));
    sort_array<KT, true>(c, tk, tt, tks, tts, m, sm_mix(seed ^ 0x52ull));
    c.nested = was_nested;
    if (c.live() && p > 1)
        OS_LAUNCH(c.st, "k_pick_splitters",
                  k_pick_splitters<KT><<<grid_for(p, 256), 256, 0, c.st>>>(tks, tts, p, s, spl_o, spl_t));
}

// Steps 2-3 of SqDet: r p regular samples from each sorted sequence of A
// (already in tag order), sorted stably by key; splitters at ranks i r p - 1.
template <class KT>
void splitters_det(Ctx& c, const typename KT::T* A, uint32_t n, uint32_t p, uint32_t r, uint64_t seed,
                   typename KT::O* spl_o, uint32_t* spl_t) {
    using T = typename KT::T;
    const uint32_t mm = r * p;
    const uint64_t m = (uint64_t)p * mm;
    T* tk = c.ar.take<T>(m);
    uint32_t* tt = c.ar.take<uint32_t>(m);
    T* tks = c.ar.take<T>(m);
    uint32_t* tts = c.ar.take<uint32_t>(m);
    if (c.live())
        OS_LAUNCH(c.st, "k_det_sample", k_det_sample<KT><<<grid_for(m, 256), 256, 0, c.st>>>(A, n, p, mm, tk, tt, c.status));
    const bool was_nested = c.nested;
    c.nested = true;
    sort_array<KT, true>(c, tk, tt, tks, tts, (uint32_t)m, sm_mix(seed ^ 0x53ull));
    c.nested = was_nested;
    if (c.live() && p > 1)
        OS_LAUNCH(c.st, "k_pick_splitters",
                  k_pick_splitters<KT><<<grid_for(p, 256), 256, 0, c.st>>>(tks, tts, p, mm, spl_o, spl_t));
}

// Sort any array (used for samples and for inputs too small to sample): one
// shared-memory sort when it fits a CTA, else an internal SqRan level with p
// chosen so that buckets are a few CTA capacities.
template <class KT, bool HV>
void sort_array(Ctx& c, const typename KT::T* src, const uint32_t* vsrc, typename KT::T* out, uint32_t* vout,
                uint32_t n, uint64_t seed) {
    using T = typename KT::T;
    using O = typename KT::O;
    constexpr uint32_t CAP = (uint32_t)Cap<O>::v;
    if (n == 0) return;
    if (n <= CAP) {
        segment_sort<KT, HV>(c, SegSpec::even(1, n), src, vsrc, out, vout, nullptr, nullptr, seed);
        return;
    }
    const uint32_t p = std::min<uint32_t>(1024, std::max<uint32_t>(2, pow2_ceil(n / (2 * CAP))));
    const uint32_t s = std::max<uint32_t>(1, CAP / p);
    O* spl_o = c.ar.take<O>(p - 1);
    uint32_t* spl_t = c.ar.take<uint32_t>(p - 1);
    uint32_t* boff = c.ar.take<uint32_t>(p + 1);
    uint32_t* bsize = c.ar.take<uint32_t>(p);
    T* w = c.ar.take<T>(n);
    uint32_t* vw = HV ? c.ar.take<uint32_t>(n) : nullptr;
    splitters_ran<KT>(c, src, n, p, s, seed, spl_o, spl_t);
    partition_top<KT, HV>(c, src, vsrc, n, spl_o, spl_t, p, w, vw, boff, bsize);
    segment_sort<KT, HV>(c, SegSpec::offsets(boff, p, n), w, vw, out, vout, w, vw, sm_mix(seed ^ 0x54ull));
}

// Device results of one user-level sort (for statistics).
struct TopResult {
    uint32_t p_used = 1;
    void* spl_o = nullptr;
    uint32_t* spl_t = nullptr;
    uint32_t* bsize = nullptr;
    const uint32_t* det_index = nullptr;   // SqDet with a payload: payloads in the order of the sorted sequences
    void* str_keys = nullptr;              // 32-byte keys: the splitters' keys (device)
    const uint32_t* str_map = nullptr;
    bool sunk = false;                     // the output already went to a HostSink
};

// A host-buffer sort copies its output to the host while buckets are still
// being sorted: the buckets are sorted in `chunks` ranges, and each range's keys
// (and payloads) are copied on `copy` as soon as that range is done; the
// caller's stream waits for the copies.
struct HostSink {
    void* keys;
    uint32_t* vals;
    cudaStream_t copy;
    uint32_t chunks;
};

template <class KT, bool HV>
void det_merge_steps(Ctx& c, const typename KT::T* w1, const uint32_t* vw1, typename KT::T* w2, uint32_t* vw2,
                     typename KT::T* kout, uint32_t* vout, uint32_t n, uint32_t p, const typename KT::O* spl_o,
                     const uint32_t* spl_t, uint32_t* boff, uint32_t* bsize);

// Step 5 on buckets [boff[b], boff[b+1]) of src into out: one segmented sort, or,
// with a HostSink, one per range of buckets, each range copied to the host while
// the next is sorted.  The measuring pass sizes one sort of all buckets, which
// bounds every range's (the arena is rewound for each).
template <class KT, bool HV>
void sort_buckets(Ctx& c, const uint32_t* boff, uint32_t p, uint32_t n, typename KT::T* src, uint32_t* vsrc,
                  typename KT::T* out, uint32_t* vout, typename KT::T* alt, uint32_t* valt, uint64_t seed,
                  const HostSink* sink, TopResult& res) {
    using T = typename KT::T;
    if (!sink || sink->chunks < 2 || p < sink->chunks || !sink->copy || c.ar.measure()) {
        segment_sort<KT, HV>(c, SegSpec::offsets(boff, p, n), src, vsrc, out, vout, alt, valt, seed);
        return;
    }
    if (!c.live()) return;
    std::vector<uint32_t> hb(p + 1);
    cudaError_t e = cudaMemcpyAsync(hb.data(), boff, sizeof(uint32_t) * (p + 1), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess || hb[0] != 0 || hb[p] != n) {   // fall back to one sort, copied by the caller
        segment_sort<KT, HV>(c, SegSpec::offsets(boff, p, n), src, vsrc, out, vout, alt, valt, seed);
        return;
    }
    const size_t mark = c.ar.used;
    size_t high = mark;
    for (uint32_t k = 0; k < sink->chunks; ++k) {
        const uint32_t b0 = (uint32_t)((uint64_t)k * p / sink->chunks), b1 = (uint32_t)((uint64_t)(k + 1) * p / sink->chunks);
        const uint32_t base = hb[b0], len = hb[b1] - base;
        if (len == 0) continue;
        c.ar.used = mark;
        segment_sort<KT, HV>(c, SegSpec::offsets_at(boff + b0, b1 - b0, len, base), src + base,
                             HV ? vsrc + base : nullptr, out + base, HV ? vout + base : nullptr, alt + base,
                             HV ? valt + base : nullptr, seed);
        high = std::max(high, c.ar.used);
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            c.ar.failed = true;
            return;
        }
        cudaEventRecord(ev, c.st);
        cudaStreamWaitEvent(sink->copy, ev, 0);
        cudaEventDestroy(ev);
        cudaMemcpyAsync(static_cast<T*>(sink->keys) + base, out + base, sizeof(T) * len, cudaMemcpyDeviceToHost,
                        sink->copy);
        if (HV) cudaMemcpyAsync(sink->vals + base, vout + base, sizeof(uint32_t) * len, cudaMemcpyDeviceToHost, sink->copy);
    }
    c.ar.used = high;
    cudaEvent_t done;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
        c.ar.failed = true;
        return;
    }
    cudaEventRecord(done, sink->copy);
    cudaStreamWaitEvent(c.st, done, 0);
    cudaEventDestroy(done);
    res.sunk = true;
}

// kin_copy (keys alone, SqRan only): kin lies in host memory the device can
// read; the sample is gathered from it directly and the top-level classify
// copies the keys into kin_copy (a device buffer of n keys, may be kout) as it
// reads them, so the keys cross the host link once and no separate copy-in
// precedes the sort.
template <class KT, bool HV>
void sort_top(Ctx& c, const typename KT::T* kin, typename KT::T* kout, const uint32_t* vin, uint32_t* vout,
              uint32_t n, const os_params& prm, TopResult& res, const HostSink* sink = nullptr,
              typename KT::T* kin_copy = nullptr) {
    using T = typename KT::T;
    using O = typename KT::O;
    const uint32_t p = prm.p, s = prm.s;
    const uint64_t ps = (uint64_t)p * s;
    const uint64_t internal_seed = sm_mix(prm.seed ^ 0xA5A5A5A5A5A5A5A5ull);
    const bool small = (p == 1) || (prm.split == OS_RAN ? ((uint64_t)n < 2 * ps)
                                                        : (((uint64_t)n + p - 1) / p < ps));
    O* spl_o = c.ar.take<O>(std::max<uint32_t>(p - 1, 1));
    uint32_t* spl_t = c.ar.take<uint32_t>(std::max<uint32_t>(p - 1, 1));
    uint32_t* boff = c.ar.take<uint32_t>(p + 1);
    uint32_t* bsize = c.ar.take<uint32_t>(p);
    res.spl_o = spl_o;
    res.spl_t = spl_t;
    res.bsize = bsize;
    res.p_used = small ? 1 : p;
    if (n == 0) return;
    if (small) {
        sort_array<KT, HV>(c, kin, vin, kout, vout, n, internal_seed);
        return;
    }
    T* w1 = c.ar.take<T>(n);
    uint32_t* vw1 = HV ? c.ar.take<uint32_t>(n) : nullptr;
    if (prm.split == OS_RAN) {
        splitters_ran<KT>(c, kin, n, p, s, prm.seed, spl_o, spl_t);
        if constexpr (!HV) {
            partition_top_v<KT>(c, kin, n, spl_o, spl_t, p, w1, boff, bsize, kin_copy);
        } else {
            partition_top<KT, HV>(c, kin, vin, n, spl_o, spl_t, p, w1, vw1, boff, bsize);
        }
        sort_buckets<KT, HV>(c, boff, p, n, w1, vw1, kout, vout, w1, vw1, internal_seed, sink, res);
    } else {
        T* w2 = c.ar.take<T>(n);
        uint32_t* vw2 = HV ? c.ar.take<uint32_t>(n) : nullptr;
        // Step 1: the p sequences sorted into w1 (stable).
        segment_sort<KT, HV>(c, SegSpec::even(p, n), kin, vin, w1, vw1, w2, vw2, internal_seed);
        res.det_index = vw1;
        splitters_det<KT>(c, w1, n, p, s, internal_seed, spl_o, spl_t);
        if (prm.flags & OS_DET_MERGE) {
            // the paper's steps 4-5: split the sorted sequences, merge every bucket
            det_merge_steps<KT, HV>(c, w1, vw1, w2, vw2, kout, vout, n, p, spl_o, spl_t, boff, bsize);
        } else {
            partition_top<KT, HV>(c, w1, vw1, n, spl_o, spl_t, p, w2, vw2, boff, bsize);
            sort_buckets<KT, HV>(c, boff, p, n, w2, vw2, kout, vout, w2, vw2, internal_seed, sink, res);
        }
    }
}

// Everything one os_sort call needs, independent of the key type.
struct RunArgs {
    const void* kin;
    void* kout;
    const uint32_t* vin;
    uint32_t* vout;
    bool has_vals;
    uint64_t n;
    os_params prm;
    void* ws;          // nullptr: measure only
    size_t ws_bytes;
    cudaStream_t st;
    int num_sms;
    const HostSink* sink;   // host-buffer sorts: where ranges of the output go as they finish
    void* kin_copy;         // host-buffer sorts read straight from host memory: the device copy (see sort_top)
    // outputs
    size_t used;
    uint32_t* status;
    TopResult res;
};

template <class KT>
int run_sort(RunArgs& a) {
    using T = typename KT::T;
    Ctx c;
    c.st = a.st;
    c.num_sms = a.num_sms;
    c.ar.base = static_cast<char*>(a.ws);
    c.ar.cap = a.ws_bytes;
    c.status = c.ar.take<uint32_t>(8);
    if (c.live()) os_memset_async(c.status, 0, 8 * sizeof(uint32_t), c.st);
    const T* kin = static_cast<const T*>(a.kin);
    T* kout = static_cast<T*>(a.kout);
    if (a.has_vals) sort_top<KT, true>(c, kin, kout, a.vin, a.vout, (uint32_t)a.n, a.prm, a.res, a.sink);
    else sort_top<KT, false>(c, kin, kout, nullptr, nullptr, (uint32_t)a.n, a.prm, a.res, a.sink,
                             static_cast<T*>(a.kin_copy));
    a.used = c.ar.used;
    a.status = c.status;
    return c.ar.failed ? OS_ERR_WS : OS_OK;
}

int run_i32(RunArgs& a);
int run_u64(RunArgs& a);
int run_f64(RunArgs& a);
int run_s32(RunArgs& a);

}  // namespace ossort

#include "detmerge.cuh"
