// SqDet in the paper's own organisation (Algorithm 1, steps 4 and 5), selected
// by OS_DET_MERGE: the p sequences sorted in step 1 stay in place; step 4 splits
// every sorted sequence by a binary search of every splitter (the pieces
// X_{k,j}, counted into the bucket sizes |Y_j| = sum_k |X_{k,j}|); step 5 merges
// the p pieces of every bucket.  The p-way merge runs as ceil(log2 p) passes of
// pairwise merges over all buckets at once: pass l merges runs of 2^(l-1)
// pieces in pairs, so a pair's left run always holds lower-numbered sequences
// than its right run, and taking the left element on equal keys is exactly the
// tagged order of Section 2.2 (no tag needs to be stored).
//
// Step 5 first copies every piece into its bucket (so every merge pass finds a
// pair's two runs at the pair's own output positions), then runs the passes.
// A merge pass is a merge-path partition (k_det_partition) and one CTA per
// DM_OT consecutive outputs (k_det_merge).
#pragma once

#include "driver.cuh"

namespace ossort {

constexpr int DM_NT = 256;

// A merge pass's tile: IT outputs per thread (odd, so that the threads' merge
// cursors, IT elements apart, start in different shared-memory banks), OT per
// CTA; MINB resident CTAs per SM (4-byte keys alone fit eight).
template <class KT, bool HV>
struct DmCfg {
    static constexpr int IT = sizeof(typename KT::O) == 4 ? 15 : 17;
    static constexpr int OT = DM_NT * IT;
    static constexpr int MINB = (sizeof(typename KT::O) == 4 && !HV) ? 8 : 4;
};

// Step 4: pos[k * (p + 1) + j] = number of elements of sorted sequence k that are
// at most splitter j in the tagged order (tag = position in A), j = 1..p-1;
// pos[k][0] = 0, pos[k][p] = |sequence k|.
template <class KT>
__global__ void k_det_split(const typename KT::T* __restrict__ A, uint64_t n, uint32_t p,
                            const typename KT::O* __restrict__ spl_o, const uint32_t* __restrict__ spl_t,
                            uint32_t* __restrict__ pos) {
    using O = typename KT::O;
    const uint64_t total = (uint64_t)p * (p + 1);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = (uint32_t)(q / (p + 1)), j = (uint32_t)(q % (p + 1));
        const uint64_t cs = (uint64_t)k * n / p, c = (uint64_t)(k + 1) * n / p - cs;
        uint64_t r;
        if (j == 0) {
            r = 0;
        } else if (j == p) {
            r = c;
        } else {
            const O so = spl_o[j - 1];
            const uint64_t st = spl_t[j - 1];
            uint64_t lo = 0, hi = c;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                const O o = KT::ord(A[cs + mid]);
                if (o < so || (o == so && cs + mid <= st)) lo = mid + 1;
                else hi = mid;
            }
            r = lo;
        }
        pos[q] = (uint32_t)r;
    }
}

// Piece sizes, bucket-major: hist[j * p + k] = |X_{k,j}|.
static __global__ void k_det_pieces(const uint32_t* __restrict__ pos, uint32_t p, uint32_t* __restrict__ hist) {
    const uint64_t total = (uint64_t)p * p;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(q / p), k = (uint32_t)(q % p);
        hist[q] = pos[(size_t)k * (p + 1) + j + 1] - pos[(size_t)k * (p + 1) + j];
    }
}

// One pair of runs of a merge pass.
struct DmPair {
    uint32_t a_src, a_len, b_src, b_len, out;
};

// Pair q of pass `level` (runs of h = 2^(level-1) pieces): bucket j = q / npb,
// pair i = q % npb, left run = pieces [2 h i, 2 h i + h), right run = the next h.
// Every pass reads the layout of the previous one (the pieces were first copied
// into their buckets), so a pair's two runs sit exactly at its output positions.
__device__ __forceinline__ DmPair dm_pair(uint32_t q, int level, uint32_t p, uint32_t npb,
                                          const uint32_t* __restrict__ col, const uint32_t* __restrict__ bsize,
                                          const uint32_t* __restrict__ boff) {
    const uint32_t h = 1u << (level - 1);
    const uint32_t j = q / npb, i = q % npb;
    const uint32_t k0 = 2 * h * i;
    const uint32_t k1 = min(k0 + h, p), k2 = min(k0 + 2 * h, p);
    auto colx = [&](uint32_t k) { return k < p ? col[(size_t)j * p + k] : bsize[j]; };
    DmPair r;
    r.out = boff[j] + colx(k0);
    r.a_len = colx(k1) - colx(k0);
    r.b_len = colx(k2) - colx(k1);
    r.a_src = r.out;
    r.b_src = r.out + r.a_len;
    return r;
}

// First index x in [lo, hi) with pred(x) true, or hi (pred monotone: false, then
// true).  Called by a whole warp: 32 probes per round, so a range of 2^20
// takes four dependent rounds of loads instead of twenty.
template <class Pred>
__device__ __forceinline__ uint32_t warp_first_true(uint32_t lo, uint32_t hi, Pred pred) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t x = min(lo + step * (uint32_t)lane, hi - 1);
        const unsigned m = __ballot_sync(0xffffffffu, pred(x));
        const int f = m ? __ffs(m) - 1 : 32;
        if (f == 0) return lo;
        const uint32_t prev = min(lo + step * (uint32_t)(f - 1), hi - 1);
        hi = f < 32 ? min(lo + step * (uint32_t)f, hi - 1) : hi;
        lo = prev + 1;
        if (lo >= hi) return hi;
    }
    const uint32_t x = lo + (uint32_t)lane;
    const unsigned m = __ballot_sync(0xffffffffu, x < hi && pred(x));
    return m ? lo + (uint32_t)(__ffs(m) - 1) : hi;
}

// Outputs of the merged pair that come from the left run among its first d
// (merge path: left element mid against right element d - 1 - mid; the left one
// comes first unless the right one is strictly smaller).  Called by a warp.
template <class KT>
__device__ __forceinline__ uint32_t dm_split(const typename KT::T* __restrict__ src, const DmPair& r, uint32_t d) {
    const uint32_t lo = d > r.b_len ? d - r.b_len : 0u, hi = min(d, r.a_len);
    return warp_first_true(lo, hi, [&](uint32_t mid) {
        return KT::ord(src[r.b_src + d - 1 - mid]) < KT::ord(src[r.a_src + mid]);
    });
}

// Step 5, first: every piece X_{k,j} copied from its sorted sequence into its
// place in bucket j (one warp per piece, bucket-major so neighbouring warps
// write neighbouring ranges).
template <class KT, bool HV>
__global__ void k_det_gather(const typename KT::T* __restrict__ A, const uint32_t* __restrict__ vA, uint64_t n,
                             uint32_t p, const uint32_t* __restrict__ pos, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ boff, typename KT::T* __restrict__ dst,
                             uint32_t* __restrict__ vdst) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t total = (uint64_t)p * p;
    for (uint64_t q = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < total; q += warps) {
        const uint32_t j = (uint32_t)(q / p), k = (uint32_t)(q % p);
        const uint32_t a = pos[(size_t)k * (p + 1) + j], len = pos[(size_t)k * (p + 1) + j + 1] - a;
        const uint64_t from = (uint64_t)k * n / p + a;
        const uint32_t to = boff[j] + col[(size_t)j * p + k];
        for (uint32_t t = lane; t < len; t += 32) {
            dst[to + t] = A[from + t];
            if (HV) vdst[to + t] = vA[from + t];
        }
    }
}

// Merge-path partition of one merge pass, one warp per tile boundary
// o = min(t OT, n), t = 0..ntiles: part[2 t] = the pair q holding output o
// (the last pair starting at or before it), part[2 t + 1] = how many of the first
// o - start(q) outputs of q come from its left run.
template <class KT, int OT>
__global__ void k_det_partition(int level, uint32_t p, uint64_t n, const typename KT::T* __restrict__ src,
                                const uint32_t* __restrict__ col, const uint32_t* __restrict__ bsize,
                                const uint32_t* __restrict__ boff, uint32_t* __restrict__ part) {
    const uint32_t h = 1u << (level - 1);
    const uint32_t npb = (p + 2 * h - 1) / (2 * h);
    const uint32_t npairs = p * npb;
    const uint32_t nb = (uint32_t)((n + OT - 1) / OT) + 1;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nb; t += warps) {
        const uint32_t o = (uint64_t)t * OT < n ? t * OT : (uint32_t)n;
        const uint32_t f = warp_first_true(0u, npairs, [&](uint32_t x) {
            return dm_pair(x, level, p, npb, col, bsize, boff).out > o;
        });
        const uint32_t q = f > 0 ? f - 1 : 0;
        const DmPair r = dm_pair(q, level, p, npb, col, bsize, boff);
        const uint32_t d = o - r.out;
        const uint32_t a = d == 0 ? 0u : d == r.a_len + r.b_len ? r.a_len : dm_split<KT>(src, r, d);
        if ((threadIdx.x & 31) == 0) {
            part[2 * (size_t)t] = q;
            part[2 * (size_t)t + 1] = a;
        }
    }
}

constexpr int DM_TBL = 1024;   // pairs one tile merges through its table (more: pair by pair)

// Step 5, one pass of pairwise merges over all buckets, one CTA per tile of
// DM_OT consecutive outputs.  Pairs wholly inside the tile find their two runs
// at their own output positions, so the tile stages its output range with one
// coalesced load; only the pairs cut by its ends are restaged from the splits
// that k_det_partition found.  A table of the tile's pairs (start, left and
// right lengths) lets every thread merge its DM_IT outputs across pairs.
template <class KT, bool HV>
__global__ void __launch_bounds__(DM_NT, (DmCfg<KT, HV>::MINB))
k_det_merge(int level, uint32_t p, uint64_t n, const typename KT::T* __restrict__ src,
            const uint32_t* __restrict__ vsrc, typename KT::T* __restrict__ dst, uint32_t* __restrict__ vdst,
            const uint32_t* __restrict__ col, const uint32_t* __restrict__ bsize, const uint32_t* __restrict__ boff,
            const uint32_t* __restrict__ part) {
    using O = typename KT::O;
    constexpr int DM_IT = DmCfg<KT, HV>::IT, DM_OT = DmCfg<KT, HV>::OT;
    extern __shared__ __align__(16) char smem[];
    O* sk = reinterpret_cast<O*>(smem);                                    // [DM_OT]
    uint32_t* tstart = reinterpret_cast<uint32_t*>(smem + sizeof(O) * DM_OT);
    uint32_t* tna = tstart + DM_TBL;
    uint32_t* tnb = tna + DM_TBL;
    uint32_t* sv = tnb + DM_TBL;                                           // [DM_OT] with a payload
    const uint32_t h = 1u << (level - 1);
    const uint32_t npb = (p + 2 * h - 1) / (2 * h);
    const uint32_t tile = blockIdx.x;
    const uint32_t o0 = tile * DM_OT;
    const uint32_t o1 = (uint64_t)o0 + DM_OT < n ? o0 + DM_OT : (uint32_t)n;
    const uint32_t total = o1 - o0;
    // the tile's own range, which is every inner pair's input
    for (uint32_t t = threadIdx.x; t < total; t += DM_NT) {
        sk[t] = KT::ord(src[o0 + t]);
        if (HV) sv[t] = vsrc[o0 + t];
    }
    const uint32_t q0 = part[2 * (size_t)tile], a0s = part[2 * (size_t)tile + 1];
    const uint32_t q1 = part[2 * (size_t)tile + 2], a1e = part[2 * (size_t)tile + 3];
    const DmPair r0 = dm_pair(q0, level, p, npb, col, bsize, boff);
    const DmPair r1 = dm_pair(q1, level, p, npb, col, bsize, boff);
    const uint32_t len0 = r0.a_len + r0.b_len, len1 = r1.a_len + r1.b_len;
    // the first pair's outputs here are its diagonals [d0s, d0e), the last one's [0, d1e)
    const uint32_t d0s = o0 - r0.out, d1e = o1 - r1.out;
    const uint32_t d0e = q1 == q0 ? d1e : len0;
    const uint32_t a0e = q1 == q0 ? a1e : r0.a_len;
    const uint32_t nseg = q1 - q0 + 1;
    const uint32_t na0 = a0e - a0s, nb0 = (d0e - d0s) - na0;
    // segment i of the tile = pair q0 + i restricted to the tile: its start in
    // the tile and its left and right lengths there
    auto seg_of = [&](uint32_t i, uint32_t& st, uint32_t& na, uint32_t& nb) {
        const uint32_t q = q0 + i;
        if (i == 0) {
            st = 0;
            na = na0;
            nb = nb0;
        } else if (q == q1) {
            st = r1.out - o0;
            na = a1e;
            nb = d1e - a1e;
        } else {
            const DmPair r = dm_pair(q, level, p, npb, col, bsize, boff);
            st = r.out - o0;
            na = r.a_len;
            nb = r.b_len;
        }
    };
    // a table of the segments when they fit (the usual case; built while the
    // tile loads); otherwise (many empty pairs: n small against p^2) every
    // segment is recomputed on use
    const bool table = nseg <= (uint32_t)DM_TBL;
    if (table) {
        for (uint32_t i = threadIdx.x; i < nseg; i += DM_NT) seg_of(i, tstart[i], tna[i], tnb[i]);
    }
    __syncthreads();
    // the cut pairs' inputs (left part, then right part) over their output range
    if (!(d0s == 0 && d0e == len0)) {
        for (uint32_t t = threadIdx.x; t < na0; t += DM_NT) {
            sk[t] = KT::ord(src[r0.a_src + a0s + t]);
            if (HV) sv[t] = vsrc[r0.a_src + a0s + t];
        }
        for (uint32_t t = threadIdx.x; t < nb0; t += DM_NT) {
            sk[na0 + t] = KT::ord(src[r0.b_src + (d0s - a0s) + t]);
            if (HV) sv[na0 + t] = vsrc[r0.b_src + (d0s - a0s) + t];
        }
    }
    if (q1 != q0 && d1e != len1) {
        const uint32_t base = r1.out - o0, nb1 = d1e - a1e;
        for (uint32_t t = threadIdx.x; t < a1e; t += DM_NT) {
            sk[base + t] = KT::ord(src[r1.a_src + t]);
            if (HV) sv[base + t] = vsrc[r1.a_src + t];
        }
        for (uint32_t t = threadIdx.x; t < nb1; t += DM_NT) {
            sk[base + a1e + t] = KT::ord(src[r1.b_src + t]);
            if (HV) sv[base + a1e + t] = vsrc[r1.b_src + t];
        }
    }
    auto seg = [&](uint32_t i, uint32_t& st, uint32_t& na, uint32_t& nb) {
        if (table) {
            st = tstart[i];
            na = tna[i];
            nb = tnb[i];
        } else {
            seg_of(i, st, na, nb);
        }
    };
    __syncthreads();
    // every thread: DM_IT consecutive outputs, across pair boundaries
    const uint32_t od = threadIdx.x * DM_IT;
    O x[DM_IT];
    uint32_t xv[HV ? DM_IT : 1];
    int cnt = 0;
    if (od < total) {
        uint32_t lo = 0, hi = nseg;                    // last segment starting at or before od
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            uint32_t st, na, nb;
            seg(mid, st, na, nb);
            if (st <= od) lo = mid;
            else hi = mid;
        }
        uint32_t sg = lo, st, na, nb;
        seg(sg, st, na, nb);
        // merge path of diagonal od - st inside pair sg
        const uint32_t dd = od - st;
        uint32_t l2 = dd > nb ? dd - nb : 0u, h2 = min(dd, na);
        while (l2 < h2) {
            const uint32_t mid = (l2 + h2) >> 1;
            if (sk[st + na + dd - 1 - mid] < sk[st + mid]) h2 = mid;
            else l2 = mid + 1;
        }
        // the two run heads stay in registers: one shared load per output
        uint32_t ai = st + l2, ae = st + na, bi = st + na + (dd - l2), be = st + na + nb;
        O ka = sk[min(ai, (uint32_t)DM_OT - 1)], kb = sk[min(bi, (uint32_t)DM_OT - 1)];
        cnt = (int)min((uint32_t)DM_IT, total - od);
#pragma unroll
        for (int i = 0; i < DM_IT; ++i) {
            if (i < cnt) {
                if (ai == ae && bi == be && sg + 1 < nseg) {   // segment done: the next non-empty one
                    do {
                        ++sg;
                        seg(sg, st, na, nb);
                    } while (na + nb == 0 && sg + 1 < nseg);
                    ai = st;
                    ae = st + na;
                    bi = ae;
                    be = ae + nb;
                    ka = sk[min(ai, (uint32_t)DM_OT - 1)];
                    kb = sk[min(bi, (uint32_t)DM_OT - 1)];
                }
                const bool take_b = ai == ae || (bi < be && kb < ka);
                x[i] = take_b ? kb : ka;
                if (HV) xv[i] = sv[take_b ? bi : ai];
                if (take_b) {
                    ++bi;
                    kb = sk[min(bi, (uint32_t)DM_OT - 1)];
                } else {
                    ++ai;
                    ka = sk[min(ai, (uint32_t)DM_OT - 1)];
                }
            }
        }
    }
    __syncthreads();                                   // staged inputs consumed
#pragma unroll
    for (int i = 0; i < DM_IT; ++i) {
        if (i < cnt) {
            sk[od + i] = x[i];
            if (HV) sv[od + i] = xv[i];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < total; t += DM_NT) {
        dst[o0 + t] = KT::key(sk[t]);
        if (HV) vdst[o0 + t] = sv[t];
    }
}

template <class KT, bool HV>
constexpr size_t det_merge_smem() {
    constexpr size_t ot = DmCfg<KT, HV>::OT;
    return sizeof(typename KT::O) * ot + sizeof(uint32_t) * 3 * DM_TBL + (HV ? sizeof(uint32_t) * ot : 0);
}

// Steps 4 and 5 of Algorithm 1 on the sorted sequences w1 (payloads vw1):
// bucket sizes and offsets into bsize / boff, the merged buckets into kout.
// w2 / vw2: scratch of n keys (and payloads) for the alternate merge passes.
template <class KT, bool HV>
void det_merge_steps(Ctx& c, const typename KT::T* w1, const uint32_t* vw1, typename KT::T* w2, uint32_t* vw2,
                     typename KT::T* kout, uint32_t* vout, uint32_t n, uint32_t p, const typename KT::O* spl_o,
                     const uint32_t* spl_t, uint32_t* boff, uint32_t* bsize) {
    uint32_t* pos = c.ar.take<uint32_t>((size_t)p * (p + 1));
    uint32_t* hist = c.ar.take<uint32_t>((size_t)p * p);
    uint32_t* col = c.ar.take<uint32_t>((size_t)p * p);
    constexpr int DM_OT = DmCfg<KT, HV>::OT;
    uint32_t* part = c.ar.take<uint32_t>(2 * ((size_t)n / DM_OT + 2));
    if (!c.live()) return;
    OS_LAUNCH(c.st, "k_det_split",
              k_det_split<KT><<<grid_for((uint64_t)p * (p + 1), 256), 256, 0, c.st>>>(w1, n, p, spl_o, spl_t, pos));
    OS_LAUNCH(c.st, "k_det_pieces", k_det_pieces<<<grid_for((uint64_t)p * p, 256), 256, 0, c.st>>>(pos, p, hist));
    OS_LAUNCH(c.st, "k_column_scan",
              k_column_scan<<<grid_for((uint64_t)p * 32, 256), 256, 0, c.st>>>(hist, p, p, col, bsize));
    OS_LAUNCH(c.st, "k_bucket_offsets", k_bucket_offsets<<<1, 1024, 0, c.st>>>(bsize, p, boff));
    int passes = 0;
    while ((1u << passes) < p) ++passes;
    const size_t sm = det_merge_smem<KT, HV>();
    smem_at_least(reinterpret_cast<const void*>(k_det_merge<KT, HV>), sm);
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + DM_OT - 1) / DM_OT);
    // the pieces into their buckets: into the buffer the first merge pass reads
    typename KT::T* lay = ((passes - 1) % 2 == 0) ? w2 : kout;
    uint32_t* vlay = ((passes - 1) % 2 == 0) ? vw2 : vout;
    OS_LAUNCH(c.st, "k_det_gather",
              k_det_gather<KT, HV><<<grid_for((uint64_t)p * p * 32, 256), 256, 0, c.st>>>(w1, vw1, n, p, pos, col,
                                                                                          boff, lay, vlay));
    const typename KT::T* src = lay;
    const uint32_t* vsrc = vlay;
    for (int l = 1; l <= passes && ntiles > 0; ++l) {
        typename KT::T* dst = ((passes - l) % 2 == 0) ? kout : w2;
        uint32_t* vdst = ((passes - l) % 2 == 0) ? vout : vw2;
        OS_LAUNCH(c.st, "k_det_partition",
                  k_det_partition<KT, DM_OT><<<grid_for((uint64_t)(ntiles + 1) * 32, 256), 256, 0, c.st>>>(
                      l, p, n, src, col, bsize, boff, part));
        OS_LAUNCH(c.st, "k_det_merge",
                  k_det_merge<KT, HV><<<ntiles, DM_NT, sm, c.st>>>(l, p, n, src, vsrc, dst, vdst, col, bsize, boff,
                                                                   part));
        src = dst;
        vsrc = vdst;
    }
}

}  // namespace ossort
