// Step 4 of Algorithms 1 and 2 at the top level, keys without a payload: the
// classify and scatter passes over 16-byte vectors of keys (4 int32 keys or 2
// 64-bit keys per load and per lane), so that every memory instruction moves a
// whole vector and the per-key work is the bucket lookup, one shared-memory
// atomic and one staged store.
//
//   k_classify_v : bucket of every key (the number of splitters below (key, tag)
//                  in the tagged order of Section 2.2, tag = position), two-byte
//                  bucket ids stored four (two) at a time, per-CTA bucket counts.
//   k_scatter_v  : the same units again: every key ranked inside its unit's part
//                  of its bucket by a shared-memory counter, staged grouped by
//                  bucket, written out as contiguous runs.
//
// Both walk the units of SUPER keys that k_classify / k_scatter walk (CTA g owns
// units [tile_lo(g), tile_lo(g+1))), so the counts of one feed the other.  Keys
// alone need no order inside a bucket (equal keys are identical), which is what
// lets one counter per bucket hand out the slots.  A key array that is not 16-byte
// aligned takes the same passes with one key per load.
#pragma once

#include "bulk.cuh"
#include "kernels.cuh"
#include "segkernels.cuh"

namespace ossort {

// Keys per 16-byte vector.
template <class T> struct VecOf { static constexpr int N = 16 / sizeof(T); };

template <class T>
__device__ __forceinline__ void unpack16(const uint4& v, T (&k)[VecOf<T>::N]) {
    if constexpr (sizeof(T) == 4) {
        k[0] = (T)v.x;
        k[1] = (T)v.y;
        k[2] = (T)v.z;
        k[3] = (T)v.w;
    } else {
        k[0] = (T)(((uint64_t)v.y << 32) | v.x);
        k[1] = (T)(((uint64_t)v.w << 32) | v.z);
    }
}

// Bucket of (o, t): as split_find, with the bin index clamped instead of the
// range tests: a key below the smallest splitter lands in bin 0, whose
// splitters all compare above it; a key above the largest lands in the last
// bin, whose splitters all compare below it.  The count is exact either way
// (the splitters below (o, t) are a prefix of every bin's range).  Bins with
// two or more splitters are binary searched.
template <class O>
__device__ __forceinline__ int split_find_clamped(const SplitTable<O>& tb, O o, uint32_t t, uint32_t last_bin) {
    const O d = o - tb.lo;
    uint32_t idx = o < tb.lo ? 0u : (uint32_t)min((O)(d >> tb.shift), (O)last_bin);
    int j = (int)tb.lut[idx];
    int k = (int)tb.lut[idx + 1];
    if (k - j > 1) {
        while (j < k) {
            const int mid = (j + k) >> 1;
            if (tb.template below<true>(mid, o, t)) j = mid + 1;
            else k = mid;
        }
        return j;
    }
    return (j < k && tb.template below<true>(j, o, t)) ? j + 1 : j;
}

// Add one lane's VEC bucket ids to the shared counters cnt: one atomic when the
// whole warp's keys share a bucket, one per lane when a lane's keys do, else one
// per key.  Ids >= p (keys past the end) go to the spare counter cnt[p].
template <int VEC>
__device__ __forceinline__ void count_vec(const uint32_t (&b)[VEC], uint32_t* cnt) {
    bool same = true;
#pragma unroll
    for (int j = 1; j < VEC; ++j) same &= b[j] == b[0];
    const uint32_t b0 = __shfl_sync(0xffffffffu, b[0], 0);
    const unsigned all = __ballot_sync(0xffffffffu, same && b[0] == b0);
    if (all == 0xffffffffu) {
        if ((threadIdx.x & 31) == 0) atomicAdd(&cnt[b0], 32u * VEC);
    } else if (same) {
        atomicAdd(&cnt[b[0]], (uint32_t)VEC);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) atomicAdd(&cnt[b[j]], 1u);
    }
}

// Slots for one lane's VEC keys among the keys of their buckets in this unit,
// taken from the shared counters cnt (as count_vec, returning the old values).
template <int VEC>
__device__ __forceinline__ void slot_vec(const uint32_t (&b)[VEC], uint32_t* cnt, uint32_t (&slot)[VEC]) {
    bool same = true;
#pragma unroll
    for (int j = 1; j < VEC; ++j) same &= b[j] == b[0];
    const int lane = threadIdx.x & 31;
    const uint32_t b0 = __shfl_sync(0xffffffffu, b[0], 0);
    const unsigned all = __ballot_sync(0xffffffffu, same && b[0] == b0);
    if (all == 0xffffffffu) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&cnt[b0], 32u * VEC);
        base = __shfl_sync(0xffffffffu, base, 0) + (uint32_t)lane * VEC;
#pragma unroll
        for (int j = 0; j < VEC; ++j) slot[j] = base + j;
    } else if (same) {
        const uint32_t base = atomicAdd(&cnt[b[0]], (uint32_t)VEC);
#pragma unroll
        for (int j = 0; j < VEC; ++j) slot[j] = base + j;
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) slot[j] = atomicAdd(&cnt[b[j]], 1u);
    }
}

// Classify, keys only or with a payload (the payload does not take part).
// Threads NT, units of SUPER keys (the scatter's).  hist is bucket-major:
// hist[b * G + g].  copy: NULL, or a device array that receives every key as it
// is read (the keys then come from host memory over the host link, read once).
template <class KT, int NT, int SUPER>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : (NT >= 512 ? 2 : 4))
k_classify_v(const typename KT::T* __restrict__ keys, uint32_t n, const typename KT::O* __restrict__ spl_o,
             const uint32_t* __restrict__ spl_t, int p, int lbits, uint32_t* __restrict__ hist,
             uint16_t* __restrict__ bid, uint32_t ntiles, typename KT::T* __restrict__ copy) {
    using T = typename KT::T;
    using O = typename KT::O;
    constexpr int VEC = VecOf<T>::N;
    constexpr int R = 16 / VEC;                      // vectors in flight per thread: 16 keys
    extern __shared__ __align__(16) char smem[];
    SplitTable<O> tb;
    tb.bind(smem, p - 1, lbits);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + split_table_bytes<O>(p - 1, lbits));   // [p + 1]
    for (int i = threadIdx.x; i < p - 1; i += NT) tb.set(i, spl_o[i], spl_t[i]);
    for (int b = threadIdx.x; b <= p; b += NT) cnt[b] = 0;
    __syncthreads();
    split_table_finish<O>(tb, p - 1, lbits);
    const uint32_t last_bin = (1u << lbits) - 1;
    const uint32_t G = gridDim.x, g = blockIdx.x;
    const uint32_t t0 = tile_lo(g, G, ntiles), t1 = tile_lo(g + 1, G, ntiles);
    const bool vec_ok = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    const uint32_t e_lo = t0 * (uint32_t)SUPER;
    const uint32_t e_hi = min(n, t1 * (uint32_t)SUPER);
    if (vec_ok) {
        constexpr uint32_t STEP = (uint32_t)NT * R * VEC;
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += STEP) {
            uint4 raw[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t e = e0 + ((uint32_t)r * NT + threadIdx.x) * VEC;
                if (e + VEC <= e_hi) {
                    raw[r] = __ldg(reinterpret_cast<const uint4*>(keys + e));
                    if (copy) *reinterpret_cast<uint4*>(copy + e) = raw[r];
                } else {
                    T tk[VEC];
#pragma unroll
                    for (int j = 0; j < VEC; ++j) tk[j] = e + j < e_hi ? keys[e + j] : T(0);
                    if (copy)
#pragma unroll
                        for (int j = 0; j < VEC; ++j)
                            if (e + j < e_hi) copy[e + j] = tk[j];
                    if constexpr (sizeof(T) == 4)
                        raw[r] = make_uint4((uint32_t)tk[0], (uint32_t)tk[1], (uint32_t)tk[2], (uint32_t)tk[3]);
                    else
                        raw[r] = make_uint4((uint32_t)(uint64_t)tk[0], (uint32_t)((uint64_t)tk[0] >> 32),
                                            (uint32_t)(uint64_t)tk[1], (uint32_t)((uint64_t)tk[1] >> 32));
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t e = e0 + ((uint32_t)r * NT + threadIdx.x) * VEC;
                T k[VEC];
                unpack16<T>(raw[r], k);
                uint32_t b[VEC];
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    b[j] = e + j < e_hi ? (uint32_t)split_find_clamped<O>(tb, KT::ord(k[j]), e + j, last_bin)
                                        : (uint32_t)p;
                if (e + VEC <= e_hi) {
                    if constexpr (VEC == 4)
                        *reinterpret_cast<uint2*>(bid + e) = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
                    else
                        *reinterpret_cast<uint32_t*>(bid + e) = b[0] | (b[1] << 16);
                } else {
#pragma unroll
                    for (int j = 0; j < VEC; ++j)
                        if (e + j < e_hi) bid[e + j] = (uint16_t)b[j];
                }
                count_vec<VEC>(b, cnt);
            }
        }
    } else {
        constexpr uint32_t STEP = (uint32_t)NT * 4;
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += STEP) {
            uint32_t b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t e = e0 + (uint32_t)r * NT + threadIdx.x;
                b[r] = p;
                if (e < e_hi) {
                    const T k = keys[e];
                    if (copy) copy[e] = k;
                    b[r] = (uint32_t)split_find_clamped<O>(tb, KT::ord(k), e, last_bin);
                    bid[e] = (uint16_t)b[r];
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t one[1] = {b[r]};
                count_vec<1>(one, cnt);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < p; b += NT) hist[(size_t)b * G + g] = cnt[b];
}

// Scatter of keys without a payload: units of SUPER keys, NT threads, each
// thread holding SUPER / NT keys of a unit as 16-byte vectors.  Two unit
// buffers in shared memory: while the CTA ranks and writes out unit t from one,
// the bulk copies of unit t + 1 (keys and bucket ids) land in the other, issued
// by thread 0 as soon as unit t - 1 left that buffer.  A unit's buffer is also
// its staging area: once every thread holds its keys in registers, the keys
// are written back grouped by bucket and streamed out as runs.  Units that are
// not whole (the array's last) or keys that are not 16-byte aligned are read
// with plain loads.
template <class T>
__host__ __device__ constexpr size_t scatter_v_smem(int p, int super) {
    return 2 * ((sizeof(T) + sizeof(uint16_t)) * (size_t)super) + 2 * sizeof(uint64_t) +
           sizeof(uint32_t) * (size_t)(3 * p + 2) + sizeof(uint32_t) * 33 + 64;
}

template <class KT, int NT, int SUPER>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : (NT >= 512 ? 2 : 4))
k_scatter_v(const typename KT::T* __restrict__ keys, const uint16_t* __restrict__ bid, uint32_t n, int p,
            const uint32_t* __restrict__ col, uint32_t cstep, const uint32_t* __restrict__ boff,
            typename KT::T* __restrict__ out, uint32_t ntiles, uint32_t* status) {
    using T = typename KT::T;
    constexpr int VEC = VecOf<T>::N;
    constexpr int NV = SUPER / (NT * VEC);           // vectors per thread per unit
    static_assert(NV * NT * VEC == SUPER, "a unit is a whole number of vectors per thread");
    constexpr uint32_t KBYTES = sizeof(T) * SUPER, BBYTES = sizeof(uint16_t) * SUPER;
    constexpr uint32_t UBYTES = KBYTES + BBYTES;      // one unit buffer: keys, then bucket ids
    extern __shared__ __align__(16) char smem[];
    char* q = smem + 2 * UBYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(q);     q += 2 * sizeof(uint64_t);
    uint32_t* toff = reinterpret_cast<uint32_t*>(q);     q += sizeof(uint32_t) * (p + 1);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(q);   q += sizeof(uint32_t) * p;
    int32_t* delta = reinterpret_cast<int32_t*>(q);      q += sizeof(uint32_t) * (p + 1);
    uint32_t* scratch = reinterpret_cast<uint32_t*>(q);  q += sizeof(uint32_t) * 32;   // one word per warp
    uint32_t* stop = reinterpret_cast<uint32_t*>(q);

    // the classify ran with cstep CTAs per scatter CTA (its CTAs 2g, 2g+1 for
    // cstep = 2 cover exactly this CTA's units): col has G * cstep columns and
    // this CTA's keys of bucket b start at column g * cstep
    const uint32_t G = gridDim.x, g = blockIdx.x;
    for (int b = threadIdx.x; b < p; b += NT) cursor[b] = boff[b] + col[((size_t)b * G + g) * cstep];
    const uint32_t t0 = tile_lo(g, G, ntiles), t1 = tile_lo(g + 1, G, ntiles);
    const bool vec_ok = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    auto whole = [&](uint32_t t) { return (uint64_t)(t + 1) * SUPER <= n; };
    auto issue = [&](uint32_t t, int sb) {           // thread 0: unit t into buffer sb
        char* u = smem + sb * UBYTES;
        mbar_arrive_expect_tx(&mbar[sb], UBYTES);
        bulk_g2s(u, keys + (size_t)t * SUPER, KBYTES, &mbar[sb]);
        bulk_g2s(u + KBYTES, bid + (size_t)t * SUPER, BBYTES, &mbar[sb]);
    };
    // copies issued into / waits completed on buffer 0 and 1 (issued: thread 0 only)
    uint32_t issued0 = 0, issued1 = 0, used0 = 0, used1 = 0;
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        *stop = 0;
        fence_mbar_init();
        if (vec_ok) {
            if (t0 < t1 && whole(t0)) {
                issue(t0, 0);
                ++issued0;
            }
            if (t0 + 1 < t1 && whole(t0 + 1)) {
                issue(t0 + 1, 1);
                ++issued1;
            }
        }
    }
    __syncthreads();
    for (uint32_t t = t0; t < t1; ++t) {
        const int sb = (int)((t - t0) & 1);
        T* sk = reinterpret_cast<T*>(smem + sb * UBYTES);
        uint16_t* sbk = reinterpret_cast<uint16_t*>(smem + sb * UBYTES + KBYTES);
        const uint32_t ubase = t * (uint32_t)SUPER;
        const uint32_t uend = min(n, ubase + (uint32_t)SUPER);
        const bool staged = vec_ok && whole(t);
        T k[NV][VEC];
        uint32_t b[NV][VEC];
        if (staged) {
            const uint32_t u = sb ? used1 : used0;
            if (!mbar_wait(&mbar[sb], u & 1)) {
                atomicOr(status, ERR_TIMEOUT);
                atomicOr(stop, 1u);
            }
            if (sb) ++used1;
            else ++used0;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint32_t li = ((uint32_t)v * NT + threadIdx.x) * VEC;     // index inside the unit
                unpack16<T>(*reinterpret_cast<const uint4*>(sk + li), k[v]);
                if constexpr (VEC == 4) {
                    const uint2 w = *reinterpret_cast<const uint2*>(sbk + li);
                    b[v][0] = w.x & 0xFFFFu;
                    b[v][1] = w.x >> 16;
                    b[v][2] = w.y & 0xFFFFu;
                    b[v][3] = w.y >> 16;
                } else {
                    const uint32_t w = *reinterpret_cast<const uint32_t*>(sbk + li);
                    b[v][0] = w & 0xFFFFu;
                    b[v][1] = w >> 16;
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint32_t e = ubase + ((uint32_t)v * NT + threadIdx.x) * VEC;
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    const bool in = e + j < uend;
                    k[v][j] = in ? keys[e + j] : T(0);
                    b[v][j] = in ? (uint32_t)bid[e + j] : (uint32_t)p;
                }
            }
        }
        for (int x = threadIdx.x; x <= p; x += NT) toff[x] = 0;
        __syncthreads();   // counters cleared; every thread holds its keys (the buffer is free for staging)
        if (*stop) break;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            uint32_t slot[VEC];
            slot_vec<VEC>(b[v], toff, slot);
#pragma unroll
            for (int j = 0; j < VEC; ++j) b[v][j] = (b[v][j] << 16) | slot[j];   // bucket, slot (both < 2^16)
        }
        const uint32_t tvalid = block_exclusive_scan(toff, p, scratch);
        // each bucket's cursor belongs to one thread (same x in both loops);
        // dst = delta[b] + staged index
        for (int x = threadIdx.x; x < p; x += NT) {
            const uint32_t lo = toff[x], hi = x + 1 < p ? toff[x + 1] : tvalid;
            delta[x] = (int32_t)(cursor[x] - lo);
            cursor[x] += hi - lo;
        }
        // Range checks without a branch per key: every access is predicated on
        // its check, and a failed check is reported once per thread afterwards.
        uint32_t bad_site = 0, bad_at = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                const uint32_t bbk = b[v][j] >> 16;
                const uint32_t loc = toff[min(bbk, (uint32_t)p)] + (b[v][j] & 0xFFFFu);
                const bool real = bbk < (uint32_t)p, ok = real && loc < (uint32_t)SUPER;
                if (ok) {
                    sk[loc] = k[v][j];
                    sbk[loc] = (uint16_t)bbk;
                }
                if (real && !ok) bad_site = 10, bad_at = loc;
            }
        __syncthreads();
        for (uint32_t jj = threadIdx.x; jj < tvalid; jj += NT) {
            const uint32_t bbk = sbk[jj];      // >= p: a slot no key was staged to (after a failed check)
            const uint32_t dst = (uint32_t)(delta[min(bbk, (uint32_t)p)] + (int32_t)jj);
            const bool ok = bbk < (uint32_t)p && dst < n;
            if (ok) out[dst] = sk[jj];
            if (!ok) bad_site = bbk < (uint32_t)p ? 11u : 12u, bad_at = bbk < (uint32_t)p ? dst : jj;
        }
        if (bad_site) flag_bounds(status, bad_site, bad_at);
        fence_proxy_async_smem();   // this thread's reads and writes of the buffer before the next copy into it
        __syncthreads();
        if (threadIdx.x == 0 && vec_ok && t + 2 < t1 && whole(t + 2)) {
            issue(t + 2, sb);
            if (sb) ++issued1;
            else ++issued0;
        }
    }
    // after a timeout: let copies still in flight land before the CTA's shared
    // memory is released (bounded again)
    if (threadIdx.x == 0) {
        while (used0 < issued0 && mbar_wait(&mbar[0], used0 & 1)) ++used0;
        while (used1 < issued1 && mbar_wait(&mbar[1], used1 & 1)) ++used1;
    }
}

// ---------------------------------------------------------------------------
// The bucket phase's classify (k_seg_classify of segkernels.cuh) over 16-byte
// vectors.  A tile [A, B) of absolute positions starts anywhere: the whole
// vector slots inside it are loaded as vectors, the at most VEC - 1 keys at
// either end one by one.
// ---------------------------------------------------------------------------

template <class KT>
size_t seg_classify_v_smem(int maxp) {
    int lb = 1;
    while ((1 << lb) < 4 * maxp && lb < 13) ++lb;
    return split_table_bytes<typename KT::O>(maxp, lb) + sizeof(uint32_t) * (maxp + 1);
}

__device__ __forceinline__ int seg_lbits_v(int p) {
    int b = 1;
    while ((1 << b) < 4 * p && b < 13) ++b;
    return b;
}

template <class KT>
__global__ void __launch_bounds__(SEG_NT, 4)
k_seg_classify_v(const typename KT::T* __restrict__ keys, const SegRec* __restrict__ rec,
                 const uint32_t* __restrict__ tile0, uint32_t nseg, const SegTotals* __restrict__ tot,
                 const typename KT::O* __restrict__ spl_o, const uint32_t* __restrict__ spl_t, int maxp,
                 uint32_t* __restrict__ hist, uint16_t* __restrict__ bid) {
    using T = typename KT::T;
    using O = typename KT::O;
    constexpr int VEC = VecOf<T>::N;
    constexpr int R = 4;
    extern __shared__ __align__(16) char smem[];
    int maxlb = 1;
    while ((1 << maxlb) < 4 * maxp && maxlb < 13) ++maxlb;
    SplitTable<O> tb;
    tb.bind(smem, maxp, maxlb);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + split_table_bytes<O>(maxp, maxlb));   // [maxp + 1]
    const uint32_t T_ = tot->tiles;
    const uint32_t t0 = tile_lo(blockIdx.x, gridDim.x, T_), t1 = tile_lo(blockIdx.x + 1, gridDim.x, T_);
    const bool vec_ok = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    SegRec r{};
    uint32_t seg_t0 = 0, seg_t1 = 0, last_bin = 0;
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
            const int lb = seg_lbits_v((int)r.p);
            split_table_finish<O>(tb, (int)r.p - 1, lb);
            last_bin = (1u << lb) - 1;
        }
        const int p = (int)r.p;
        const uint32_t tl = t - seg_t0;
        for (int b = threadIdx.x; b <= p; b += SEG_NT) cnt[b] = 0;
        __syncthreads();
        const uint32_t A = r.beg + tl * r.tile, B = r.beg + min(r.len, (tl + 1) * r.tile);
        // whole vector slots [fa, fb) without range tests; the at most 2 (VEC - 1)
        // keys of [A, B) outside them (and every key when the keys are not
        // 16-byte aligned) key by key
        const uint32_t fa = vec_ok ? (A + VEC - 1) / VEC : B / VEC + 1;
        const uint32_t fb = vec_ok ? max(B / VEC, fa) : fa;
        for (uint32_t v0 = fa; v0 < fb; v0 += (uint32_t)SEG_NT * R) {
            uint4 raw[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const uint32_t vs = v0 + (uint32_t)q * SEG_NT + threadIdx.x;
                if (vs < fb) raw[q] = __ldg(reinterpret_cast<const uint4*>(keys + (size_t)vs * VEC));
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const uint32_t vs = v0 + (uint32_t)q * SEG_NT + threadIdx.x;
                const uint32_t e = vs * VEC;
                uint32_t b[VEC];
                if (vs < fb) {
                    T k[VEC];
                    unpack16<T>(raw[q], k);
#pragma unroll
                    for (int j = 0; j < VEC; ++j)
                        b[j] = (uint32_t)split_find_clamped<O>(tb, KT::ord(k[j]), e + j - r.beg, last_bin);
                    if constexpr (VEC == 4)
                        *reinterpret_cast<uint2*>(bid + e) = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
                    else
                        *reinterpret_cast<uint32_t*>(bid + e) = b[0] | (b[1] << 16);
                } else {
#pragma unroll
                    for (int j = 0; j < VEC; ++j) b[j] = (uint32_t)p;     // the spare counter
                }
                count_vec<VEC>(b, cnt);
            }
        }
        {
            const uint32_t lo_end = min(B, fa * VEC);                 // keys [A, lo_end) before the slots
            const uint32_t hi_beg = max(lo_end, min(B, fb * VEC));    // keys [hi_beg, B) after them
            const uint32_t nlo = lo_end - A, nedge = nlo + (B - hi_beg);
            for (uint32_t i = threadIdx.x; i < nedge; i += SEG_NT) {
                const uint32_t e = i < nlo ? A + i : hi_beg + (i - nlo);
                const uint32_t bk = (uint32_t)split_find_clamped<O>(tb, KT::ord(keys[e]), e - r.beg, last_bin);
                bid[e] = (uint16_t)bk;
                atomicAdd(&cnt[bk], 1u);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < p; b += SEG_NT) hist[r.hist0 + (size_t)b * r.ntile + tl] = cnt[b];
        __syncthreads();
    }
}

}  // namespace ossort
