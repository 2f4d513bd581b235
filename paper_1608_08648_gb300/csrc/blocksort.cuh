// Stable block-wide merge sort in registers and shared memory (the bucket
// sort of step 5).  NT threads each own IT consecutive keys and sort them in
// registers: with a payload by an odd-even transposition network (adjacent
// compare-exchange on strict '>', hence stable); keys only by Batcher's
// odd-even merge sort network (equal keys are indistinguishable there).  Then
// log2(NT) rounds merge pairs of sorted runs: every thread finds where its IT
// outputs start with a merge-path binary search over the two runs in shared
// memory and merges them serially, taking from the left run on ties (stable).
#pragma once

#include "common.cuh"

namespace ossort {

// Padded shared-memory index: one spare slot per 128 bytes, so that a thread
// reading its IT consecutive elements does not collide with its neighbours.
template <class X> __device__ __forceinline__ int pad_idx(int i) {
    return i + (i >> (sizeof(X) == 4 ? 5 : 4));
}
template <class X> __host__ __device__ constexpr int padded_len(int n) {
    return n + (n >> (sizeof(X) == 4 ? 5 : 4)) + 1;
}

// Sorts sk[0, total) (and the payload sv alongside when HV), where total is a
// power-of-two multiple of IT no larger than NT*IT; the caller fills unused slots
// of [0, total) with the maximum key.  Both arrays use pad_idx addressing.
// Must be called by all NT threads; starts and ends with a __syncthreads.
template <class O, bool HV, int NT, int IT>
__device__ void block_merge_sort(O* sk, uint32_t* sv, int total) {
    const int tid = threadIdx.x;
    const bool active = tid * IT < total;
    O k[IT];
    uint32_t v[IT];
    __syncthreads();
    if (active) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            k[i] = sk[pad_idx<O>(tid * IT + i)];
            if (HV) v[i] = sv[pad_idx<uint32_t>(tid * IT + i)];
        }
        if (HV) {
            // Odd-even transposition sort of the IT keys: adjacent compare-exchange
            // on strict '>' keeps equal keys in order (stable, so payloads follow
            // the stable order).
#pragma unroll
            for (int r = 0; r < IT; ++r) {
#pragma unroll
                for (int j = r & 1; j + 1 < IT; j += 2) {
                    if (k[j + 1] < k[j]) {
                        O t = k[j]; k[j] = k[j + 1]; k[j + 1] = t;
                        uint32_t w = v[j]; v[j] = v[j + 1]; v[j + 1] = w;
                    }
                }
            }
        } else {
            // Keys only: equal keys are identical bit patterns, so any sorting
            // network will do; Batcher's odd-even merge sort (63 compare-exchanges
            // for 16 keys, 19 for 8), branch-free with min / max.
#pragma unroll
            for (int pp = 1; pp < IT; pp <<= 1)
#pragma unroll
                for (int kk = pp; kk >= 1; kk >>= 1)
#pragma unroll
                    for (int j = kk % pp; j + kk < IT; j += 2 * kk)
#pragma unroll
                        for (int i = 0; i < kk; ++i)
                            if (i + j + kk < IT && (i + j) / (2 * pp) == (i + j + kk) / (2 * pp)) {
                                const O a = k[i + j], b = k[i + j + kk];
                                k[i + j] = a < b ? a : b;
                                k[i + j + kk] = a < b ? b : a;
                            }
        }
    }
    for (int run = IT; run < total; run *= 2) {
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                sk[pad_idx<O>(tid * IT + i)] = k[i];
                if (HV) sv[pad_idx<uint32_t>(tid * IT + i)] = v[i];
            }
        }
        __syncthreads();
        if (active) {
            const int me = tid * IT;
            const int base = me & ~(2 * run - 1);
            const int d = me - base;           // output diagonal inside the pair
            const int A = base, B = base + run;
            int lo = d > run ? d - run : 0;
            int hi = d < run ? d : run;
            while (lo < hi) {                  // count of left-run keys among the first d outputs
                int mid = (lo + hi) >> 1;
                if (sk[pad_idx<O>(A + mid)] <= sk[pad_idx<O>(B + d - 1 - mid)]) lo = mid + 1;
                else hi = mid;
            }
            int ai = lo, bi = d - lo;
            O ka = sk[pad_idx<O>(A + min(ai, run - 1))];
            O kb = sk[pad_idx<O>(B + min(bi, run - 1))];
            uint32_t va = 0, vb = 0;
            if (HV) {
                va = sv[pad_idx<uint32_t>(A + min(ai, run - 1))];
                vb = sv[pad_idx<uint32_t>(B + min(bi, run - 1))];
            }
            // Branch-free serial merge: one shared-memory read per output.
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const bool takeA = (bi >= run) || (ai < run && ka <= kb);
                k[i] = takeA ? ka : kb;
                if (HV) v[i] = takeA ? va : vb;
                ai += takeA ? 1 : 0;
                bi += takeA ? 0 : 1;
                const int q = takeA ? A + min(ai, run - 1) : B + min(bi, run - 1);
                const O nk = sk[pad_idx<O>(q)];
                ka = takeA ? nk : ka;
                kb = takeA ? kb : nk;
                if (HV) {
                    const uint32_t nv = sv[pad_idx<uint32_t>(q)];
                    va = takeA ? nv : va;
                    vb = takeA ? vb : nv;
                }
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            sk[pad_idx<O>(tid * IT + i)] = k[i];
            if (HV) sv[pad_idx<uint32_t>(tid * IT + i)] = v[i];
        }
    }
    __syncthreads();
}

// Smallest power-of-two multiple of IT that holds n keys.
template <int IT> __device__ __forceinline__ int sort_extent(int n) {
    int t = IT;
    while (t < n) t <<= 1;
    return t;
}

}  // namespace ossort
