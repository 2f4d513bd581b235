/*
 * CPU oracle for the oversampling sample sort of Gerbessiotis,
 * "Using parallelism techniques to improve sequential and multi-core sorting
 * performance" (SqDet, Algorithm 1; SqRan, Algorithm 2; duplicate handling,
 * Section 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library under test may include,
 * link or call this code; only the tests, the smoke check and the bench's CPU
 * baseline use it.  It is deliberately plain and slow: it follows the paper's
 * five steps in the paper's order (sort p chunks, sample, pick splitters,
 * binary-search the splitters into every sorted chunk, p-way merge per bucket)
 * with textbook merge sort and binary heaps, in plain C.
 */
#ifndef OSSORT_ORACLE_H
#define OSSORT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_I32 = 0, ORC_U64 = 1, ORC_F64 = 2, ORC_S32 = 3 };   /* key types; S32: 32-byte strings */
enum { ORC_DET = 0, ORC_RAN = 1 };                /* splitter choice */

/* SplitMix64 (Steele, Lea, Flood 2014) in counter form: the (i+1)-th output of the
 * sequential generator whose state starts at `state`, mix(state + (i+1) * GAMMA). */
uint64_t oracle_splitmix64_raw(uint64_t state, uint64_t i);

/* Output i of stream `stream` of `seed`: the raw generator started at
 * mix(seed + (stream + 1) * GAMMA). */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t stream, uint64_t i);

/* Random sample position j of SqRan: floor(u_j * n / 2^64) with u_j the j-th output
 * of stream 1 (sampling with replacement over original positions). */
uint64_t oracle_ran_index(uint64_t seed, uint64_t j, uint64_t n);

/* Three-way compare of two keys of type kt given as raw bit patterns (the value's
 * own bytes, zero-extended to 64 bits).  i32: signed order; u64: unsigned order;
 * f64: IEEE 754 total order without NaN (sign first, then magnitude). */
int oracle_key_cmp(int kt, uint64_t a_bits, uint64_t b_bits);

/* Three-way compare of two 32-byte string keys: memcmp order (unsigned bytes,
 * lexicographic), the order of the paper's experiments (Section 3). */
int oracle_str_cmp(const void* a, const void* b);

/*
 * SqDet / SqRan.  keys: n values of type kt (ORC_S32: n records of 32 bytes);
 * vals: n uint32 payloads or NULL.  Not reentrant for ORC_S32 (the key array
 * is held in a file-scope pointer during the call).
 * p >= 1 sequences / buckets; s >= 1 is the regular oversampling factor r of
 * Algorithm 1 (DET) or the random oversampling factor s of Algorithm 2 (RAN).
 *
 * Outputs (each may be NULL):
 *   out_keys / out_vals : the concatenation Y of the merged buckets (step 5);
 *                         when out_keys is NULL step 5 is skipped entirely.
 *   spl_keys, spl_tags  : the p-1 tagged splitters of step 3 (raw key values of
 *                         type kt).  DET tag: the flattened (sequence k, local
 *                         index l) tag of Section 2.2, i.e. start_k + l; RAN tag:
 *                         the original input position of the sampled key.
 *   bucket_sizes        : p sizes |Y_j| (step 4 counts summed over sequences).
 *   p_used              : p, or 1 when the input is too small to sample
 *                         (RAN: n < 2ps; DET: ceil(n/p) < s*p; or p == 1).
 * Returns 0 on success, -1 on a bad argument, -2 on allocation failure.
 */
int oracle_sort(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                int split, uint32_t p, uint32_t s, uint64_t seed,
                void* out_keys, uint32_t* out_vals,
                void* spl_keys, uint64_t* spl_tags, uint64_t* bucket_sizes,
                uint32_t* p_used);

/*
 * The multi-core adaptation of Section 2.4 (McDet / McRan): the same call with
 * the p sorts of step 1 split over `threads` POSIX threads (worker w takes the
 * sequences [w p / t, (w+1) p / t), t = min(threads, p)) and, when par_step5 is
 * non-zero, the p merges of step 5 split the same way (the paper's measured
 * McRan leaves step 5 sequential).  Same outputs as oracle_sort, bit for bit.
 */
int oracle_sort_mc(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                   int split, uint32_t p, uint32_t s, uint64_t seed,
                   void* out_keys, uint32_t* out_vals,
                   void* spl_keys, uint64_t* spl_tags, uint64_t* bucket_sizes,
                   uint32_t* p_used, uint32_t threads, int par_step5);

/* SomeSort alone on the whole input (the stable merge sort of step 1), the
 * stand-alone column of the paper's tables: (key, original index) order. */
int oracle_some_sort(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                     void* out_keys, uint32_t* out_vals);

#ifdef __cplusplus
}
#endif
#endif
