/*
 * ossort: oversampling sample sort for one GB300 (sm_103a), after Gerbessiotis,
 * "Using parallelism techniques to improve sequential and multi-core sorting
 * performance" (arXiv 1608.08648).
 *
 * The library sorts n keys of one type, optionally carrying a uint32 payload,
 * with the paper's partitioning template: choose p-1 splitters by deterministic
 * regular oversampling (SqDet, Algorithm 1: sort p sequences, take r p regular
 * samples from each) or by random oversampling (SqRan, Algorithm 2: p s - 1
 * random keys), sort the sample, put every key into the bucket the splitters
 * give it, and sort every bucket.  Duplicate keys are handled with the tags of
 * Section 2.2: keys compare as (key, tag), where the tag is the key's original
 * position (SqRan) or its position in the concatenation of the sorted
 * sequences (SqDet), so equal keys spread over buckets exactly as distinct keys
 * would and the bucket-size bound of Lemma 1 holds for any input.
 *
 * Conventions shared by every entry point:
 *  - Device pointers are plain CUDA device (or managed) addresses.  The caller
 *    owns every buffer; the library never allocates device or pinned memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it and the call returns without waiting, except where
 *    an entry point says it synchronizes.
 *  - Order: int32 signed; uint64 unsigned; float64 IEEE 754 totalOrder
 *    (-inf < negatives < -0 < +0 < positives < +inf).  NaN keys are not
 *    supported (their position is unspecified, never an error).
 *  - The sort is stable: equal keys keep their input order, so a payload comes
 *    out in the order of a stable sort.
 *  - Limits: n <= OS_MAX_N, 1 <= p <= OS_MAX_P, 1 <= s, p * s <= OS_MAX_PS.
 *  - Every function returns an os_status code; nothing is thrown or aborted.
 */
#ifndef OSSORT_H
#define OSSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OSSORT_VERSION 10000           /* 1.0.0 */
#define OS_MAX_N   (1ull << 31)        /* largest n accepted */
#define OS_MAX_P   4096u               /* largest p accepted */
#define OS_MAX_PS  (1u << 24)          /* largest p * s accepted */

/* Key types. */
typedef enum { OS_I32 = 0, OS_U64 = 1, OS_F64 = 2 } os_key_t;

/* Splitter choice: SqDet (Algorithm 1) or SqRan (Algorithm 2). */
typedef enum { OS_DET = 0, OS_RAN = 1 } os_split_t;

/* Status codes. */
typedef enum {
    OS_OK = 0,
    OS_ERR_ARG = 1,          /* null pointer, bad type, p or s out of range, bad flags */
    OS_ERR_WS = 2,           /* workspace missing or smaller than os_workspace_size */
    OS_ERR_UNSUPPORTED = 3,  /* n, p or p s above the limits */
    OS_ERR_CUDA = 4,         /* a CUDA call failed; see os_last_cuda_error */
    OS_ERR_DEVICE = 5        /* a kernel reported an internal error in the status word */
} os_status;

/* Flags of os_params.flags. */
#define OS_STABLE 1u         /* accepted for clarity: the sort is always stable */

/*
 * Parameters of one sort (Algorithm 1 / Algorithm 2 call SqDet(X, n, p, SomeSort)).
 *   split : OS_DET or OS_RAN.
 *   p     : number of sequences and buckets (the paper's p).
 *   s     : OS_DET: the regular oversampling factor r = ceil(omega_n) of
 *           Algorithm 1, so each of the p sorted sequences gives r p samples,
 *           the sample holds r p^2 keys and the splitters are its (i r p)-th
 *           smallest, i = 1..p-1.  OS_RAN: the random oversampling factor s of
 *           Algorithm 2: the sample holds p s - 1 keys and the splitters are its
 *           (i s)-th smallest.
 *   seed  : OS_RAN only: sample position j is floor(u_j n / 2^64), u_j the j-th
 *           output of stream 1 of the counter-based SplitMix64 keyed by seed
 *           (sampling with replacement over the original positions).
 *   flags : 0 or OS_STABLE.
 * When the input is too small to sample (OS_RAN: n < 2 p s, the condition
 * p s < n/2 of Claim 1; OS_DET: ceil(n/p) < r p; or p = 1) the whole input is
 * one bucket: the call still sorts, and the statistics report p_used = 1.
 */
typedef struct {
    int32_t  split;
    uint32_t p;
    uint32_t s;
    uint32_t flags;
    uint64_t seed;
} os_params;

/*
 * Optional statistics of one sort.  The three arrays are HOST memory owned by
 * the caller (each may be NULL).  Filling them makes os_sort synchronize.
 *   p_used        : p, or 1 under the too-small rule above.
 *   depth         : deepest in-bucket repartition level any bucket needed
 *                   (0: every bucket was sorted directly in shared memory).
 *   max_bucket    : largest bucket |Y_j|.
 *   repart_keys   : keys moved by in-bucket repartitions, summed over levels
 *                   (every repartitioned key is read twice and written once).
 *   splitter_keys : p-1 keys of the key type (step 3), or unused when p_used = 1.
 *   splitter_tags : p-1 tags of the splitters (original position for OS_RAN,
 *                   position in the sorted-sequence concatenation for OS_DET).
 *   bucket_sizes  : p sizes |Y_j| (all of the input in bucket 0 when p_used = 1).
 */
typedef struct {
    uint32_t  p_used;
    uint32_t  depth;
    uint64_t  max_bucket;
    uint64_t  repart_keys;
    void*     splitter_keys;
    uint64_t* splitter_tags;
    uint64_t* bucket_sizes;
} os_stats;

/*
 * Workspace bytes os_sort needs for this key type, n, payload presence and
 * parameters.  The workspace is device memory, 256-byte aligned, that the caller
 * allocates once and may reuse for any later call with the same or smaller needs.
 * Errors: OS_ERR_ARG (bytes NULL or bad parameters), OS_ERR_UNSUPPORTED.
 */
int os_workspace_size(int key_type, uint64_t n, int has_vals, const os_params* prm,
                      size_t* bytes);

/*
 * Sort n keys (Algorithms 1 and 2 with the data-parallel organisation of the
 * traditional oversampling sort: sample, splitters, classify every key, scatter
 * the keys into contiguous buckets, sort every bucket).
 *   d_keys_in  : n keys, device.  Read only, unless it equals d_keys_out.
 *   d_keys_out : n keys, device; may equal d_keys_in (in place).
 *   d_vals_in  : n uint32 payloads or NULL; d_vals_out must then be non-NULL
 *                (may equal d_vals_in).
 *   d_ws, ws_bytes : workspace of at least os_workspace_size bytes.
 *   stats      : NULL, or statistics to fill (this synchronizes the stream and
 *                also returns OS_ERR_DEVICE if a kernel flagged an error).
 * Buffers must not overlap other than in the in-place cases named above.
 */
int os_sort(int key_type, const void* d_keys_in, void* d_keys_out,
            const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
            const os_params* prm, void* d_ws, size_t ws_bytes, void* stream,
            os_stats* stats);

/*
 * Bytes of workspace os_sort_host needs: os_workspace_size plus room for the
 * device copies of the keys (and payloads).
 */
int os_workspace_size_host(int key_type, uint64_t n, int has_vals, const os_params* prm,
                           size_t* bytes);

/*
 * Same sort on HOST buffers: copies the keys (and payloads) to the device
 * workspace, sorts, copies the result back and synchronizes the stream.  Host
 * buffers should be pinned for full copy bandwidth; h_keys_out may equal
 * h_keys_in.  Returns OS_ERR_DEVICE if a kernel flagged an error.
 */
int os_sort_host(int key_type, const void* h_keys_in, void* h_keys_out,
                 const uint32_t* h_vals_in, uint32_t* h_vals_out, uint64_t n,
                 const os_params* prm, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Sort without any device allocation by the caller.  (An addition of this
 * library with no counterpart in the paper.)  For callers that may not
 * allocate device memory -- code inside a framework that owns all device
 * memory, or a path that must not allocate after start-up -- and so cannot
 * provide the workspace os_sort asks for.  Same arguments and semantics as
 * os_sort without d_ws, ws_bytes and stats; the workspace is a scratch array of
 * OS_NOALLOC_SCRATCH_BYTES compiled into the library, held on every device
 * where this entry point has been called until the process exits.
 *  - A sort whose os_workspace_size exceeds OS_NOALLOC_SCRATCH_BYTES is refused
 *    with OS_ERR_UNSUPPORTED before any work is enqueued (64 MiB holds, e.g.,
 *    about 8.2 million int32 keys for SqRan p = 1024, s = 16 without payload).
 *  - The first call on a device, with that device current, looks up the
 *    scratch's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture on the device.
 *  - All calls on a device share the scratch: calls that overlap on the GPU
 *    (on different streams without ordering) race and must be avoided.
 *    Whatever must start at zero is cleared by every call.
 *  - Device-side error flags stay in the scratch and are not reported here.
 * Calls no allocating routine.
 */
#define OS_NOALLOC_SCRATCH_BYTES (64u << 20)

int os_sort_noalloc(int key_type, const void* d_keys_in, void* d_keys_out,
                    const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                    const os_params* prm, void* stream);

/*
 * Synchronize `stream` and read the device status word in the workspace of the
 * last sort enqueued with it: OS_OK, or OS_ERR_DEVICE with the raw error bits in
 * *bits (may be NULL).
 */
int os_check(const void* d_ws, void* stream, uint32_t* bits);

/*
 * Launch accounting (Section 3 of the paper times whole runs; the library also
 * reports where device time goes).  os_launch_count returns the number of
 * kernels this library has launched in the process.  Between os_profile_start
 * and os_profile_stop every launch is bracketed by a CUDA event pair on its
 * stream; os_profile_stop synchronizes on those events and returns, per kernel
 * name, the launches, total and longest device time (up to max_entries
 * entries; *n_entries receives the number of distinct kernels).  Profiling is
 * process-wide and meant for one benchmarking thread.
 */
typedef struct {
    char     name[48];
    uint64_t launches;
    double   total_ms;
    double   max_ms;
} os_kernel_time;

uint64_t os_launch_count(void);
int os_profile_start(void);
int os_profile_stop(os_kernel_time* out, int max_entries, int* n_entries);

/* The cudaError_t of the last failed CUDA call in this thread (0 if none). */
int os_last_cuda_error(void);

/* Text of a status code. */
const char* os_strerror(int status);

/* OSSORT_VERSION of the loaded library. */
int os_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OSSORT_H */
