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
 *    owns every buffer; the sort entry points allocate no memory (the server
 *    keeps a small pinned status array per in-flight slot, os_sort_noalloc a
 *    static device array, and os_sort_host one copy stream per device).
 *  - Calls may come from several host threads at once, each with its own
 *    workspace.  The library's only process-wide device settings are its
 *    kernels' shared-memory limits, each written once per device before the
 *    kernel's first launch there, so no call changes state another call's
 *    launches depend on.
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

/* Key types.  OS_S32: 32-byte strings compared as memcmp does (unsigned bytes,
 * lexicographic) -- the keys of the paper's experiments (Section 3).  A sort of
 * OS_S32 keys partitions by the tagged order (first 8 bytes, tag), then orders
 * the keys that tie on their first 8 (16, 24) bytes by the next 8; it reads a
 * small count back from the device after each of those steps, so it
 * synchronizes its stream, and it is not accepted by the batched sort or the
 * server. */
typedef enum { OS_I32 = 0, OS_U64 = 1, OS_F64 = 2, OS_S32 = 3 } os_key_t;

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
#define OS_DET_MERGE 2u      /* OS_DET only: steps 4-5 as in Algorithm 1 -- split every sorted
                                sequence by a binary search of the splitters, then merge the p
                                pieces of every bucket -- instead of classifying and scattering
                                every key and sorting every bucket again.  Same output, same
                                splitters and bucket sizes. */

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
 *   flags : 0, OS_STABLE, OS_DET_MERGE (with OS_DET), or their or.
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
 *   splitter_keys : p-1 keys of the key type (step 3; 32 bytes each for OS_S32),
 *                   or unused when p_used = 1.
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
 * workspace, sorts, copies the result back and synchronizes the stream.  From
 * 2^22 keys on (except 32-byte strings) the buckets are sorted in eight ranges
 * and each range is copied back, on a stream the library creates once per
 * device, while the later ranges are still being sorted.  An OS_RAN sort of
 * keys alone from page-locked (device-addressable) host memory skips the
 * copy-in: it gathers its sample from the host buffer and its first classify
 * pass reads the keys from there once, writing the device copy as it goes.
 * Host buffers should be pinned for full copy bandwidth; h_keys_out may equal
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
 * os_sort without d_ws and ws_bytes; the workspace is a scratch array of
 * OS_NOALLOC_SCRATCH_BYTES compiled into the library.
 *  - A sort whose os_workspace_size exceeds OS_NOALLOC_SCRATCH_BYTES is refused
 *    with OS_ERR_UNSUPPORTED before any work is enqueued (64 MiB holds, e.g.,
 *    about 8.2 million int32 keys for SqRan p = 1024, s = 16 without payload).
 *  - The scratch is device memory of the library's module: under CUDA's default
 *    lazy module loading it is reserved on a device when the library's kernels
 *    are first loaded there; under eager loading (CUDA_MODULE_LOADING=EAGER) on
 *    every device context the library touches, whether or not this entry point
 *    is called.  Either way it stays until the process exits and counts against
 *    the device memory other users (e.g. a serving arena) can have.
 *  - The first call on a device, with that device current, looks up the
 *    scratch's device address (cudaGetSymbolAddress) and remembers it; make that
 *    first call before any stream capture on the device.  Calls after a
 *    cudaDeviceReset are not supported (the remembered address is stale).
 *  - All calls on a device share the scratch: calls that overlap on the GPU
 *    (on different streams without ordering) race and must be avoided.
 *    Whatever must start at zero is cleared by every call.
 *  - stats: NULL (asynchronous), or filled exactly as by os_sort; then the call
 *    synchronizes `stream` and returns OS_ERR_DEVICE if a kernel flagged an
 *    error in the status word (a skipped access or a bucket left too large).
 * Calls no allocating routine.
 */
#define OS_NOALLOC_SCRATCH_BYTES (64u << 20)

int os_sort_noalloc(int key_type, const void* d_keys_in, void* d_keys_out,
                    const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                    const os_params* prm, void* stream, os_stats* stats);

/*
 * ---- Batched segmented sort -------------------------------------------------
 * Many independent arrays held back to back in one buffer ("segments"), every
 * one sorted on its own by one fixed sequence of persistent kernels, each of
 * which walks the whole segment table.  (The paper sorts one array; the
 * batched form applies its SqRan template, Algorithm 2, to every segment, with
 * p and s chosen per length class as the paper's calibration of omega_n
 * through n suggests.)
 *
 * Segment g is [off[g], off[g+1]) of the buffer; it is sorted exactly as
 * os_sort sorts it alone with split = OS_RAN, the p and s of its length class
 * and seed u(seed, 2, g) (output g of stream 2 of the counter-based
 * SplitMix64 keyed by seed): the same splitters (tags are positions inside the
 * segment), the same bucket sizes, the same output.  A segment whose class has
 * p = 1, or that is shorter than 2 p s, is one bucket (the too-small rule of
 * os_params).
 *
 * Length classes: segment g belongs to the first class k with
 * len_g <= classes[k].max_len, or to the last class when it is longer than every
 * max_len.  max_len must increase strictly from class to class.
 *   p    : buckets per segment, 1 <= p <= OS_MAX_P (1: the segment is sorted
 *          whole, directly in shared memory when it fits one CTA).
 *   s    : random oversampling factor; p s <= OS_SEG_MAX_PS when p > 1.
 *   tile : keys per classify / scatter tile (a CTA's unit of work), a multiple
 *          of 2048 up to 16384.
 */
#define OS_SEG_MAX_CLASSES 32u
#define OS_SEG_MAX_PS      4096u
#define OS_SEG_MAX_NSEG    (1u << 26)

typedef struct {
    uint64_t max_len;
    uint32_t p;
    uint32_t s;
    uint32_t tile;
    uint32_t reserved;   /* must be 0 */
} os_seg_class;

/*
 * Optional per-segment statistics, written to DEVICE arrays owned by the caller
 * (each may be NULL) on the sort's stream, without synchronizing.
 *   bucket_base   : [nseg + 1]: first bucket of segment g in the two arrays
 *                   below; bucket_base[nseg] = total buckets.  Segment g has
 *                   bucket_base[g+1] - bucket_base[g] buckets (its p, or 1).
 *   bucket_sizes  : [bucket_cap] bucket sizes, in bucket order.
 *   splitter_keys : [bucket_cap] keys: segment g's p - 1 splitters sit at
 *                   bucket_base[g] .. bucket_base[g] + p - 2.
 *   splitter_tags : [bucket_cap] their positions inside the segment.
 *   bucket_cap    : capacity of the three bucket arrays; entries beyond it are
 *                   not written.
 */
typedef struct {
    uint32_t* bucket_base;
    uint32_t* bucket_sizes;
    void*     splitter_keys;
    uint32_t* splitter_tags;
    uint64_t  bucket_cap;
} os_seg_stats;

/*
 * Workspace bytes os_sort_segmented needs for n keys in nseg segments with this
 * class table.  With classes == NULL (nclass ignored): the most any table that
 * os_tune_segmented may return can need.
 * Errors: OS_ERR_ARG (bytes NULL, bad class table), OS_ERR_UNSUPPORTED (n above
 * OS_MAX_N, nseg above OS_SEG_MAX_NSEG, or planned totals beyond 32 bits).
 */
int os_workspace_size_segmented(int key_type, uint64_t n, uint32_t nseg, int has_vals,
                                const os_seg_class* classes, uint32_t nclass, size_t* bytes);

/*
 * Sort every segment of d_keys_in into the same range of d_keys_out.
 *   d_keys_in     : n keys, device, read only.  Must not overlap d_keys_out.
 *   d_keys_out    : n keys, device.
 *   d_vals_in/out : n uint32 payloads each, or both NULL; stable order.
 *   d_seg_offsets : nseg + 1 uint64, DEVICE: off[0] = 0, non-decreasing,
 *                   off[nseg] = n (a violation sets an error bit in the status
 *                   word and the offending segments are left unsorted).
 *   classes       : HOST array of nclass length classes (read during the call).
 *   seed          : batch seed; segment g's sample uses u(seed, 2, g).
 *   stats         : NULL, or device arrays to fill (see os_seg_stats).
 * Enqueues a fixed sequence of kernels whose shape depends only on n, nseg,
 * the payload and the classes, never on the offsets (no synchronization, no
 * host read of device data), so the call may be captured in a CUDA graph.
 * Device-side errors are read with os_check on the same workspace.
 */
int os_sort_segmented(int key_type, const void* d_keys_in, void* d_keys_out,
                      const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                      const uint64_t* d_seg_offsets, uint32_t nseg,
                      const os_seg_class* classes, uint32_t nclass, uint64_t seed,
                      void* d_ws, size_t ws_bytes, void* stream, const os_seg_stats* stats);

/*
 * CUDA graph of one os_sort_segmented call: captured once, launched many times.
 * The graph reads the keys, payloads and offsets at the captured addresses
 * every time it runs, so the caller may rewrite their contents between launches
 * (any offsets with the same n and nseg).  Capture runs on a private stream
 * and enqueues no work; os_graph_launch enqueues the whole sort on `stream`.
 * The workspace must stay allocated and unused by other calls while the graph
 * may run.
 */
typedef struct os_graph_s* os_graph;

int os_graph_capture_segmented(os_graph* graph, int key_type, const void* d_keys_in, void* d_keys_out,
                               const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                               const uint64_t* d_seg_offsets, uint32_t nseg,
                               const os_seg_class* classes, uint32_t nclass, uint64_t seed,
                               void* d_ws, size_t ws_bytes, const os_seg_stats* stats);
int os_graph_launch(os_graph graph, void* stream);
/* Kernels one launch of the graph runs. */
uint64_t os_graph_kernels(os_graph graph);
int os_graph_destroy(os_graph graph);

/*
 * Starting class table for segments up to max_len: one class of whole
 * segments up to the shared-memory sort's capacity (8192 int32 keys, 4096
 * 64-bit keys) with p = 1, then classes doubling in length, each with p a power
 * of two giving buckets near 60% of that capacity and s = 16.
 * Writes at most max_classes entries; *nclass receives the count.
 */
int os_seg_default_classes(int key_type, uint64_t max_len, os_seg_class* classes,
                           uint32_t max_classes, uint32_t* nclass);

/*
 * Autotuner: times os_sort_segmented on the caller's own batch and chooses the
 * class table (the whole-segment cutoff, and p, s and tile per length class)
 * by coordinate descent from os_seg_default_classes: cutoff in {capacity/2,
 * capacity, 2 capacity}; per class (largest share of keys first)
 * p in {p/4, p/2, 2p, 4p}, s in {4, 8, 16, 32, 64}, tile in {2048, 4096, 8192, 16384},
 * keeping a change only when it lowers the median of `reps` timed runs.
 *   h_seg_offsets : the same offsets as d_seg_offsets, in HOST memory.
 *   d_keys_out, d_vals_out : scratch the trial sorts write.
 *   d_ws, ws_bytes : os_workspace_size_segmented(..., NULL, ...) bytes cover
 *                   every candidate; candidates needing more are skipped.
 *   classes, max_classes, nclass : the chosen table.
 *   best_ms       : median time of the chosen table (may be NULL).
 * Synchronizes `stream` after every trial.
 */
int os_tune_segmented(int key_type, const void* d_keys_in, void* d_keys_out,
                      const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                      const uint64_t* d_seg_offsets, const uint64_t* h_seg_offsets, uint32_t nseg,
                      uint64_t seed, void* d_ws, size_t ws_bytes, void* stream, uint32_t reps,
                      os_seg_class* classes, uint32_t max_classes, uint32_t* nclass, float* best_ms);

/*
 * ---- Serving loop ------------------------------------------------------------
 * A sort server for requests that arrive over time (an addition of this
 * library; the paper sorts one array at a time).  The caller gives it one
 * device arena -- the HBM budget -- and it keeps every request's output and
 * workspace (splitters, buckets, work lists) inside it.  A dispatcher thread
 * admits queued requests in arrival order as soon as an in-flight slot is free
 * and the arena holds the request's output plus workspace, and enqueues each
 * admitted sort (os_sort with the request's parameters) on one of several CUDA
 * streams, so requests that arrive while others run overlap on the GPU.  A
 * stream callback marks the request done, time-stamps it and returns its
 * workspace to the arena at once; its output stays until os_server_release.
 * Results are bit-identical to os_sort of the same request alone.
 */
typedef struct os_server_s* os_server;

typedef struct {
    void*    d_arena;       /* device memory the server sub-allocates: the HBM budget */
    size_t   arena_bytes;
    uint32_t streams;       /* CUDA streams the admitted sorts are spread over, 1..64 */
    uint32_t max_inflight;  /* admitted, unfinished requests at most, >= 1 */
} os_server_config;

/* Flags of os_request.flags. */
#define OS_REQ_HOST_INPUT 1u   /* d_keys_in is HOST memory (pinned for full copy speed): the server copies
                                  the keys into the request's output block on the request's stream when it
                                  admits the request, then sorts them there in place; the copy counts in the
                                  request's latency.  The host keys are read until the request is done. */

typedef struct {
    int32_t     key_type;
    uint32_t    flags;      /* 0 or OS_REQ_HOST_INPUT */
    const void* d_keys_in;  /* n keys, resident on the device outside the arena (or on the host with
                               OS_REQ_HOST_INPUT); read until the request is done */
    uint64_t    n;
    os_params   prm;
} os_request;

typedef struct {
    uint64_t ticket;
    int32_t  status;        /* OS_OK, or the error of the request's sort */
    uint32_t stream;        /* stream index the sort ran on */
    void*    d_keys_out;    /* sorted keys inside the arena, valid until os_server_release */
    uint64_t n;
    uint64_t bytes;         /* arena bytes the request held while running (output + workspace) */
    double   submit_s;      /* host steady-clock times, seconds */
    double   admit_s;
    double   done_s;
} os_result;

typedef struct {
    uint64_t submitted, admitted, completed, released;
    uint32_t queued, inflight;
    uint64_t arena_in_use, arena_peak, arena_bytes;
    uint32_t max_inflight_seen;
} os_server_stats;

/*
 * Create a server on the current device.  Errors: OS_ERR_ARG (NULL arena,
 * streams or max_inflight out of range), OS_ERR_CUDA.
 */
int os_server_create(const os_server_config* cfg, os_server* server);

/*
 * Queue one request; *ticket identifies it.  Never blocks on the GPU.
 * Errors: OS_ERR_ARG (bad request), OS_ERR_UNSUPPORTED (its output plus
 * workspace exceed the whole arena: it could never be admitted).
 */
int os_server_submit(os_server server, const os_request* req, uint64_t* ticket);

/*
 * Completed requests not returned before, oldest completion first: up to
 * max_results into `results`, *count receives how many.  With timeout_us > 0
 * waits up to that long for at least one completion.
 */
int os_server_poll(os_server server, os_result* results, uint32_t max_results, int64_t timeout_us,
                   uint32_t* count);

/* Return a completed request's output to the arena (after the caller used it). */
int os_server_release(os_server server, uint64_t ticket);

int os_server_get_stats(os_server server, os_server_stats* stats);

/*
 * Open-loop replay of a request trace (benchmarking): request i is submitted at
 * arrival_s[i] seconds after the call starts (non-decreasing), completions are
 * collected and released at once, and results[i] receives request i's record
 * (d_keys_out is no longer valid).  Returns when every request is done.
 */
int os_server_replay(os_server server, const os_request* reqs, const double* arrival_s, uint32_t count,
                     os_result* results);

/*
 * Stop the dispatcher, wait for in-flight sorts and free the server.  Queued
 * requests that were never admitted are dropped.
 */
int os_server_destroy(os_server server);

/*
 * Synchronize `stream` and read the device status word in the workspace of the
 * last sort enqueued with it: OS_OK, or OS_ERR_DEVICE with the raw error bits in
 * *bits (may be NULL).
 */
int os_check(const void* d_ws, void* stream, uint32_t* bits);

/*
 * Counters of the last sort (plain or segmented) enqueued with this workspace,
 * read after synchronizing `stream`:
 *   errors      : the device error bits (0 when none; os_check's word).
 *   depth       : deepest in-bucket repartition level used.
 *   repart_keys : keys moved by in-bucket repartitions, summed over levels.
 *   bad_site, bad_index : first failed range check (0 when none).
 *   split_keys  : the part of repart_keys moved by the first in-bucket level
 *                 (the SqRan split of every oversized bucket).
 */
typedef struct {
    uint32_t errors;
    uint32_t depth;
    uint64_t repart_keys;
    uint32_t bad_site;
    uint32_t bad_index;
    uint64_t split_keys;
} os_counters;

int os_read_counters(const void* d_ws, void* stream, os_counters* counters);

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
