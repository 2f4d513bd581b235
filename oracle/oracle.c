/*
 * CPU oracle for SqDet (Algorithm 1) and SqRan (Algorithm 2) of Gerbessiotis,
 * "Using parallelism techniques to improve sequential and multi-core sorting
 * performance", with the duplicate handling of Section 2.2.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the bench; never by the library.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Readings of the paper taken here (each is listed with the design notes):
 *  - Tags (Section 2.2): every key is ordered by (key, tag).  Inside a sorted
 *    sequence the paper's implicit tag is (sequence id k, local index l); it is
 *    flattened to start_k + l, which orders exactly as the pair.  Before
 *    step 1 the tag is the original index, and the stable SomeSort keeps equal
 *    keys in that order, so (key, start_k + l) and (key, original index) are
 *    the same total order.
 *  - Sequences (step 1): sequence k is [floor(k n/p), floor((k+1) n/p)).
 *  - DET sample (step 2): with r = s and m = r p samples per sequence, sample j
 *    (j = 1..m) of a sequence of c keys is its key of local rank ceil(j c/m) - 1,
 *    so the m segments differ in size by at most one and j = m is the maximum.
 *  - RAN sample (step 2): p s - 1 keys drawn with replacement over original
 *    positions, position j = floor(u_j n / 2^64) with u_j from stream 1 of the
 *    counter-based SplitMix64 below; the tag is that original position.
 *  - Splitters (step 3): S_i is the (i * stride)-th smallest element of the
 *    sorted sample T, stride = r p (DET) or s (RAN), i = 1..p-1.
 *  - Split (step 4): a key x belongs to bucket j when S_j < x <= S_{j+1} in the
 *    tagged order (S_0 = -inf, S_p = +inf): an element equal to a splitter
 *    closes the lower bucket.
 *  - Too small to sample: RAN needs p s < n/2 (Claim 1), DET needs
 *    ceil(n/p) >= r p; otherwise, and for p = 1, the whole input is one bucket.
 *  - float64 order is IEEE 754 totalOrder restricted to non-NaN values.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define SM_GAMMA 0x9E3779B97F4A7C15ULL

/* ---- SplitMix64 (Steele, Lea, Flood 2014), counter form --------------------- */
static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_raw(uint64_t state, uint64_t i) {
    return sm_mix(state + (i + 1) * SM_GAMMA);
}

uint64_t oracle_splitmix64(uint64_t seed, uint64_t stream, uint64_t i) {
    return oracle_splitmix64_raw(sm_mix(seed + (stream + 1) * SM_GAMMA), i);
}

uint64_t oracle_ran_index(uint64_t seed, uint64_t j, uint64_t n) {
    uint64_t u = oracle_splitmix64(seed, 1, j);
    return (uint64_t)(((unsigned __int128)u * (unsigned __int128)n) >> 64);
}

/* ---- key order --------------------------------------------------------------- */
int oracle_key_cmp(int kt, uint64_t a, uint64_t b) {
    if (kt == ORC_I32) {
        int32_t x = (int32_t)(uint32_t)a, y = (int32_t)(uint32_t)b;
        return (x > y) - (x < y);
    }
    if (kt == ORC_U64) return (a > b) - (a < b);
    /* float64: a negative sign is below a positive one (so -0 < +0); with equal
     * signs, a larger magnitude is larger for positives and smaller for negatives. */
    double x, y;
    memcpy(&x, &a, sizeof x);
    memcpy(&y, &b, sizeof y);
    int na = (int)(a >> 63), nb = (int)(b >> 63);
    if (na != nb) return na ? -1 : 1;
    double ax = fabs(x), ay = fabs(y);
    if (ax == ay) return 0;
    int mag = ax < ay ? -1 : 1;
    return na ? -mag : mag;
}

/* 32-byte string keys (ORC_S32): a record holds the key's index into the input
 * array, and keys compare as memcmp of their 32 bytes (unsigned bytes,
 * lexicographic).  The input array of the sort being run: */
static const unsigned char* g_str_keys = NULL;

int oracle_str_cmp(const void* a, const void* b) {
    const int c = memcmp(a, b, 32);
    return (c > 0) - (c < 0);
}

static int key_cmp(int kt, uint64_t a, uint64_t b) {
    if (kt == ORC_S32) return oracle_str_cmp(g_str_keys + 32 * a, g_str_keys + 32 * b);
    return oracle_key_cmp(kt, a, b);
}

typedef struct {
    uint64_t key;   /* raw bits of the key (ORC_S32: its index in the input) */
    uint64_t tag;   /* duplicate-handling tag */
    uint32_t val;   /* payload */
} rec_t;

/* The tagged order of Section 2.2: key first, tag second. */
static int rec_cmp(int kt, const rec_t* a, const rec_t* b) {
    int c = key_cmp(kt, a->key, b->key);
    if (c) return c;
    return (a->tag > b->tag) - (a->tag < b->tag);
}

/* ---- SomeSort: textbook top-down merge sort (stable) ------------------------- */
static void merge_sort_rec(int kt, rec_t* a, rec_t* tmp, uint64_t n) {
    if (n < 2) return;
    uint64_t h = n / 2;
    merge_sort_rec(kt, a, tmp, h);
    merge_sort_rec(kt, a + h, tmp, n - h);
    uint64_t i = 0, j = h, o = 0;
    while (i < h && j < n) {
        if (rec_cmp(kt, &a[j], &a[i]) < 0) tmp[o++] = a[j++];
        else tmp[o++] = a[i++];
    }
    while (i < h) tmp[o++] = a[i++];
    while (j < n) tmp[o++] = a[j++];
    memcpy(a, tmp, n * sizeof(rec_t));
}

static int some_sort(int kt, rec_t* a, uint64_t n) {
    if (n < 2) return 0;
    rec_t* tmp = (rec_t*)malloc(n * sizeof(rec_t));
    if (!tmp) return -2;
    merge_sort_rec(kt, a, tmp, n);
    free(tmp);
    return 0;
}

/* ---- p-way merge with a binary min-heap (Knuth, Vol. 3, 5.4.1) --------------- */
typedef struct {
    const rec_t* cur;
    const rec_t* end;
} run_t;

static int heap_less(int kt, const run_t* runs, uint32_t a, uint32_t b) {
    int c = rec_cmp(kt, runs[a].cur, runs[b].cur);
    if (c) return c < 0;
    return a < b;
}

static void heap_down(int kt, const run_t* runs, uint32_t* h, uint32_t sz, uint32_t i) {
    for (;;) {
        uint32_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < sz && heap_less(kt, runs, h[l], h[m])) m = l;
        if (r < sz && heap_less(kt, runs, h[r], h[m])) m = r;
        if (m == i) return;
        uint32_t t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
}

/* Merge q sorted runs into out (which has room for all of them). */
static int multiway_merge(int kt, run_t* runs, uint32_t q, rec_t* out) {
    uint32_t* h = (uint32_t*)malloc((q ? q : 1) * sizeof(uint32_t));
    if (!h) return -2;
    uint32_t sz = 0;
    for (uint32_t k = 0; k < q; ++k)
        if (runs[k].cur < runs[k].end) h[sz++] = k;
    for (uint32_t i = sz; i-- > 0;) heap_down(kt, runs, h, sz, i);
    uint64_t o = 0;
    while (sz) {
        uint32_t k = h[0];
        out[o++] = *runs[k].cur++;
        if (runs[k].cur == runs[k].end) h[0] = h[--sz];
        heap_down(kt, runs, h, sz, 0);
    }
    free(h);
    return 0;
}

/* ---- key I/O ------------------------------------------------------------------ */
static uint64_t load_key(int kt, const void* k, uint64_t i) {
    if (kt == ORC_S32) return i;
    if (kt == ORC_I32) return (uint64_t)((const uint32_t*)k)[i];
    return ((const uint64_t*)k)[i];
}

static void store_key(int kt, void* k, uint64_t i, uint64_t bits) {
    if (kt == ORC_S32) memcpy((unsigned char*)k + 32 * i, g_str_keys + 32 * bits, 32);
    else if (kt == ORC_I32) ((uint32_t*)k)[i] = (uint32_t)bits;
    else ((uint64_t*)k)[i] = bits;
}

/* Number of elements of the sorted run a[0, c) that are <= x in the tagged order. */
static uint64_t count_le(int kt, const rec_t* a, uint64_t c, const rec_t* x) {
    uint64_t lo = 0, hi = c;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (rec_cmp(kt, &a[mid], x) <= 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static void write_outputs(int kt, const rec_t* y, uint64_t n, void* out_keys, uint32_t* out_vals) {
    if (out_keys)
        for (uint64_t i = 0; i < n; ++i) store_key(kt, out_keys, i, y[i].key);
    if (out_vals)
        for (uint64_t i = 0; i < n; ++i) out_vals[i] = y[i].val;
}

/* ---- the multi-core adaptation (Section 2.4): whole steps split over threads -- */
/* Worker w of t takes the sequences (step 1) or buckets (step 5) [w p / t, (w+1) p / t). */
typedef struct {
    int kt, rc;
    uint32_t p, lo, hi;
    rec_t* X;
    const uint64_t* cs;
    const uint64_t* pos;      /* step 5: split positions, p x (p + 1) */
    const uint64_t* yoff;     /* step 5: first output position of every bucket */
    rec_t* Y;
} work_t;

static void* step1_worker(void* arg) {
    work_t* w = (work_t*)arg;
    for (uint32_t k = w->lo; k < w->hi && !w->rc; ++k)
        w->rc = some_sort(w->kt, w->X + w->cs[k], w->cs[k + 1] - w->cs[k]);
    return NULL;
}

static void* step5_worker(void* arg) {
    work_t* w = (work_t*)arg;
    run_t* runs = (run_t*)malloc((size_t)w->p * sizeof(run_t));
    if (!runs) { w->rc = -2; return NULL; }
    for (uint32_t j = w->lo; j < w->hi && !w->rc; ++j) {
        for (uint32_t k = 0; k < w->p; ++k) {
            const uint64_t* pk = w->pos + (size_t)k * (w->p + 1);
            runs[k].cur = w->X + w->cs[k] + pk[j];
            runs[k].end = w->X + w->cs[k] + pk[j + 1];
        }
        w->rc = multiway_merge(w->kt, runs, w->p, w->Y + w->yoff[j]);
    }
    free(runs);
    return NULL;
}

/* Run fn over t workers (t = 1: inline, no thread).  Returns the first error. */
static int run_workers(void* (*fn)(void*), work_t* proto, uint32_t t) {
    if (t <= 1) {
        proto->lo = 0;
        proto->hi = proto->p;
        fn(proto);
        return proto->rc;
    }
    work_t* ws = (work_t*)malloc((size_t)t * sizeof(work_t));
    pthread_t* th = (pthread_t*)malloc((size_t)t * sizeof(pthread_t));
    int rc = 0;
    if (!ws || !th) { free(ws); free(th); return -2; }
    uint32_t started = 0;
    for (uint32_t w = 0; w < t; ++w) {
        ws[w] = *proto;
        ws[w].rc = 0;
        ws[w].lo = (uint32_t)(((uint64_t)w * proto->p) / t);
        ws[w].hi = (uint32_t)(((uint64_t)(w + 1) * proto->p) / t);
        if (pthread_create(&th[w], NULL, fn, &ws[w]) != 0) { rc = -2; break; }
        ++started;
    }
    for (uint32_t w = 0; w < started; ++w) {
        pthread_join(th[w], NULL);
        if (!rc) rc = ws[w].rc;
    }
    free(th);
    free(ws);
    return rc;
}

static int sort_impl(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                     int split, uint32_t p, uint32_t s, uint64_t seed,
                     void* out_keys, uint32_t* out_vals,
                     void* spl_keys, uint64_t* spl_tags, uint64_t* bucket_sizes,
                     uint32_t* p_used, uint32_t threads, int par_step5) {
    if (kt < ORC_I32 || kt > ORC_S32 || (split != ORC_DET && split != ORC_RAN)) return -1;
    if (p < 1 || s < 1 || (n > 0 && !keys)) return -1;
    const uint32_t t = threads < 1 ? 1 : (threads > p ? p : threads);
    g_str_keys = kt == ORC_S32 ? (const unsigned char*)keys : NULL;

    rec_t* X = (rec_t*)malloc((n ? n : 1) * sizeof(rec_t));
    if (!X) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        X[i].key = load_key(kt, keys, i);
        X[i].tag = i;
        X[i].val = vals ? vals[i] : 0u;
    }
    if (bucket_sizes) memset(bucket_sizes, 0, (size_t)p * sizeof(uint64_t));

    uint64_t ps = (uint64_t)p * s;
    uint64_t ceil_np = (n + p - 1) / p;
    int too_small = (p == 1) || (split == ORC_RAN ? (n < 2 * ps) : (ceil_np < ps));
    if (too_small) {
        int rc = some_sort(kt, X, n);
        if (rc) { free(X); return rc; }
        write_outputs(kt, X, n, out_keys, out_vals);
        if (bucket_sizes) bucket_sizes[0] = n;
        if (p_used) *p_used = 1;
        free(X);
        return 0;
    }

    /* Step 1, BaselineSorting: p sequences, each sorted by SomeSort (over t
     * threads in the multi-core form). */
    uint64_t* cs = (uint64_t*)malloc(((size_t)p + 1) * sizeof(uint64_t));
    if (!cs) { free(X); return -2; }
    for (uint64_t k = 0; k <= p; ++k) cs[k] = (uint64_t)(((unsigned __int128)k * n) / p);
    {
        work_t w1 = {kt, 0, p, 0, p, X, cs, NULL, NULL, NULL};
        int rc = run_workers(step1_worker, &w1, t);
        if (rc) { free(cs); free(X); return rc; }
    }
    if (split == ORC_DET)
        for (uint64_t i = 0; i < n; ++i) X[i].tag = i;   /* (k, l) flattened to start_k + l */

    /* Steps 2 and 3: the sample T and the splitters S_1..S_{p-1}. */
    rec_t* S = (rec_t*)malloc(((size_t)p) * sizeof(rec_t));
    rec_t* T = NULL;
    uint64_t tn = 0, stride = 0;
    int rc = 0;
    if (!S) { free(cs); free(X); return -2; }
    if (split == ORC_DET) {
        uint64_t m = ps;                               /* r p keys per sequence */
        tn = (uint64_t)p * m;
        stride = m;                                    /* s = r p in Algorithm 1 */
        rec_t* Tk = (rec_t*)malloc(tn * sizeof(rec_t));
        T = (rec_t*)malloc(tn * sizeof(rec_t));
        run_t* runs = (run_t*)malloc((size_t)p * sizeof(run_t));
        if (!Tk || !T || !runs) rc = -2;
        if (!rc) {
            for (uint32_t k = 0; k < p; ++k) {
                uint64_t c = cs[k + 1] - cs[k];
                for (uint64_t j = 1; j <= m; ++j) {
                    uint64_t l = (uint64_t)(((unsigned __int128)j * c + m - 1) / m) - 1;
                    Tk[(uint64_t)k * m + (j - 1)] = X[cs[k] + l];
                }
                runs[k].cur = Tk + (uint64_t)k * m;
                runs[k].end = Tk + (uint64_t)(k + 1) * m;
            }
            rc = multiway_merge(kt, runs, p, T);       /* merge all T_k into T */
        }
        free(runs);
        free(Tk);
    } else {
        tn = ps - 1;
        stride = s;
        T = (rec_t*)malloc(tn * sizeof(rec_t));
        if (!T) rc = -2;
        if (!rc) {
            for (uint64_t j = 0; j < tn; ++j) {
                uint64_t idx = oracle_ran_index(seed, j, n);
                T[j].key = load_key(kt, keys, idx);
                T[j].tag = idx;
                T[j].val = 0;
            }
            rc = some_sort(kt, T, tn);                 /* sort T using SomeSort */
        }
    }
    if (!rc)
        for (uint32_t i = 1; i < p; ++i) S[i] = T[(uint64_t)i * stride - 1];
    free(T);
    if (rc) { free(S); free(cs); free(X); return rc; }

    if (spl_keys || spl_tags)
        for (uint32_t i = 1; i < p; ++i) {
            if (spl_keys) store_key(kt, spl_keys, i - 1, S[i].key);
            if (spl_tags) spl_tags[i - 1] = S[i].tag;
        }

    /* Step 4: split every sorted sequence X_k around S by binary search. */
    uint64_t* pos = (uint64_t*)malloc((size_t)p * ((size_t)p + 1) * sizeof(uint64_t));
    if (!pos) { free(S); free(cs); free(X); return -2; }
    for (uint32_t k = 0; k < p; ++k) {
        uint64_t c = cs[k + 1] - cs[k];
        uint64_t* pk = pos + (size_t)k * (p + 1);
        pk[0] = 0;
        pk[p] = c;
        for (uint32_t j = 1; j < p; ++j) pk[j] = count_le(kt, X + cs[k], c, &S[j]);
        for (uint32_t j = 0; j < p; ++j)
            if (bucket_sizes) bucket_sizes[j] += pk[j + 1] - pk[j];
    }
    if (p_used) *p_used = p;

    /* Step 5: p-way merge of X_{0..p-1, j} into Y_j; Y is their concatenation
     * (bucket j starts after buckets 0..j-1).  The multi-core form may give
     * every thread its own buckets. */
    if (out_keys) {
        rec_t* Y = (rec_t*)malloc((n ? n : 1) * sizeof(rec_t));
        uint64_t* yoff = (uint64_t*)malloc(((size_t)p + 1) * sizeof(uint64_t));
        if (!Y || !yoff) rc = -2;
        if (!rc) {
            yoff[0] = 0;
            for (uint32_t j = 0; j < p; ++j) {
                uint64_t len = 0;
                for (uint32_t k = 0; k < p; ++k) {
                    const uint64_t* pk = pos + (size_t)k * (p + 1);
                    len += pk[j + 1] - pk[j];
                }
                yoff[j + 1] = yoff[j] + len;
            }
            work_t w5 = {kt, 0, p, 0, p, X, cs, pos, yoff, Y};
            rc = run_workers(step5_worker, &w5, par_step5 ? t : 1);
        }
        if (!rc) write_outputs(kt, Y, n, out_keys, out_vals);
        free(yoff);
        free(Y);
    }
    free(pos);
    free(S);
    free(cs);
    free(X);
    return rc;
}

int oracle_sort(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                int split, uint32_t p, uint32_t s, uint64_t seed,
                void* out_keys, uint32_t* out_vals,
                void* spl_keys, uint64_t* spl_tags, uint64_t* bucket_sizes,
                uint32_t* p_used) {
    return sort_impl(kt, keys, vals, n, split, p, s, seed, out_keys, out_vals, spl_keys, spl_tags,
                     bucket_sizes, p_used, 1, 0);
}

int oracle_sort_mc(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                   int split, uint32_t p, uint32_t s, uint64_t seed,
                   void* out_keys, uint32_t* out_vals,
                   void* spl_keys, uint64_t* spl_tags, uint64_t* bucket_sizes,
                   uint32_t* p_used, uint32_t threads, int par_step5) {
    return sort_impl(kt, keys, vals, n, split, p, s, seed, out_keys, out_vals, spl_keys, spl_tags,
                     bucket_sizes, p_used, threads, par_step5);
}

int oracle_some_sort(int kt, const void* keys, const uint32_t* vals, uint64_t n,
                     void* out_keys, uint32_t* out_vals) {
    if (kt < ORC_I32 || kt > ORC_S32 || (n > 0 && !keys)) return -1;
    g_str_keys = kt == ORC_S32 ? (const unsigned char*)keys : NULL;
    rec_t* X = (rec_t*)malloc((n ? n : 1) * sizeof(rec_t));
    if (!X) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        X[i].key = load_key(kt, keys, i);
        X[i].tag = i;
        X[i].val = vals ? vals[i] : 0u;
    }
    int rc = some_sort(kt, X, n);
    if (!rc) write_outputs(kt, X, n, out_keys, out_vals);
    free(X);
    return rc;
}
