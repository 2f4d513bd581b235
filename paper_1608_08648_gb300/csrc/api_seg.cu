// The batched segmented entry points of include/ossort.h: class-table checks,
// workspace planning, dispatch on the key type, CUDA-graph capture and the
// autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ossort.h"
#include "api_util.h"
#include "segmented.cuh"

using namespace ossort;

struct os_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
};

namespace {

constexpr uint32_t TUNE_S[] = {4, 8, 16, 32, 64};
constexpr uint32_t TUNE_TILE[] = {2048, 4096, 8192, 16384};
constexpr uint32_t TUNE_MAX_P = OS_SEG_MAX_PS / 4;   // p s <= OS_SEG_MAX_PS with s >= 4

uint64_t leaf_cap(int kt) { return kt == OS_I32 ? 8192 : 4096; }

int check_classes(const os_seg_class* classes, uint32_t nclass, SegClasses& out) {
    if (!classes || nclass < 1 || nclass > OS_SEG_MAX_CLASSES) return OS_ERR_ARG;
    static_assert(OS_SEG_MAX_CLASSES == (unsigned)SEG_MAX_CLASSES, "class table size");
    static_assert(OS_SEG_MAX_PS == (unsigned)SEG_SAMPLE, "largest sample of a segment");
    out = SegClasses{};
    out.n = nclass;
    for (uint32_t k = 0; k < nclass; ++k) {
        const os_seg_class& c = classes[k];
        if (c.reserved != 0 || c.p < 1 || c.p > OS_MAX_P || c.s < 1) return OS_ERR_ARG;
        if (c.tile < (uint32_t)SEG_SUB || c.tile > 16384u || c.tile % SEG_SUB) return OS_ERR_ARG;
        if (c.p > 1 && (uint64_t)c.p * c.s > OS_SEG_MAX_PS) return OS_ERR_ARG;
        if (k > 0 && c.max_len <= classes[k - 1].max_len) return OS_ERR_ARG;
        out.c[k] = SegClass{c.max_len, c.p, c.s, c.tile, 0u};
    }
    return OS_OK;
}

// A table whose workspace bounds cover every table the tuner can return:
// p <= TUNE_MAX_P, s >= 4, tile >= 2048.
SegClasses tuner_bound_table() {
    SegClasses t{};
    t.n = 1;
    t.c[0] = SegClass{~0ull, TUNE_MAX_P, 4u, (uint32_t)SEG_SUB, 0u};
    return t;
}

int run_seg(int kt, SegArgs& a) {
    switch (kt) {
        case OS_I32: return run_seg_i32(a);
        case OS_U64: return run_seg_u64(a);
        default: return run_seg_f64(a);
    }
}

int check_sizes(int kt, uint64_t n, uint32_t nseg, const SegClasses& cls) {
    if (kt == OS_S32) return OS_ERR_UNSUPPORTED;
    if (kt < OS_I32 || kt > OS_F64) return OS_ERR_ARG;
    if (n > OS_MAX_N || nseg > OS_SEG_MAX_NSEG) return OS_ERR_UNSUPPORTED;
    const SegBounds b = seg_bounds_of(n, nseg, cls);
    if (b.tiles >= (1ull << 32) || b.buckets >= (1ull << 32) || b.hist >= (1ull << 32)) return OS_ERR_UNSUPPORTED;
    return OS_OK;
}

size_t seg_plan_bytes(int kt, uint64_t n, uint32_t nseg, bool hv, const SegClasses& cls) {
    SegArgs a{};
    a.n = n;
    a.nseg = nseg;
    a.has_vals = hv;
    a.cls = cls;
    a.ws = nullptr;
    run_seg(kt, a);
    return a.used + 256;
}

// Argument checks shared by the sort and the graph capture.
int prepare(int kt, const void* kin, void* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
            const uint64_t* off, uint32_t nseg, const os_seg_class* classes, uint32_t nclass, uint64_t seed,
            void* ws, size_t ws_bytes, const os_seg_stats* stats, SegArgs& a) {
    SegClasses cls;
    int rc = check_classes(classes, nclass, cls);
    if (rc) return rc;
    rc = check_sizes(kt, n, nseg, cls);
    if (rc) return rc;
    if (nseg == 0 && n != 0) return OS_ERR_ARG;
    if (n > 0 && (!kin || !kout)) return OS_ERR_ARG;
    if (nseg > 0 && !off) return OS_ERR_ARG;
    if ((vin != nullptr) != (vout != nullptr)) return OS_ERR_ARG;
    if (n > 0 && (kin == kout || (vin && static_cast<const void*>(vin) == static_cast<void*>(vout))))
        return OS_ERR_ARG;
    const bool hv = vin != nullptr;
    const size_t need = seg_plan_bytes(kt, n, nseg, hv, cls);
    if (!ws || ws_bytes < need) return OS_ERR_WS;
    a = SegArgs{};
    a.kin = kin;
    a.kout = kout;
    a.vin = vin;
    a.vout = vout;
    a.has_vals = hv;
    a.n = n;
    a.off = off;
    a.nseg = nseg;
    a.cls = cls;
    a.seed = seed;
    a.ws = ws;
    a.ws_bytes = ws_bytes;
    a.num_sms = num_sms_of_current_device();
    a.stats = stats;
    return OS_OK;
}

// Starting class table (see os_seg_default_classes) with a given cutoff for
// whole segments.
std::vector<os_seg_class> default_table(int kt, uint64_t max_len, uint64_t cutoff, uint32_t max_classes) {
    std::vector<os_seg_class> t;
    if (max_classes == 0) return t;
    t.push_back(os_seg_class{cutoff, 1u, 1u, 4096u, 0u});
    const double target = 0.6 * (double)leaf_cap(kt);
    uint64_t lo = cutoff;
    while (lo < max_len && t.size() < max_classes) {
        uint64_t hi = (t.size() + 1 == max_classes || 2 * lo >= max_len) ? max_len : 2 * lo;
        const double mid = 0.5 * ((double)lo + (double)hi);
        const int e = (int)std::lround(std::log2(std::max(mid / target, 2.0)));
        uint32_t p = 1u << std::min(e, 8);
        const uint32_t s = 16;
        while (p > 2 && 2ull * p * s > lo + 1) p >>= 1;
        t.push_back(os_seg_class{hi, p, s, 4096u, 0u});
        lo = hi;
    }
    return t;
}

}  // namespace

extern "C" {

int os_workspace_size_segmented(int key_type, uint64_t n, uint32_t nseg, int has_vals,
                                const os_seg_class* classes, uint32_t nclass, size_t* bytes) {
    if (!bytes) return OS_ERR_ARG;
    SegClasses cls;
    if (classes) {
        const int rc = check_classes(classes, nclass, cls);
        if (rc) return rc;
    } else {
        cls = tuner_bound_table();
    }
    const int rc = check_sizes(key_type, n, nseg, cls);
    if (rc) return rc;
    *bytes = seg_plan_bytes(key_type, n, nseg, has_vals != 0, cls);
    return OS_OK;
}

int os_sort_segmented(int key_type, const void* d_keys_in, void* d_keys_out, const uint32_t* d_vals_in,
                      uint32_t* d_vals_out, uint64_t n, const uint64_t* d_seg_offsets, uint32_t nseg,
                      const os_seg_class* classes, uint32_t nclass, uint64_t seed, void* d_ws, size_t ws_bytes,
                      void* stream, const os_seg_stats* stats) {
    SegArgs a;
    int rc = prepare(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, d_seg_offsets, nseg, classes, nclass,
                     seed, d_ws, ws_bytes, stats, a);
    if (rc) return rc;
    if (nseg == 0) return OS_OK;
    a.st = static_cast<cudaStream_t>(stream);
    rc = run_seg(key_type, a);
    if (rc) return rc;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OS_OK : cuda_fail(e);
}

int os_graph_capture_segmented(os_graph* graph, int key_type, const void* d_keys_in, void* d_keys_out,
                               const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                               const uint64_t* d_seg_offsets, uint32_t nseg, const os_seg_class* classes,
                               uint32_t nclass, uint64_t seed, void* d_ws, size_t ws_bytes,
                               const os_seg_stats* stats) {
    if (!graph) return OS_ERR_ARG;
    *graph = nullptr;
    SegArgs a;
    int rc = prepare(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, d_seg_offsets, nseg, classes, nclass,
                     seed, d_ws, ws_bytes, stats, a);
    if (rc) return rc;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
    auto* g = new os_graph_s();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        a.st = cs;
        rc = nseg > 0 ? run_seg(key_type, a) : OS_OK;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (e2 != cudaSuccess && rc == OS_OK) rc = cuda_fail(e2);
    } else {
        rc = cuda_fail(e);
    }
    if (rc == OS_OK) {
        size_t nn = 0;
        e = cudaGraphGetNodes(g->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g->graph, nodes.data(), &nn);
        for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++g->kernels;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    cudaStreamDestroy(cs);
    if (rc != OS_OK) {
        os_graph_destroy(g);
        return rc;
    }
    *graph = g;
    return OS_OK;
}

int os_graph_launch(os_graph graph, void* stream) {
    if (!graph || !graph->exec) return OS_ERR_ARG;
    const cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    add_launches(graph->kernels);
    return OS_OK;
}

uint64_t os_graph_kernels(os_graph graph) { return graph ? graph->kernels : 0; }

int os_graph_destroy(os_graph graph) {
    if (!graph) return OS_ERR_ARG;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return OS_OK;
}

int os_seg_default_classes(int key_type, uint64_t max_len, os_seg_class* classes, uint32_t max_classes,
                           uint32_t* nclass) {
    if (key_type < OS_I32 || key_type > OS_F64 || !classes || !nclass || max_classes < 1) return OS_ERR_ARG;
    const std::vector<os_seg_class> t =
        default_table(key_type, max_len, leaf_cap(key_type), std::min(max_classes, OS_SEG_MAX_CLASSES));
    for (size_t k = 0; k < t.size(); ++k) classes[k] = t[k];
    *nclass = (uint32_t)t.size();
    return OS_OK;
}

int os_tune_segmented(int key_type, const void* d_keys_in, void* d_keys_out, const uint32_t* d_vals_in,
                      uint32_t* d_vals_out, uint64_t n, const uint64_t* d_seg_offsets,
                      const uint64_t* h_seg_offsets, uint32_t nseg, uint64_t seed, void* d_ws, size_t ws_bytes,
                      void* stream, uint32_t reps, os_seg_class* classes, uint32_t max_classes, uint32_t* nclass,
                      float* best_ms) {
    if (!h_seg_offsets || !classes || !nclass || max_classes < 1 || reps < 1 || nseg < 1) return OS_ERR_ARG;
    if (key_type == OS_S32) return OS_ERR_UNSUPPORTED;
    if (key_type < OS_I32 || key_type > OS_F64) return OS_ERR_ARG;
    if (h_seg_offsets[0] != 0 || h_seg_offsets[nseg] != n) return OS_ERR_ARG;
    uint64_t max_len = 0;
    for (uint32_t g = 0; g < nseg; ++g) {
        if (h_seg_offsets[g + 1] < h_seg_offsets[g]) return OS_ERR_ARG;
        max_len = std::max<uint64_t>(max_len, h_seg_offsets[g + 1] - h_seg_offsets[g]);
    }
    const uint32_t mc = std::min(max_classes, OS_SEG_MAX_CLASSES);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError());
    }
    int err = OS_OK;
    // Median of `reps` timed runs after one untimed run; +inf when the table
    // does not fit the workspace.
    auto time_table = [&](const std::vector<os_seg_class>& t) -> float {
        size_t need = 0;
        if (os_workspace_size_segmented(key_type, n, nseg, d_vals_in != nullptr, t.data(), (uint32_t)t.size(),
                                        &need) != OS_OK ||
            need > ws_bytes)
            return INFINITY;
        std::vector<float> ms;
        for (uint32_t r = 0; r <= reps && err == OS_OK; ++r) {
            cudaEventRecord(e0, st);
            const int rc = os_sort_segmented(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n,
                                             d_seg_offsets, nseg, t.data(), (uint32_t)t.size(), seed, d_ws,
                                             ws_bytes, stream, nullptr);
            cudaEventRecord(e1, st);
            if (rc != OS_OK) {
                err = rc;
                break;
            }
            const cudaError_t ce = cudaEventSynchronize(e1);
            float x = 0.f;
            if (ce == cudaSuccess) cudaEventElapsedTime(&x, e0, e1);
            else err = cuda_fail(ce);
            if (r > 0) ms.push_back(x);
        }
        if (err != OS_OK || ms.empty()) return INFINITY;
        std::sort(ms.begin(), ms.end());
        return ms[ms.size() / 2];
    };
    const uint64_t cap = leaf_cap(key_type);
    std::vector<os_seg_class> best = default_table(key_type, max_len, cap, mc);
    float best_t = time_table(best);
    for (uint64_t cut : {cap / 2, 2 * cap}) {
        const std::vector<os_seg_class> t = default_table(key_type, max_len, cut, mc);
        const float x = time_table(t);
        if (x < best_t) {
            best_t = x;
            best = t;
        }
    }
    // Classes in order of the keys they hold.
    std::vector<std::pair<uint64_t, size_t>> order;
    for (size_t k = 0; k < best.size(); ++k) {
        const uint64_t lo = k ? best[k - 1].max_len : 0;
        const uint64_t hi = k + 1 < best.size() ? best[k].max_len : ~0ull;
        uint64_t keys = 0;
        for (uint32_t g = 0; g < nseg; ++g) {
            const uint64_t len = h_seg_offsets[g + 1] - h_seg_offsets[g];
            if (len > lo && len <= hi) keys += len;
        }
        if (best[k].p > 1) order.push_back({keys, k});
    }
    std::sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    auto try_change = [&](size_t k, uint32_t p, uint32_t s, uint32_t tile) {
        if (p < 2 || p > TUNE_MAX_P || (uint64_t)p * s > OS_SEG_MAX_PS) return;
        std::vector<os_seg_class> t = best;
        if (t[k].p == p && t[k].s == s && t[k].tile == tile) return;
        t[k].p = p;
        t[k].s = s;
        t[k].tile = tile;
        const float x = time_table(t);
        if (x < best_t) {
            best_t = x;
            best = t;
        }
    };
    for (const auto& ok : order) {
        const size_t k = ok.second;
        const uint32_t p0 = best[k].p;
        for (uint32_t p : {p0 / 4, p0 / 2, p0 * 2, p0 * 4}) try_change(k, p, best[k].s, best[k].tile);
        for (uint32_t s : TUNE_S) try_change(k, best[k].p, s, best[k].tile);
        for (uint32_t tile : TUNE_TILE) try_change(k, best[k].p, best[k].s, tile);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != OS_OK) return err;
    if (!std::isfinite(best_t)) return OS_ERR_WS;
    for (size_t k = 0; k < best.size(); ++k) classes[k] = best[k];
    *nclass = (uint32_t)best.size();
    if (best_ms) *best_ms = best_t;
    return OS_OK;
}

}  // extern "C"
