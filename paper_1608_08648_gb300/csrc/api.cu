// The C ABI of include/ossort.h: argument checks, workspace planning, dispatch
// on the key type, statistics and the host-buffer variant.
#include <atomic>
#include <cstdio>
#include <map>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ossort.h"
#include "api_util.h"
#include "driver.cuh"

using namespace ossort;

// ---- launch accounting and per-kernel event profiling ------------------------
namespace {
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
std::atomic<uint64_t> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local const char* g_pending_name = nullptr;
thread_local cudaEvent_t g_pending_a = nullptr;

cudaEvent_t pool_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

namespace ossort {
// A launch enqueued while its stream is being captured into a graph runs only
// when the graph is launched: it is counted then (add_launches), not here.
static bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}
void add_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void prof_before(cudaStream_t st, const char* name) {
    if (capturing(st)) return;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    g_pending_name = name;
    g_pending_a = pool_event();
    cudaEventRecord(g_pending_a, st);
}
void prof_after(cudaStream_t st, const char* name) {
    static const bool debug_sync = [] {
        const char* e = std::getenv("OSSORT_DEBUG_SYNC");
        return e && e[0] == '1';
    }();
    if (capturing(st)) return;
    if (debug_sync) {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) std::fprintf(stderr, "ossort: kernel %s failed: %s\n", name, cudaGetErrorString(e));
        else std::fprintf(stderr, "ossort: kernel %s ok\n", name);
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || !g_pending_a) return;
    cudaEvent_t b = pool_event();
    cudaEventRecord(b, st);
    g_recs.push_back(ProfRec{g_pending_name, g_pending_a, b});
    g_pending_a = nullptr;
}
}  // namespace ossort

namespace {
thread_local int g_last_cuda = 0;
}  // namespace

namespace ossort {
int cuda_fail(cudaError_t e) {
    g_last_cuda = (int)e;
    return OS_ERR_CUDA;
}

int num_sms_of_current_device() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    return sms > 0 ? sms : 152;
}
}  // namespace ossort

namespace {

size_t key_bytes(int kt) { return kt == OS_I32 ? 4 : (kt == OS_S32 ? 32 : 8); }

int check_params(int kt, uint64_t n, const os_params* prm) {
    if (kt < OS_I32 || kt > OS_S32 || !prm) return OS_ERR_ARG;
    if (prm->split != OS_DET && prm->split != OS_RAN) return OS_ERR_ARG;
    if (prm->p < 1 || prm->s < 1) return OS_ERR_ARG;
    if (prm->flags & ~(OS_STABLE | OS_DET_MERGE)) return OS_ERR_ARG;
    if ((prm->flags & OS_DET_MERGE) && prm->split != OS_DET) return OS_ERR_ARG;
    if (n > OS_MAX_N || prm->p > OS_MAX_P || (uint64_t)prm->p * prm->s > OS_MAX_PS)
        return OS_ERR_UNSUPPORTED;
    return OS_OK;
}

int dispatch(int kt, RunArgs& a) {
    switch (kt) {
        case OS_I32: return run_i32(a);
        case OS_U64: return run_u64(a);
        case OS_S32: return run_s32(a);
        default: return run_f64(a);
    }
}

// Workspace bytes of one sort: the planning pass (the driver run with a measuring
// arena).  Its result depends on the key type, n, the payload and p, s, split and
// flags (not on the seed, the device or the buffers), so the last results are kept
// in a small cache under a lock: a caller sorting many arrays of a few shapes
// plans each shape once.
size_t plan_bytes(int kt, uint64_t n, bool has_vals, const os_params* prm) {
    using Key = std::tuple<int, uint64_t, bool, int32_t, uint32_t, uint32_t, uint32_t>;
    static std::mutex mu;
    static std::map<Key, size_t> cache;
    const Key key{kt, n, has_vals, prm->split, prm->p, prm->s, prm->flags};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    RunArgs a{};
    a.n = n;
    a.has_vals = has_vals;
    a.prm = *prm;
    a.ws = nullptr;
    dispatch(kt, a);
    const size_t bytes = a.used + 256;
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 4096) cache.clear();
    cache[key] = bytes;
    return bytes;
}

template <class KT>
void splitters_to_host(const std::vector<typename KT::O>& o, void* dst) {
    auto* d = static_cast<typename KT::T*>(dst);
    for (size_t i = 0; i < o.size(); ++i) d[i] = KT::key(o[i]);
}

int fill_stats(int kt, const RunArgs& a, cudaStream_t st, os_stats* stats) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t status[8];
    e = cudaMemcpy(status, a.status, sizeof status, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint32_t p = a.prm.p, pu = a.res.p_used;
    stats->p_used = pu;
    stats->depth = status[1];
    stats->repart_keys = ((uint64_t)status[2] | ((uint64_t)status[3] << 32)) +
                         ((uint64_t)status[4] | ((uint64_t)status[5] << 32));
    if (pu == 1) {
        stats->max_bucket = a.n;
        if (stats->bucket_sizes) {
            for (uint32_t j = 0; j < p; ++j) stats->bucket_sizes[j] = 0;
            stats->bucket_sizes[0] = a.n;
        }
    } else {
        std::vector<uint32_t> b(p);
        e = cudaMemcpy(b.data(), a.res.bsize, p * sizeof(uint32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e);
        uint64_t mx = 0;
        for (uint32_t j = 0; j < p; ++j) {
            if (stats->bucket_sizes) stats->bucket_sizes[j] = b[j];
            mx = b[j] > mx ? b[j] : mx;
        }
        stats->max_bucket = mx;
        if (stats->splitter_tags) {
            std::vector<uint32_t> t(p - 1);
            e = cudaMemcpy(t.data(), a.res.spl_t, (p - 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e);
            for (uint32_t j = 0; j + 1 < p; ++j) stats->splitter_tags[j] = t[j];
        }
        if (stats->splitter_keys) {
            if (kt == OS_S32) {
                e = cudaMemcpy(stats->splitter_keys, a.res.str_keys, (size_t)(p - 1) * 32, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_fail(e);
            } else if (kt == OS_I32) {
                std::vector<uint32_t> o(p - 1);
                e = cudaMemcpy(o.data(), a.res.spl_o, (p - 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_fail(e);
                splitters_to_host<KeyI32>(o, stats->splitter_keys);
            } else {
                std::vector<uint64_t> o(p - 1);
                e = cudaMemcpy(o.data(), a.res.spl_o, (p - 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_fail(e);
                if (kt == OS_U64) splitters_to_host<KeyU64>(o, stats->splitter_keys);
                else splitters_to_host<KeyF64>(o, stats->splitter_keys);
            }
        }
    }
    return status[0] ? OS_ERR_DEVICE : OS_OK;
}

}  // namespace

namespace {

// os_sort, optionally handing ranges of the output to a HostSink as they finish
// (a.res.sunk tells whether it did).
int sort_device(int key_type, const void* d_keys_in, void* d_keys_out, const uint32_t* d_vals_in,
                uint32_t* d_vals_out, uint64_t n, const os_params* prm, void* d_ws, size_t ws_bytes, void* stream,
                os_stats* stats, const HostSink* sink, RunArgs& a, void* kin_copy = nullptr) {
    int rc = check_params(key_type, n, prm);
    if (rc) return rc;
    if (n > 0 && (!d_keys_in || !d_keys_out)) return OS_ERR_ARG;
    if ((d_vals_in != nullptr) != (d_vals_out != nullptr)) return OS_ERR_ARG;
    const bool hv = d_vals_in != nullptr;
    const size_t need = plan_bytes(key_type, n, hv, prm);
    if (!d_ws || ws_bytes < need) return OS_ERR_WS;
    a = RunArgs{};
    a.kin = d_keys_in;
    a.kout = d_keys_out;
    a.vin = d_vals_in;
    a.vout = d_vals_out;
    a.has_vals = hv;
    a.n = n;
    a.prm = *prm;
    a.ws = d_ws;
    a.ws_bytes = ws_bytes;
    a.st = static_cast<cudaStream_t>(stream);
    a.num_sms = num_sms_of_current_device();
    a.sink = sink;
    a.kin_copy = kin_copy;
    rc = dispatch(key_type, a);
    if (rc) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    if (stats) return fill_stats(key_type, a, a.st, stats);
    return OS_OK;
}

// The stream on which host-buffer sorts copy finished ranges out (one per device,
// created on first use), or nullptr.
cudaStream_t host_copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

constexpr uint32_t HOST_CHUNKS = 8;            // bucket ranges of a host-buffer sort (measured: 4, 8, 16)
constexpr uint64_t HOST_CHUNK_MIN_N = 1u << 22;  // below this, one range

}  // namespace

extern "C" {

uint64_t os_launch_count(void) { return g_launches.load(); }

int os_profile_start(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_prof_on = true;
    return OS_OK;
}

int os_profile_stop(os_kernel_time* out, int max_entries, int* n_entries) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_on = false;
        recs.swap(g_recs);
    }
    std::vector<os_kernel_time> agg;
    int rc = OS_OK;
    for (auto& r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e);
        size_t i = 0;
        while (i < agg.size() && std::strncmp(agg[i].name, r.name, sizeof(agg[i].name)) != 0) ++i;
        if (i == agg.size()) {
            os_kernel_time t{};
            std::strncpy(t.name, r.name, sizeof(t.name) - 1);
            agg.push_back(t);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
        if (ms > agg[i].max_ms) agg[i].max_ms = ms;
    }
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& r : recs) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
    }
    if (n_entries) *n_entries = (int)agg.size();
    if (out)
        for (int i = 0; i < (int)agg.size() && i < max_entries; ++i) out[i] = agg[i];
    return rc;
}

int os_version(void) { return OSSORT_VERSION; }

int os_last_cuda_error(void) { return g_last_cuda; }

const char* os_strerror(int status) {
    switch (status) {
        case OS_OK: return "ok";
        case OS_ERR_ARG: return "invalid argument";
        case OS_ERR_WS: return "workspace missing or too small";
        case OS_ERR_UNSUPPORTED: return "size or parameter beyond the supported limits";
        case OS_ERR_CUDA: return "CUDA call failed";
        case OS_ERR_DEVICE: return "a kernel reported an internal error";
        default: return "unknown status";
    }
}

int os_workspace_size(int key_type, uint64_t n, int has_vals, const os_params* prm, size_t* bytes) {
    if (!bytes) return OS_ERR_ARG;
    int rc = check_params(key_type, n, prm);
    if (rc) return rc;
    *bytes = plan_bytes(key_type, n, has_vals != 0, prm);
    return OS_OK;
}


int os_sort(int key_type, const void* d_keys_in, void* d_keys_out, const uint32_t* d_vals_in, uint32_t* d_vals_out,
            uint64_t n, const os_params* prm, void* d_ws, size_t ws_bytes, void* stream, os_stats* stats) {
    RunArgs a{};
    return sort_device(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, prm, d_ws, ws_bytes, stream, stats,
                       nullptr, a);
}

int os_workspace_size_host(int key_type, uint64_t n, int has_vals, const os_params* prm, size_t* bytes) {
    size_t inner = 0;
    int rc = os_workspace_size(key_type, n, has_vals, prm, &inner);
    if (rc) return rc;
    const size_t kb = ((n * key_bytes(key_type)) + 255) & ~size_t(255);
    const size_t vb = has_vals ? ((n * 4 + 255) & ~size_t(255)) : 0;
    *bytes = ((inner + 255) & ~size_t(255)) + kb + vb;
    return OS_OK;
}

int os_sort_host(int key_type, const void* h_keys_in, void* h_keys_out, const uint32_t* h_vals_in,
                 uint32_t* h_vals_out, uint64_t n, const os_params* prm, void* d_ws, size_t ws_bytes,
                 void* stream) {
    int rc = check_params(key_type, n, prm);
    if (rc) return rc;
    if (n > 0 && (!h_keys_in || !h_keys_out)) return OS_ERR_ARG;
    if ((h_vals_in != nullptr) != (h_vals_out != nullptr)) return OS_ERR_ARG;
    const bool hv = h_vals_in != nullptr;
    size_t need = 0;
    os_workspace_size_host(key_type, n, hv, prm, &need);
    if (!d_ws || ws_bytes < need) return OS_ERR_WS;
    const size_t inner = (plan_bytes(key_type, n, hv, prm) + 255) & ~size_t(255);
    char* base = static_cast<char*>(d_ws);
    void* dk = base + inner;
    uint32_t* dv = hv ? reinterpret_cast<uint32_t*>(base + inner + (((n * key_bytes(key_type)) + 255) & ~size_t(255)))
                      : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t kbytes = n * key_bytes(key_type);
    cudaError_t e = cudaSuccess;
    // Keys alone, SqRan, large enough to sample: when the device can address the
    // host buffer (page-locked memory: the host link of a Grace-Blackwell node is
    // coherent), the sort reads the keys from it directly -- the sample by a
    // gather, the top-level classify by a pass that also leaves the device copy
    // the scatter uses -- instead of waiting for a separate copy-in first.
    const void* hdev = nullptr;
    if (!hv && key_type != OS_S32 && prm->split == OS_RAN && prm->p > 1 && n >= HOST_CHUNK_MIN_N &&
        n >= 2ull * prm->p * prm->s) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, h_keys_in) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer != nullptr)
            hdev = pa.devicePointer;
        cudaGetLastError();
    }
    if (n > 0 && !hdev) {
        e = cudaMemcpyAsync(dk, h_keys_in, kbytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && hv) e = cudaMemcpyAsync(dv, h_vals_in, n * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // the output goes back range by range while the buckets are sorted (32-byte
    // strings and small inputs: in one copy after the sort)
    HostSink sink{h_keys_out, h_vals_out, nullptr, 1u};
    if (key_type != OS_S32 && n >= HOST_CHUNK_MIN_N) {
        sink.copy = host_copy_stream();
        sink.chunks = sink.copy ? HOST_CHUNKS : 1u;
    }
    RunArgs a{};
    rc = sort_device(key_type, hdev ? hdev : dk, dk, dv, dv, n, prm, d_ws, inner, stream, nullptr,
                     sink.chunks > 1 ? &sink : nullptr, a, hdev ? dk : nullptr);
    if (rc) return rc;
    if (n > 0 && !a.res.sunk) {
        e = cudaMemcpyAsync(h_keys_out, dk, kbytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && hv) e = cudaMemcpyAsync(h_vals_out, dv, n * 4, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return os_check(d_ws, stream, nullptr);
}

int os_check(const void* d_ws, void* stream, uint32_t* bits) {
    if (!d_ws) return OS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t word = 0;
    e = cudaMemcpy(&word, d_ws, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    if (bits) *bits = word;
    return word ? OS_ERR_DEVICE : OS_OK;
}

int os_read_counters(const void* d_ws, void* stream, os_counters* counters) {
    if (!d_ws || !counters) return OS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t w[8];
    e = cudaMemcpy(w, d_ws, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    counters->errors = w[0];
    counters->depth = w[1];
    counters->split_keys = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
    counters->repart_keys = counters->split_keys + ((uint64_t)w[4] | ((uint64_t)w[5] << 32));
    counters->bad_site = w[6];
    counters->bad_index = w[7];
    return OS_OK;
}

}  // extern "C"
