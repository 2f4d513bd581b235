// Serving loop of include/ossort.h: a FIFO of sort requests, admission by
// in-flight slots and free arena bytes, sorts spread over several CUDA
// streams, completion through stream callbacks.
//
// Locking: one mutex guards the queue, the allocator and the request records.
// CUDA calls are made only by the dispatcher thread with the mutex released;
// the stream callback (a CUDA-owned thread) touches host state only.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ossort.h"
#include "api_util.h"
#include "arena_alloc.h"

using namespace ossort;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t key_bytes_of(int kt) { return kt == OS_I32 ? 4 : (kt == OS_S32 ? 32 : 8); }

constexpr uint32_t STATUS_WORDS = 8;   // pinned copy of a request's status block

struct Req;

}  // namespace

struct os_server_s {
    int device = 0;
    char* arena = nullptr;
    ArenaAlloc alloc;
    std::vector<cudaStream_t> streams;
    std::vector<uint32_t> stream_load;
    uint32_t max_inflight = 1;
    uint32_t* h_status = nullptr;          // pinned: STATUS_WORDS per in-flight slot
    std::vector<uint32_t> free_slots;
    std::mutex mu;
    std::condition_variable cv_dispatch;   // a request queued or finished, a slot or arena bytes freed, stop
    std::condition_variable cv_done;       // a request finished
    std::deque<Req*> queue;
    std::deque<Req*> done;                 // finished, not yet returned by poll
    std::unordered_map<uint64_t, Req*> live;   // not yet released
    uint64_t next_ticket = 1;
    uint32_t inflight = 0, max_inflight_seen = 0;
    uint64_t submitted = 0, admitted = 0, completed = 0, released = 0;
    bool stop = false;
    std::thread th;
};

namespace {

struct Req {
    os_server_s* srv = nullptr;
    uint64_t ticket = 0;
    os_request r{};
    size_t out_bytes = 0, ws_bytes = 0;
    size_t off = SIZE_MAX;      // arena block: output, then workspace
    uint32_t slot = 0, stream = 0;
    int state = 0;              // 0 queued, 1 running, 2 done, 3 returned by poll
    int status = OS_OK;
    double submit_s = 0, admit_s = 0, done_s = 0;
};

void fill_result(const Req* q, os_result* r) {
    r->ticket = q->ticket;
    r->status = q->status;
    r->stream = q->stream;
    r->d_keys_out = q->srv->arena + q->off;
    r->n = q->r.n;
    r->bytes = q->out_bytes + q->ws_bytes;
    r->submit_s = q->submit_s;
    r->admit_s = q->admit_s;
    r->done_s = q->done_s;
}

// Runs on a CUDA callback thread once the request's sort and status copy are done.
void CUDART_CB on_done(void* p) {
    Req* q = static_cast<Req*>(p);
    os_server_s* s = q->srv;
    std::lock_guard<std::mutex> lk(s->mu);
    q->done_s = now_s();
    if (q->status == OS_OK && s->h_status[q->slot * STATUS_WORDS] != 0) q->status = OS_ERR_DEVICE;
    q->state = 2;
    s->alloc.shrink(q->off, q->out_bytes);   // the workspace goes back at once
    s->free_slots.push_back(q->slot);
    --s->inflight;
    --s->stream_load[q->stream];
    ++s->completed;
    s->done.push_back(q);
    s->cv_dispatch.notify_one();
    s->cv_done.notify_all();
}

bool head_admissible(os_server_s* s) {
    if (s->queue.empty() || s->inflight >= s->max_inflight) return false;
    const Req* q = s->queue.front();
    return s->alloc.largest_free() >= ArenaAlloc::round(q->out_bytes + q->ws_bytes);
}

void dispatch_loop(os_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_dispatch.wait(lk, [s] { return s->stop || head_admissible(s); });
        if (s->stop) return;
        Req* q = s->queue.front();
        const size_t off = s->alloc.alloc(q->out_bytes + q->ws_bytes);
        if (off == SIZE_MAX) continue;   // cannot happen after head_admissible; re-check
        s->queue.pop_front();
        q->off = off;
        q->state = 1;
        q->admit_s = now_s();
        q->slot = s->free_slots.back();
        s->free_slots.pop_back();
        uint32_t best = 0;
        for (uint32_t i = 1; i < s->streams.size(); ++i)
            if (s->stream_load[i] < s->stream_load[best]) best = i;
        q->stream = best;
        ++s->stream_load[best];
        ++s->inflight;
        ++s->admitted;
        s->max_inflight_seen = std::max(s->max_inflight_seen, s->inflight);
        lk.unlock();
        cudaStream_t st = s->streams[best];
        char* out = s->arena + off;
        char* ws = out + q->out_bytes;
        int rc = OS_OK;
        const void* kin = q->r.d_keys_in;
        if ((q->r.flags & OS_REQ_HOST_INPUT) && q->r.n > 0) {
            // host keys: copied into the output block, then sorted there in place
            const cudaError_t ce = cudaMemcpyAsync(out, kin, q->r.n * key_bytes_of(q->r.key_type),
                                                   cudaMemcpyHostToDevice, st);
            if (ce != cudaSuccess) rc = cuda_fail(ce);
            kin = out;
        }
        if (rc == OS_OK)
            rc = os_sort(q->r.key_type, kin, out, nullptr, nullptr, q->r.n, &q->r.prm, ws, q->ws_bytes, st,
                         nullptr);
        uint32_t* hs = s->h_status + q->slot * STATUS_WORDS;
        hs[0] = 0;
        q->status = rc;   // written before the callback is enqueued
        cudaError_t e = cudaSuccess;
        if (rc == OS_OK) e = cudaMemcpyAsync(hs, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_done, q);
        lk.lock();
        if (e != cudaSuccess) {
            // the callback will not run: finish the request here
            q->status = cuda_fail(e);
            lk.unlock();
            on_done(q);
            lk.lock();
        }
    }
}

int check_request(const os_request* req, size_t& ws_bytes) {
    if (!req || (req->flags & ~OS_REQ_HOST_INPUT) != 0) return OS_ERR_ARG;
    if (req->key_type == OS_S32) return OS_ERR_UNSUPPORTED;   // its sort synchronizes its stream
    if (req->n > 0 && !req->d_keys_in) return OS_ERR_ARG;
    return os_workspace_size(req->key_type, req->n, 0, &req->prm, &ws_bytes);
}

}  // namespace

extern "C" {

int os_server_create(const os_server_config* cfg, os_server* server) {
    if (!cfg || !server || !cfg->d_arena || cfg->arena_bytes < ArenaAlloc::ALIGN) return OS_ERR_ARG;
    if (cfg->streams < 1 || cfg->streams > 64 || cfg->max_inflight < 1 || cfg->max_inflight > 4096)
        return OS_ERR_ARG;
    *server = nullptr;
    auto* s = new os_server_s();
    cudaError_t e = cudaGetDevice(&s->device);
    s->arena = static_cast<char*>(cfg->d_arena);
    s->alloc.reset(cfg->arena_bytes);
    s->max_inflight = cfg->max_inflight;
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_status), sizeof(uint32_t) * STATUS_WORDS * cfg->max_inflight,
                          cudaHostAllocDefault);
    for (uint32_t i = 0; e == cudaSuccess && i < cfg->streams; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        if (s->h_status) cudaFreeHost(s->h_status);
        delete s;
        return cuda_fail(e);
    }
    s->stream_load.assign(s->streams.size(), 0);
    for (uint32_t i = cfg->max_inflight; i-- > 0;) s->free_slots.push_back(i);
    s->th = std::thread(dispatch_loop, s);
    *server = s;
    return OS_OK;
}

int os_server_submit(os_server s, const os_request* req, uint64_t* ticket) {
    if (!s || !ticket) return OS_ERR_ARG;
    size_t ws = 0;
    const int rc = check_request(req, ws);
    if (rc) return rc;
    auto* q = new Req();
    q->srv = s;
    q->r = *req;
    q->out_bytes = ArenaAlloc::round(req->n * key_bytes_of(req->key_type));
    q->ws_bytes = ws;
    if (ArenaAlloc::round(q->out_bytes + q->ws_bytes) > s->alloc.capacity()) {
        delete q;
        return OS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    q->submit_s = now_s();
    s->queue.push_back(q);
    s->live[q->ticket] = q;
    ++s->submitted;
    *ticket = q->ticket;
    s->cv_dispatch.notify_one();
    return OS_OK;
}

int os_server_poll(os_server s, os_result* results, uint32_t max_results, int64_t timeout_us, uint32_t* count) {
    if (!s || !count || (max_results > 0 && !results)) return OS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [s] { return !s->done.empty(); });
    uint32_t k = 0;
    while (k < max_results && !s->done.empty()) {
        Req* q = s->done.front();
        s->done.pop_front();
        q->state = 3;
        fill_result(q, &results[k++]);
    }
    *count = k;
    return OS_OK;
}

int os_server_release(os_server s, uint64_t ticket) {
    if (!s) return OS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end() || it->second->state < 2) return OS_ERR_ARG;
    Req* q = it->second;
    if (q->state == 2) {   // finished but never polled: drop it from the done list
        auto d = std::find(s->done.begin(), s->done.end(), q);
        if (d != s->done.end()) s->done.erase(d);
    }
    s->alloc.release(q->off);
    s->live.erase(it);
    ++s->released;
    delete q;
    s->cv_dispatch.notify_one();
    return OS_OK;
}

int os_server_get_stats(os_server s, os_server_stats* st) {
    if (!s || !st) return OS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->released = s->released;
    st->queued = (uint32_t)s->queue.size();
    st->inflight = s->inflight;
    st->arena_in_use = s->alloc.in_use();
    st->arena_peak = s->alloc.peak();
    st->arena_bytes = s->alloc.capacity();
    st->max_inflight_seen = s->max_inflight_seen;
    return OS_OK;
}

int os_server_replay(os_server s, const os_request* reqs, const double* arrival_s, uint32_t count,
                     os_result* results) {
    if (!s || (count > 0 && (!reqs || !arrival_s || !results))) return OS_ERR_ARG;
    for (uint32_t i = 1; i < count; ++i)
        if (arrival_s[i] < arrival_s[i - 1]) return OS_ERR_ARG;
    std::unordered_map<uint64_t, uint32_t> index;
    std::vector<os_result> buf(256);
    const double t0 = now_s();
    uint32_t next = 0, finished = 0;
    while (finished < count) {
        const double t = now_s() - t0;
        while (next < count && arrival_s[next] <= t) {
            uint64_t ticket = 0;
            const int rc = os_server_submit(s, &reqs[next], &ticket);
            if (rc == OS_OK) {
                index[ticket] = next;
            } else {
                std::memset(&results[next], 0, sizeof(os_result));
                results[next].status = rc;
                results[next].n = reqs[next].n;
                results[next].submit_s = results[next].admit_s = results[next].done_s = now_s();
                ++finished;
            }
            ++next;
        }
        int64_t wait_us = 1000;
        if (next < count) {
            const double gap = arrival_s[next] - (now_s() - t0);
            wait_us = gap > 0 ? (int64_t)(gap * 1e6) : 0;
        }
        uint32_t k = 0;
        os_server_poll(s, buf.data(), (uint32_t)buf.size(), wait_us > 100 ? wait_us - 50 : 0, &k);
        for (uint32_t j = 0; j < k; ++j) {
            auto it = index.find(buf[j].ticket);
            if (it == index.end()) continue;   // a request submitted outside this replay
            results[it->second] = buf[j];
            results[it->second].d_keys_out = nullptr;
            os_server_release(s, buf[j].ticket);
            index.erase(it);
            ++finished;
        }
    }
    return OS_OK;
}

int os_server_destroy(os_server s) {
    if (!s) return OS_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_dispatch.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);   // in-flight sorts and their callbacks
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->h_status) cudaFreeHost(s->h_status);
    for (auto& kv : s->live) delete kv.second;
    delete s;
    return OS_OK;
}

}  // extern "C"
