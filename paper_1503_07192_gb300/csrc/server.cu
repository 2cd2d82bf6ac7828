// Native continuous-batching query server (the serving pattern in the library itself).
//
// Requests (a resident graph, a host batch of pairs, a host output buffer) are queued by
// any thread; a scheduler thread keeps up to `slots` launches in flight, each on its own
// CUDA stream with pinned staging buffers and preallocated device buffers and query
// scratch: whenever a slot is free it takes the oldest waiting request and every other
// waiting request for the same graph (up to max_pairs pairs), copies their pairs to the
// device, answers them with one query launch (Algorithm 2, grouped by component pair),
// copies the distances back, and completes each request with its own slice once the
// slot's event has fired.  Requests that arrive while others are on the GPU join the next
// free slot; launches of different slots overlap on the device.  Latency is measured on
// the host from submission to completion.  Graphs are admitted against a device-memory
// budget by their table footprint.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int64_t ticket;
    int32_t gid;
    std::vector<int32_t> pairs;  // copied at submission
    int64_t q;
    void* out;                   // caller's buffer, q x 4 bytes
    Clock::time_point t0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t* h_pairs = nullptr;
    int32_t* h_out = nullptr;
    int32_t* d_pairs = nullptr;
    int32_t* d_out = nullptr;
    uint32_t* scratch = nullptr;
    std::vector<Req*> reqs;
    std::vector<int64_t> offs;
    bool busy = false;
};

}  // namespace

struct spq_server {
    int device = 0;
    int64_t max_pairs = 0;
    size_t budget = 0, resident = 0;
    std::mutex mu;
    std::condition_variable cv;       // new requests / stop
    std::condition_variable done_cv;  // completions
    bool stop = false;
    std::deque<Req*> queue;
    std::unordered_map<int32_t, spq_handle*> graphs;
    std::unordered_map<int64_t, int> state;  // ticket -> 0 pending, 1 done
    std::vector<Slot> slots;
    std::thread th;
    std::vector<double> lat_ms;
    int64_t pairs_done = 0;
    int64_t next_ticket = 1;
    cudaError_t failed = cudaSuccess;  // first CUDA error of the scheduler
};

namespace {

// (sl.reqs holds the batch already; h is its graph)
cudaError_t launch_slot(Slot& sl, spq_handle* h) {
    int64_t total = 0;
    sl.offs.clear();
    for (Req* r : sl.reqs) {
        memcpy(sl.h_pairs + 2 * total, r->pairs.data(), (size_t)r->q * 8);
        sl.offs.push_back(total);
        total += r->q;
    }
    cudaError_t e = cudaMemcpyAsync(sl.d_pairs, sl.h_pairs, (size_t)total * 8, cudaMemcpyHostToDevice, sl.st);
    if (e != cudaSuccess) return e;
    spq::QueryCtx<int32_t> ci;
    spq::QueryCtx<float> cf;
    bool f32store = false, out_f32 = false;
    int32_t k = 0;
    spq::handle_query_view(h, &ci, &cf, &f32store, &out_f32, &k);
    uint32_t* scratch = (total >= 4096 && k <= 65535 && h->query_grouped) ? sl.scratch : nullptr;
    e = f32store ? spq::launch_query<float>(cf, sl.d_pairs, total, sl.d_out, out_f32, (uint32_t)k, scratch, sl.st)
                 : spq::launch_query<int32_t>(ci, sl.d_pairs, total, sl.d_out, out_f32, (uint32_t)k, scratch, sl.st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)total * 4, cudaMemcpyDeviceToHost, sl.st)) != cudaSuccess)
        return e;
    if ((e = cudaEventRecord(sl.ev, sl.st)) != cudaSuccess) return e;
    sl.busy = true;
    return cudaSuccess;
}

// The oldest request and every other waiting request for its graph, up to max_pairs
// pairs (called with the lock held).
std::vector<Req*> take_batch(spq_server* s) {
    std::vector<Req*> batch{s->queue.front()};
    s->queue.pop_front();
    int64_t total = batch[0]->q;
    std::deque<Req*> keep;
    while (!s->queue.empty()) {
        Req* r = s->queue.front();
        s->queue.pop_front();
        if (r->gid == batch[0]->gid && total + r->q <= s->max_pairs) {
            batch.push_back(r);
            total += r->q;
        } else {
            keep.push_back(r);
        }
    }
    s->queue.swap(keep);
    return batch;
}

void scheduler(spq_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        // completions (outside the lock: the slots belong to this thread)
        for (Slot& sl : s->slots) {
            if (!sl.busy || cudaEventQuery(sl.ev) != cudaSuccess) continue;
            const Clock::time_point now = Clock::now();
            std::vector<double> lat;
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                Req* r = sl.reqs[i];
                memcpy(r->out, sl.h_out + sl.offs[i], (size_t)r->q * 4);
                lat.push_back(std::chrono::duration<double, std::milli>(now - r->t0).count());
            }
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (size_t i = 0; i < sl.reqs.size(); ++i) {
                    s->state[sl.reqs[i]->ticket] = 1;
                    s->pairs_done += sl.reqs[i]->q;
                    delete sl.reqs[i];
                }
                s->lat_ms.insert(s->lat_ms.end(), lat.begin(), lat.end());
                sl.reqs.clear();
                sl.busy = false;
            }
            s->done_cv.notify_all();
            progressed = true;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        bool any_busy = false;
        for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
        if (s->stop && s->queue.empty() && !any_busy) return;
        for (Slot& sl : s->slots) {
            if (sl.busy || s->queue.empty()) continue;
            sl.reqs = take_batch(s);  // visible to spq_server_remove_graph from here on
            spq_handle* h = s->graphs.at(sl.reqs[0]->gid);
            lk.unlock();
            const cudaError_t e = launch_slot(sl, h);
            lk.lock();
            if (e != cudaSuccess) {
                if (s->failed == cudaSuccess) s->failed = e;
                for (Req* r : sl.reqs) {  // answered as failed: out untouched
                    s->state[r->ticket] = -1;
                    delete r;
                }
                sl.reqs.clear();
                sl.busy = false;
                s->done_cv.notify_all();
            }
            progressed = true;
            any_busy = true;
        }
        if (!progressed) {
            if (!any_busy)
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(10));
            }
        }
    }
}

void free_slots(spq_server* s) {
    for (Slot& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.h_pairs) cudaFreeHost(sl.h_pairs);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.d_pairs) cudaFree(sl.d_pairs);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.scratch) cudaFree(sl.scratch);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

spq_status spq_server_create(int device, int32_t slots, int64_t max_pairs, size_t memory_budget, spq_server** out) {
    if (!out || slots < 1 || slots > 64 || max_pairs < 1 || max_pairs > ((int64_t)1 << 28)) return SPQ_EINVAL;
    *out = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return SPQ_EINVAL;
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};
    spq_server* s = new (std::nothrow) spq_server();
    if (!s) return SPQ_ENOMEM;
    s->device = device;
    s->max_pairs = max_pairs;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = memory_budget ? memory_budget : (size_t)(0.9 * (double)free_b);
    s->slots.resize((size_t)slots);
    cudaError_t e = cudaSuccess;
    const size_t scratch_words = (size_t)spq::query_scratch_words(max_pairs);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_pairs, (size_t)max_pairs * 8, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_out, (size_t)max_pairs * 4, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_pairs, (size_t)max_pairs * 8);
        if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_out, (size_t)max_pairs * 4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&sl.scratch, scratch_words * 4);
    }
    if (e != cudaSuccess) {
        spq::note_cuda_error(e);
        free_slots(s);
        delete s;
        return SPQ_ECUDA;
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return SPQ_OK;
}

spq_status spq_server_add_graph(spq_server* s, int32_t gid, spq_handle* h) {
    if (!s || !h) return SPQ_EINVAL;
    if (h->device != s->device) return SPQ_EINVAL;  // the server's slots run on its own device
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->graphs.count(gid)) return SPQ_EINVAL;
    const size_t fp = h->bytes;
    if (s->resident + fp > s->budget) return SPQ_ENOMEM;
    s->graphs[gid] = h;
    s->resident += fp;
    return SPQ_OK;
}

spq_status spq_server_remove_graph(spq_server* s, int32_t gid) {
    if (!s) return SPQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->graphs.find(gid);
    if (it == s->graphs.end()) return SPQ_EINVAL;
    // wait until no queued or running request uses the graph
    for (;;) {
        bool used = false;
        for (Req* r : s->queue) used = used || r->gid == gid;
        for (Slot& sl : s->slots)
            for (Req* r : sl.reqs) used = used || r->gid == gid;
        if (!used) break;
        s->done_cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    s->resident -= it->second->bytes;
    s->graphs.erase(it);
    return SPQ_OK;
}

spq_status spq_server_submit(spq_server* s, int32_t gid, const int32_t* pairs, int64_t q, void* out, int64_t* ticket) {
    if (!s || !ticket || q < 1 || !pairs || !out) return SPQ_EINVAL;
    if (q > s->max_pairs) return SPQ_ENOMEM;
    Req* r = new (std::nothrow) Req();
    if (!r) return SPQ_ENOMEM;
    r->gid = gid;
    r->q = q;
    r->out = out;
    r->pairs.assign(pairs, pairs + 2 * q);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->graphs.find(gid);
        bool ok = it != s->graphs.end();
        const int32_t n = ok ? it->second->n : 0;
        for (int64_t i = 0; ok && i < 2 * q; ++i) ok = r->pairs[i] >= 0 && r->pairs[i] < n;
        if (!ok) {
            delete r;
            return SPQ_EINVAL;
        }
        r->ticket = s->next_ticket++;
        r->t0 = Clock::now();
        s->state[r->ticket] = 0;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return SPQ_OK;
}

int32_t spq_server_poll(spq_server* s, int64_t ticket) {
    if (!s) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return -1;
    const int v = it->second;
    if (v != 0) s->state.erase(it);
    return v;
}

spq_status spq_server_wait(spq_server* s, int64_t ticket, double timeout_s) {
    if (!s) return SPQ_EINVAL;
    if (!(timeout_s >= 0.0)) timeout_s = 0.0;  // (NaN too)
    timeout_s = std::min(timeout_s, 1e7);
    std::unique_lock<std::mutex> lk(s->mu);
    const Clock::time_point until =
        Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    for (;;) {
        auto it = s->state.find(ticket);
        if (it == s->state.end()) return SPQ_EINVAL;
        if (it->second != 0) {
            const int v = it->second;
            s->state.erase(it);
            return v == 1 ? SPQ_OK : SPQ_ECUDA;
        }
        if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout) return SPQ_ETIMEOUT;
    }
}

spq_status spq_server_stats(spq_server* s, double* p50_ms, double* p99_ms, int64_t* requests, int64_t* pairs,
                            int32_t reset) {
    if (!s) return SPQ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v = s->lat_ms;
    if (requests) *requests = (int64_t)v.size();
    if (pairs) *pairs = s->pairs_done;
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + (ptrdiff_t)i, v.end());
        return v[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (reset) {
        s->lat_ms.clear();
        s->pairs_done = 0;
    }
    return s->failed == cudaSuccess ? SPQ_OK : SPQ_ECUDA;
}

void spq_server_destroy(spq_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    free_slots(s);
    for (Req* r : s->queue) delete r;
    delete s;
}

}  // extern "C"
