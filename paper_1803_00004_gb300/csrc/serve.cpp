// Serving: continuous batching of filter requests on one device.
//
// A submission is stamped and queued at once; it never waits for the GPU or
// for its plan.  Plan threads take queued requests in arrival order, find
// each one's plan in the server's cache or build it (the host FP64 fit of
// the coefficients, Sec. IV / App. B), and mark the request ready; the plan
// build is therefore inside the request's latency.  A worker thread admits
// ready requests in order while the device arena (one allocation made when
// the server starts, the "free HBM" the server admits by) has room for their
// buffers and a slot is free, merges the requests admitted together into one
// persistent batched launch (bf_filter_batch's kernel, its parameters, work
// list and partial planes placed in the arena block, so no allocation
// happens per request), and issues each group on the next of a few streams:
// host->device copies (host requests), the launch, device->host copies, and a
// completion event.  Groups on different streams overlap on the device;
// requests that arrive while others run are admitted as soon as arena memory
// and slots free up.  The worker polls completion events, returns the
// group's arena block and slots, and wakes pollers.  Each image's result
// depends only on its own plan and pixels, so it equals a lone bf_filter call
// up to fp32 rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t ns_between(Clock::time_point a, Clock::time_point b) {
    return b > a ? (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(b - a).count() : 0;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over the server's device arena (offsets in bytes, 256-byte granules); freed blocks
// merge with their neighbours.
class Arena {
public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t *off) {
        n = align_up(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align_up(std::max<size_t>(n, 1));
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }

private:
    size_t size_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct PlanEntry {
    bf_plan *plan = nullptr;
    int refs = 0;                 // requests holding the plan
    uint64_t last_use = 0;
};

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> key;     // the plan cache key (the descriptor's bytes)
    bf_plan_desc desc{};
    bf_plan *plan = nullptr;
    const float *in = nullptr;
    float *out = nullptr;
    size_t in_pitch = 0, out_pitch = 0;
    int h = 0, w = 0, host = 0;
    Clock::time_point t_submit, t_admit, t_done;
    uint64_t plan_ns = 0, device_ns = 0;
    int status = BF_OK;
    bool ready = false, done = false, cancelled = false;
};

struct Group {
    std::vector<uint64_t> tickets;
    size_t off = 0, bytes = 0;    // the group's arena block
    int stream = 0;
    cudaEvent_t start = nullptr, end = nullptr;
    bf_status launch_status = BF_OK;
};

constexpr size_t kMaxCachedPlans = 256;

}  // namespace

struct bf_server {
    bf_serve_config cfg{};
    Arena arena;
    uint8_t *d_arena = nullptr;
    int slots_in_use = 0;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_plan, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1, use_clock = 0;
    std::deque<uint64_t> pending;  // waiting for their plan (plan thread)
    std::deque<uint64_t> queue;    // plan ready, waiting for arena memory and a slot (worker)
    std::unordered_map<uint64_t, Request> reqs;
    std::map<std::vector<uint8_t>, PlanEntry> plans;
    std::list<Group> inflight;
    std::thread worker;
    std::vector<std::thread> planners;
};

namespace {

// Arena bytes of a group: the staging of its host requests' images, then its batched launch's buffer.
size_t staging_bytes(const Request &r) { return r.host ? 2 * align_up((size_t)r.h * r.w * sizeof(float)) : 0; }

size_t group_bytes(const std::vector<const Request *> &g) {
    std::vector<const bf_plan *> ps;
    std::vector<bf_image> ims;
    size_t stage = 0;
    uintptr_t fake = kAlign;  // the layout's size does not depend on the image addresses
    for (const Request *r : g) {
        stage += staging_bytes(*r);
        const size_t n = (size_t)r->h * r->w * sizeof(float);
        ims.push_back(bf_image{reinterpret_cast<const float *>(fake), (size_t)r->w * sizeof(float),
                               reinterpret_cast<float *>(fake + align_up(n)), (size_t)r->w * sizeof(float), r->h, r->w});
        fake += 2 * align_up(n);
        ps.push_back(r->plan);
    }
    const size_t batch = bfi::batch_device_bytes(ps.data(), ims.data(), (int)ps.size());
    return batch ? stage + align_up(batch) : 0;  // 0: the batch layout failed
}

void release_plan(bf_server *S, const Request &r) {
    auto it = S->plans.find(r.key);
    if (it != S->plans.end() && it->second.refs > 0) --it->second.refs;
}

// Least recently used plans no request holds go once the cache is over its size.
void trim_plans(bf_server *S) {
    while (S->plans.size() > kMaxCachedPlans) {
        auto victim = S->plans.end();
        for (auto it = S->plans.begin(); it != S->plans.end(); ++it)
            if (it->second.refs == 0 && (victim == S->plans.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == S->plans.end()) return;
        bf_plan_destroy(victim->second.plan);
        S->plans.erase(victim);
    }
}

void complete_locked(bf_server *S, Request &r, int status) {
    r.status = status;
    r.done = true;
    r.t_done = Clock::now();
    S->cv_done.notify_all();
}

// Plan thread: arrival order; cache hit or host build (outside the lock); then the request is ready.
void planner_main(bf_server *S) {
    cudaSetDevice(S->cfg.device);  // launch geometries are looked up for the current device
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_plan.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        if (S->pending.empty()) {
            if (S->stop) return;
            continue;
        }
        const uint64_t t = S->pending.front();
        S->pending.pop_front();
        auto rit = S->reqs.find(t);
        if (rit == S->reqs.end() || rit->second.done) continue;
        std::vector<uint8_t> key = rit->second.key;
        bf_plan_desc desc = rit->second.desc;
        bf_plan *plan = nullptr;
        bf_status st = BF_OK;
        auto pit = S->plans.find(key);
        if (pit == S->plans.end()) {
            lk.unlock();
            st = bf_plan_create(&desc, &plan);
            lk.lock();
            if (st == BF_OK) {
                pit = S->plans.find(key);
                if (pit != S->plans.end()) {
                    bf_plan_destroy(plan);  // built meanwhile for another request
                } else {
                    pit = S->plans.emplace(key, PlanEntry{plan, 0, 0}).first;
                }
            }
        }
        rit = S->reqs.find(t);
        if (rit == S->reqs.end()) continue;
        Request &r = rit->second;
        if (r.done) continue;  // cancelled while its plan was built
        if (st != BF_OK) {
            complete_locked(S, r, st);
            continue;
        }
        pit->second.refs++;
        pit->second.last_use = ++S->use_clock;
        r.plan = pit->second.plan;
        r.plan_ns = ns_between(r.t_submit, Clock::now());
        trim_plans(S);
        std::vector<const Request *> alone{&r};
        const size_t need = group_bytes(alone);
        if (need == 0 || need > S->arena.size()) {
            release_plan(S, r);
            complete_locked(S, r, need == 0 ? BF_ERR_UNSUPPORTED : BF_ERR_ADMISSION);
            continue;
        }
        r.ready = true;
        S->queue.push_back(t);
        S->cv_work.notify_one();
    }
}

}  // namespace

namespace {

// Issues one admitted group on its stream (worker thread, no lock held; the group's requests are not touched
// by other threads until the group completes).
void launch_group(bf_server *S, Group &g, const std::vector<Request *> &rs) {
    cudaStream_t s = S->streams[g.stream];
    if (cudaEventCreate(&g.start) != cudaSuccess || cudaEventCreate(&g.end) != cudaSuccess) {
        cudaGetLastError();
        g.launch_status = bfi::fail(BF_ERR_CUDA, "server events");
        return;
    }
    bf_status st = BF_OK;
    if (cudaEventRecord(g.start, s) != cudaSuccess) st = BF_ERR_CUDA;
    uint8_t *block = S->d_arena + g.off, *cur = block;
    std::vector<const bf_plan *> ps;
    std::vector<bf_image> ims;
    for (Request *r : rs) {
        const size_t row = (size_t)r->w * sizeof(float), n = align_up(row * r->h);
        bf_image im{r->in, r->in_pitch, r->out, r->out_pitch, r->h, r->w};
        if (r->host) {
            float *din = reinterpret_cast<float *>(cur), *dout = reinterpret_cast<float *>(cur + n);
            cur += 2 * n;
            if (st == BF_OK &&
                cudaMemcpy2DAsync(din, row, r->in, r->in_pitch, row, r->h, cudaMemcpyHostToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                st = bfi::fail(BF_ERR_CUDA, "server upload");
            }
            im = bf_image{din, row, dout, row, r->h, r->w};
        }
        ps.push_back(r->plan);
        ims.push_back(im);
    }
    if (st == BF_OK)
        st = bfi::enqueue_batch_into(ps.data(), ims.data(), (int)ps.size(), s, cur, g.bytes - (size_t)(cur - block));
    for (size_t i = 0; i < rs.size() && st == BF_OK; ++i)
        if (rs[i]->host && cudaMemcpy2DAsync(rs[i]->out, rs[i]->out_pitch, ims[i].d_out, ims[i].out_pitch_bytes,
                                             (size_t)rs[i]->w * sizeof(float), rs[i]->h, cudaMemcpyDeviceToHost,
                                             s) != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_CUDA, "server download");
        }
    if (cudaEventRecord(g.end, s) != cudaSuccess) {
        cudaGetLastError();
        if (st == BF_OK) st = BF_ERR_CUDA;
    }
    g.launch_status = st;
}

void finish_group(bf_server *S, Group &g, bf_status st) {
    float ms = 0.f;
    if (st == BF_OK && cudaEventElapsedTime(&ms, g.start, g.end) != cudaSuccess) cudaGetLastError();
    if (g.start) cudaEventDestroy(g.start);
    if (g.end) cudaEventDestroy(g.end);
    std::lock_guard<std::mutex> lk(S->mu);
    S->arena.release(g.off, g.bytes);
    S->slots_in_use -= (int)g.tickets.size();
    for (uint64_t t : g.tickets) {
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;
        it->second.device_ns = (uint64_t)(ms * 1e6);
        release_plan(S, it->second);
        complete_locked(S, it->second, st);
    }
    S->cv_work.notify_one();  // memory and slots came back
}

void worker_main(bf_server *S) {
    cudaSetDevice(S->cfg.device);
    for (;;) {
        Group g;
        std::vector<Request *> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->inflight.empty(); });
            if (S->stop && S->queue.empty() && S->inflight.empty() && S->pending.empty()) return;
            // admission: order of readiness, while the group's arena block fits and slots are free
            std::vector<const Request *> cand;
            size_t bytes = 0;
            while (!S->queue.empty() && (int)admitted.size() < S->cfg.max_batch &&
                   S->slots_in_use + (int)admitted.size() < S->cfg.max_slots) {
                Request &r = S->reqs[S->queue.front()];
                cand.push_back(&r);
                const size_t need = group_bytes(cand);
                size_t off = 0;
                if (need == 0 || !S->arena.alloc(need, &off)) {  // probe: does the grown block fit?
                    cand.pop_back();
                    break;
                }
                S->arena.release(off, need);
                bytes = need;
                S->queue.pop_front();
                r.t_admit = Clock::now();
                admitted.push_back(&r);
                g.tickets.push_back(r.ticket);
            }
            if (!admitted.empty()) {
                S->arena.alloc(bytes, &g.off);  // fits: the probe above just found the block
                g.bytes = bytes;
                S->slots_in_use += (int)admitted.size();
                g.stream = S->next_stream;
                S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
            }
        }
        if (!admitted.empty()) {
            launch_group(S, g, admitted);
            std::lock_guard<std::mutex> lk(S->mu);
            S->inflight.push_back(std::move(g));
        }
        // completions
        std::vector<Group> finished;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto it = S->inflight.begin(); it != S->inflight.end();) {
                cudaError_t q = it->end ? cudaEventQuery(it->end) : cudaSuccess;
                if (q == cudaErrorNotReady) {
                    ++it;
                    continue;
                }
                if (q != cudaSuccess) cudaGetLastError();
                if (q != cudaSuccess && it->launch_status == BF_OK) it->launch_status = BF_ERR_CUDA;
                finished.push_back(std::move(*it));
                it = S->inflight.erase(it);
            }
        }
        for (auto &f : finished) finish_group(S, f, f.launch_status);
        if (admitted.empty() && finished.empty()) {
            // work in flight, or ready requests waiting for memory, but nothing changed: poll again shortly
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

std::vector<uint8_t> desc_key(const bf_plan_desc &d) {
    std::vector<uint8_t> k(sizeof(d));
    std::memcpy(k.data(), &d, sizeof(d));
    return k;
}

}  // namespace

extern "C" {

bf_status bf_serve_create(const bf_serve_config *cfg, bf_server **out) {
    if (!cfg || !out) return bfi::fail(BF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return bfi::fail(BF_ERR_NO_DEVICE, "server device not available");
    }
    if (cfg->max_slots < 0 || cfg->n_streams < 0 || cfg->max_batch < 0 || cfg->plan_threads < 0 ||
        cfg->plan_threads > 64)
        return bfi::fail(BF_ERR_INVALID_ARG, "negative server limits");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(cfg->device);
    bf_server *S = new (std::nothrow) bf_server();
    if (!S) {
        cudaSetDevice(prev);
        return bfi::fail(BF_ERR_OOM, "server allocation");
    }
    S->cfg = *cfg;
    if (S->cfg.max_slots == 0) S->cfg.max_slots = 64;
    if (S->cfg.n_streams == 0) S->cfg.n_streams = 4;
    if (S->cfg.max_batch == 0) S->cfg.max_batch = 16;
    if (S->cfg.plan_threads <= 0) S->cfg.plan_threads = 4;
    size_t budget = cfg->hbm_budget_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
        budget = std::min<size_t>(fr / 4, (size_t)16 << 30);
    }
    budget = budget / kAlign * kAlign;
    bf_status st = BF_OK;
    if (budget == 0 || cudaMalloc((void **)&S->d_arena, budget) != cudaSuccess) {
        cudaGetLastError();
        st = bfi::fail(BF_ERR_OOM, "server arena of " + std::to_string(budget) + " bytes");
    }
    S->arena.init(budget);
    for (int i = 0; i < S->cfg.n_streams && st == BF_OK; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_CUDA, "server streams");
            break;
        }
        S->streams.push_back(s);
    }
    if (st != BF_OK) {
        for (auto x : S->streams) cudaStreamDestroy(x);
        if (S->d_arena) cudaFree(S->d_arena);
        delete S;
        cudaSetDevice(prev);
        return st;
    }
    for (int i = 0; i < S->cfg.plan_threads; ++i) S->planners.emplace_back(planner_main, S);
    S->worker = std::thread(worker_main, S);
    cudaSetDevice(prev);
    *out = S;
    return BF_OK;
}

bf_status bf_serve_submit(bf_server *S, const bf_request *req, uint64_t *ticket) {
    const Clock::time_point t0 = Clock::now();
    if (!S || !req || !ticket) return bfi::fail(BF_ERR_INVALID_ARG, "NULL argument");
    if (req->memory != BF_MEM_DEVICE && req->memory != BF_MEM_HOST) return bfi::fail(BF_ERR_INVALID_ARG, "memory kind");
    if (req->height < 1 || req->width < 1) return bfi::fail(BF_ERR_INVALID_ARG, "bad request image");
    bf_status st = bfi::check_image(req->in, req->in_pitch_bytes, req->out, req->out_pitch_bytes, req->height,
                                    req->width);
    if (st != BF_OK) return st;
    Request r;
    r.desc = req->desc;
    r.desc.device = S->cfg.device;
    r.key = desc_key(r.desc);
    r.in = req->in;
    r.out = req->out;
    r.in_pitch = req->in_pitch_bytes;
    r.out_pitch = req->out_pitch_bytes;
    r.h = req->height;
    r.w = req->width;
    r.host = req->memory == BF_MEM_HOST ? 1 : 0;
    r.t_submit = t0;
    if (staging_bytes(r) > S->arena.size())
        return bfi::fail(BF_ERR_ADMISSION, "request needs more device memory than the server's arena");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return bfi::fail(BF_ERR_INVALID_ARG, "server is shutting down");
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    S->pending.push_back(r.ticket);
    S->reqs.emplace(r.ticket, std::move(r));
    S->cv_plan.notify_one();
    return BF_OK;
}

bf_status bf_serve_poll(bf_server *S, uint64_t ticket, int timeout_ms, bf_result *out) {
    if (!S || !out) return bfi::fail(BF_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return bfi::fail(BF_ERR_NOT_FOUND, "unknown ticket");
    auto is_done = [&] {
        auto j = S->reqs.find(ticket);
        return j == S->reqs.end() || j->second.done;
    };
    if (timeout_ms < 0) S->cv_done.wait(lk, is_done);
    else if (timeout_ms > 0) S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), is_done);
    it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return bfi::fail(BF_ERR_NOT_FOUND, "unknown ticket");
    if (!it->second.done) return BF_ERR_TIMEOUT;
    const Request &r = it->second;
    const bool admitted = r.t_admit != Clock::time_point();
    out->status = r.cancelled ? BF_ERR_CANCELLED : r.status;
    out->latency_ns = ns_between(r.t_submit, r.t_done);
    out->queue_ns = admitted ? ns_between(r.t_submit, r.t_admit) : 0;
    out->plan_ns = r.plan_ns;
    out->device_ns = r.device_ns;
    const bool cancelled = r.cancelled;
    S->reqs.erase(it);
    return cancelled ? BF_ERR_CANCELLED : BF_OK;
}

bf_status bf_serve_cancel(bf_server *S, uint64_t ticket) {
    if (!S) return bfi::fail(BF_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second.done || it->second.t_admit != Clock::time_point())
        return bfi::fail(BF_ERR_NOT_FOUND, "request not pending");
    Request &r = it->second;
    for (auto *q : {&S->pending, &S->queue})
        for (auto j = q->begin(); j != q->end(); ++j)
            if (*j == ticket) {
                q->erase(j);
                break;
            }
    if (r.ready) release_plan(S, r);  // held its plan while waiting for admission
    r.cancelled = true;
    complete_locked(S, r, BF_ERR_CANCELLED);
    return BF_OK;
}

void bf_serve_destroy(bf_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &kv : S->reqs) {  // never admitted: cancelled (the plan thread skips them)
            Request &r = kv.second;
            if (r.done || r.t_admit != Clock::time_point()) continue;
            if (r.ready) release_plan(S, r);
            r.cancelled = true;
            complete_locked(S, r, BF_ERR_CANCELLED);
        }
        S->pending.clear();
        S->queue.clear();
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_plan.notify_all();
        S->cv_done.notify_all();
    }
    for (auto &t : S->planners)
        if (t.joinable()) t.join();
    if (S->worker.joinable()) S->worker.join();
    for (auto s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (S->d_arena) cudaFree(S->d_arena);
    for (auto &kv : S->plans) bf_plan_destroy(kv.second.plan);
    delete S;
}

}  // extern "C"
