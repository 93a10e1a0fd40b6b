// Serving: continuous batching of filter requests on one device.
//
// Submitting only queues a request (and builds or reuses its plan).  A worker
// thread admits queued requests in arrival order while the device-memory
// budget and the slot count allow, merges the requests admitted together
// into one persistent batched launch (bf_filter_batch's kernel, without graph
// capture because every group has new buffers), and issues each group on the
// next of a few streams: host->device copies, the launch, device->host
// copies, then a completion event.  Groups on different streams overlap on
// the device, and requests that arrive while others run are admitted as soon
// as memory and slots free up.  The worker polls completion events, releases
// the group's memory and slots, and wakes pollers.  Results are identical to
// a lone bf_filter call up to fp32 rounding: each image's work depends only on
// its own plan and pixels.
#include <cuda_runtime.h>

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

double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket;
    bf_plan *plan;
    const float *h_in;
    float *h_out;
    int h, w;
    size_t bytes;  // device bytes while admitted
    Clock::time_point t_submit, t_admit, t_done;
    double device_ms = 0;
    int status = BF_OK;
    bool done = false, cancelled = false;
};

struct Group {
    std::vector<uint64_t> tickets;
    std::vector<float *> bufs;
    size_t bytes = 0;
    int stream = 0;
    cudaEvent_t start = nullptr, end = nullptr;
    bf_status launch_status = BF_OK;
};

}  // namespace

struct bf_server {
    bf_serve_config cfg{};
    size_t budget = 0, in_use = 0;
    int slots_in_use = 0;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::map<std::vector<uint8_t>, bf_plan *> plans;
    std::list<Group> inflight;
    std::thread worker;
};

namespace {

void finish_group(bf_server *S, Group &g, bf_status st) {
    float ms = 0.f;
    if (st == BF_OK && cudaEventElapsedTime(&ms, g.start, g.end) != cudaSuccess) cudaGetLastError();
    cudaStream_t s = S->streams[g.stream];
    for (float *b : g.bufs) cudaFreeAsync(b, s);
    cudaEventDestroy(g.start);
    cudaEventDestroy(g.end);
    auto now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= g.bytes;
    S->slots_in_use -= (int)g.tickets.size();
    for (uint64_t t : g.tickets) {
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;
        it->second.done = true;
        it->second.status = st;
        it->second.device_ms = ms;
        it->second.t_done = now;
    }
    S->cv_done.notify_all();
}

// Issues one admitted group on its stream (worker thread, no lock held).
void launch_group(bf_server *S, Group &g, std::vector<Request *> &rs) {
    cudaStream_t s = S->streams[g.stream];
    bf_status st = BF_OK;
    if (cudaEventCreate(&g.start) != cudaSuccess || cudaEventCreate(&g.end) != cudaSuccess) {
        cudaGetLastError();
        g.launch_status = bfi::fail(BF_ERR_CUDA, "server events");
        return;
    }
    cudaEventRecord(g.start, s);
    std::vector<const bf_plan *> ps;
    std::vector<bf_image> ims;
    for (Request *r : rs) {
        size_t n = (size_t)r->h * r->w * sizeof(float);
        float *din = nullptr, *dout = nullptr;
        if (cudaMallocAsync((void **)&din, n, s) != cudaSuccess || cudaMallocAsync((void **)&dout, n, s) != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_OOM, "server buffers");
            if (din) g.bufs.push_back(din);
            break;
        }
        g.bufs.push_back(din);
        g.bufs.push_back(dout);
        if (cudaMemcpyAsync(din, r->h_in, n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_CUDA, "server upload");
            break;
        }
        ps.push_back(r->plan);
        ims.push_back(bf_image{din, (size_t)r->w * sizeof(float), dout, (size_t)r->w * sizeof(float), r->h, r->w});
    }
    if (st == BF_OK) st = bfi::enqueue_batch_direct(ps.data(), ims.data(), (int)ps.size(), s);
    if (st == BF_OK)
        for (size_t i = 0; i < rs.size(); ++i)
            if (cudaMemcpyAsync(rs[i]->h_out, ims[i].d_out, (size_t)rs[i]->h * rs[i]->w * sizeof(float),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess) {
                cudaGetLastError();
                st = bfi::fail(BF_ERR_CUDA, "server download");
                break;
            }
    cudaEventRecord(g.end, s);
    g.launch_status = st;
}

void worker_main(bf_server *S) {
    cudaSetDevice(S->cfg.device);
    for (;;) {
        Group g;
        std::vector<Request *> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto ready = [&] { return S->stop || !S->queue.empty() || !S->inflight.empty(); };
            S->cv_work.wait(lk, ready);
            if (S->stop && S->queue.empty() && S->inflight.empty()) return;
            // admission: arrival order, within the memory budget and the slot count
            while (!S->queue.empty() && (int)admitted.size() < S->cfg.max_batch) {
                Request &r = S->reqs[S->queue.front()];
                if (S->in_use + r.bytes > S->budget || S->slots_in_use >= S->cfg.max_slots) break;
                S->queue.pop_front();
                S->in_use += r.bytes;
                S->slots_in_use += 1;
                r.t_admit = Clock::now();
                admitted.push_back(&r);
                g.tickets.push_back(r.ticket);
                g.bytes += r.bytes;
            }
            if (!admitted.empty()) {
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
            // work is in flight but nothing finished or could be admitted: poll again shortly
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
    if (cfg->max_slots < 0 || cfg->n_streams < 0 || cfg->max_batch < 0)
        return bfi::fail(BF_ERR_INVALID_ARG, "negative server limits");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(cfg->device);
    bf_server *S = new (std::nothrow) bf_server();
    if (!S) return bfi::fail(BF_ERR_OOM, "server allocation");
    S->cfg = *cfg;
    if (S->cfg.max_slots == 0) S->cfg.max_slots = 64;
    if (S->cfg.n_streams == 0) S->cfg.n_streams = 4;
    if (S->cfg.max_batch == 0) S->cfg.max_batch = 16;
    S->budget = cfg->hbm_budget_bytes;
    if (S->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
        S->budget = fr / 2;
    }
    for (int i = 0; i < S->cfg.n_streams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto x : S->streams) cudaStreamDestroy(x);
            delete S;
            cudaSetDevice(prev);
            return bfi::fail(BF_ERR_CUDA, "server streams");
        }
        S->streams.push_back(s);
    }
    S->worker = std::thread(worker_main, S);
    cudaSetDevice(prev);
    *out = S;
    return BF_OK;
}

bf_status bf_serve_submit(bf_server *S, const bf_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket) return bfi::fail(BF_ERR_INVALID_ARG, "NULL argument");
    if (req->height < 1 || req->width < 1 || !req->h_in || !req->h_out)
        return bfi::fail(BF_ERR_INVALID_ARG, "bad request image");
    bf_plan_desc d = req->desc;
    d.device = S->cfg.device;
    if (d.policy == BF_RANGE_PAPER_3D)
        return bfi::fail(BF_ERR_UNSUPPORTED, "the 3-D form (BF_RANGE_PAPER_3D) runs through bf_filter, not the server");
    bf_plan *plan = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto k = desc_key(d);
        auto it = S->plans.find(k);
        if (it != S->plans.end()) plan = it->second;
    }
    if (!plan) {
        bf_status st = bf_plan_create(&d, &plan);
        if (st != BF_OK) return st;
        std::lock_guard<std::mutex> lk(S->mu);
        auto k = desc_key(d);
        auto it = S->plans.find(k);
        if (it != S->plans.end()) {
            bf_plan_destroy(plan);
            plan = it->second;
        } else {
            S->plans[k] = plan;
        }
    }
    bf_image probe{reinterpret_cast<const float *>(256), (size_t)req->width * 4,
                   reinterpret_cast<float *>(256 + (size_t)req->width * req->height * 4 + 256),
                   (size_t)req->width * 4, req->height, req->width};
    const bf_plan *pp = plan;
    size_t bytes = 2 * (size_t)req->height * req->width * sizeof(float) + bfi::batch_device_bytes(&pp, &probe, 1);
    std::lock_guard<std::mutex> lk(S->mu);
    if (bytes > S->budget) return bfi::fail(BF_ERR_ADMISSION, "request needs more device memory than the budget");
    Request r;
    r.ticket = S->next_ticket++;
    r.plan = plan;
    r.h_in = req->h_in;
    r.h_out = req->h_out;
    r.h = req->height;
    r.w = req->width;
    r.bytes = bytes;
    r.t_submit = Clock::now();
    S->reqs[r.ticket] = r;
    S->queue.push_back(r.ticket);
    *ticket = r.ticket;
    S->cv_work.notify_one();
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
    out->status = r.cancelled ? BF_ERR_CANCELLED : r.status;
    out->latency_ms = ms_since(r.t_submit, r.t_done);
    out->queue_ms = r.cancelled ? 0.0 : ms_since(r.t_submit, r.t_admit);
    out->device_ms = r.device_ms;
    S->reqs.erase(it);
    return r.cancelled ? BF_ERR_CANCELLED : BF_OK;
}

bf_status bf_serve_cancel(bf_server *S, uint64_t ticket) {
    if (!S) return bfi::fail(BF_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if (*it == ticket) {
            S->queue.erase(it);
            Request &r = S->reqs[ticket];
            r.cancelled = true;
            r.done = true;
            r.status = BF_ERR_CANCELLED;
            r.t_done = Clock::now();
            S->cv_done.notify_all();
            return BF_OK;
        }
    return bfi::fail(BF_ERR_NOT_FOUND, "request not pending");
}

void bf_serve_destroy(bf_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (uint64_t t : S->queue) {  // never admitted: cancelled
            Request &r = S->reqs[t];
            r.cancelled = true;
            r.done = true;
            r.status = BF_ERR_CANCELLED;
        }
        S->queue.clear();
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (auto &kv : S->plans) bf_plan_destroy(kv.second);
    delete S;
}

}  // extern "C"
