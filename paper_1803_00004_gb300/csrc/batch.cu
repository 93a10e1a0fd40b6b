// bf_filter_batch: many images (each with its own plan) in one persistent
// launch per kernel class.
//
// The host builds a work list of (image, tile, term group) items, largest
// first, with one launch geometry per kernel class: a fixed number of column
// threads, and per image the widest tile that fits them next to its halo.
// Per-image parameters, image descriptors, the work list and one cursor per
// class live in one device buffer uploaded by a single copy.  Images whose
// terms are split into groups get partial planes in the same buffer and are
// finalized by one batched launch.  The sequence (upload, cursor reset,
// persistent launches, finalize) is captured into a CUDA graph the first time
// a batch signature (plans, image pointers and sizes) is seen and replayed
// afterwards; replays of one graph are ordered on the device by an event.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bf_internal.h"

namespace bfi {
namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct ClassLaunch {
    int m, nk, ncols, n_items, grid;
    bool packed;
    size_t item_off;   // byte offset of the class's first item in the buffer
    size_t cursor_off;
};

// Geometry of one batch class: column threads = the widest halo plus `extra` (whole warps, at most 448),
// tile height at least th_min (and the window span), at most nk_cap terms per CTA (0: as many as fit).
// bf_autotune_batch fills the table; classes without an entry take the defaults.
struct BatchTune {
    int extra = 128, th_min = 48, nk_cap = 0;
};
using ClassId = std::pair<int, int>;                    // (windows per axis, packed family)
using TuneKey = std::tuple<int, int, int, int>;         // device, windows per axis, packed family, widest reach
using TuneOverride = std::map<ClassId, BatchTune>;
std::mutex g_tmu;
std::map<TuneKey, BatchTune> g_tune;

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        d = -1;
    }
    return d;
}

// Branch streams of a device for the batch's direct launches (the 3-D form, 16-bit basis storage): they are
// independent (each image has its own scratch), so they run side by side on up to kDirectStreams streams forked
// from and joined back to the batch's stream (inside a captured graph: parallel branches).  Created once per
// device, before any capture; the mutex orders the fork and join of concurrent callers.
constexpr int kDirectStreams = 8;
constexpr int kMaxDirectDevices = 64;
struct DirectStreams {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s[kDirectStreams] = {};
    cudaEvent_t fork = nullptr, join[kDirectStreams] = {};
};
DirectStreams g_direct[kMaxDirectDevices];

DirectStreams *direct_streams(int device) {
    if (device < 0 || device >= kMaxDirectDevices) return nullptr;
    DirectStreams &d = g_direct[device];
    std::lock_guard<std::mutex> lk(d.mu);
    if (d.ready) return &d;
    cudaError_t e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming);
    for (int k = 0; k < kDirectStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&d.s[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    d.ready = true;
    return &d;
}

}  // namespace

// Host-side layout of one batch; fill() writes the staging bytes for a device base address.
struct BatchLayout {
    int n = 0;
    std::vector<FilterParams> params;
    std::vector<BatchImage> imgs;
    std::vector<WorkItem> items;      // grouped by class, each class's items contiguous
    std::vector<int> list;            // images that need the finalize pass
    std::vector<ClassLaunch> launches;
    size_t off_params = 0, off_imgs = 0, off_items = 0, off_list = 0, off_cursors = 0, off_scratch = 0, total = 0;
    std::vector<size_t> scratch_off;  // per image, relative to off_scratch (or SIZE_MAX)
    int max_h = 0, max_w = 0;
    // Images of plans the persistent kernel does not run (the 3-D form; 16-bit basis storage): launched after the
    // persistent launches, side by side on the branch streams, in their own geometry, with their scratch in the
    // buffer's scratch area.
    struct Direct {
        FilterParams kp;
        int precision, kahan;
        TileConfig tc;
        bf_image im;
        size_t scratch_off;  // relative to off_scratch
        size_t scratch_bytes;
    };
    std::vector<Direct> direct;

    void fill(uint8_t *staging, uintptr_t d_base) {
        std::vector<BatchImage> im = imgs;
        for (int i = 0; i < n; ++i)
            im[i].part = scratch_off[i] == SIZE_MAX ? nullptr
                                                    : reinterpret_cast<float *>(d_base + off_scratch + scratch_off[i]);
        std::memcpy(staging + off_params, params.data(), params.size() * sizeof(FilterParams));
        std::memcpy(staging + off_imgs, im.data(), im.size() * sizeof(BatchImage));
        std::memcpy(staging + off_items, items.data(), items.size() * sizeof(WorkItem));
        if (!list.empty()) std::memcpy(staging + off_list, list.data(), list.size() * sizeof(int));
        std::memset(staging + off_cursors, 0, launches.size() * sizeof(int));
    }
    size_t upload_bytes() const { return off_scratch; }
};

using LayoutDirect = BatchLayout::Direct;

bf_status build_batch(const bf_plan *const *plans, const bf_image *images, int n, BatchLayout &L,
                      const TuneOverride *ov = nullptr) {
    L = BatchLayout();
    L.n = n;
    const int sms = device_sm_count();
    // one persistent launch per (windows per axis, kernel family): plans whose selected terms are
    // consecutive use the packed-pair family, the others the scalar family (no padded term groups)
    std::map<std::pair<int, int>, std::vector<int>> by_class;
    size_t scratch = 0;
    for (int i = 0; i < n; ++i) {
        const FilterParams &kp = plans[i]->kp;
        if (kp.zbins > 0 || plans[i]->desc.precision != BF_PREC_FP32) {
            LayoutDirect d;
            d.kp = kp;
            d.precision = plans[i]->desc.precision;
            d.kahan = plans[i]->desc.kahan;
            d.tc = choose_tile(kp, images[i].height, images[i].width, d.precision);
            if (d.tc.ncols == 0) return fail(BF_ERR_UNSUPPORTED, "no launch geometry for a batched 3-D or 16-bit plan");
            d.im = images[i];
            d.scratch_bytes = scratch_bytes(d.tc, images[i].height, images[i].width, kp.zbins);
            d.scratch_off = scratch;
            scratch = align_up(scratch + d.scratch_bytes, 256);
            L.direct.push_back(d);
            continue;
        }
        by_class[{plans[i]->m, kp.k[kp.nr - 1] - kp.k[0] + 1 == kp.nr ? 1 : 0}].push_back(i);
    }
    L.params.resize(n);
    L.imgs.resize(n);
    L.scratch_off.assign(n, SIZE_MAX);
    std::vector<std::vector<WorkItem>> class_items;
    for (auto &kv : by_class) {
        const int m = kv.first.first;
        const bool packed = kv.first.second != 0;
        int rx_max = 0;
        for (int i : kv.second) rx_max = std::max(rx_max, plans[i]->kp.rx);
        BatchTune tn;
        if (ov && ov->count(kv.first)) {
            tn = ov->at(kv.first);
        } else {
            std::lock_guard<std::mutex> lk(g_tmu);
            const auto it = g_tune.find(TuneKey{current_device(), m, packed ? 1 : 0, rx_max});
            if (it != g_tune.end()) tn = it->second;
        }
        // column threads: room for a tile of `extra` columns next to the widest halo
        int ncols = std::min(448, ((2 * rx_max + tn.extra + 31) / 32) * 32);
        int nk = batch_class_nk(m, ncols, packed, tn.nk_cap);
        while (nk == 0 && ncols > 2 * rx_max + 32) {
            ncols -= 32;
            nk = batch_class_nk(m, ncols, packed, tn.nk_cap);
        }
        if (nk == 0 || ncols < 2 * rx_max + 8) return fail(BF_ERR_UNSUPPORTED, "batched tile cannot hold this reach");
        std::vector<std::pair<double, WorkItem>> its;
        for (int i : kv.second) {
            const bf_plan *p = plans[i];
            const bf_image &im = images[i];
            const FilterParams &kp = p->kp;
            const int groups = packed ? term_groups(kp, nk) : (kp.nr + nk - 1) / nk;
            int tw = ((ncols - 2 * kp.rx) / 8) * 8;
            tw = std::min(tw, ((im.width + 7) / 8) * 8);
            const int vspan = kp.vhi - kp.vlo + 1;
            const int th = std::min(im.height, std::max(tn.th_min, vspan));
            if (!packed) L.params[i] = kp;
            else if (!term_layout(kp, nk, L.params[i]))
                return fail(BF_ERR_UNSUPPORTED, "the plan's terms need more than 128 slots at this class");
            BatchImage &b = L.imgs[i];
            b.in = im.d_in;
            b.out = im.d_out;
            b.part = nullptr;
            b.in_pitch = im.in_pitch_bytes / sizeof(float);
            b.out_pitch = im.out_pitch_bytes / sizeof(float);
            b.H = im.height;
            b.W = im.width;
            b.params = i;
            b.groups = groups;
            if (groups > 1) {
                L.scratch_off[i] = scratch;
                scratch = align_up(scratch + sizeof(float) * 2 * (size_t)groups * im.height * im.width, 256);
                L.list.push_back(i);
            }
            L.max_h = std::max(L.max_h, im.height);
            L.max_w = std::max(L.max_w, im.width);
            const double cost = (double)ncols * (th + 0.3 * vspan);
            for (int g = 0; g < groups; ++g)
                for (int y0 = 0; y0 < im.height; y0 += th)
                    for (int x0 = 0; x0 < im.width; x0 += tw)
                        its.push_back({cost * std::min(th, im.height - y0), WorkItem{i, x0, y0, tw, th, g}});
        }
        std::stable_sort(its.begin(), its.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
        std::vector<WorkItem> items;
        for (auto &e : its) items.push_back(e.second);
        ClassLaunch cl;
        cl.m = m;
        cl.nk = nk;
        cl.packed = packed;
        cl.ncols = ncols;
        cl.n_items = (int)items.size();
        cl.grid = std::max(1, std::min(cl.n_items, sms * batch_ctas_per_sm(m, nk, ncols)));
        cl.item_off = L.items.size();  // index for now; converted to bytes below
        cl.cursor_off = L.launches.size();
        L.items.insert(L.items.end(), items.begin(), items.end());
        L.launches.push_back(cl);
    }
    L.off_params = 0;
    L.off_imgs = align_up(L.off_params + L.params.size() * sizeof(FilterParams), 256);
    L.off_items = align_up(L.off_imgs + L.imgs.size() * sizeof(BatchImage), 256);
    L.off_list = align_up(L.off_items + L.items.size() * sizeof(WorkItem), 256);
    L.off_cursors = align_up(L.off_list + L.list.size() * sizeof(int), 256);
    L.off_scratch = align_up(L.off_cursors + L.launches.size() * sizeof(int), 256);
    L.total = L.off_scratch + scratch;
    for (auto &cl : L.launches) {
        cl.item_off = L.off_items + cl.item_off * sizeof(WorkItem);
        cl.cursor_off = L.off_cursors + cl.cursor_off * sizeof(int);
    }
    return BF_OK;
}

// Enqueues upload + launches of a built batch whose device buffer is d_buf and
// whose staging bytes (already filled for d_buf) are at h_staging.
bf_status enqueue_batch(const BatchLayout &L, uint8_t *d_buf, const uint8_t *h_staging, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(d_buf, h_staging, L.upload_bytes(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(BF_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    const auto *d_params = reinterpret_cast<const FilterParams *>(d_buf + L.off_params);
    const auto *d_imgs = reinterpret_cast<const BatchImage *>(d_buf + L.off_imgs);
    for (const auto &cl : L.launches) {
        bf_status st = launch_batch_class(cl.m, cl.nk, cl.packed, cl.ncols, d_imgs, d_params,
                                          reinterpret_cast<const WorkItem *>(d_buf + cl.item_off), cl.n_items,
                                          reinterpret_cast<int *>(d_buf + cl.cursor_off), cl.grid, s);
        if (st != BF_OK) return st;
    }
    bf_status st = launch_batch_finalize(d_imgs, reinterpret_cast<const int *>(d_buf + L.off_list), (int)L.list.size(),
                                         L.max_h, L.max_w, d_params, s);
    if (st != BF_OK || L.direct.empty()) return st;
    // the direct launches, side by side on the device's branch streams (one after another if they cannot be had)
    DirectStreams *ds = direct_streams(current_device());
    std::unique_lock<std::mutex> lk;
    int K = 0;
    if (ds) {
        lk = std::unique_lock<std::mutex>(ds->mu);
        K = (int)std::min<size_t>(kDirectStreams, L.direct.size());
        e = cudaEventRecord(ds->fork, s);
        for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ds->s[k], ds->fork, 0);
        if (e != cudaSuccess) return fail(BF_ERR_CUDA, std::string("batch fork: ") + cudaGetErrorString(e));
    }
    for (size_t i = 0; i < L.direct.size() && st == BF_OK; ++i) {
        const auto &d = L.direct[i];
        float *scr = d.scratch_bytes ? reinterpret_cast<float *>(d_buf + L.off_scratch + d.scratch_off) : nullptr;
        st = launch_filter(d.kp, d.precision, d.kahan, d.tc, d.im.d_in, d.im.in_pitch_bytes / sizeof(float), d.im.d_out,
                           d.im.out_pitch_bytes / sizeof(float), scr, d.im.height, d.im.width,
                           K ? ds->s[i % K] : s);
    }
    // join (also after a failure, so that the branch streams end inside the stream's order or the capture)
    for (int k = 0; k < K; ++k) {
        e = cudaEventRecord(ds->join[k], ds->s[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ds->join[k], 0);
        if (e != cudaSuccess && st == BF_OK) st = fail(BF_ERR_CUDA, std::string("batch join: ") + cudaGetErrorString(e));
    }
    return st;
}

bf_status enqueue_batch_with(const bf_plan *const *plans, const bf_image *images, int n, void *stream,
                             const TuneOverride *ov) {
    BatchLayout L;
    bf_status st = build_batch(plans, images, n, L, ov);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *d_buf = nullptr;
    if (cudaMallocAsync((void **)&d_buf, L.total, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_OOM, "batch buffer");
    }
    // pageable staging: the runtime has copied it out when cudaMemcpyAsync returns
    std::vector<uint8_t> staging(std::max<size_t>(L.upload_bytes(), 1));
    L.fill(staging.data(), reinterpret_cast<uintptr_t>(d_buf));
    st = enqueue_batch(L, d_buf, staging.data(), s);
    cudaFreeAsync(d_buf, s);
    return st;
}

bf_status enqueue_batch_into(const bf_plan *const *plans, const bf_image *images, int n, void *stream, void *d_buf,
                             size_t cap) {
    BatchLayout L;
    bf_status st = build_batch(plans, images, n, L);
    if (st != BF_OK) return st;
    if (L.total > cap) return fail(BF_ERR_OOM, "batch needs more than its reserved buffer");
    std::vector<uint8_t> staging(std::max<size_t>(L.upload_bytes(), 1));
    L.fill(staging.data(), reinterpret_cast<uintptr_t>(d_buf));
    return enqueue_batch(L, static_cast<uint8_t *>(d_buf), staging.data(), (cudaStream_t)stream);
}

bf_status enqueue_batch_direct(const bf_plan *const *plans, const bf_image *images, int n, void *stream) {
    return enqueue_batch_with(plans, images, n, stream, nullptr);
}

size_t batch_device_bytes(const bf_plan *const *plans, const bf_image *images, int n) {
    BatchLayout L;
    if (build_batch(plans, images, n, L) != BF_OK) return 0;
    return L.total;
}

namespace {

struct GraphEntry {
    std::vector<uint8_t> key;
    int device = 0;
    uint8_t *d_buf = nullptr;
    uint8_t *h_staging = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    ~GraphEntry() {
        if (done) cudaEventSynchronize(done);
        if (exec) cudaGraphExecDestroy(exec);
        if (done) cudaEventDestroy(done);
        if (d_buf) cudaFree(d_buf);
        if (h_staging) cudaFreeHost(h_staging);
    }
};

std::mutex g_gmu;
std::list<std::unique_ptr<GraphEntry>> g_graphs;  // most recently used first
constexpr size_t kMaxGraphs = 8;

std::vector<uint8_t> signature(const bf_plan *const *plans, const bf_image *images, int n, int device) {
    std::vector<uint8_t> k;
    auto put = [&](const void *p, size_t b) {
        const uint8_t *c = static_cast<const uint8_t *>(p);
        k.insert(k.end(), c, c + b);
    };
    put(&device, sizeof(device));
    put(&n, sizeof(n));
    for (int i = 0; i < n; ++i) {
        put(&plans[i]->kp, sizeof(FilterParams));
        put(&plans[i]->desc.precision, sizeof(int));
        put(&images[i], sizeof(bf_image));
    }
    return k;
}

bf_status make_entry(const bf_plan *const *plans, const bf_image *images, int n, int device,
                     std::vector<uint8_t> key, GraphEntry *&out) {
    BatchLayout L;
    bf_status st = build_batch(plans, images, n, L);
    if (st != BF_OK) return st;
    auto ent = std::make_unique<GraphEntry>();
    ent->key = std::move(key);
    ent->device = device;
    if (cudaMalloc((void **)&ent->d_buf, L.total) != cudaSuccess ||
        cudaHostAlloc((void **)&ent->h_staging, std::max<size_t>(L.upload_bytes(), 1), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_OOM, "batch buffers");
    }
    L.fill(ent->h_staging, reinterpret_cast<uintptr_t>(ent->d_buf));
    if (!L.direct.empty()) direct_streams(device);  // the branch streams exist before the capture begins
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_CUDA, "capture stream");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_batch(L, ent->d_buf, ent->h_staging, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (st == BF_OK && e != cudaSuccess) st = fail(BF_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    } else {
        st = fail(BF_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    cudaStreamDestroy(cap);
    if (st == BF_OK) {
        e = cudaGraphInstantiate(&ent->exec, graph, 0);
        if (e != cudaSuccess) st = fail(BF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    if (graph) cudaGraphDestroy(graph);
    if (st == BF_OK && cudaEventCreateWithFlags(&ent->done, cudaEventDisableTiming) != cudaSuccess)
        st = fail(BF_ERR_CUDA, "graph event");
    if (st != BF_OK) {
        cudaGetLastError();
        return st;
    }
    g_graphs.push_front(std::move(ent));
    while (g_graphs.size() > kMaxGraphs) g_graphs.pop_back();
    out = g_graphs.front().get();
    return BF_OK;
}

}  // namespace

bf_status check_image(const float *d_in, size_t in_pitch, const float *d_out, size_t out_pitch, int h, int w);

}  // namespace bfi

using namespace bfi;

namespace {

// Argument checks shared by bf_filter_batch and bf_autotune_batch; the non-empty images and their plans go to
// ps / ims, and their device to *device.
bf_status collect_batch(const bf_plan *const *plans, const bf_image *images, int n, std::vector<const bf_plan *> &ps,
                        std::vector<bf_image> &ims, int *device) {
    if (n < 0) return fail(BF_ERR_INVALID_ARG, "negative batch size");
    if (n == 0) return BF_OK;
    if (!plans || !images) return fail(BF_ERR_INVALID_ARG, "NULL batch arrays");
    *device = -2;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(BF_ERR_INVALID_ARG, "NULL plan in batch");
        if (plans[i]->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan in batch");
        if (*device == -2) *device = plans[i]->desc.device;
        if (plans[i]->desc.device != *device) return fail(BF_ERR_INVALID_ARG, "plans of one batch must share a device");
        const bf_image &im = images[i];
        bf_status st = check_image(im.d_in, im.in_pitch_bytes, im.d_out, im.out_pitch_bytes, im.height, im.width);
        if (st != BF_OK) return st;
        if (im.height == 0 || im.width == 0) continue;  // nothing to do for empty images
        ps.push_back(plans[i]);
        ims.push_back(im);
    }
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_autotune_batch(const bf_plan *const *plans, const bf_image *images, int n, void *stream) {
    std::vector<const bf_plan *> ps;
    std::vector<bf_image> ims;
    int device = -2;
    bf_status st = collect_batch(plans, images, n, ps, ims, &device);
    if (st != BF_OK || ps.empty()) return st;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || (prev != device && cudaSetDevice(device) != cudaSuccess)) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plans' device");
    }
    const int nb = (int)ps.size();
    // the classes of this batch, their widest reach, and their current geometry (table entry or defaults)
    std::map<ClassId, int> reach;
    for (const bf_plan *p : ps) {
        const ClassId c{p->m, p->kp.k[p->kp.nr - 1] - p->kp.k[0] + 1 == p->kp.nr ? 1 : 0};
        reach[c] = std::max(reach.count(c) ? reach[c] : 0, p->kp.rx);
    }
    TuneOverride cur;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        for (const auto &kv : reach) {
            const auto it = g_tune.find(TuneKey{device, kv.first.first, kv.first.second, kv.second});
            cur[kv.first] = it != g_tune.end() ? it->second : BatchTune();
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = fail(BF_ERR_CUDA, "batch-autotune events");
    }
    // device time of the whole batch (upload, persistent launches, finalize): the faster of two runs after a warm-up
    auto time_batch = [&]() -> float {
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, s);
            if (enqueue_batch_with(ps.data(), ims.data(), nb, s, &cur) != BF_OK) return 1e30f;
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                return 1e30f;
            }
            if (r > 0) best = std::min(best, ms);
        }
        return best;
    };
    if (st == BF_OK) {
        // coordinate descent, one class and one parameter at a time, two sweeps; a change must win by 1 %
        const int extras[] = {64, 128, 192, 256, 384};
        const int heights[] = {24, 48, 96, 192};
        const int caps[] = {0, 4, 2};
        float best = time_batch();
        for (int sweep = 0; sweep < 2; ++sweep)
            for (auto &kv : cur)
                for (int dim = 0; dim < 3; ++dim) {
                    const BatchTune keep = kv.second;
                    BatchTune win = keep;
                    const int nv = dim == 0 ? 5 : dim == 1 ? 4 : 3;
                    for (int v = 0; v < nv; ++v) {
                        BatchTune t = keep;
                        if (dim == 0) t.extra = extras[v];
                        else if (dim == 1) t.th_min = heights[v];
                        else t.nk_cap = caps[v];
                        if (t.extra == keep.extra && t.th_min == keep.th_min && t.nk_cap == keep.nk_cap) continue;
                        kv.second = t;
                        const float ms = time_batch();
                        if (ms < best * 0.99f) {
                            best = ms;
                            win = t;
                        }
                    }
                    kv.second = win;
                }
        if (best >= 1e30f) st = fail(BF_ERR_CUDA, "no batch geometry ran");
    }
    if (st == BF_OK) {
        {
            std::lock_guard<std::mutex> lk(g_tmu);
            for (const auto &kv : cur) g_tune[TuneKey{device, kv.first.first, kv.first.second, reach[kv.first]}] = kv.second;
        }
        // captured batches of this device were built with the old geometry
        std::lock_guard<std::mutex> lk(g_gmu);
        g_graphs.remove_if([&](const std::unique_ptr<GraphEntry> &g) { return g->device == device; });
    }
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (prev != device) cudaSetDevice(prev);
    return st;
}

extern "C" bf_status bf_filter_batch(const bf_plan *const *plans, const bf_image *images, int n, void *stream) {
    std::vector<const bf_plan *> ps;
    std::vector<bf_image> ims;
    int device = -2;
    bf_status st0 = collect_batch(plans, images, n, ps, ims, &device);
    if (st0 != BF_OK) return st0;
    if (ps.empty()) return BF_OK;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || (prev != device && cudaSetDevice(device) != cudaSuccess)) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plans' device");
    }
    bf_status st = BF_OK;
    {
        std::lock_guard<std::mutex> lk(g_gmu);
        std::vector<uint8_t> key = signature(ps.data(), ims.data(), (int)ps.size(), device);
        GraphEntry *ent = nullptr;
        for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
            if ((*it)->key == key) {
                g_graphs.splice(g_graphs.begin(), g_graphs, it);
                ent = g_graphs.front().get();
                break;
            }
        if (!ent) st = make_entry(ps.data(), ims.data(), (int)ps.size(), device, std::move(key), ent);
        if (st == BF_OK && debug_consume_launch_failure()) st = fail(BF_ERR_CUDA, "injected launch failure (test hook)");
        if (st == BF_OK) {
            cudaStream_t s = (cudaStream_t)stream;
            cudaError_t e = cudaStreamWaitEvent(s, ent->done, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ent->exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(ent->done, s);
            if (e != cudaSuccess) st = fail(BF_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        }
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
