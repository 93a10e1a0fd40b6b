// Autotuner for the fused filter's launch geometry (tile width and height,
// cosine terms per CTA).  Candidates come ranked from the cost model; each is
// timed with CUDA events on a synthetic image of the requested size, and the
// fastest is remembered per (device, kernel class, reach, image size) for
// later bf_filter / bf_filter_batch calls.  BF_TUNE_CACHE=<file> persists the
// table across processes (one line per entry).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bf_internal.h"

namespace bfi {
namespace {

// (device, M, terms, reach, vlo, vhi, h, w, precision, selection kind): the kind is 1 for a gapped term
// selection (the families on offer differ) plus 2 for the 3-D form (no ring) plus 4 for its Haar range
// series (NK = 2 only)
using Key = std::tuple<int, int, int, int, int, int, int, int, int, int>;

std::mutex g_mu;
std::map<Key, TileConfig> g_table;
bool g_loaded = false;

Key make_key(const FilterParams &p, int h, int w, int precision) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const int kind = (p.k[p.nr - 1] - p.k[0] + 1 != p.nr ? 1 : 0) + (p.zbins > 0 ? 2 : 0) + (p.zmode == 2 ? 4 : 0);
    return Key{dev, p.m, p.nr, p.rx, p.vlo, p.vhi, h, w, precision, kind};
}

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("BF_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int k[10];
    TileConfig tc;
    unsigned long smem;
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lu %d", &k[0], &k[1], &k[2], &k[3],
                       &k[4], &k[5], &k[6], &k[7], &k[8], &k[9], &tc.tw, &tc.th, &tc.ncols, &tc.threads, &tc.nk,
                       &tc.groups, &tc.ring, &tc.depth, &tc.packed, &smem, &tc.pre) == 21) {
        tc.smem = smem;
        g_table[Key{k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], k[8], k[9]}] = tc;
    }
    std::fclose(f);
}

void save_locked(const Key &key, const TileConfig &tc) {
    const char *path = std::getenv("BF_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lu %d\n", std::get<0>(key),
                 std::get<1>(key), std::get<2>(key), std::get<3>(key), std::get<4>(key), std::get<5>(key),
                 std::get<6>(key), std::get<7>(key), std::get<8>(key), std::get<9>(key), tc.tw, tc.th, tc.ncols,
                 tc.threads, tc.nk, tc.groups, tc.ring, tc.depth, tc.packed, (unsigned long)tc.smem, tc.pre);
    std::fclose(f);
}

// Deterministic pseudo-random pixels in [lo, hi] (a hash of the index).  smooth = 0: uniform over the
// range.  smooth = 1 (the 3-D form, whose cost grows with the distinct intensity slices per tile): a
// slowly varying field plus 3% noise, closer to natural images than white noise.
__global__ void fill_kernel(float *img, size_t n, int width, float lo, float hi, int smooth) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u + 0x9e3779b9u;
        x ^= x >> 16;
        x *= 0x85ebca6bu;
        x ^= x >> 13;
        float u = (float)(x >> 8) * (1.0f / 16777216.0f);
        if (smooth) {
            const float c = (float)(i % (size_t)width), r = (float)(i / (size_t)width);
            u = 0.5f + 0.4f * __sinf(c * 0.011f) * __sinf(r * 0.017f) + 0.06f * (u - 0.5f);
        }
        img[i] = lo + (hi - lo) * u;
    }
}

// The geometries the tuners time: the cost model's best four of every family (ring, exchange depth, kernel
// family, terms per CTA) within every residency class (1, 2, or 3 and more CTAs per SM by shared memory).
// The model ranks well within a residency class; across classes it misjudges how much latency the extra
// resident CTAs hide.
std::vector<TileConfig> timed_candidates(const FilterParams &p, int height, int width, int precision) {
    int smem_sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        smem_sm <= 0) {
        cudaGetLastError();
        smem_sm = 228 * 1024;
    }
    std::vector<TileConfig> ranked = tile_candidates(p, height, width, precision, 100000), out;
    std::map<std::tuple<int, int, int>, int> per_class;
    for (const auto &c : ranked) {
        const int res = (int)std::min<size_t>(3, (size_t)smem_sm / (c.smem + 1024));  // 1 KiB reserved per CTA
        if (per_class[std::make_tuple(c.ring * 4 + c.depth + 8 * c.packed + 32 * c.pre, c.nk, res)]++ < 4) out.push_back(c);
    }
    return out;
}

}  // namespace

TileConfig choose_tile(const FilterParams &p, int height, int width, int precision) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_locked();
        auto it = g_table.find(make_key(p, height, width, precision));
        // an entry stays usable only while its term grouping matches the library's current layout
        if (it != g_table.end() &&
            it->second.packed >= 0 && it->second.packed <= 2 &&
            it->second.groups == family_groups(p, it->second.nk, it->second.packed) &&
            (p.zbins == 0 || (it->second.packed == 1 && !it->second.ring)) && pre_allowed(precision, it->second.pre) &&
            (it->second.pre == 0 || (it->second.packed == 1 && !it->second.ring && p.zbins == 0)))
            return it->second;
    }
    return model_tile(p, height, width, precision);
}

void remember_tile(const FilterParams &p, int height, int width, int precision, const TileConfig &tc) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    Key k = make_key(p, height, width, precision);
    g_table[k] = tc;
    save_locked(k, tc);
}

}  // namespace bfi

using namespace bfi;

namespace {

// Times the candidates on `sample` (pitch in floats; nullptr: a synthetic image in the plan's data range)
// and pins the fastest.
bf_status autotune_plan(const bf_plan *plan, const float *sample, size_t sample_pitch, int height, int width,
                        void *stream, int *info) {
    if (!plan || height < 1 || width < 1) return fail(BF_ERR_INVALID_ARG, "bad autotune arguments");
    if (plan->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(plan->desc.device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plan's device");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const std::vector<TileConfig> cands = timed_candidates(plan->kp, height, width, plan->desc.precision);
    bf_status st = BF_OK;
    float *in = nullptr, *out = nullptr, *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    size_t n = (size_t)height * width, need = 0;
    for (const auto &c : cands) need = std::max(need, scratch_bytes(c, height, width, plan->kp.zbins));
    if (cands.empty()) st = fail(BF_ERR_UNSUPPORTED, "no launch geometry for this plan");
    if (st == BF_OK && ((!sample && cudaMalloc((void **)&in, n * sizeof(float)) != cudaSuccess) ||
                        cudaMalloc((void **)&out, n * sizeof(float)) != cudaSuccess ||
                        (need && cudaMalloc((void **)&scratch, need) != cudaSuccess))) {
        cudaGetLastError();
        st = fail(BF_ERR_OOM, "autotune buffers");
    }
    if (st == BF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(BF_ERR_CUDA, "autotune events");
    }
    TileConfig best{};
    float best_ms = 1e30f;
    if (st == BF_OK) {
        const float *src = sample ? sample : in;
        const size_t src_pitch = sample ? sample_pitch : (size_t)width;
        if (!sample)
            fill_kernel<<<256, 256, 0, s>>>(in, n, width, plan->desc.i_lo, plan->desc.i_hi, plan->kp.zbins > 0 ? 1 : 0);
        for (const auto &c : cands) {
            bf_status r = launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, c, src, src_pitch, out, width,
                                        scratch, height, width, stream);  // warm-up
            if (r != BF_OK) continue;
            float t[3];
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                cudaEventRecord(e0, s);
                ok = launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, c, src, src_pitch, out, width,
                                   scratch, height, width, stream) == BF_OK;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
                else cudaEventElapsedTime(&t[rep], e0, e1);
            }
            if (!ok) continue;
            std::sort(t, t + 3);
            if (t[1] < best_ms) {
                best_ms = t[1];
                best = c;
            }
        }
        if (best.ncols == 0) st = fail(BF_ERR_CUDA, "no candidate geometry ran");
    }
    if (st == BF_OK) {
        remember_tile(plan->kp, height, width, plan->desc.precision, best);
        if (info) {
            fill_info(best, height, width, info, plan->kp.zbins);
        }
    }
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    cudaFree(scratch);
    cudaSetDevice(prev);
    return st;
}

}  // namespace

extern "C" bf_status bf_autotune(const bf_plan *plan, int height, int width, void *stream, int *info) {
    return autotune_plan(plan, nullptr, 0, height, width, stream, info);
}

extern "C" bf_status bf_autotune_image(const bf_plan *plan, const float *d_in, size_t in_pitch, int height, int width,
                                       void *stream, int *info) {
    if (!d_in || height < 1 || width < 1 || in_pitch % sizeof(float) || in_pitch < (size_t)width * sizeof(float))
        return fail(BF_ERR_INVALID_ARG, "bad sample image (NULL, empty, or pitch not a multiple of 4 bytes >= width * 4)");
    return autotune_plan(plan, d_in, in_pitch / sizeof(float), height, width, stream, info);
}

extern "C" bf_status bf_autotune_group(const bf_plan *const *plans, int n, int height, int width, int n_streams,
                                       int *infos) {
    if (!plans || n < 1 || n > 256 || height < 1 || width < 1 || n_streams < 1 || n_streams > 16)
        return fail(BF_ERR_INVALID_ARG, "bad group-autotune arguments");
    for (int i = 0; i < n; ++i)
        if (!plans[i]) return fail(BF_ERR_INVALID_ARG, "null plan in the group");
    for (int i = 0; i < n; ++i) {
        if (plans[i]->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
        if (plans[i]->desc.device != plans[0]->desc.device)
            return fail(BF_ERR_INVALID_ARG, "the group's plans are on different devices");
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(plans[0]->desc.device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plans' device");
    }
    // plans with one table key (kernel class, reach, image size, precision) share one geometry
    std::vector<Key> keys;
    std::vector<int> cls(n), rep;
    for (int i = 0; i < n; ++i) {
        const Key k = make_key(plans[i]->kp, height, width, plans[i]->desc.precision);
        const auto it = std::find(keys.begin(), keys.end(), k);
        cls[i] = (int)(it - keys.begin());
        if (it == keys.end()) {
            keys.push_back(k);
            rep.push_back(i);
        }
    }
    const int nc = (int)keys.size();
    std::vector<std::vector<TileConfig>> cands(nc);
    std::vector<TileConfig> cur(nc);
    bf_status st = BF_OK;
    bool smooth = false;
    for (int c = 0; c < nc && st == BF_OK; ++c) {
        const bf_plan *pl = plans[rep[c]];
        cands[c] = timed_candidates(pl->kp, height, width, pl->desc.precision);
        cur[c] = choose_tile(pl->kp, height, width, pl->desc.precision);  // the pinned or modelled start
        if (cands[c].empty()) st = fail(BF_ERR_UNSUPPORTED, "no launch geometry for a plan of the group");
        smooth = smooth || pl->kp.zbins > 0;
    }
    // one input, one output per plan, and per plan the largest scratch any of its class's geometries needs
    const size_t npx = (size_t)height * width;
    std::vector<size_t> soff(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        size_t need = scratch_bytes(cur[cls[i]], height, width, plans[i]->kp.zbins);
        for (const auto &c : cands[cls[i]]) need = std::max(need, scratch_bytes(c, height, width, plans[i]->kp.zbins));
        soff[i + 1] = soff[i] + (need + 255) / 256 * 256;
    }
    float *in = nullptr, *out = nullptr;
    char *scratch = nullptr;
    std::vector<cudaStream_t> ss(n_streams, nullptr);
    std::vector<cudaEvent_t> join(n_streams, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == BF_OK && (cudaMalloc((void **)&in, npx * sizeof(float)) != cudaSuccess ||
                        cudaMalloc((void **)&out, (size_t)n * npx * sizeof(float)) != cudaSuccess ||
                        (soff[n] && cudaMalloc((void **)&scratch, soff[n]) != cudaSuccess))) {
        cudaGetLastError();
        st = fail(BF_ERR_OOM, "group-autotune buffers");
    }
    for (int j = 0; j < n_streams && st == BF_OK; ++j)
        if (cudaStreamCreateWithFlags(&ss[j], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[j], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st = fail(BF_ERR_CUDA, "group-autotune streams");
        }
    if (st == BF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(BF_ERR_CUDA, "group-autotune events");
    }
    // the group as a caller runs it: plan i on stream i mod n_streams, in the given order, forked from and
    // joined to the first stream; the time is the first stream's, from the fork to the join
    auto run_group = [&](float *ms) -> bool {
        bool ok = cudaEventRecord(e0, ss[0]) == cudaSuccess;
        for (int j = 1; j < n_streams; ++j) ok = ok && cudaStreamWaitEvent(ss[j], e0, 0) == cudaSuccess;
        for (int i = 0; i < n && ok; ++i)
            ok = launch_filter(plans[i]->kp, plans[i]->desc.precision, plans[i]->desc.kahan, cur[cls[i]], in, width,
                               out + (size_t)i * npx, width, reinterpret_cast<float *>(scratch ? scratch + soff[i] : nullptr),
                               height, width, ss[i % n_streams]) == BF_OK;
        for (int j = 1; j < n_streams; ++j) {
            cudaEventRecord(join[j], ss[j]);
            cudaStreamWaitEvent(ss[0], join[j], 0);
        }
        cudaEventRecord(e1, ss[0]);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (ms) cudaEventElapsedTime(ms, e0, e1);
        return ok;
    };
    auto time_group = [&]() -> float {
        float t[5];
        if (!run_group(nullptr)) return 1e30f;  // warm-up
        for (int r = 0; r < 5; ++r)
            if (!run_group(&t[r])) return 1e30f;
        std::sort(t, t + 5);
        return t[2];
    };
    if (st == BF_OK) {
        fill_kernel<<<256, 256, 0, ss[0]>>>(in, npx, width, plans[0]->desc.i_lo, plans[0]->desc.i_hi, smooth ? 1 : 0);
        // coordinate descent: one class at a time over its candidates, the others held; two sweeps.  A change
        // must win by 0.5 %, so timing noise does not move a class off a geometry that is as good.
        float best = time_group();
        for (int sweep = 0; sweep < 2; ++sweep)
            for (int c = 0; c < nc; ++c) {
                TileConfig keep = cur[c];
                for (const auto &cand : cands[c]) {
                    cur[c] = cand;
                    const float t = time_group();
                    if (t < best * 0.995f) {
                        best = t;
                        keep = cand;
                    }
                }
                cur[c] = keep;
            }
        // tile-height refinement: the cost model ranks geometries by a launch's own cost, so its best
        // candidates rarely include a taller tile; in a concurrent group one can win (fewer CTAs leave SMs to the
        // other streams, and the window start-up is spread over more rows).  Each class keeps its chosen width,
        // family and terms per CTA and tries every tile height.
        for (int c = 0; c < nc && best < 1e30f; ++c) {
            const bf_plan *pl = plans[rep[c]];
            TileConfig keep = cur[c];
            for (const auto &cand : tile_candidates(pl->kp, height, width, pl->desc.precision, 1 << 20)) {
                if (cand.tw != keep.tw || cand.ncols != keep.ncols || cand.nk != keep.nk || cand.ring != keep.ring ||
                    cand.depth != keep.depth || cand.packed != keep.packed || cand.pre != keep.pre || cand.th == keep.th ||
                    scratch_bytes(cand, height, width, pl->kp.zbins) > scratch_bytes(keep, height, width, pl->kp.zbins))
                    continue;
                cur[c] = cand;
                const float t = time_group();
                if (t < best * 0.995f) {
                    best = t;
                    keep = cand;
                }
            }
            cur[c] = keep;
        }
        if (best >= 1e30f) st = fail(BF_ERR_CUDA, "no geometry of the group ran");
    }
    if (st == BF_OK) {
        for (int c = 0; c < nc; ++c)
            remember_tile(plans[rep[c]]->kp, height, width, plans[rep[c]]->desc.precision, cur[c]);
        if (infos)
            for (int i = 0; i < n; ++i) fill_info(cur[cls[i]], height, width, infos + kInfoInts * i, plans[i]->kp.zbins);
    }
    for (int j = 0; j < n_streams; ++j) {
        if (ss[j]) {
            cudaStreamSynchronize(ss[j]);
            cudaStreamDestroy(ss[j]);
        }
        if (join[j]) cudaEventDestroy(join[j]);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    cudaFree(scratch);
    cudaSetDevice(prev);
    return st;
}

namespace {

// Selects the plan's device for a table look-up (the table is keyed per device);
// host-only plans use whatever device is current.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int device) {
        if (device < 0) return;
        if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            prev = -1;
        }
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" bf_status bf_launch_candidates(const bf_plan *plan, int height, int width, int max_n, int *infos,
                                          int *n_out) {
    if (!plan || height < 1 || width < 1 || max_n < 0 || !n_out || (max_n > 0 && !infos))
        return fail(BF_ERR_INVALID_ARG, "bad launch-candidate arguments");
    std::vector<TileConfig> c = tile_candidates(plan->kp, height, width, plan->desc.precision, max_n);
    for (size_t i = 0; i < c.size(); ++i) fill_info(c[i], height, width, infos + kInfoInts * i, plan->kp.zbins);
    *n_out = (int)c.size();
    return BF_OK;
}

extern "C" bf_status bf_set_launch(const bf_plan *plan, int height, int width, const int *info) {
    if (!plan || height < 1 || width < 1 || !info) return fail(BF_ERR_INVALID_ARG, "bad set-launch arguments");
    DeviceScope dev(plan->desc.device);
    if (!dev.ok) return fail(BF_ERR_NO_DEVICE, "cannot select the plan's device");
    for (const auto &c : tile_candidates(plan->kp, height, width, plan->desc.precision, 100000)) {
        int got[kInfoInts];
        fill_info(c, height, width, got, plan->kp.zbins);
        // the fields a caller chooses; the rest (threads, launches, bytes) follow from them
        if (got[0] == info[0] && got[1] == info[1] && got[3] == info[3] && got[8] == info[8] && got[9] == info[9] &&
            got[10] == info[10] && got[11] == info[11] && got[12] == info[12]) {
            remember_tile(plan->kp, height, width, plan->desc.precision, c);
            return BF_OK;
        }
    }
    return fail(BF_ERR_INVALID_ARG, "not a launch geometry of this plan and image size (see bf_launch_candidates)");
}
