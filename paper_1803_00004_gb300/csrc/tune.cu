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
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lu", &k[0], &k[1], &k[2], &k[3], &k[4],
                       &k[5], &k[6], &k[7], &k[8], &k[9], &tc.tw, &tc.th, &tc.ncols, &tc.threads, &tc.nk, &tc.groups,
                       &tc.ring, &tc.depth, &tc.packed, &smem) == 20) {
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
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lu\n", std::get<0>(key), std::get<1>(key),
                 std::get<2>(key), std::get<3>(key), std::get<4>(key), std::get<5>(key), std::get<6>(key),
                 std::get<7>(key), std::get<8>(key), std::get<9>(key), tc.tw, tc.th, tc.ncols, tc.threads, tc.nk, tc.groups, tc.ring,
                 tc.depth, tc.packed, (unsigned long)tc.smem);
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

}  // namespace

TileConfig choose_tile(const FilterParams &p, int height, int width, int precision) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_locked();
        auto it = g_table.find(make_key(p, height, width, precision));
        // an entry stays usable only while its term grouping matches the library's current layout
        if (it != g_table.end() &&
            it->second.groups == (it->second.packed ? term_groups(p, it->second.nk) : (p.nr + it->second.nk - 1) / it->second.nk) &&
            (p.zbins == 0 || (it->second.packed && !it->second.ring)))
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

extern "C" bf_status bf_autotune(const bf_plan *plan, int height, int width, void *stream, int *info) {
    if (!plan || height < 1 || width < 1) return fail(BF_ERR_INVALID_ARG, "bad autotune arguments");
    if (plan->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(plan->desc.device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plan's device");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the cost model is coarse: keep the best few of every family (ring or not, terms per CTA)
    std::vector<TileConfig> ranked = tile_candidates(plan->kp, height, width, plan->desc.precision, 100000), cands;
    std::map<std::pair<int, int>, int> per_family;
    for (const auto &c : ranked)
        if (per_family[{c.ring * 4 + c.depth + 8 * c.packed, c.nk}]++ < 4) cands.push_back(c);
    bf_status st = BF_OK;
    float *in = nullptr, *out = nullptr, *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    size_t n = (size_t)height * width, need = 0;
    for (const auto &c : cands) need = std::max(need, scratch_bytes(c, height, width, plan->kp.zbins));
    if (cands.empty()) st = fail(BF_ERR_UNSUPPORTED, "no launch geometry for this plan");
    if (st == BF_OK && (cudaMalloc((void **)&in, n * sizeof(float)) != cudaSuccess ||
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
        fill_kernel<<<256, 256, 0, s>>>(in, n, width, plan->desc.i_lo, plan->desc.i_hi, plan->kp.zbins > 0 ? 1 : 0);
        for (const auto &c : cands) {
            bf_status r = launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, c, in, width, out, width,
                                        scratch, height, width, stream);  // warm-up
            if (r != BF_OK) continue;
            float t[3];
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                cudaEventRecord(e0, s);
                ok = launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, c, in, width, out, width, scratch,
                                   height, width, stream) == BF_OK;
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
            got[10] == info[10] && got[11] == info[11]) {
            remember_tile(plan->kp, height, width, plan->desc.precision, c);
            return BF_OK;
        }
    }
    return fail(BF_ERR_INVALID_ARG, "not a launch geometry of this plan and image size (see bf_launch_candidates)");
}
