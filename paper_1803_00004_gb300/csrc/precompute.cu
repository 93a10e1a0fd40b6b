// Pre-computation for later parameter settings (Sec. V-C, Case 1): the image
// is given first and the range parameters later.  With the cosine half-period
// P and the spatial kernel fixed (a fixed truncation T_r, or P = dI), the basis
// frequencies pi k / P do not depend on sigma_r; only the weights a_k do.
// bf_precompute runs the fused kernel once over the frequencies k < kmax and
// stores, per pixel, the four window sums of each (Eq. (36) before the
// weighting: sums of cos I, sin I, cos, sin over the spatial boxes).
// bf_filter_cached then filters with any plan sharing P and the spatial
// kernel by weighting those sums with its a_k cos/sin(pi k I(x) / P): one read
// of 16 bytes per selected term per pixel, no box filtering.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "bf_classes.h"
#include "bf_internal.h"

struct bf_cache {
    bfi::FilterParams basis;  // the plan's parameters the sums were computed with
    int kslots = 0;           // frequencies 0 .. kslots - 1 are stored
    int height = 0, width = 0, device = 0;
    int precision = 0;        // bf_precision of the stored sums
    float *planes = nullptr;  // [kslots][height][width][4]: sums of cos I, sin I, cos, sin (fp32, fp16 or bf16)
    size_t bytes = 0;
};

namespace bfi {
namespace {

// Weighting of the cached sums (Eq. (36)): for each selected term k, (cos, sin)(pi k t) at the centre pixel
// (t = (I(x) - i_lo) / P carried as two floats, sincospi corrected to first order in the low part), then
// num / den.  Guard as the fused kernel: den <= den_eps -> I(x).
// The four sums of one pixel and frequency, side by side: one 16-byte (fp32) or 8-byte (16-bit) load of the
// raw bits, widened to fp32 when used.
template <typename T> struct Raw { using type = uint2; };
template <> struct Raw<float> { using type = float4; };
__device__ __forceinline__ float4 load_raw(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ uint2 load_raw(const __half *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
__device__ __forceinline__ uint2 load_raw(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
__device__ __forceinline__ float4 widen(float4 v, const float *) { return v; }
__device__ __forceinline__ float4 widen(uint2 u, const __half *) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 widen(uint2 u, const __nv_bfloat16 *) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

template <typename T>
__global__ void bf_cached_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out,
                                 size_t out_pitch, const T *__restrict__ planes, int H, int W,
                                 const __grid_constant__ FilterParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    constexpr float kPiF = 3.14159265358979f;
    const float ix = __ldg(in + (size_t)y * in_pitch + x);
    const float v = ix - p.i_lo;
    const float th = v * p.inv_p;
    const float tl = fmaf(v, p.inv_p, -th) + v * p.inv_p_lo;
    const size_t plane = (size_t)H * W, px = (size_t)y * W + x;
    float num = 0.f, den = 0.f;
    // each term's sums are loaded one term ahead of its arithmetic
    typename Raw<T>::type fn = load_raw(planes + ((size_t)p.k[0] * plane + px) * 4);
    for (int j = 0; j < p.nr; ++j) {
        const typename Raw<T>::type f = fn;
        if (j + 1 < p.nr) fn = load_raw(planes + ((size_t)p.k[j + 1] * plane + px) * 4);
        const float kf = (float)p.k[j];
        const float kh = kf * th;
        const float kl = fmaf(kf, th, -kh) + kf * tl;
        float s, c;
        sincospif(kh, &s, &c);
        const float d = kPiF * kl;
        const float ck = fmaf(-d, s, c), sk = fmaf(d, c, s);
        const float a = p.a[j];
        const float4 w = widen(f, planes);
        num = fmaf(a, fmaf(ck, w.x, sk * w.y), num);
        den = fmaf(a, fmaf(ck, w.z, sk * w.w), den);
    }
    out[(size_t)y * out_pitch + x] = den > p.den_eps ? num / den + p.i_lo : ix;
}

// The parameters that fix the basis images and their box sums: P, the intensity origin and the spatial
// box windows with their weights.
bool same_basis(const FilterParams &a, const FilterParams &b) {
    if (a.inv_p != b.inv_p || a.inv_p_lo != b.inv_p_lo || a.i_lo != b.i_lo || a.m != b.m || a.rx != b.rx ||
        a.vlo != b.vlo || a.vhi != b.vhi)
        return false;
    for (int r = 0; r < a.m; ++r) {
        if (a.v0[r] != b.v0[r] || a.v1[r] != b.v1[r] || a.u0[r] != b.u0[r] || a.u1[r] != b.u1[r]) return false;
        for (int q = 0; q < a.m; ++q)
            if (a.C[r][q] != b.C[r][q]) return false;
    }
    return true;
}

}  // namespace
}  // namespace bfi

using namespace bfi;

extern "C" {

bf_status bf_precompute(const bf_plan *plan, const float *d_in, size_t in_pitch, int height, int width, int kmax,
                        int precision, void *stream, bf_cache **out) {
    if (out) *out = nullptr;
    if (!plan || !out || kmax < 2 || kmax > kMaxSlots || precision < BF_PREC_FP32 || precision > BF_PREC_FP16)
        return fail(BF_ERR_INVALID_ARG, "bad pre-computation arguments");
    if (height < 1 || width < 1) return fail(BF_ERR_INVALID_ARG, "empty image");
    if (!d_in || in_pitch % sizeof(float) || in_pitch < (size_t)width * sizeof(float) || in_pitch > 0xffffffffu)
        return fail(BF_ERR_INVALID_ARG, "NULL input or bad pitch");
    bf_status st = BF_OK;
    if (plan->kp.zbins > 0)
        return fail(BF_ERR_UNSUPPORTED, "the 3-D form (BF_RANGE_PAPER_3D) has no pre-computation cache");
    if (plan->desc.device < 0) return fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(plan->desc.device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the plan's device");
    }
    // the plan's basis with the frequencies 0 .. kmax - 1 (consecutive: the packed family)
    FilterParams pv = plan->kp;
    pv.nr = kmax;
    for (int i = 0; i < kmax; ++i) {
        pv.k[i] = i;
        pv.a[i] = 1.f;
    }
    // the cost model's best packed-family geometry (consecutive frequencies: every candidate is packed) that
    // computes its basis in the kernel (the cache modes have no pre-pass variant)
    TileConfig tc{};
    for (const auto &c : tile_candidates(pv, height, width, BF_PREC_FP32, 1 << 20))
        if (c.pre == 0) {
            tc = c;
            break;
        }
    bf_cache *c = nullptr;
    if (tc.ncols == 0 || tc.packed != 1) st = fail(BF_ERR_UNSUPPORTED, "no launch geometry for the pre-computation");
    if (st == BF_OK) {
        c = new bf_cache;
        c->basis = plan->kp;
        c->kslots = tc.groups * tc.nk;  // the groups' frequencies, kmax rounded up to whole groups
        c->height = height;
        c->width = width;
        c->device = plan->desc.device;
        c->precision = precision;
        c->bytes = (precision == BF_PREC_FP32 ? 4 : 2) * 4 * (size_t)c->kslots * height * width;
        if (cudaMalloc((void **)&c->planes, c->bytes) != cudaSuccess) {
            cudaGetLastError();
            st = fail(BF_ERR_OOM, "pre-computation cache (" + std::to_string(c->bytes >> 20) + " MiB)");
        }
    }
    if (st == BF_OK)
        st = launch_filter(pv, plan->desc.precision, plan->desc.kahan, tc, d_in, in_pitch / sizeof(float), nullptr, 0,
                           c->planes, height, width, stream,
                           precision == BF_PREC_FP16   ? kModeCacheF16
                           : precision == BF_PREC_BF16 ? kModeCacheBF16
                                                       : kModeCache);
    if (st == BF_OK) {
        *out = c;
    } else if (c) {
        cudaFree(c->planes);
        delete c;
    }
    cudaSetDevice(prev);
    return st;
}

bf_status bf_filter_cached(const bf_cache *cache, const bf_plan *plan, const float *d_in, size_t in_pitch,
                           float *d_out, size_t out_pitch, void *stream) {
    if (!cache || !plan) return fail(BF_ERR_INVALID_ARG, "NULL cache or plan");
    bf_status st = check_image(d_in, in_pitch, d_out, out_pitch, cache->height, cache->width);
    if (st != BF_OK) return st;
    if (plan->desc.device != cache->device) return fail(BF_ERR_INVALID_ARG, "plan and cache are on different devices");
    if (!same_basis(plan->kp, cache->basis))
        return fail(BF_ERR_INVALID_ARG, "the plan's period, intensity origin or spatial kernel differs from the cache's");
    if (plan->kp.k[plan->kp.nr - 1] >= cache->kslots)
        return fail(BF_ERR_RANGE, "the plan selects a frequency beyond the cache's (raise kmax)");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(cache->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(BF_ERR_NO_DEVICE, "cannot select the cache's device");
    }
    if (debug_consume_launch_failure()) {
        st = fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    } else {
        dim3 grid((cache->width + 255) / 256, cache->height);
        const size_t ip = in_pitch / sizeof(float), op = out_pitch / sizeof(float);
        cudaStream_t s = (cudaStream_t)stream;
        if (cache->precision == BF_PREC_FP16)
            bf_cached_kernel<<<grid, 256, 0, s>>>(d_in, ip, d_out, op, reinterpret_cast<const __half *>(cache->planes),
                                                  cache->height, cache->width, plan->kp);
        else if (cache->precision == BF_PREC_BF16)
            bf_cached_kernel<<<grid, 256, 0, s>>>(d_in, ip, d_out, op,
                                                  reinterpret_cast<const __nv_bfloat16 *>(cache->planes), cache->height,
                                                  cache->width, plan->kp);
        else
            bf_cached_kernel<<<grid, 256, 0, s>>>(d_in, ip, d_out, op, cache->planes, cache->height, cache->width,
                                                  plan->kp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(BF_ERR_CUDA, std::string("cached filter launch: ") + cudaGetErrorString(e));
    }
    cudaSetDevice(prev);
    return st;
}

void bf_cache_destroy(bf_cache *cache) {
    if (!cache) return;
    int prev = 0;
    const bool sel = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(cache->device) == cudaSuccess;
    cudaFree(cache->planes);
    if (sel) cudaSetDevice(prev);
    cudaGetLastError();
    delete cache;
}

size_t bf_cache_bytes(const bf_cache *cache) { return cache ? cache->bytes : 0; }

}  // extern "C"
