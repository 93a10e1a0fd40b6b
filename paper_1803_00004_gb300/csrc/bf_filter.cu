// Fused single-pass evaluation of the box-filter form of the bilateral filter
// (Eq. (36) and the final divide of Eq. (1)) for sm_103a.
//
// Per CTA: a tile of `tw` output columns and `th` output rows.  One thread per
// image column of the tile plus a horizontal halo of `rx` columns on each side
// walks down the rows:
//
//  1. Vertical pass.  For every cosine term k of the pass and every basis image
//     g in {cos(w_k I) I, sin(w_k I) I, cos(w_k I), sin(w_k I)} (Eq. (34)), the
//     thread keeps one running sum per vertical box window [v0, v1]:
//         V(y) = V(y-1) + g(y + v1) - g(y + v0 - 1).
//     The basis values at the entering / leaving rows are recomputed from the
//     input pixel (sincospi of the base angle, then the angle-addition
//     recurrence up to k), so only the raw image is read and no basis image is
//     ever stored.
//  2. The vertical sums are mixed into one value per horizontal window,
//     Z_q = sum_r C[r][q] V_r, and published in shared memory.
//  3. Horizontal pass.  Work items (term, segment of `seg` output columns) run
//     horizontal running sums over the published row and weight the four
//     filtered images with a_k cos(w_k I(x)), a_k sin(w_k I(x)) into partial
//     numerator / denominator (Eq. (36)).
//  4. One thread per output column sums the partials over the terms and
//     divides (or accumulates into a scratch buffer for multi-pass plans).
//
// Rows above the first window of the tile are treated as zero, so the walk
// starts (vhi - vlo) rows early and needs no explicit initialisation; pixels
// outside the image contribute zero to numerator and denominator.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "bf_internal.h"

namespace bfi {

namespace {

std::atomic<int> g_fail_launches{0};

// Basis at one pixel: base rotation (cos, sin)(pi t) and the starting value
// (cos, sin)(pi k0 t), t = v / P.  t is carried as th + tl (two floats; the
// rounding of v / P would otherwise cost pi k |t| 2^-24 of phase at term k)
// and each sincospi is corrected to first order in its low part.  Invalid
// pixels start from (0, 0), so every basis image is zero there.
__device__ __forceinline__ void basis_start(float v, float inv_p, float inv_p_lo, int k0, bool valid, float &c1,
                                            float &s1, float &c0, float &s0) {
    constexpr float kPiF = 3.14159265358979f;
    const float th = v * inv_p;
    const float tl = fmaf(v, inv_p, -th) + v * inv_p_lo;
    float sb, cb;
    sincospif(th, &sb, &cb);
    const float d = kPiF * tl;
    c1 = fmaf(-d, sb, cb);
    s1 = fmaf(d, cb, sb);
    if (!valid) {
        c0 = 0.f;
        s0 = 0.f;
    } else if (k0 == 0) {
        c0 = 1.f;
        s0 = 0.f;
    } else if (k0 == 1) {
        c0 = c1;
        s0 = s1;
    } else {
        const float kf = (float)k0;
        const float kh = kf * th;
        const float kl = fmaf(kf, th, -kh) + kf * tl;
        float sk, ck;
        sincospif(kh, &sk, &ck);
        const float dk = kPiF * kl;
        c0 = fmaf(-dk, sk, ck);
        s0 = fmaf(dk, ck, sk);
    }
}

template <int NK, int M>
__global__ void __launch_bounds__(512, 1)
bf_fused_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                float *__restrict__ acc, int H, int W, int tw, int th, int seg, int mode, const FilterParams p) {
    extern __shared__ float smem[];
    const int nthr = blockDim.x;
    const int ZP = nthr + 1;
    const int WP = tw + 1;
    float *zbuf = smem;                      // [M][NK][4][ZP]
    float *wbuf = zbuf + M * NK * 4 * ZP;    // [NK][2][WP]
    float *pbuf = wbuf + NK * 2 * WP;        // [NK][2][WP]

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * tw;
    const int y0 = blockIdx.y * th;
    const int xcol = x0 - p.rx + tid;
    const bool colv = (tid < tw + 2 * p.rx) && xcol >= 0 && xcol < W;
    const int y_end = min(y0 + th, H);
    const int y_lo = max(0, y0 + p.vlo);
    const int ys = y0 + p.vlo - p.vhi;
    const int nseg = tw / seg;
    constexpr int NE = 2 * M + 1;  // edges: M entering rows, M leaving rows, the centre row

    float V[NK][4][M];
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < M; ++r) V[i][t][r] = 0.f;

    for (int y = ys; y < y_end; ++y) {
        const bool outrow = (y >= y0);
        float Ie[NE], c1[NE], s1[NE], ce[NE], se[NE];
        const int k0 = p.k[0];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int off = e < M ? p.v1[e] : (e < 2 * M ? p.v0[e - M] - 1 : 0);
            const int row = y + off;
            const bool valid = (e < 2 * M) ? (colv && row >= y_lo && row < H) : (colv && outrow);
            const float v = valid ? __ldg(in + (size_t)row * in_pitch + xcol) - p.i_lo : 0.f;
            Ie[e] = v;
            basis_start(v, p.inv_p, p.inv_p_lo, k0, valid, c1[e], s1[e], ce[e], se[e]);
        }
        int kcur = k0;
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            const int steps = p.k[i] - kcur;
            kcur = p.k[i];
            for (int s = 0; s < steps; ++s) {
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                    const float c = ce[e] * c1[e] - se[e] * s1[e];
                    const float sv = se[e] * c1[e] + ce[e] * s1[e];
                    ce[e] = c;
                    se[e] = sv;
                }
            }
#pragma unroll
            for (int r = 0; r < M; ++r) {
                const int ei = r, eo = M + r;
                V[i][0][r] += ce[ei] * Ie[ei] - ce[eo] * Ie[eo];
                V[i][1][r] += se[ei] * Ie[ei] - se[eo] * Ie[eo];
                V[i][2][r] += ce[ei] - ce[eo];
                V[i][3][r] += se[ei] - se[eo];
            }
            if (outrow) {
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int q = 0; q < M; ++q) {
                        float z = 0.f;
#pragma unroll
                        for (int r = 0; r < M; ++r) z += p.C[r][q] * V[i][t][r];
                        zbuf[((q * NK + i) * 4 + t) * ZP + tid] = z;
                    }
                const int xl = tid - p.rx;
                if (xl >= 0 && xl < tw) {
                    wbuf[(i * 2 + 0) * WP + xl] = p.a[i] * ce[2 * M];
                    wbuf[(i * 2 + 1) * WP + xl] = p.a[i] * se[2 * M];
                }
            }
        }
        if (!outrow) continue;  // warm-up rows: uniform over the CTA
        __syncthreads();

        // horizontal pass: items (term i, segment sg)
        for (int item = tid; item < NK * nseg; item += nthr) {
            const int i = item % NK, sg = item / NK;
            const int xs = sg * seg;
            float S[4][M];
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float *zr = zbuf + ((q * NK + i) * 4 + t) * ZP + xs + p.rx;
                    float s = 0.f;
                    for (int dx = p.u0[q]; dx <= p.u1[q]; ++dx) s += zr[dx];
                    S[t][q] = s;
                }
            for (int j = 0; j < seg; ++j) {
                const int xl = xs + j;
                float F[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float f = 0.f;
#pragma unroll
                    for (int q = 0; q < M; ++q) f += S[t][q];
                    F[t] = f;
                }
                const float wc = wbuf[(i * 2 + 0) * WP + xl], ws = wbuf[(i * 2 + 1) * WP + xl];
                pbuf[(i * 2 + 0) * WP + xl] = wc * F[0] + ws * F[1];
                pbuf[(i * 2 + 1) * WP + xl] = wc * F[2] + ws * F[3];
                if (j + 1 < seg) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int q = 0; q < M; ++q) {
                            const float *zr = zbuf + ((q * NK + i) * 4 + t) * ZP + xl + p.rx;
                            S[t][q] += zr[p.u1[q] + 1] - zr[p.u0[q]];
                        }
                }
            }
        }
        __syncthreads();

        if (tid < tw) {
            const int x = x0 + tid;
            if (x < W) {
                float num = 0.f, den = 0.f;
#pragma unroll
                for (int i = 0; i < NK; ++i) {
                    num += pbuf[(i * 2 + 0) * WP + tid];
                    den += pbuf[(i * 2 + 1) * WP + tid];
                }
                const size_t plane = (size_t)H * W;
                float *an = acc + (size_t)y * W + x;
                if (mode == kPassFirst) {
                    an[0] = num;
                    an[plane] = den;
                } else if (mode == kPassMid) {
                    an[0] += num;
                    an[plane] += den;
                } else {
                    if (mode == kPassLast) {
                        num += an[0];
                        den += an[plane];
                    }
                    const float ix = __ldg(in + (size_t)y * in_pitch + x);
                    out[(size_t)y * out_pitch + x] = (den > p.den_eps) ? num / den + p.i_lo : ix;
                }
            }
        }
    }
}

// Slots (cosine terms) per pass for each window count: keeps the per-thread
// running-sum state at 4 * slots * M <= 64 floats.
constexpr int kSlots[kMaxWin + 1] = {0, 16, 8, 5, 4, 3, 2};

template <int M>
void *kernel_for_m() {
    return (void *)bf_fused_kernel<kSlots[M], M>;
}

void *kernel_ptr(int m) {
    switch (m) {
        case 1: return kernel_for_m<1>();
        case 2: return kernel_for_m<2>();
        case 3: return kernel_for_m<3>();
        case 4: return kernel_for_m<4>();
        case 5: return kernel_for_m<5>();
        case 6: return kernel_for_m<6>();
    }
    return nullptr;
}

// ---------------------------------------------------------------- exact BF

__global__ void bf_exact_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out,
                                size_t out_pitch, int H, int W, int spatial, float inv2ss, int R, int range,
                                float sigma_r) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const float ix = in[(size_t)y * in_pitch + x];
    const float inv2sr = 1.0f / (2.0f * sigma_r * sigma_r);
    float num = 0.f, den = 0.f;
    for (int dy = -R; dy <= R; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= H) continue;
        const float *row = in + (size_t)yy * in_pitch;
        for (int dx = -R; dx <= R; ++dx) {
            const int xx = x + dx;
            if (xx < 0 || xx >= W) continue;
            const float iy = __ldg(row + xx);
            const float t = ix - iy;
            float kr;
            if (range == BF_KERNEL_GAUSSIAN) kr = expf(-t * t * inv2sr);
            else if (range == BF_KERNEL_EXPONENTIAL) kr = expf(-fabsf(t) / sigma_r);
            else kr = fabsf(t) <= sigma_r ? 1.f : 0.f;
            const float ks = spatial == BF_KERNEL_BOX ? 1.f : expf(-(float)(dx * dx + dy * dy) * inv2ss);
            const float wgt = ks * kr;
            num += wgt * iy;
            den += wgt;
        }
    }
    out[(size_t)y * out_pitch + x] = num / den;
}

bf_status cuda_fail(cudaError_t e, const char *what) {
    return fail(BF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

bool debug_consume_launch_failure() {
    int n = g_fail_launches.load();
    while (n > 0) {
        if (g_fail_launches.compare_exchange_weak(n, n - 1)) return true;
    }
    return false;
}

void debug_set_fail_launches(int n) { g_fail_launches.store(n > 0 ? n : 0); }

bool kernel_class_supported(int m) { return m >= 1 && m <= kMaxWin; }

int slots_per_pass(int m) { return (m >= 1 && m <= kMaxWin) ? kSlots[m] : 0; }

TileConfig choose_tile(int m, int rx, int vspan, int height, int width, int precision) {
    (void)precision;
    TileConfig tc;
    tc.seg = 16;
    int tw = 128;
    if (width < tw) tw = ((width + tc.seg - 1) / tc.seg) * tc.seg;
    if (tw < tc.seg) tw = tc.seg;
    tc.tw = tw;
    int th = 64;
    if (vspan > 64) th = 128;
    if (vspan > 128) th = 256;
    if (height < th) th = height > 0 ? height : 1;
    tc.th = th;
    int thr = tw + 2 * rx;
    tc.threads = ((thr + 31) / 32) * 32;
    const int nk = kSlots[m];
    tc.smem = sizeof(float) * ((size_t)m * nk * 4 * (tc.threads + 1) + (size_t)nk * 4 * (tw + 1));
    return tc;
}

bf_status launch_filter_pass(const FilterParams &p, int precision, int kahan, const TileConfig &tc,
                             const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, float *d_acc,
                             int height, int width, int mode, void *stream) {
    (void)precision;
    (void)kahan;
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    void *fn = kernel_ptr(p.m);
    if (!fn) return fail(BF_ERR_UNSUPPORTED, "no kernel for this window count");
    if (tc.threads > 512) return fail(BF_ERR_UNSUPPORTED, "horizontal reach too large for one CTA (radius > 192)");
    if (tc.smem > 227 * 1024) return fail(BF_ERR_UNSUPPORTED, "tile needs more than 227 KB of shared memory");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc.smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    dim3 grid((width + tc.tw - 1) / tc.tw, (height + tc.th - 1) / tc.th);
    int tw = tc.tw, th = tc.th, seg = tc.seg, H = height, W = width;
    const float *in = d_in;
    float *out = d_out, *acc = d_acc;
    FilterParams pp = p;
    void *args[] = {(void *)&in, (void *)&in_pitch, (void *)&out, (void *)&out_pitch, (void *)&acc, (void *)&H,
                    (void *)&W, (void *)&tw, (void *)&th, (void *)&seg, (void *)&mode, (void *)&pp};
    e = cudaLaunchKernel(fn, grid, dim3(tc.threads), args, tc.smem, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    return BF_OK;
}

bf_status launch_exact(const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, int height, int width,
                       int spatial, float sigma_s, int radius, int range, float sigma_r, void *stream) {
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    dim3 block(128), grid((width + 127) / 128, height);
    bf_exact_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(d_in, in_pitch, d_out, out_pitch, height, width, spatial,
                                                             1.0f / (2.0f * sigma_s * sigma_s), radius, range, sigma_r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "exact launch");
    return BF_OK;
}

}  // namespace bfi
