// Tile body of the fused filter and its kernel templates, shared by the
// translation units that instantiate the kernel classes (kernels_m*.cu) so
// that they compile in parallel.  See bf_filter.cu for the algorithm.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "bf_internal.h"

namespace bfi {

constexpr int kScanThreads = 64;  // two warps: one exchange row per lane (<= 64 rows)

namespace {

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

__device__ __forceinline__ int pos_mod(int a, int d) {
    const int r = a % d;
    return r < 0 ? r + d : r;
}

__device__ __forceinline__ void ring_put(float *ring, int D, int ncols, int row, int tid, float v, float c1, float s1,
                                         float c0, float s0) {
    float *r = ring + (size_t)(pos_mod(row, D) * 5) * ncols + tid;
    r[0] = v;
    r[ncols] = c1;
    r[2 * ncols] = s1;
    r[3 * ncols] = c0;
    r[4 * ncols] = s0;
}

// Compensated (Kahan) accumulation s += x with running error term c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Adds x to the sliding sum s: compensated, or plain (c then stays 0).
__device__ __forceinline__ void sum_add(float &s, float &c, int compensated, float x) {
    if (compensated) kahan_add(s, c, x);
    else s += x;
}

// Advances (c, s) = (cos, sin)(pi k t) by `steps` multiples of the base rotation.
__device__ __forceinline__ void rotate(float &c, float &s, float c1, float s1, int steps) {
    if (steps == 1) {  // consecutive terms (the usual case): no loop
        const float cn = fmaf(c, c1, -s * s1);
        s = fmaf(s, c1, c * s1);
        c = cn;
        return;
    }
    for (int n = 0; n < steps; ++n) {
        const float cn = fmaf(c, c1, -s * s1);
        const float sn = fmaf(s, c1, c * s1);
        c = cn;
        s = sn;
    }
}

// One tile: output columns [x0, x0 + tw) x rows [y0, y0 + th) of one image,
// cosine terms [g NK, g NK + NK) of p.  All threads of the CTA call it; it
// ends on a barrier, so the shared memory can be reused right after.  `grouped`:
// store partial numerator / denominator planes (part) instead of dividing.
template <int NK, int M, bool RING, bool CL>
__device__ __forceinline__ void tile_body(const FilterParams &p, const float *__restrict__ in, size_t in_pitch,
                                          float *__restrict__ out, size_t out_pitch, float *__restrict__ part, int H,
                                          int W, int x0, int y0, int tw, int th, int ncols, int g, bool grouped,
                                          int depth, float *smem) {
    constexpr int NROW = M * NK * 4;  // exchange rows per image row: windows x terms x basis images
    constexpr int NE = 2 * M + 1;     // edges per step: M entering rows, M leaving rows, the output row
    constexpr int NRP = NROW + 1;     // column pitch of the exchange, odd: a warp's lanes hit distinct banks
    const int ZC = ncols + 2;         // exchange columns: tile column c at index c + 1; 0 and ncols + 1 stay 0
    // `depth` exchange buffers: 2 -> the output phase reads the row the scan finished in the same step (two
    // barriers per row); 3 -> it reads the row scanned one step earlier (one barrier per row)
    // exchange [depth][ZC][NRP], column-major so that every row offset is a compile-time constant: column
    // threads store a column, scan lanes walk along a row, output threads read a column
    float *zb0 = smem;
    float *wb0 = smem + depth * ZC * NRP;  // [depth][NK][2][tw]: a_k cos, a_k sin at the output row
    // RING: per column, the basis inputs of the last D rows (v, cos/sin(pi t), cos/sin(pi k0 t)), so each
    // row's sincospi and load happen once instead of at every window edge: [D][5][ncols]
    const int D = p.vhi - p.vlo + 2;
    float *ring = wb0 + depth * NK * 2 * tw;
    // CL (thread-block cluster across the image width): no halo columns; the scan reads the
    // neighbouring CTAs' exchange rows through distributed shared memory and writes its window
    // sums to sb ([tw][NRP]) because the neighbours still read the raw rows
    float *sb = ring + (RING ? 5 * (size_t)D * ncols : 0);
    const int halo = CL ? 0 : p.rx;

    const int tid = threadIdx.x;
    const bool is_col = tid < ncols;
    const int xcol = x0 - halo + tid;
    const bool colv = is_col && tid < tw + 2 * halo && xcol >= 0 && xcol < W;
    const int nout = min(y0 + th, H) - y0;
    const int xl = tid - halo;
    const bool is_out = is_col && xl >= 0 && xl < tw && x0 + xl < W;

    for (int i = tid; i < depth * NRP; i += blockDim.x) {
        const int b = i / NRP, r = i - b * NRP;
        zb0[(b * ZC) * NRP + r] = 0.f;
        zb0[(b * ZC + ncols + 1) * NRP + r] = 0.f;
    }

    // this group's terms
    int kk[NK];
    float aa[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        const int j = g * NK + i;
        const bool ok = j < p.nr;
        kk[i] = p.k[ok ? j : p.nr - 1];
        aa[i] = ok ? p.a[j] : 0.f;
    }

    float V[NK][4][M];
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < M; ++r) V[i][t][r] = 0.f;

    // window sums at the first output row: every row of the span once
    if (is_col) {
        for (int off = p.vlo; off <= p.vhi; ++off) {
            const int row = y0 + off;
            if (row < 0 || row >= H) continue;
            const float v = colv ? __ldg(in + (size_t)row * in_pitch + xcol) - p.i_lo : 0.f;
            float c1, s1, c, s;
            basis_start(v, p.inv_p, p.inv_p_lo, kk[0], colv, c1, s1, c, s);
            if (RING) ring_put(ring, D, ncols, row, tid, v, c1, s1, c, s);
            int kc = kk[0];
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                rotate(c, s, c1, s1, kk[i] - kc);
                kc = kk[i];
                const float gi[4] = {c * v, s * v, c, s};
#pragma unroll
                for (int r = 0; r < M; ++r)
                    if (off >= p.v0[r] && off <= p.v1[r]) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) V[i][t][r] += gi[t];
                    }
            }
        }
    }

    const int lag = depth - 1;  // steps between a row's vertical pass and its output phase
    for (int j = 0; j < nout + lag; ++j) {
        const int y = y0 + j;
        if (is_col && j < nout) {
            float Ie[NE], c1[NE], s1[NE], ce[NE], se[NE];
            if (RING && j > 0) {  // the newest row of the span enters the ring
                const int row = y + p.vhi;
                if (row < H) {
                    const float v = colv ? __ldg(in + (size_t)row * in_pitch + xcol) - p.i_lo : 0.f;
                    float a, b, c, s;
                    basis_start(v, p.inv_p, p.inv_p_lo, kk[0], colv, a, b, c, s);
                    ring_put(ring, D, ncols, row, tid, v, a, b, c, s);
                }
            }
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int off = e < M ? p.v1[e] : (e < 2 * M ? p.v0[e - M] - 1 : 0);
                const int row = y + off;
                // at j == 0 the sums already hold row y0: only the output-row edge is live
                const bool valid = colv && row >= 0 && row < H && (j > 0 || e == 2 * M);
                if (RING) {
                    // slots of rows outside the image were never written: do not read them
                    const float *rr = ring + (size_t)(pos_mod(row, D) * 5) * ncols + tid;
                    Ie[e] = valid ? rr[0] : 0.f;
                    c1[e] = valid ? rr[ncols] : 1.f;
                    s1[e] = valid ? rr[2 * ncols] : 0.f;
                    ce[e] = valid ? rr[3 * ncols] : 0.f;
                    se[e] = valid ? rr[4 * ncols] : 0.f;
                } else {
                    const float v = valid ? __ldg(in + (size_t)row * in_pitch + xcol) - p.i_lo : 0.f;
                    Ie[e] = v;
                    basis_start(v, p.inv_p, p.inv_p_lo, kk[0], valid, c1[e], s1[e], ce[e], se[e]);
                }
            }
            float *zb = zb0 + ((j % depth) * ZC + tid + 1) * NRP;
            float *wb = wb0 + (j % depth) * NK * 2 * tw;
            int kc = kk[0];
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                const int steps = kk[i] - kc;
                kc = kk[i];
#pragma unroll
                for (int e = 0; e < NE; ++e) rotate(ce[e], se[e], c1[e], s1[e], steps);
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    const int ei = r, eo = M + r;
                    V[i][0][r] += fmaf(ce[ei], Ie[ei], -ce[eo] * Ie[eo]);
                    V[i][1][r] += fmaf(se[ei], Ie[ei], -se[eo] * Ie[eo]);
                    V[i][2][r] += ce[ei] - ce[eo];
                    V[i][3][r] += se[ei] - se[eo];
                }
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int q = 0; q < M; ++q) {
                        float z = 0.f;
#pragma unroll
                        for (int r = 0; r < M; ++r) z = fmaf(p.C[r][q], V[i][t][r], z);
                        zb[(q * NK + i) * 4 + t] = z;
                    }
                if (is_out) {
                    wb[(i * 2 + 0) * tw + xl] = aa[i] * ce[2 * M];
                    wb[(i * 2 + 1) * tw + xl] = aa[i] * se[2 * M];
                }
            }
        } else if (CL && !is_col && j >= 1 && j - 1 < nout) {
            const int r = tid - ncols;
            if (r < NROW) {
                // sliding sum of window q over this CTA's columns; columns left of 0 / right of tw
                // live in the neighbouring CTAs of the cluster (zero at the image border)
                namespace cg = cooperative_groups;
                cg::cluster_group cl = cg::this_cluster();
                const int rank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
                const int q = r / (NK * 4);
                const int u0 = p.u0[q], u1 = p.u1[q];
                float *own = zb0 + ((j - 1) % depth) * ZC * NRP + r;
                const float *lft = rank > 0 ? cl.map_shared_rank(own, rank - 1) : nullptr;
                const float *rgt = rank + 1 < csize ? cl.map_shared_rank(own, rank + 1) : nullptr;
                auto fetch = [&](int pos) -> float {
                    if (pos < 0) return lft ? lft[(tw + pos + 1) * NRP] : 0.f;
                    if (pos < tw) return own[(pos + 1) * NRP];
                    return rgt ? rgt[(pos - tw + 1) * NRP] : 0.f;
                };
                float S = 0.f, comp = 0.f;
                int b = u0;
                for (; b + 7 <= u1; b += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = fetch(b + u);
                    sum_add(S, comp, p.kahan, ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
                }
                float rest = 0.f;
                for (; b <= u1; ++b) rest += fetch(b);
                sum_add(S, comp, p.kahan, rest);
                float *outr = sb + r;
                for (int c0 = 0; c0 < tw; c0 += 8) {
                    float d[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) d[u] = fetch(c0 + u + u1 + 1) - fetch(c0 + u + u0);
                    float pd = -comp;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        outr[(c0 + u) * NRP] = S + pd;
                        pd += d[u];
                    }
                    sum_add(S, comp, p.kahan, pd + comp);
                }
            }
        } else if (!CL && !is_col && j >= 1 && j - 1 < nout) {
            const int r = tid - ncols;
            if (r < NROW) {
                // sliding sum of window q over the row; S(c) replaces Z(c + u0), which the
                // slide has consumed (index c + u0 + 1 in buffer coordinates)
                const int q = r / (NK * 4);
                const int u0 = p.u0[q], u1 = p.u1[q];
                float *row = zb0 + ((j - 1) % depth) * ZC * NRP + r;
                float S = 0.f, comp = 0.f;
                int b = p.rx + u0 + 1;
                const int bend = p.rx + u1 + 1;
                for (; b + 7 <= bend; b += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = row[(b + u) * NRP];
                    sum_add(S, comp, p.kahan, ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
                }
                float rest = 0.f;
                for (; b <= bend; ++b) rest += row[b * NRP];
                sum_add(S, comp, p.kahan, rest);
                for (int c0 = p.rx; c0 < p.rx + tw; c0 += 8) {
                    float d[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) d[u] = row[(c0 + u + u1 + 2) * NRP] - row[(c0 + u + u0 + 1) * NRP];
                    float pd = -comp;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        row[(c0 + u + u0 + 1) * NRP] = S + pd;
                        pd += d[u];
                    }
                    sum_add(S, comp, p.kahan, pd + comp);
                }
            }
        }
        if (depth == 2) __syncthreads();
        if (is_out && j >= lag) {
            const int yo = y - lag;
            const float *zp = zb0 + ((j - lag) % depth) * ZC * NRP + tid * NRP;
            const float *wp = wb0 + ((j - lag) % depth) * NK * 2 * tw + xl;
            float num = 0.f, den = 0.f;
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                float F[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float f = 0.f;
#pragma unroll
                    for (int q = 0; q < M; ++q) {
                        if (CL) f += sb[xl * NRP + (q * NK + i) * 4 + t];
                        else f += zp[(p.u0[q] + 1) * NRP + (q * NK + i) * 4 + t];
                    }
                    F[t] = f;
                }
                const float wc = wp[(i * 2 + 0) * tw], ws = wp[(i * 2 + 1) * tw];
                num = fmaf(wc, F[0], fmaf(ws, F[1], num));
                den = fmaf(wc, F[2], fmaf(ws, F[3], den));
            }
            const int x = x0 + xl;
            if (grouped) {
                const size_t plane = (size_t)H * W;
                float *pp = part + (size_t)(2 * g) * plane + (size_t)yo * W + x;
                pp[0] = num;
                pp[plane] = den;
            } else {
                const float ix = __ldg(in + (size_t)yo * in_pitch + x);
                out[(size_t)yo * out_pitch + x] = (den > p.den_eps) ? num / den + p.i_lo : ix;
            }
        }
        if (CL) {
            // neighbours must have read this step's rows before they are overwritten, and must see the
            // next rows before scanning them
            cooperative_groups::this_cluster().sync();
        } else {
            __syncthreads();
        }
    }
}

template <int NK, int M, bool RING, bool CL>
__global__ void __launch_bounds__(512, 1)
bf_fused_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth,
                const __grid_constant__ FilterParams p) {
    extern __shared__ float smem[];
    tile_body<NK, M, RING, CL>(p, in, in_pitch, out, out_pitch, part, H, W, blockIdx.x * tw, blockIdx.y * th, tw, th, ncols,
                           blockIdx.z, gridDim.z > 1, depth, smem);
}

// Persistent batched form: each CTA repeatedly takes the next work item from
// the cursor (largest items first, as the host ordered them) and runs the
// tile body with that image's parameters staged in shared memory.  The loop is
// bounded by the item count.
template <int NK, int M>
__global__ void __launch_bounds__(512, 1)
bf_batch_kernel(const BatchImage *__restrict__ imgs, const FilterParams *__restrict__ params,
                const WorkItem *__restrict__ items, int n_items, int *__restrict__ cursor, int ncols) {
    extern __shared__ float smem[];
    __shared__ FilterParams sp;
    __shared__ int s_item;
    for (int iter = 0; iter < n_items; ++iter) {
        if (threadIdx.x == 0) s_item = atomicAdd(cursor, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        const BatchImage im = imgs[w.img];
        const int *src = reinterpret_cast<const int *>(params + im.params);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(FilterParams) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        tile_body<NK, M, false, false>(sp, im.in, im.in_pitch, im.out, im.out_pitch, im.part, im.H, im.W, w.x0, w.y0, w.tw,
                                w.th, ncols, w.g, im.groups > 1, 2, smem);
    }
}


}  // namespace

// Kernel classes: windows per axis M and terms per group NK (NK * M <= 16, and
// no class spills registers).
struct KernelClass {
    int m, nk;
    const void *fn[2][2];  // [ring][cluster] tile kernels
    const void *batch_fn;
};

#define BF_CLASS(M, NK)                                                                                    \
    {M,                                                                                                    \
     NK,                                                                                                   \
     {{(const void *)bf_fused_kernel<NK, M, false, false>, (const void *)bf_fused_kernel<NK, M, false, true>}, \
      {(const void *)bf_fused_kernel<NK, M, true, false>, (const void *)bf_fused_kernel<NK, M, true, true>}},   \
     (const void *)bf_batch_kernel<NK, M>}

// Per-TU class tables (kernels_m*.cu).
extern const KernelClass kClassesM1[];
extern const KernelClass kClassesM2[];
extern const KernelClass kClassesM3[];
extern const KernelClass kClassesM4to6[];
extern const int kNumClassesM1, kNumClassesM2, kNumClassesM3, kNumClassesM4to6;

}  // namespace bfi
