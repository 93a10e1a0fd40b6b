// Fused evaluation of the box-filter form of the bilateral filter (Eq. (36)
// and the final divide of Eq. (1)) for sm_103a.
//
// One CTA covers `tw` output columns x `th` output rows for one group of
// cosine terms (blockIdx.z).  It has `ncols` column threads (one per image
// column of the tile plus a horizontal halo of `rx` columns each side) and two
// scan warps.  Per output row y:
//
//  1. Vertical pass (column threads).  For every term k of the group and basis
//     image g in {cos(w_k I) I, sin(w_k I) I, cos(w_k I), sin(w_k I)} (Eq. (34))
//     a column thread keeps one running sum per vertical box window [v0, v1]:
//         V(y) = V(y-1) + g(y + v1) - g(y + v0 - 1).
//     Basis values at the entering / leaving rows are recomputed from the raw
//     pixel (sincospi of the base angle, angle-addition recurrence), so only
//     the image itself is read and no basis image exists in memory.  The sums
//     are mixed per horizontal window, Z_q = sum_r C[r][q] V_r, and published
//     in one of two shared-memory exchange buffers.
//  2. Horizontal pass (scan warps, one exchange row per lane, concurrently with
//     the next row's vertical pass): the sliding window sum of the row's
//     window, Kahan-compensated per block of 8 columns, written in place over
//     the values it has consumed.
//  3. Range accumulation (column threads of output columns): the filtered images are
//     weighted with a_k cos(w_k I(x)), a_k sin(w_k I(x)) into numerator and
//     denominator (Eq. (36)), then divided (one group) or stored as partial
//     planes that a finalize kernel sums in a fixed order (several groups).
//
// The running sums of the first output row are initialised directly (one
// basis evaluation per row of the window span); pixels outside the image
// contribute zero to numerator and denominator.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "bf_internal.h"

namespace bfi {

namespace {

constexpr int kScanThreads = 64;  // two warps: one exchange row per lane (<= 64 rows)

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
template <int NK, int M, bool RING>
__device__ __forceinline__ void tile_body(const FilterParams &p, const float *__restrict__ in, size_t in_pitch,
                                          float *__restrict__ out, size_t out_pitch, float *__restrict__ part, int H,
                                          int W, int x0, int y0, int tw, int th, int ncols, int g, bool grouped,
                                          int depth, float *smem) {
    constexpr int NROW = M * NK * 4;  // exchange rows per image row: windows x terms x basis images
    constexpr int NE = 2 * M + 1;     // edges per step: M entering rows, M leaving rows, the output row
    const int ZP = ncols + 3;         // odd: scan lanes (rows) hit distinct banks
    // `depth` exchange buffers: 2 -> the output phase reads the row the scan finished in the same step (two
    // barriers per row); 3 -> it reads the row scanned one step earlier (one barrier per row)
    float *zb0 = smem;                    // [depth][NROW][ZP]: tile column c at index c + 1; 0, ncols+1, ncols+2 stay 0
    float *wb0 = smem + depth * NROW * ZP;  // [depth][NK][2][tw]: a_k cos, a_k sin at the output row
    // RING: per column, the basis inputs of the last D rows (v, cos/sin(pi t), cos/sin(pi k0 t)), so each
    // row's sincospi and load happen once instead of at every window edge: [D][5][ncols]
    const int D = p.vhi - p.vlo + 2;
    float *ring = wb0 + depth * NK * 2 * tw;

    const int tid = threadIdx.x;
    const bool is_col = tid < ncols;
    const int xcol = x0 - p.rx + tid;
    const bool colv = is_col && tid < tw + 2 * p.rx && xcol >= 0 && xcol < W;
    const int nout = min(y0 + th, H) - y0;
    const int xl = tid - p.rx;
    const bool is_out = is_col && xl >= 0 && xl < tw && x0 + xl < W;

    for (int i = tid; i < depth * NROW; i += blockDim.x) {
        zb0[i * ZP] = 0.f;
        zb0[i * ZP + ncols + 1] = 0.f;
        zb0[i * ZP + ncols + 2] = 0.f;
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
            float *zb = zb0 + (j % depth) * NROW * ZP + tid + 1;
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
                        zb[((q * NK + i) * 4 + t) * ZP] = z;
                    }
                if (is_out) {
                    wb[(i * 2 + 0) * tw + xl] = aa[i] * ce[2 * M];
                    wb[(i * 2 + 1) * tw + xl] = aa[i] * se[2 * M];
                }
            }
        } else if (!is_col && j >= 1 && j - 1 < nout) {
            const int r = tid - ncols;
            if (r < NROW) {
                // sliding sum of window q over the row; S(c) replaces Z(c + u0), which the
                // slide has consumed (index c + u0 + 1 in buffer coordinates)
                const int q = r / (NK * 4);
                const int u0 = p.u0[q], u1 = p.u1[q];
                float *row = zb0 + ((j - 1) % depth) * NROW * ZP + r * ZP;
                float S = 0.f, comp = 0.f;
                int b = p.rx + u0 + 1;
                const int bend = p.rx + u1 + 1;
                for (; b + 7 <= bend; b += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = row[b + u];
                    kahan_add(S, comp, ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
                }
                float rest = 0.f;
                for (; b <= bend; ++b) rest += row[b];
                kahan_add(S, comp, rest);
                for (int c0 = p.rx; c0 < p.rx + tw; c0 += 8) {
                    float d[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) d[u] = row[c0 + u + u1 + 2] - row[c0 + u + u0 + 1];
                    float pd = -comp;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        row[c0 + u + u0 + 1] = S + pd;
                        pd += d[u];
                    }
                    kahan_add(S, comp, pd + comp);
                }
            }
        }
        if (depth == 2) __syncthreads();
        if (is_out && j >= lag) {
            const int yo = y - lag;
            const float *zp = zb0 + ((j - lag) % depth) * NROW * ZP + tid;
            const float *wp = wb0 + ((j - lag) % depth) * NK * 2 * tw + xl;
            float num = 0.f, den = 0.f;
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                float F[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float f = 0.f;
#pragma unroll
                    for (int q = 0; q < M; ++q) f += zp[((q * NK + i) * 4 + t) * ZP + p.u0[q] + 1];
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
        __syncthreads();
    }
}

template <int NK, int M, bool RING>
__global__ void __launch_bounds__(512, 1)
bf_fused_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth,
                const __grid_constant__ FilterParams p) {
    extern __shared__ float smem[];
    tile_body<NK, M, RING>(p, in, in_pitch, out, out_pitch, part, H, W, blockIdx.x * tw, blockIdx.y * th, tw, th, ncols,
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
        tile_body<NK, M, false>(sp, im.in, im.in_pitch, im.out, im.out_pitch, im.part, im.H, im.W, w.x0, w.y0, w.tw,
                                w.th, ncols, w.g, im.groups > 1, 2, smem);
    }
}

__global__ void bf_batch_finalize_kernel(const BatchImage *__restrict__ imgs, const int *__restrict__ list,
                                         const FilterParams *__restrict__ params) {
    const BatchImage im = imgs[list[blockIdx.z]];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= im.W || y >= im.H) return;
    const FilterParams &p = params[im.params];
    const size_t plane = (size_t)im.H * im.W, o = (size_t)y * im.W + x;
    float num = 0.f, den = 0.f;
    for (int g = 0; g < im.groups; ++g) {
        num += im.part[(size_t)(2 * g) * plane + o];
        den += im.part[(size_t)(2 * g + 1) * plane + o];
    }
    im.out[(size_t)y * im.out_pitch + x] = (den > p.den_eps) ? num / den + p.i_lo : im.in[(size_t)y * im.in_pitch + x];
}

// Sums the partial numerator / denominator planes of the term groups (in group
// order, so the result does not depend on scheduling) and divides.
__global__ void bf_finalize_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out,
                                   size_t out_pitch, const float *__restrict__ part, int H, int W, int groups,
                                   float den_eps, float i_lo) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t plane = (size_t)H * W, o = (size_t)y * W + x;
    float num = 0.f, den = 0.f;
    for (int g = 0; g < groups; ++g) {
        num += part[(size_t)(2 * g) * plane + o];
        den += part[(size_t)(2 * g + 1) * plane + o];
    }
    out[(size_t)y * out_pitch + x] = (den > den_eps) ? num / den + i_lo : in[(size_t)y * in_pitch + x];
}

// Kernel classes: windows per axis M and terms per group NK (NK * M <= 16, and
// no class spills registers).
struct KernelClass {
    int m, nk;
    const void *fn;       // tile kernel, edges recomputed
    const void *fn_ring;  // tile kernel with the per-column basis ring
    const void *batch_fn;
};

#define BF_CLASS(M, NK)                                                                                   \
    {M, NK, (const void *)bf_fused_kernel<NK, M, false>, (const void *)bf_fused_kernel<NK, M, true>,     \
     (const void *)bf_batch_kernel<NK, M>}
const KernelClass kClasses[] = {
    BF_CLASS(1, 16), BF_CLASS(1, 8), BF_CLASS(1, 4), BF_CLASS(1, 2),
    BF_CLASS(2, 8),  BF_CLASS(2, 4), BF_CLASS(2, 2), BF_CLASS(3, 5), BF_CLASS(3, 4), BF_CLASS(3, 2),
    BF_CLASS(4, 2),  BF_CLASS(5, 1), BF_CLASS(6, 1),
};
#undef BF_CLASS

const void *find_kernel(int m, int nk, bool ring) {
    for (const auto &c : kClasses)
        if (c.m == m && c.nk == nk) return ring ? c.fn_ring : c.fn;
    return nullptr;
}

size_t smem_bytes(int m, int nk, int ncols, int tw, int depth = 2) {
    return sizeof(float) * ((size_t)depth * m * nk * 4 * (ncols + 3) + (size_t)depth * nk * 2 * tw);
}

size_t ring_bytes(const FilterParams &p, int ncols) {
    return sizeof(float) * 5 * (size_t)(p.vhi - p.vlo + 2) * ncols;
}

int device_sms() {
    static int sms = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 152;
        }
        return n;
    }();
    return sms;
}

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

// Launch geometries ranked by a simple cost model: per-CTA work ~ columns x
// (rows + 0.3 x window span for the initialisation) x (edge cost + per-term
// cost), times the number of waves the grid needs on this device.
std::vector<TileConfig> tile_candidates(const FilterParams &p, int height, int width, int precision, int max_n) {
    (void)precision;
    const int sms = device_sms();
    const int vspan = p.vhi - p.vlo + 1;
    const int wpad = ((width + 7) / 8) * 8;
    std::vector<std::pair<double, TileConfig>> all;
    for (const auto &cls : kClasses) {
        if (cls.m != p.m) continue;
        const int groups = (p.nr + cls.nk - 1) / cls.nk;
        // column threads in whole warps; the tile takes what the halo leaves
        for (int ncols = 32; ncols + kScanThreads <= 512; ncols += 32) {
            int tw = ((ncols - 2 * p.rx) / 8) * 8;
            if (tw < 8) continue;
            tw = std::min(tw, wpad);
            if (ncols > ((tw + 2 * p.rx + 31) / 32) * 32) break;  // wider tiles than the image gain nothing
            for (int variant = 0; variant < 4; ++variant) {
                const int ring = variant & 1, depth = 2 + (variant >> 1);
                // the ring serves the output row too, so it must lie inside the window span
                if (ring && !(p.vlo <= 0 && p.vhi >= 0)) continue;
                const size_t smem = smem_bytes(p.m, cls.nk, ncols, tw, depth) + (ring ? ring_bytes(p, ncols) : 0);
                if (smem > 227 * 1024) continue;
                const int by_smem = (int)((228 * 1024) / (smem + 1024));
                const int by_threads = 2048 / (ncols + kScanThreads);
                const int by_regs = 65536 / (128 * (ncols + kScanThreads));
                const int cps = std::max(1, std::min({by_smem, by_threads, by_regs}));
                const double edge = (ring ? 60.0 + 12.0 * (2 * p.m + 1) : 60.0 * (2 * p.m + 1)) * (depth == 3 ? 0.9 : 1.0);
                for (int th : {16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 1024}) {
                    const int the = std::min(th, std::max(height, 1));
                    const long ctas = (long)((width + tw - 1) / tw) * ((height + the - 1) / the) * groups;
                    const double per_cta = (double)ncols * (the + 0.3 * vspan) * (edge + 40.0 * cls.nk * p.m);
                    const double waves = std::ceil((double)ctas / (sms * cps));
                    const double cost =
                        waves * per_cta * cps + (groups > 1 ? 16.0 * groups * (double)height * width : 0.0);
                    TileConfig tc;
                    tc.tw = tw;
                    tc.th = the;
                    tc.ncols = ncols;
                    tc.threads = ncols + kScanThreads;
                    tc.nk = cls.nk;
                    tc.groups = groups;
                    tc.ring = ring;
                    tc.depth = depth;
                    tc.smem = smem;
                    all.push_back({cost, tc});
                    if (the >= height) break;
                }
            }
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    std::vector<TileConfig> out;
    for (size_t i = 0; i < all.size() && (int)out.size() < max_n; ++i) out.push_back(all[i].second);
    return out;
}

TileConfig model_tile(const FilterParams &p, int height, int width, int precision) {
    std::vector<TileConfig> c = tile_candidates(p, height, width, precision, 1);
    return c.empty() ? TileConfig{} : c[0];
}

int device_sm_count() { return device_sms(); }

size_t batch_smem_bytes(int m, int nk, int ncols) { return smem_bytes(m, nk, ncols, ncols); }

int batch_class_nk(int m, int ncols) {
    for (const auto &c : kClasses)  // classes are listed with the largest term count first
        if (c.m == m && batch_smem_bytes(m, c.nk, ncols) <= 220 * 1024) return c.nk;
    return 0;
}

int batch_ctas_per_sm(int m, int nk, int ncols) {
    const size_t smem = batch_smem_bytes(m, nk, ncols) + sizeof(FilterParams) + 64;
    const int threads = ncols + kScanThreads;
    const int by_smem = (int)((228 * 1024) / (smem + 1024));
    const int by_threads = 2048 / threads;
    const int by_regs = 65536 / (128 * threads);
    return std::max(1, std::min({by_smem, by_threads, by_regs}));
}

bf_status launch_batch_class(int m, int nk, int ncols, const BatchImage *d_imgs, const FilterParams *d_params,
                             const WorkItem *d_items, int n_items, int *d_cursor, int grid, void *stream) {
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    const void *fn = nullptr;
    for (const auto &c : kClasses)
        if (c.m == m && c.nk == nk) fn = c.batch_fn;
    if (!fn) return fail(BF_ERR_UNSUPPORTED, "no batched kernel for this class");
    const size_t smem = batch_smem_bytes(m, nk, ncols);
    if (ncols + kScanThreads > 512 || smem > 220 * 1024) return fail(BF_ERR_UNSUPPORTED, "batched tile too large");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    void *args[] = {(void *)&d_imgs, (void *)&d_params, (void *)&d_items, (void *)&n_items, (void *)&d_cursor,
                    (void *)&ncols};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(ncols + kScanThreads), args, smem, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched filter launch");
    return BF_OK;
}

bf_status launch_batch_finalize(const BatchImage *d_imgs, const int *d_list, int n_list, int max_h, int max_w,
                                const FilterParams *d_params, void *stream) {
    if (n_list == 0) return BF_OK;
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    dim3 grid((max_w + 255) / 256, max_h, n_list);
    bf_batch_finalize_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_imgs, d_list, d_params);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batched finalize launch");
    return BF_OK;
}

size_t scratch_bytes(const TileConfig &tc, int height, int width) {
    return tc.groups > 1 ? sizeof(float) * 2 * (size_t)tc.groups * height * width : 0;
}

bf_status launch_filter(const FilterParams &p, int precision, int kahan, const TileConfig &tc, const float *d_in,
                        size_t in_pitch, float *d_out, size_t out_pitch, float *d_scratch, int height, int width,
                        void *stream) {
    (void)precision;
    (void)kahan;
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    const void *fn = find_kernel(p.m, tc.nk, tc.ring != 0);
    if (!fn || tc.ncols <= 0) return fail(BF_ERR_UNSUPPORTED, "no kernel class for this plan and image");
    if (tc.threads > 512) return fail(BF_ERR_UNSUPPORTED, "horizontal reach too large for one CTA");
    if (tc.smem > 227 * 1024) return fail(BF_ERR_UNSUPPORTED, "tile needs more than 227 KB of shared memory");
    if (tc.groups > 1 && !d_scratch) return fail(BF_ERR_INVALID_ARG, "missing scratch for grouped launch");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc.smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    dim3 grid((width + tc.tw - 1) / tc.tw, (height + tc.th - 1) / tc.th, tc.groups);
    int tw = tc.tw, th = tc.th, ncols = tc.ncols, H = height, W = width, depth = tc.depth;
    const float *in = d_in;
    float *out = d_out, *part = d_scratch;
    FilterParams pp = p;
    void *args[] = {(void *)&in, (void *)&in_pitch, (void *)&out, (void *)&out_pitch, (void *)&part, (void *)&H,
                    (void *)&W, (void *)&tw, (void *)&th, (void *)&ncols, (void *)&depth, (void *)&pp};
    e = cudaLaunchKernel(fn, grid, dim3(tc.threads), args, tc.smem, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    if (tc.groups > 1) {
        if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
        dim3 fg((width + 255) / 256, height);
        bf_finalize_kernel<<<fg, 256, 0, (cudaStream_t)stream>>>(d_in, in_pitch, d_out, out_pitch, d_scratch, height,
                                                                 width, tc.groups, p.den_eps, p.i_lo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
    }
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
