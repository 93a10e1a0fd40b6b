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
#include <cstdlib>
#include <string>
#include <vector>

#include "bf_tile.cuh"

namespace bfi {

namespace {

std::atomic<int> g_fail_launches{0};

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

// All kernel classes of a family, largest term count first within a window count.
struct ClassList {
    std::vector<KernelClass> v[2];  // [packed]
    ClassList() {
        auto add = [&](int f, const KernelClass *a, int n) { v[f].insert(v[f].end(), a, a + n); };
        add(1, kClassesM1, kNumClassesM1);
        add(1, kClassesM2, kNumClassesM2);
        add(1, kClassesM3, kNumClassesM3);
        add(1, kClassesM4to6, kNumClassesM4to6);
        add(0, kScalarClassesM1M2, kNumScalarClassesM1M2);
        add(0, kScalarClassesM3to6, kNumScalarClassesM3to6);
    }
};
const std::vector<KernelClass> &classes(bool packed) {
    static ClassList c;
    return c.v[packed ? 1 : 0];
}

const void *find_kernel(int m, int nk, bool ring, bool packed) {
    for (const auto &c : classes(packed))
        if (c.m == m && c.nk == nk) return c.fn[ring ? 1 : 0];
    return nullptr;
}

// The hybrid layout's kernel of class (m, nk), nullptr where none is built (M = 1 and 2).
const void *find_hybrid_kernel(int m, int nk, bool ring) {
    for (const auto *t : {kHybridClassesM1, kHybridClassesM2}) {
        const int n = t == kHybridClassesM1 ? kNumHybridClassesM1 : kNumHybridClassesM2;
        for (int i = 0; i < n; ++i)
            if (t[i].m == m && t[i].nk == nk) return t[i].fn[ring ? 1 : 0];
    }
    return nullptr;
}

// The pre-pass variant `pre` (1 fp32, 2 fp16, 3 bf16) of packed class (m, nk), nullptr where none is built.
const void *find_pre_kernel(int m, int nk, int pre) {
    if (pre < 1 || pre > 3) return nullptr;
    for (const auto *t : {kPreClassesM1, kPreClassesM2M3, kPreClassesM4to6}) {
        const int n = t == kPreClassesM1 ? kNumPreClassesM1 : t == kPreClassesM2M3 ? kNumPreClassesM2M3 : kNumPreClassesM4to6;
        for (int i = 0; i < n; ++i)
            if (t[i].m == m && t[i].nk == nk) return t[i].fn[pre - 1];
    }
    return nullptr;
}

const ZKernelClass *find_zclass(int m, int nk) {
    for (const auto *t : {kZClassesM1M2, kZClassesM3to6}) {
        const int n = t == kZClassesM1M2 ? kNumZClassesM1M2 : kNumZClassesM3to6;
        for (int i = 0; i < n; ++i)
            if (t[i].m == m && t[i].nk == nk) return &t[i];
    }
    return nullptr;
}

// The 3-D form's persistent slice kernel of class (m, nk): zmode 1 the range box, 2 the Haar range
// series' weights (nullptr where the class has none); `threads` <= 256 picks the register-bounded kernel
// where the class has one, and for the Haar series `threads` <= 512 its 512-thread form.  *regs: the
// registers per thread the cost model assumes.
const void *find_zkernel(int m, int nk, int zmode, int threads = 512, int *regs = nullptr) {
    const ZKernelClass *c = find_zclass(m, nk);
    if (regs) *regs = 128;
    if (!c) return nullptr;
    const void *small = zmode == 2 ? c->haar_small : c->box_small;
    if (threads <= 256 && small) {
        if (regs) *regs = zmode == 2 ? c->haar_small_regs : c->box_small_regs;
        return small;
    }
    if (zmode == 2 && threads <= 512 && c->haar_mid) {
        if (regs) *regs = c->haar_small_regs;
        return c->haar_mid;
    }
    return zmode == 2 ? c->haar : c->box;
}

// Bytes of the Haar range series' weight table in the slice kernel's shared memory (16-byte multiple).
size_t zweights_bytes(const FilterParams &p) {
    return p.zmode == 2 ? ((sizeof(float) * (2 * (size_t)p.rz + 1) + 15) & ~(size_t)15) : 0;
}

// The 3-D form's work list: one CTA per tile marks the slices of the tile's output pixels in a shared
// bitmap (the same slice rule as the tile body) and appends one item (tile, slice) per marked slice at
// the position counters[0] hands out.  At most `cap` items are stored.
__global__ void __launch_bounds__(256) bf_zlist_kernel(const float *__restrict__ in, size_t in_pitch, int H, int W,
                                                       int tw, int th, int tiles_x, int2 *__restrict__ items, int cap,
                                                       int *__restrict__ counters,
                                                       const __grid_constant__ FilterParams p) {
    __shared__ unsigned bits[kMaxZBins / 32];
    __shared__ int woff[kMaxZBins / 32];
    __shared__ int base;
    const int tile = blockIdx.x, ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int x0 = tx * tw, y0 = ty * th, nx = min(tw, W - x0), ny = min(th, H - y0);
    const int words = (p.zbins + 31) >> 5;
    for (int i = threadIdx.x; i < words; i += blockDim.x) bits[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int r = i / nx, c = i - r * nx;
        const int n = z_slice(__ldg(in + (size_t)(y0 + r) * in_pitch + x0 + c) - p.i_lo, p);
        atomicOr(&bits[n >> 5], 1u << (n & 31));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < words; ++w) {
            woff[w] = t;
            t += __popc(bits[w]);
        }
        base = atomicAdd(counters, t);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        unsigned b = bits[w];
        int o = base + woff[w];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            if (o < cap) items[o] = make_int2(tile, w * 32 + bit);
            ++o;
        }
    }
}

// The two launches of a hybrid layout: pk, the packed groups (windows of NK consecutive frequencies, slots
// zero-weight where the selection has no term): the window from the lowest selected frequency, then every later
// window of NK consecutive selected frequencies, taken greedily in ascending order; sc, the other selected terms
// (the scalar family's term set).  Returns the number of packed groups (0: no hybrid layout: nothing left for
// the scalar family, or more than kMaxSlots packed slots).
int hybrid_split(const FilterParams &p, int nk, FilterParams &pk, FilterParams &sc) {
    if (nk < 1 || nk > kMaxSlots || p.nr < 1) return 0;
    pk = p;
    sc = p;
    pk.nr = 0;
    sc.nr = 0;
    int gp = 0;
    for (int i = 0; i < p.nr;) {
        const bool dense = i + nk <= p.nr && p.k[i + nk - 1] - p.k[i] == nk - 1;
        if (i == 0 || dense) {
            if (pk.nr + nk > kMaxSlots) return 0;
            const int k0 = p.k[i];
            for (int s = 0; s < nk; ++s) {
                pk.k[pk.nr + s] = k0 + s;
                if (i < p.nr && p.k[i] == k0 + s) {
                    pk.a[pk.nr + s] = p.a[i];
                    ++i;
                } else {
                    pk.a[pk.nr + s] = 0.f;
                }
            }
            pk.nr += nk;
            ++gp;
        } else {
            sc.k[sc.nr] = p.k[i];
            sc.a[sc.nr] = p.a[i];
            ++sc.nr;
            ++i;
        }
    }
    return sc.nr > 0 ? gp : 0;
}

// The selection has gaps (the packed family then pads groups with zero-weight frequencies).
bool gapped_terms(const FilterParams &p) { return p.k[p.nr - 1] - p.k[0] + 1 != p.nr; }

// Shared memory of a tile: the exchange, the output weights (not with the packed family's ring, which
// recomputes them from the ring) and the ring.
size_t smem_bytes(int m, int nk, int ncols, int tw, int depth = 2, bool weights = true) {
    return sizeof(float) * ((size_t)depth * (m * nk * 4 + 2) * (ncols + 2) + (weights ? (size_t)depth * nk * 2 * tw : 0));
}

// The ring: (v, cos, sin of the base angle, pad) per row and column, plus the anchor (cos, sin)(pi k0 t) when
// some term group starts at k0 >= 2 (the scalar family always keeps it).
size_t ring_bytes(const FilterParams &p, int ncols, bool anchor = true) {
    return (16 + (anchor ? 8 : 0)) * (size_t)(p.vhi - p.vlo + 2) * ncols;
}

// Some group of the launch's term layout starts at frequency 2 or more.
bool groups_need_anchor(const FilterParams &p, int nk, bool packed) {
    if (!packed) return true;
    for (int i = 0; i < p.nr;) {
        const int k0 = p.k[i];
        if (k0 >= 2) return true;
        while (i < p.nr && p.k[i] < k0 + nk) ++i;
    }
    return false;
}

// Dynamic shared memory a geometry needs (hybrid: what both of its kernels need).
size_t tile_smem_bytes(const FilterParams &p, int nk, int ncols, int tw, int depth, int ring, int packed) {
    const bool pring = ring && packed == 1;
    return smem_bytes(p.m, nk, ncols, tw, depth, !pring) +
           (ring ? ring_bytes(p, ncols, packed != 1 || groups_need_anchor(p, nk, true)) : 0);
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

// Brute-force Eq. (1) with the range kernel read from a table (the look-up-table baseline of Sec. V,
// Case 2): lut[n] = K_r(n step), n = 0 .. levels - 1, read at the entry nearest to |I(x) - I(y)| (the
// index rounded to nearest-even in fp32); spatial weights from a (2R + 1)^2 table.  A 32 x 8 block of
// outputs with its (32 + 2R) x (8 + 2R) input tile, the two tables and the tile in shared memory.
__global__ void __launch_bounds__(256) bf_bft_kernel(const float *__restrict__ in, size_t in_pitch,
                                                     float *__restrict__ out, size_t out_pitch, int H, int W,
                                                     int spatial, float sigma_s, int R, int range, float sigma_r,
                                                     int levels, float step, float inv_step) {
    extern __shared__ float sm[];
    const int sw_n = (2 * R + 1) * (2 * R + 1);
    const int pw = 32 + 2 * R, ph = 8 + 2 * R;
    float *lut = sm, *sw = sm + levels, *tile = sw + sw_n;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int n = tid; n < levels; n += 256) {
        const float t = n * step;
        lut[n] = range == BF_KERNEL_GAUSSIAN      ? expf(-t * t / (2.f * sigma_r * sigma_r))
                 : range == BF_KERNEL_EXPONENTIAL ? expf(-t / sigma_r)
                                                  : (t <= sigma_r ? 1.f : 0.f);
    }
    for (int i = tid; i < sw_n; i += 256) {
        const int dy = i / (2 * R + 1) - R, dx = i % (2 * R + 1) - R;
        const float r2 = (float)(dx * dx + dy * dy);
        sw[i] = spatial == BF_KERNEL_BOX           ? 1.f
                : spatial == BF_KERNEL_EXPONENTIAL ? expf(-sqrtf(r2) / sigma_s)
                                                   : expf(-r2 / (2.f * sigma_s * sigma_s));
    }
    const int xb = blockIdx.x * 32 - R, yb = blockIdx.y * 8 - R;
    for (int i = tid; i < pw * ph; i += 256) {
        const int gy = yb + i / pw, gx = xb + i % pw;
        tile[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? __ldg(in + (size_t)gy * in_pitch + gx) : 0.f;
    }
    __syncthreads();
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const float *c = tile + (threadIdx.y + R) * pw + threadIdx.x + R;
    const float ix = c[0];
    // neighbours outside the image are excluded (the loop bounds stop at the border)
    const int dy0 = max(-R, -y), dy1 = min(R, H - 1 - y), dx0 = max(-R, -x), dx1 = min(R, W - 1 - x);
    float num = 0.f, den = 0.f;
    for (int dy = dy0; dy <= dy1; ++dy) {
        const float *row = c + dy * pw;
        const float *swr = sw + (dy + R) * (2 * R + 1) + R;
        for (int dx = dx0; dx <= dx1; ++dx) {
            const float iy = row[dx];
            const int n = min(__float2int_rn(fabsf(ix - iy) * inv_step), levels - 1);
            const float wgt = swr[dx] * lut[n];
            num = fmaf(wgt, iy, num);
            den += wgt;
        }
    }
    out[(size_t)y * out_pitch + x] = num / den;
}

__global__ void bf_exact_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out,
                                size_t out_pitch, int H, int W, int spatial, float sigma_s, int R, int range,
                                float sigma_r) {
    const float inv2ss = 1.0f / (2.0f * sigma_s * sigma_s);
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
            const float r2 = (float)(dx * dx + dy * dy);
            const float ks = spatial == BF_KERNEL_BOX           ? 1.f
                             : spatial == BF_KERNEL_EXPONENTIAL ? expf(-sqrtf(r2) / sigma_s)
                                                                : expf(-r2 * inv2ss);
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

// Term groups of a launch: packed family (1), greedy windows of NK consecutive frequencies; scalar family (0),
// consecutive slices of NK selected terms; hybrid (2), the packed windows of hybrid_split, then the other selected
// terms in slices of NK in the scalar family.
int family_groups(const FilterParams &p, int nk, int packed) {
    if (packed == 2) {
        FilterParams pk, sc;
        const int gp = hybrid_split(p, nk, pk, sc);
        return gp > 0 ? gp + (sc.nr + nk - 1) / nk : 0;
    }
    return packed ? term_groups(p, nk) : (p.nr + nk - 1) / nk;
}

// The input range check of bf_debug_range_checks: pixels outside [lo, hi] (NaN included), counted into one
// per-device counter.
__device__ unsigned long long g_out_of_range;

__global__ void bf_range_count_kernel(const float *__restrict__ in, size_t in_pitch, int H, int W, float lo, float hi) {
    unsigned long long n = 0;
    const size_t total = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float v = __ldg(in + (i / W) * in_pitch + i % W);
        n += (v >= lo && v <= hi) ? 0 : 1;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&g_out_of_range, n);
}

std::atomic<int> g_range_checks{-1};  // -1: not yet read from the environment

bool debug_range_checks() {
    int v = g_range_checks.load();
    if (v < 0) {
        const char *e = std::getenv("BF_DEBUG_RANGE");
        int want = (e && e[0] == '1') ? 1 : 0;
        g_range_checks.compare_exchange_strong(v, want);
        v = g_range_checks.load();
    }
    return v > 0;
}

void debug_set_range_checks(bool on) { g_range_checks.store(on ? 1 : 0); }

bf_status count_out_of_range(const float *d_in, size_t in_pitch, int h, int w, float lo, float hi, void *stream,
                             unsigned long long *count) {
    cudaStream_t s = (cudaStream_t)stream;
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_out_of_range);
    if (e == cudaSuccess) e = cudaMemsetAsync(addr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "range check");
    const int blocks = (int)std::min<size_t>(((size_t)h * w + 255) / 256, (size_t)device_sms() * 8);
    bf_range_count_kernel<<<std::max(blocks, 1), 256, 0, s>>>(d_in, in_pitch, h, w, lo, hi);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, addr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "range check");
    return BF_OK;
}

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
    // the scalar family competes only for gapped selections (otherwise it does the same groups, slower);
    // the 3-D form runs the packed family without the ring
    const bool z3d = p.zbins > 0;
    // families: packed (1); for gapped selections also hybrid (2: windows of consecutive frequencies packed, the
    // other terms scalar) and scalar (0)
    const bool gapped = gapped_terms(p) && !z3d;
    for (int packed : {1, 2, 0})
    for (const auto &cls : classes(packed != 0)) {
        if (packed != 1 && !gapped) break;
        if (cls.m != p.m) continue;
        if (z3d && !find_zkernel(cls.m, cls.nk, p.zmode)) continue;  // the Haar series runs NK = 2 only
        const int groups = family_groups(p, cls.nk, packed);
        if (packed == 1 && groups * cls.nk > kMaxSlots) continue;
        if (packed == 2 && (groups < 2 || !find_hybrid_kernel(cls.m, cls.nk, false))) continue;
        // per term and window: the scalar family has no pairing; hybrid: the mean over its packed and scalar groups
        double term_cost = packed == 1 ? 40.0 : 60.0;
        if (packed == 2) {
            FilterParams pk, ps;
            const int gp = hybrid_split(p, cls.nk, pk, ps);
            term_cost = (40.0 * gp + 60.0 * (groups - gp)) / groups;
        }
        // column threads in whole warps; the tile takes what the halo leaves
        for (int ncols = 32; ncols + kScanThreads <= 512; ncols += 32) {
            int tw = ((ncols - 2 * p.rx) / 8) * 8;
            if (tw < 8) continue;
            tw = std::min(tw, wpad);
            if (ncols > ((tw + 2 * p.rx + 31) / 32) * 32) break;  // wider tiles than the image gain nothing
            for (int variant = 0; variant < 8; ++variant) {
                // variants 4..7: the basis inputs read from the pre-pass buffer in the plan's storage precision
                const int ring = variant & 1, depth = 2 + ((variant >> 1) & 1);
                const int pre = variant < 4 ? 0 : precision == BF_PREC_FP16 ? 2 : precision == BF_PREC_BF16 ? 3 : 1;
                if (!pre_allowed(precision, pre)) continue;
                if (pre && (ring || z3d || packed != 1 || !find_pre_kernel(cls.m, cls.nk, pre))) continue;
                if (packed == 2 && !find_hybrid_kernel(cls.m, cls.nk, ring)) continue;
                if (ring && z3d) continue;
                // the ring serves the output row too, so it must lie inside the window span
                if (ring && !(p.vlo <= 0 && p.vhi >= 0)) continue;
                // the packed ring's output phase reads row y - lag back from the ring: lag <= 1 - vlo
                if (ring && packed && depth - 1 > 1 - p.vlo) continue;
                const size_t smem = tile_smem_bytes(p, cls.nk, ncols, tw, depth, ring, packed);
                // the slice kernel keeps a few bytes of static shared memory besides the tile's
                if (smem + zweights_bytes(p) > 227 * 1024 - (z3d ? 256 : 0)) continue;
                const int by_smem = (int)((228 * 1024) / (smem + 1024));
                const int by_threads = 2048 / (ncols + kScanThreads);
                int regs = 128;
                if (z3d) find_zkernel(cls.m, cls.nk, p.zmode, ncols + kScanThreads, &regs);
                const int by_regs = 65536 / (regs * (ncols + kScanThreads));
                const int cps = std::max(1, std::min({by_smem, by_threads, by_regs}));
                // three exchange buffers save a barrier per row; the slice kernel measured no gain from them
                // (pre-pass variants: ranked just behind the in-kernel basis of the same geometry)
                const double edge = (ring ? 60.0 + 12.0 * (2 * p.m + 1) : 60.0 * (2 * p.m + 1)) *
                                    (depth == 3 && !z3d ? 0.9 : 1.0) * (pre == 1 ? 1.02 : 1.0);
                for (int th : {16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 1024}) {
                    const int the = std::min(th, std::max(height, 1));
                    const long tiles = (long)((width + tw - 1) / tw) * ((height + the - 1) / the);
                    const long ctas = tiles * groups;
                    const double per_cta = (double)ncols * (the + 0.3 * vspan) * (edge + term_cost * cls.nk * p.m);
                    const double waves = std::ceil((double)ctas / (sms * cps));
                    double cost = waves * per_cta * cps + (groups > 1 ? 16.0 * groups * (double)height * width : 0.0);
                    if (z3d) {
                        // the 3-D form passes over a tile once per distinct slice among its output pixels; the
                        // count is modelled as 7.5 (tw th)^0.27 (a fit on noisy piecewise-constant images),
                        // at most zbins.  The persistent launch balances the items, so waves do not matter;
                        // two resident CTAs hide latency better, fewer than 256 resident threads worse.
                        const double slices = std::min((double)p.zbins, 7.5 * std::pow((double)tw * the, 0.27));
                        const int resident = cps * (ncols + kScanThreads);
                        const double occ = (cps > 1 ? 1.3 : 1.0) / (resident < 256 ? 1.35 : 1.0);
                        cost = (double)ctas * slices * per_cta / (sms * occ) +
                               (groups > 1 ? 16.0 * groups * (double)height * width : 0.0);
                    }
                    TileConfig tc;
                    tc.tw = tw;
                    tc.th = the;
                    tc.ncols = ncols;
                    tc.threads = ncols + kScanThreads;
                    tc.nk = cls.nk;
                    tc.groups = groups;
                    tc.ring = ring;
                    tc.depth = depth;
                    tc.packed = packed;
                    tc.smem = smem;
                    tc.pre = pre;
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

// The model's pick.
TileConfig model_tile(const FilterParams &p, int height, int width, int precision) {
    const auto c = tile_candidates(p, height, width, precision, 1);
    return c.empty() ? TileConfig{} : c[0];
}

int device_sm_count() { return device_sms(); }

size_t batch_smem_bytes(int m, int nk, int ncols) { return smem_bytes(m, nk, ncols, ncols); }

int batch_class_nk(int m, int ncols, bool packed, int cap) {
    for (const auto &c : classes(packed))  // classes are listed with the largest term count first
        if (c.m == m && (cap <= 0 || c.nk <= cap) && batch_smem_bytes(m, c.nk, ncols) <= 220 * 1024) return c.nk;
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

bf_status launch_batch_class(int m, int nk, bool packed, int ncols, const BatchImage *d_imgs, const FilterParams *d_params,
                             const WorkItem *d_items, int n_items, int *d_cursor, int grid, void *stream) {
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    const void *fn = nullptr;
    for (const auto &c : classes(packed))
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

int term_groups(const FilterParams &p, int nk) {
    int groups = 0;
    for (int i = 0; i < p.nr;) {
        const int k0 = p.k[i];
        ++groups;
        while (i < p.nr && p.k[i] < k0 + nk) ++i;
    }
    return groups;
}

bool term_layout(const FilterParams &p, int nk, FilterParams &out) {
    out = p;
    int slot = 0;
    for (int i = 0; i < p.nr;) {
        const int k0 = p.k[i];
        if (slot + nk > kMaxSlots) return false;
        for (int s = 0; s < nk; ++s) {
            out.k[slot + s] = k0 + s;
            if (i < p.nr && p.k[i] == k0 + s) {
                out.a[slot + s] = p.a[i];
                ++i;
            } else {
                out.a[slot + s] = 0.f;
            }
        }
        slot += nk;
    }
    out.nr = slot;
    return true;
}

void fill_info(const TileConfig &tc, int height, int width, int *info, int zbins) {
    info[0] = tc.tw;
    info[1] = tc.th;
    info[2] = tc.threads;
    info[3] = tc.nk;
    info[4] = tc.groups;
    // kernel launches: the basis pre-pass, the filter (3-D form: the slice list and the slice kernel), the
    // finalize of a grouped launch
    info[5] = (tc.pre ? 1 : 0) + (zbins > 0 ? 2 : 1) + (tc.groups > 1 ? 1 : 0);
    info[6] = (int)tc.smem;
    info[7] = (int)(scratch_bytes(tc, height, width, zbins) >> 10);
    info[8] = tc.ring ? 1 : 0;
    info[9] = tc.depth;
    info[10] = tc.ncols;
    info[11] = tc.packed;
    info[12] = tc.pre;
}

namespace {
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t partial_bytes(const TileConfig &tc, int height, int width) {
    return tc.groups > 1 ? sizeof(float) * 2 * (size_t)tc.groups * height * width : 0;
}

// Work items of the 3-D form: each tile holds at most min(zbins, its pixels) slices.
size_t zlist_cap(const TileConfig &tc, int height, int width, int zbins) {
    if (tc.tw < 1 || tc.th < 1) return 0;
    const size_t tiles = (size_t)((width + tc.tw - 1) / tc.tw) * ((height + tc.th - 1) / tc.th);
    return std::min(tiles * (size_t)zbins, (size_t)height * width);
}
}  // namespace

// The pre-pass buffer of a PRE geometry: one element per pixel (16 bytes fp32, 8 bytes 16-bit), after the
// partial planes.
size_t pre_bytes(const TileConfig &tc, int height, int width) {
    return tc.pre ? (size_t)(tc.pre == 1 ? 16 : 8) * height * width : 0;
}

size_t scratch_bytes(const TileConfig &tc, int height, int width, int zbins) {
    const size_t part = partial_bytes(tc, height, width);
    if (tc.pre) return align256(part) + pre_bytes(tc, height, width);
    if (zbins <= 0) return part;
    // [partial planes][counters: 2 ints, 256 bytes reserved][items: int2 each]
    return align256(part) + 256 + sizeof(int2) * zlist_cap(tc, height, width, zbins);
}

// The 3-D form (Sec. IV-D): the work list of (tile, slice) items, the persistent slice kernel over it, and
// the finalize of a grouped launch.  Geometry already checked by launch_filter.
bf_status launch_filter_z3d(const FilterParams &p, const TileConfig &tc, const float *d_in, size_t in_pitch,
                            float *d_out, size_t out_pitch, float *d_scratch, int height, int width, void *stream) {
    if (p.zbins < 2 || p.zbins > kMaxZBins || p.rz < 0) return fail(BF_ERR_INVALID_ARG, "bad slice count");
    if (tc.ring || !tc.packed) return fail(BF_ERR_INVALID_ARG, "the 3-D form runs the packed family without the ring");
    if (p.zmode == 2 && (!p.zw || 2 * p.rz + 1 > kMaxZWeights))
        return fail(BF_ERR_INVALID_ARG, "missing or oversized Haar range weight table");
    const size_t zwb = zweights_bytes(p), smem = tc.smem + zwb;
    if (smem > 227 * 1024 - 256) return fail(BF_ERR_UNSUPPORTED, "tile too large for the slice kernel");
    const void *fn = find_zkernel(p.m, tc.nk, p.zmode, tc.threads);
    if (!fn) return fail(BF_ERR_UNSUPPORTED, "no slice kernel for this class");
    FilterParams pp;
    if (!term_layout(p, tc.nk, pp) || pp.nr != tc.groups * tc.nk)
        return fail(BF_ERR_INVALID_ARG, "launch geometry does not match the plan's term groups");
    cudaStream_t s = (cudaStream_t)stream;
    const int tiles_x = (width + tc.tw - 1) / tc.tw, tiles_y = (height + tc.th - 1) / tc.th;
    const size_t cap_sz = zlist_cap(tc, height, width, p.zbins);
    if (cap_sz > (size_t)INT32_MAX / std::max(tc.groups, 1) || (size_t)tiles_x * tiles_y > (size_t)INT32_MAX)
        return fail(BF_ERR_UNSUPPORTED, "image too large for the slice work list");
    int cap = (int)cap_sz;
    char *base = reinterpret_cast<char *>(d_scratch);
    float *part = tc.groups > 1 ? d_scratch : nullptr;
    int *counters = reinterpret_cast<int *>(base + align256(partial_bytes(tc, height, width)));
    int2 *items = reinterpret_cast<int2 *>(reinterpret_cast<char *>(counters) + 256);
    cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "slice counters");
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    bf_zlist_kernel<<<tiles_x * tiles_y, 256, 0, s>>>(d_in, in_pitch, height, width, tc.tw, tc.th, tiles_x, items,
                                                      cap, counters, pp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "slice list launch");
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int cps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, fn, tc.threads, smem);
    if (e != cudaSuccess || cps < 1) {
        cudaGetLastError();
        cps = 1;
    }
    const long want = (long)cap * tc.groups;
    const int grid = (int)std::max(1L, std::min((long)device_sms() * cps, want));
    int tw = tc.tw, th = tc.th, ncols = tc.ncols, H = height, W = width, depth = tc.depth, groups = tc.groups;
    int max_iter = cap * tc.groups, zw_off = (int)(tc.smem / sizeof(float));
    const float *in = d_in;
    float *out = d_out;
    static thread_local ZWeights zwp;  // the table travels as a kernel parameter (copied at launch)
    if (p.zmode == 2) std::copy(p.zw, p.zw + 2 * p.rz + 1, zwp.w);
    void *args[] = {(void *)&in, (void *)&in_pitch, (void *)&out, (void *)&out_pitch, (void *)&part, (void *)&H,
                    (void *)&W, (void *)&tw, (void *)&th, (void *)&ncols, (void *)&depth, (void *)&tiles_x,
                    (void *)&groups, (void *)&items, (void *)&cap, (void *)&counters, (void *)&max_iter,
                    (void *)&zw_off, (void *)&pp, (void *)&zwp};
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    e = cudaLaunchKernel(fn, dim3(grid), dim3(tc.threads), args, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "slice filter launch");
    if (tc.groups > 1) {
        if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
        dim3 fg((width + 255) / 256, height);
        bf_finalize_kernel<<<fg, 256, 0, s>>>(d_in, in_pitch, d_out, out_pitch, d_scratch, height, width, tc.groups,
                                               p.den_eps, p.i_lo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
    }
    return BF_OK;
}

bf_status launch_filter(const FilterParams &p, int precision, int kahan, const TileConfig &tc, const float *d_in,
                        size_t in_pitch, float *d_out, size_t out_pitch, float *d_scratch, int height, int width,
                        void *stream, int cache_mode) {
    (void)precision;
    (void)kahan;
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    if (tc.pre < 0 || tc.pre > 3 || (tc.pre && (tc.packed != 1 || tc.ring || p.zbins > 0 || cache_mode)))
        return fail(BF_ERR_INVALID_ARG, "malformed launch geometry (pre-pass variant)");
    if (tc.packed < 0 || tc.packed > 2 || (tc.packed == 2 && (p.zbins > 0 || cache_mode)))
        return fail(BF_ERR_INVALID_ARG, "malformed launch geometry (family)");
    const void *fn = tc.pre                ? find_pre_kernel(p.m, tc.nk, tc.pre)
                     : tc.packed == 2      ? find_hybrid_kernel(p.m, tc.nk, tc.ring != 0)
                                           : find_kernel(p.m, tc.nk, tc.ring != 0, tc.packed != 0);
    if (!fn || tc.ncols <= 0) return fail(BF_ERR_UNSUPPORTED, "no kernel class for this plan and image");
    if (tc.threads > 512) return fail(BF_ERR_UNSUPPORTED, "horizontal reach too large for one CTA");
    // the tile body needs whole warps of column threads (its two scan warps meet on a 64-thread named
    // barrier) and tile widths in blocks of 8 columns; geometries from a cache file are checked here
    if (tc.ncols % 32 != 0 || tc.threads != tc.ncols + kScanThreads || tc.tw < 8 || tc.tw % 8 != 0 ||
        tc.tw + 2 * p.rx > tc.ncols || tc.th < 1 || (tc.depth != 2 && tc.depth != 3) || tc.nk < 1 ||
        (tc.packed && tc.nk % 2 != 0))
        return fail(BF_ERR_INVALID_ARG, "malformed launch geometry");
    if (tc.smem > 227 * 1024) return fail(BF_ERR_UNSUPPORTED, "tile needs more than 227 KB of shared memory");
    if (p.zbins == 0 && tc.smem < tile_smem_bytes(p, tc.nk, tc.ncols, tc.tw, tc.depth, tc.ring, tc.packed))
        return fail(BF_ERR_INVALID_ARG, "malformed launch geometry (shared memory below the tile's)");
    if ((tc.groups > 1 || cache_mode || p.zbins > 0 || tc.pre) && !d_scratch)
        return fail(BF_ERR_INVALID_ARG, "missing scratch for grouped launch");
    if (cache_mode && tc.packed != 1) return fail(BF_ERR_INVALID_ARG, "the pre-computation runs the packed family");
    if (p.zbins > 0) {
        if (cache_mode) return fail(BF_ERR_UNSUPPORTED, "the 3-D form has no pre-computation cache");
        return launch_filter_z3d(p, tc, d_in, in_pitch, d_out, out_pitch, d_scratch, height, width, stream);
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc.smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    dim3 grid((width + tc.tw - 1) / tc.tw, (height + tc.th - 1) / tc.th, tc.groups);
    int tw = tc.tw, th = tc.th, ncols = tc.ncols, H = height, W = width, depth = tc.depth;
    const float *in = d_in;
    float *out = d_out, *part = d_scratch;
    FilterParams pp = p;  // scalar family: the selection as the plan holds it
    if (tc.packed == 2) {
        // hybrid: one launch over all groups, the packed tile body for groups 0 .. gp - 1 (the windows of NK
        // consecutive frequencies, their partial planes first), the scalar one for the others, then the finalize
        FilterParams ps;
        const int gp = hybrid_split(p, tc.nk, pp, ps);
        if (gp < 1 || tc.groups < 2 || tc.groups != family_groups(p, tc.nk, 2))
            return fail(BF_ERR_INVALID_ARG, "launch geometry does not match the plan's term groups");
        void *args_h[] = {(void *)&in,  (void *)&in_pitch, (void *)&out,   (void *)&out_pitch, (void *)&part,
                          (void *)&H,   (void *)&W,        (void *)&tw,    (void *)&th,        (void *)&ncols,
                          (void *)&depth, (void *)&gp,     (void *)&pp,    (void *)&ps};
        e = cudaLaunchKernel(fn, grid, dim3(tc.threads), args_h, tc.smem, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "filter launch (hybrid)");
        if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
        dim3 fg((width + 255) / 256, height);
        bf_finalize_kernel<<<fg, 256, 0, (cudaStream_t)stream>>>(d_in, in_pitch, d_out, out_pitch, d_scratch, height,
                                                                 width, tc.groups, p.den_eps, p.i_lo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
        return BF_OK;
    }
    if (tc.packed ? !term_layout(p, tc.nk, pp) || pp.nr != tc.groups * tc.nk
                  : tc.groups != (p.nr + tc.nk - 1) / tc.nk)
        return fail(BF_ERR_INVALID_ARG, "launch geometry does not match the plan's term groups");
    int mode = cache_mode ? cache_mode : tc.groups > 1 ? kModePartial : kModeFinal;
    // the pre-pass: basis inputs of every pixel, after the partial planes in the scratch
    const void *pre = nullptr;
    if (tc.pre) {
        void *buf = reinterpret_cast<char *>(d_scratch) + align256(partial_bytes(tc, height, width));
        pre = buf;
        if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
        const int blocks = (int)std::max<size_t>(1, std::min<size_t>(((size_t)height * width + 255) / 256,
                                                                    (size_t)device_sms() * 8));
        cudaStream_t s = (cudaStream_t)stream;
        if (tc.pre == 1)
            bf_basis_kernel<1><<<blocks, 256, 0, s>>>(d_in, in_pitch, buf, height, width, p.inv_p, p.inv_p_lo, p.i_lo);
        else if (tc.pre == 2)
            bf_basis_kernel<2><<<blocks, 256, 0, s>>>(d_in, in_pitch, buf, height, width, p.inv_p, p.inv_p_lo, p.i_lo);
        else
            bf_basis_kernel<3><<<blocks, 256, 0, s>>>(d_in, in_pitch, buf, height, width, p.inv_p, p.inv_p_lo, p.i_lo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "basis pre-pass launch");
    }
    void *args[] = {(void *)&in,  (void *)&in_pitch, (void *)&out,   (void *)&out_pitch, (void *)&part,
                    (void *)&H,   (void *)&W,        (void *)&tw,    (void *)&th,        (void *)&ncols,
                    (void *)&depth, (void *)&mode,   (void *)&pp,    (void *)&pre};
    e = cudaLaunchKernel(fn, grid, dim3(tc.threads), args, tc.smem, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    if (tc.groups > 1 && !cache_mode) {
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
                                                             sigma_s, radius, range, sigma_r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "exact launch");
    return BF_OK;
}

bf_status launch_exact_lut(const float *d_in, size_t in_pitch, float *d_out, size_t out_pitch, int height, int width,
                           int spatial, float sigma_s, int radius, int range, float sigma_r, float data_range,
                           int levels, void *stream) {
    if (debug_consume_launch_failure()) return fail(BF_ERR_CUDA, "injected launch failure (test hook)");
    const size_t smem = sizeof(float) * ((size_t)levels + (size_t)(2 * radius + 1) * (2 * radius + 1) +
                                         (size_t)(32 + 2 * radius) * (8 + 2 * radius));
    cudaError_t e = cudaFuncSetAttribute(bf_bft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const float inv_step = (float)((levels - 1) / (double)data_range), step = (float)(data_range / (levels - 1));
    dim3 block(32, 8), grid((width + 31) / 32, (height + 7) / 8);
    bf_bft_kernel<<<grid, block, smem, (cudaStream_t)stream>>>(d_in, in_pitch, d_out, out_pitch, height, width,
                                                               spatial, sigma_s, radius, range, sigma_r, levels,
                                                               step, inv_step);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "look-up-table exact launch");
    return BF_OK;
}

}  // namespace bfi
