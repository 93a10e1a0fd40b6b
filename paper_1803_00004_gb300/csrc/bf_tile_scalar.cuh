// Scalar tile body of the fused filter: one cosine term per instruction lane, any set of terms per group
// (steps between consecutive terms taken from the plan).  Used for plans whose selected terms are not
// consecutive, where the packed-pair family (bf_tile.cuh) would need extra term groups.  Same algorithm,
// layout of shared memory and launch geometry as the packed family; the exchange rows are ordered
// (window, term, basis image) here.
#pragma once

#include <cuda_runtime.h>

#include "bf_classes.h"
#include "bf_internal.h"

namespace bfi {
// The scalar family lives in its own namespace, so that a translation unit can hold both families' tile bodies
// (the hybrid layout's kernel runs either).
namespace sc {

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

// j mod depth for j >= 0 and the exchange depths the launch accepts (2 or 3): a mask or a division by the
// constant 3, not a division by a runtime value.
__device__ __forceinline__ int mod_depth(int j, int depth) {
    return depth == 2 ? (j & 1) : (int)((unsigned)j % 3u);
}

// Ring slot of row y + off given ys = y mod D and off in [-D, D].
__device__ __forceinline__ int ring_slot(int ys, int off, int D) {
    int s = ys + off;
    s += s < 0 ? D : 0;
    s -= s >= D ? D : 0;
    return s;
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

// The same on a pair of sums (Blackwell's two-wide fp32 instructions; each lane rounded as the scalar
// instruction would round it): the horizontal pass slides two exchange rows per lane.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 x) {
    const float2 y = sub2(x, c);
    const float2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}
__device__ __forceinline__ void sum_add2(float2 &s, float2 &c, int compensated, float2 x) {
    if (compensated) kahan_add2(s, c, x);
    else s = add2(s, x);
}

// (c, s) = (cos, sin)(pi k t) advanced by one multiple of the base rotation (c1, s1) = (cos, sin)(pi t).
__device__ __forceinline__ void rot1(float &c, float &s, float c1, float s1) {
    const float cn = fmaf(c, c1, -s * s1);
    s = fmaf(s, c1, c * s1);
    c = cn;
}

// The same by `steps` multiples (terms that are not consecutive).
__device__ __forceinline__ void rotn(float &c, float &s, float c1, float s1, int steps) {
    for (int n = 0; n < steps; ++n) rot1(c, s, c1, s1);
}

// The same with the double rotation (c2, s2) = (cos, sin)(2 pi t) at hand: steps / 2 double steps, then one
// single step if `steps` is odd (a step of 2, the commonest gap of a best-N selection, is one rotation).
__device__ __forceinline__ void rotn2(float &c, float &s, float c1, float s1, float c2, float s2, int steps) {
    for (int n = 0; n + 1 < steps; n += 2) rot1(c, s, c2, s2);
    if (steps & 1) rot1(c, s, c1, s1);
}

// (cos, sin) of twice an angle from its (cos, sin).
__device__ __forceinline__ void double_angle(float c1, float s1, float &c2, float &s2) {
    c2 = fmaf(c1, c1, -s1 * s1);
    s2 = 2.f * c1 * s1;
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
    // Exchange [depth][ZC][NRP], column-major so that every row offset is a compile-time constant: column
    // threads store a column, scan lanes walk along a row, output threads read a column.  NRP is even so
    // that row pairs move as float2, and NRP / 2 is odd so that a warp's float2 accesses to consecutive
    // columns, and its lanes' float accesses along a column, hit distinct banks.
    constexpr int NRP = NROW + 2;
    constexpr int NP2 = NRP / 2;  // column pitch in float2 (odd: a warp's float2 accesses along a column hit distinct banks)
    const int ZC = ncols + 2;  // tile column c at index c + 1; columns 0 and ncols + 1 stay 0
    // `depth` exchange buffers: 2 -> the output phase reads the row the scan finished in the same step (two
    // barriers per row); 3 -> it reads the row scanned one step earlier (one barrier per row)
    float *zb0 = smem;
    float2 *wb0 = reinterpret_cast<float2 *>(smem + depth * ZC * NRP);  // [depth][NK][tw]: a_k (cos, sin) at the output row
    // RING: per column, the basis inputs of the last D rows, so each row's load and sincospi happen once
    // instead of at every window edge: (v, cos pi t, sin pi t) in ringA, (cos, sin)(pi k0 t) in ringB
    const int D = p.vhi - p.vlo + 2;
    float4 *ringA = reinterpret_cast<float4 *>(wb0 + depth * NK * tw);  // [D][ncols]
    float2 *ringB = reinterpret_cast<float2 *>(ringA + (RING ? D * ncols : 0));  // [D][ncols]
    const int halo = p.rx;

    const int tid = threadIdx.x;
    const bool is_col = tid < ncols;
    const int xcol = x0 - halo + tid;
    const bool colv = is_col && tid < tw + 2 * halo && xcol >= 0 && xcol < W;
    const int nout = min(y0 + th, H) - y0;
    const int xl = tid - halo;
    const bool is_out = is_col && xl >= 0 && xl < tw && x0 + xl < W;
    // the two scan warps: warp 0 slides left to right over tile columns [0, cB), warp 1 right to left over
    // [cB, tw); each writes its sums in place (left: into the slot of Z(c + u0), right: of Z(c + u1))
    const int cB = (tw >> 4) << 3;

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
    const int k0 = kk[0];
    // the group steps by 2 or more between some of its frequencies: the double rotation is then computed once per
    // pixel and edge and used for those steps (uniform over the CTA)
    bool wide = false;
#pragma unroll
    for (int i = 1; i < NK; ++i) wide = wide || kk[i] - kk[i - 1] >= 2;

    float V[NK][4][M];
#pragma unroll
    for (int i = 0; i < NK; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < M; ++r) V[i][t][r] = 0.f;

    // window sums at the first output row: every row of the span once
    // pixel (minus i_lo) of this thread's column at image row `row`, 0 outside the image
    // row addresses as one 32 x 32 -> 64-bit multiply-add on this column's base address (the launch keeps row
    // pitches below 2^32 bytes; rows are loaded only inside [0, H))
    const char *col_in = reinterpret_cast<const char *>(in + (colv ? xcol : 0));
    const unsigned in_pb = (unsigned)(in_pitch * sizeof(float));
    auto pixel = [&](int row) -> float {
        return (colv && (unsigned)row < (unsigned)H)
                   ? __ldg(reinterpret_cast<const float *>(col_in + (size_t)(unsigned)row * in_pb)) - p.i_lo
                   : 0.f;
    };
    if (is_col) {
        float vn = pixel(y0 + p.vlo);  // the next row's pixel is loaded one iteration ahead
        for (int off = p.vlo; off <= p.vhi; ++off) {
            const int row = y0 + off;
            const float v = vn;
            if (off < p.vhi) vn = pixel(row + 1);
            if (row < 0 || row >= H) continue;
            float c1, s1, c, s;
            basis_start(v, p.inv_p, p.inv_p_lo, k0, colv, c1, s1, c, s);
            if (RING) {
                const int sl = pos_mod(row, D) * ncols + tid;
                ringA[sl] = make_float4(v, c1, s1, 0.f);
                ringB[sl] = make_float2(c, s);
            }
            bool in_w[M];
#pragma unroll
            for (int r = 0; r < M; ++r) in_w[r] = off >= p.v0[r] && off <= p.v1[r];
            float c2 = 0.f, s2 = 0.f;
            if (wide) double_angle(c1, s1, c2, s2);
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                if (i > 0) {
                    if (wide) rotn2(c, s, c1, s1, c2, s2, kk[i] - kk[i - 1]);
                    else rotn(c, s, c1, s1, kk[i] - kk[i - 1]);
                }
                const float gi[4] = {c * v, s * v, c, s};
#pragma unroll
                for (int r = 0; r < M; ++r)
                    if (in_w[r]) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) V[i][t][r] += gi[t];
                    }
            }
        }
    }

    const int lag = depth - 1;  // steps between a row's vertical pass and its output phase
    int ys = RING ? pos_mod(y0, D) : 0;  // ring slot of row y (advanced each step)
    const float2 *zq[M];                 // output thread: column of window q's sliding sum
#pragma unroll
    for (int q = 0; q < M; ++q)
        zq[q] = reinterpret_cast<const float2 *>(zb0 + (tid + (xl < cB ? p.u0[q] : p.u1[q]) + 1) * NRP);
    // edge offsets: M entering rows, M leaving rows, the output row
    auto edge_off = [&](int e) -> int { return e < M ? p.v1[e] : (e < 2 * M ? p.v0[e - M] - 1 : 0); };
    // The pixels a step needs from global memory are loaded one step ahead, so their latency overlaps the
    // previous step: RING: the row entering the ring; otherwise the 2M + 1 edge rows.
    float pf[RING ? 1 : NE];
    if (RING) {
        pf[0] = pixel(y0 + 1 + p.vhi);
    } else {
#pragma unroll
        for (int e = 0; e < NE; ++e) pf[e] = e == 2 * M ? pixel(y0) : 0.f;  // at j == 0 only the output edge is live
    }
    for (int j = 0; j < nout + lag; ++j) {
        const int y = y0 + j;
        if (is_col && j < nout) {
            float Ie[NE], c1[NE], s1[NE], ce[NE], se[NE];
            float vr = 0.f;
            if (RING) {
                // pf[0] holds row y + vhi from step 1 on; step 0 inserts nothing
                if (j > 0) {
                    vr = pf[0];
                    if (j + 1 < nout) pf[0] = pixel(y + 1 + p.vhi);
                }
            } else {
#pragma unroll
                for (int e = 0; e < NE; ++e) Ie[e] = pf[e];
                if (j + 1 < nout) {
#pragma unroll
                    for (int e = 0; e < NE; ++e) pf[e] = pixel(y + 1 + edge_off(e));
                }
            }
            if (RING && j > 0) {  // the newest row of the span enters the ring
                const int row = y + p.vhi;
                if (row < H) {
                    const float v = vr;
                    float a, b, c, s;
                    basis_start(v, p.inv_p, p.inv_p_lo, k0, colv, a, b, c, s);
                    const int sl = ring_slot(ys, p.vhi, D) * ncols + tid;
                    ringA[sl] = make_float4(v, a, b, 0.f);
                    ringB[sl] = make_float2(c, s);
                }
            }
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int off = edge_off(e);
                const int row = y + off;
                // at j == 0 the sums already hold row y0: only the output-row edge is live
                const bool valid = colv && row >= 0 && row < H && (j > 0 || e == 2 * M);
                if (RING) {
                    // slots of rows outside the image were never written: do not read them
                    const int sl = ring_slot(ys, off, D) * ncols + tid;
                    const float4 A = valid ? ringA[sl] : make_float4(0.f, 1.f, 0.f, 0.f);
                    Ie[e] = A.x;
                    c1[e] = A.y;
                    s1[e] = A.z;
                    if (k0 == 0) {
                        ce[e] = valid ? 1.f : 0.f;
                        se[e] = 0.f;
                    } else if (k0 == 1) {
                        ce[e] = valid ? A.y : 0.f;
                        se[e] = valid ? A.z : 0.f;
                    } else {
                        const float2 B = valid ? ringB[sl] : make_float2(0.f, 0.f);
                        ce[e] = B.x;
                        se[e] = B.y;
                    }
                } else {
                    // the prefetched value is 0 outside the image; `valid` also masks the rows that the
                    // sums already hold at j == 0
                    if (!valid) Ie[e] = 0.f;
                    basis_start(Ie[e], p.inv_p, p.inv_p_lo, k0, valid, c1[e], s1[e], ce[e], se[e]);
                }
            }
            // per edge double rotations for the classes with few windows (more edges would spill registers)
            constexpr bool DBL = M <= 2;
            float c2[NE], s2[NE];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                c2[e] = 0.f;
                s2[e] = 0.f;
                if (DBL && wide) double_angle(c1[e], s1[e], c2[e], s2[e]);
            }
            float2 *zb = reinterpret_cast<float2 *>(zb0 + (mod_depth(j, depth) * ZC + tid + 1) * NRP);
            float2 *wb = wb0 + mod_depth(j, depth) * NK * tw;
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                if (i > 0) {  // one uniform branch per term
                    const int steps = kk[i] - kk[i - 1];
                    if (steps == 1) {
#pragma unroll
                        for (int e = 0; e < NE; ++e) rot1(ce[e], se[e], c1[e], s1[e]);
                    } else if (DBL && steps == 2) {
#pragma unroll
                        for (int e = 0; e < NE; ++e) rot1(ce[e], se[e], c2[e], s2[e]);
                    } else if (DBL) {
#pragma unroll
                        for (int e = 0; e < NE; ++e) rotn2(ce[e], se[e], c1[e], s1[e], c2[e], s2[e], steps);
                    } else {
#pragma unroll
                        for (int e = 0; e < NE; ++e) rotn(ce[e], se[e], c1[e], s1[e], steps);
                    }
                }
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    const int ei = r, eo = M + r;
                    V[i][0][r] = fmaf(-ce[eo], Ie[eo], fmaf(ce[ei], Ie[ei], V[i][0][r]));
                    V[i][1][r] = fmaf(-se[eo], Ie[eo], fmaf(se[ei], Ie[ei], V[i][1][r]));
                    V[i][2][r] += ce[ei] - ce[eo];
                    V[i][3][r] += se[ei] - se[eo];
                }
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    float z[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        z[t] = 0.f;
#pragma unroll
                        for (int r = 0; r < M; ++r) z[t] = fmaf(p.C[r][q], V[i][t][r], z[t]);
                    }
                    zb[(q * NK + i) * 2 + 0] = make_float2(z[0], z[1]);
                    zb[(q * NK + i) * 2 + 1] = make_float2(z[2], z[3]);
                }
                if (is_out) wb[i * tw + xl] = make_float2(aa[i] * ce[2 * M], aa[i] * se[2 * M]);
            }
        } else if (!is_col && j >= 1 && j - 1 < nout) {
            const int st = tid - ncols;
            const int seg = st >> 5, l = st & 31;  // scan warp, lane = row pair (rows 2l, 2l + 1)
            float2 held = make_float2(0.f, 0.f);
            float2 *hp = nullptr;
            if (l < NROW / 2) {
                const int q = (2 * l) / (4 * NK);
                const int u0 = p.u0[q], u1 = p.u1[q];
                float2 *row = reinterpret_cast<float2 *>(zb0 + mod_depth(j - 1, depth) * ZC * NRP) + l;
                // tile column c is buffer column c + rx + 1; Z(c) at row[(c + rx + 1) * NP2]
                float2 S = make_float2(0.f, 0.f), comp = make_float2(0.f, 0.f);
                if (seg == 0 && cB > 0) {
                    // left to right: S(c + 1) = S(c) + Z(c + 1 + u1) - Z(c + u0); S(c) replaces Z(c + u0)
                    int b = p.rx + u0 + 1;
                    const int bend = p.rx + u1 + 1;
                    for (; b + 7 <= bend; b += 8) {
                        float2 v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) v[u] = row[(b + u) * NP2];
                        sum_add2(S, comp, p.kahan, add2(add2(add2(v[0], v[1]), add2(v[2], v[3])),
                                                        add2(add2(v[4], v[5]), add2(v[6], v[7]))));
                    }
                    float2 rest = make_float2(0.f, 0.f);
                    for (; b <= bend; ++b) rest = add2(rest, row[b * NP2]);
                    sum_add2(S, comp, p.kahan, rest);
                    for (int c0 = p.rx; c0 < p.rx + cB; c0 += 8) {
                        float2 d[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) d[u] = sub2(row[(c0 + u + u1 + 2) * NP2], row[(c0 + u + u0 + 1) * NP2]);
                        float2 pd = make_float2(-comp.x, -comp.y);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            row[(c0 + u + u0 + 1) * NP2] = add2(S, pd);
                            pd = add2(pd, d[u]);
                        }
                        sum_add2(S, comp, p.kahan, add2(pd, comp));
                    }
                } else if (seg == 1) {
                    // right to left from c = tw - 1: S(c - 1) = S(c) + Z(c - 1 + u0) - Z(c + u1); S(c) replaces
                    // Z(c + u1).  The last sum, S(cB), goes into the slot of Z(cB + u1), which the left
                    // warp reads last: it is held until both warps pass the named barrier below.
                    int b = p.rx + tw - 1 + u0 + 1;
                    const int bend = p.rx + tw - 1 + u1 + 1;
                    for (; b + 7 <= bend; b += 8) {
                        float2 v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) v[u] = row[(b + u) * NP2];
                        sum_add2(S, comp, p.kahan, add2(add2(add2(v[0], v[1]), add2(v[2], v[3])),
                                                        add2(add2(v[4], v[5]), add2(v[6], v[7]))));
                    }
                    float2 rest = make_float2(0.f, 0.f);
                    for (; b <= bend; ++b) rest = add2(rest, row[b * NP2]);
                    sum_add2(S, comp, p.kahan, rest);
                    for (int c0 = p.rx + tw - 1; c0 >= p.rx + cB; c0 -= 8) {
                        float2 d[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) d[u] = sub2(row[(c0 - u + u0) * NP2], row[(c0 - u + u1 + 1) * NP2]);
                        float2 pd = make_float2(-comp.x, -comp.y);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float2 o = add2(S, pd);
                            if (u == 7 && c0 - 7 == p.rx + cB) {
                                held = o;
                                hp = &row[(c0 - u + u1 + 1) * NP2];
                            } else {
                                row[(c0 - u + u1 + 1) * NP2] = o;
                            }
                            pd = add2(pd, d[u]);
                        }
                        sum_add2(S, comp, p.kahan, add2(pd, comp));
                    }
                }
            }
            asm volatile("bar.sync 1, 64;" ::: "memory");  // the two scan warps only
            if (hp) *hp = held;
        }
        if (depth == 2) __syncthreads();
        if (is_out && j >= lag) {
            const int yo = y - lag;
            const int zo = mod_depth(j - lag, depth) * ZC * (NRP / 2);
            const float2 *wp = wb0 + mod_depth(j - lag, depth) * NK * tw + xl;
            float num = 0.f, den = 0.f;
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                float F[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float2 a = zq[q][zo + (q * NK + i) * 2 + 0];
                    const float2 b = zq[q][zo + (q * NK + i) * 2 + 1];
                    F[0] += a.x;
                    F[1] += a.y;
                    F[2] += b.x;
                    F[3] += b.y;
                }
                const float2 w = wp[i * tw];
                num = fmaf(w.x, F[0], fmaf(w.y, F[1], num));
                den = fmaf(w.x, F[2], fmaf(w.y, F[3], den));
            }
            const int x = x0 + xl;
            if (grouped) {
                const size_t plane = (size_t)H * W;
                float *pp = part + (size_t)(2 * g) * plane + (size_t)yo * W + x;
                pp[0] = num;
                pp[plane] = den;
            } else {
                float r;
                if (den > p.den_eps) r = num / den + p.i_lo;
                else r = __ldg(in + (size_t)yo * in_pitch + x);  // guard (rare): the input pixel
                out[(size_t)yo * out_pitch + x] = r;
            }
        }
        if (RING) ys = ys + 1 == D ? 0 : ys + 1;
        __syncthreads();
    }
}

template <int NK, int M, bool RING>
__global__ void __launch_bounds__(512, 1)
bf_fused_scalar_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth, int mode,
                const __grid_constant__ FilterParams p) {
    extern __shared__ __align__(16) float smem[];
    tile_body<NK, M, RING>(p, in, in_pitch, out, out_pitch, part, H, W, blockIdx.x * tw, blockIdx.y * th, tw, th, ncols,
                           blockIdx.z, mode == kModePartial, depth, smem);
}

// Persistent batched form: each CTA repeatedly takes the next work item from
// the cursor (largest items first, as the host ordered them) and runs the
// tile body with that image's parameters staged in shared memory.  The loop is
// bounded by the item count.
template <int NK, int M>
__global__ void __launch_bounds__(512, 1)
bf_batch_scalar_kernel(const BatchImage *__restrict__ imgs, const FilterParams *__restrict__ params,
                const WorkItem *__restrict__ items, int n_items, int *__restrict__ cursor, int ncols) {
    extern __shared__ __align__(16) float smem[];
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


}  // namespace
}  // namespace sc

#define BF_SCALAR_CLASS(M, NK)                                                                                  \
    {M, NK, {(const void *)sc::bf_fused_scalar_kernel<NK, M, false>, (const void *)sc::bf_fused_scalar_kernel<NK, M, true>}, \
     (const void *)sc::bf_batch_scalar_kernel<NK, M>}

}  // namespace bfi
