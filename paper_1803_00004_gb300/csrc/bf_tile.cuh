// Tile body of the fused filter and its kernel templates, shared by the
// translation units that instantiate the kernel classes (kernels_m*.cu) so
// that they compile in parallel.  See bf_filter.cu for the algorithm.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "bf_classes.h"
#include "bf_internal.h"

namespace bfi {


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

// Basis inputs stored by the pre-pass (bf_basis_kernel) for the PRE variants of the tile body, one element per
// pixel, [H][W]: PRE = 1: float4 (v, cos pi t, sin pi t, 0) in fp32, the values basis_start computes; PRE = 2 / 3:
// v in fp32 and the base rotation (cos, sin)(pi t) as one fp16 / bf16 pair, 8 bytes (x = v, y = the pair's bits).
// v is the pixel minus i_lo, t = v / P.
template <int PRE>
struct PreElem {
    using T = float2;
};
template <>
struct PreElem<0> {
    using T = float;  // PRE = 0: the pixel itself; the basis is computed in the tile body
};
template <>
struct PreElem<1> {
    using T = float4;
};

// (v, cos pi t, sin pi t) from a stored element.  The 16-bit pair is rescaled to unit length, so that its
// rounding moves only the angle (by at most ~2^-12 rad in fp16, ~2^-9 in bf16), not the magnitude that the
// recurrence would raise to the power of the term offset.
template <int PRE>
__device__ __forceinline__ void pre_basis(const typename PreElem<PRE>::T &e, float &v, float &c1, float &s1) {
    if constexpr (PRE == 1) {
        v = e.x;
        c1 = e.y;
        s1 = e.z;
    } else if constexpr (PRE >= 2) {
        v = e.x;
        const unsigned u = __float_as_uint(e.y);
        float2 f;
        if constexpr (PRE == 2) f = __half22float2(*reinterpret_cast<const __half2 *>(&u));
        else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
        const float n2 = fmaf(f.x, f.x, f.y * f.y);
        const float r = n2 > 0.f ? rsqrtf(n2) : 0.f;
        c1 = f.x * r;
        s1 = f.y * r;
    }
}

// The starting value (cos, sin)(pi k0 t) of a term group from stored basis inputs: k0 = 0, 1 from the stored
// base rotation; k0 >= 2 by a direct sincospi of the two-float angle (as basis_start), so every group's
// recurrence runs at most NK - 1 steps from an fp32 anchor.  Invalid pixels start from (0, 0).
__device__ __forceinline__ void pre_anchor(float v, float inv_p, float inv_p_lo, int k0, bool valid, float c1, float s1,
                                           float &c0, float &s0) {
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
        constexpr float kPiF = 3.14159265358979f;
        const float th = v * inv_p;
        const float tl = fmaf(v, inv_p, -th) + v * inv_p_lo;
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

// Slice of the 3-D form's z axis holding intensity v (minus i_lo): the nearest of the zbins levels,
// rint(v zscale) in fp32 (ties to even), clamped to [0, zbins - 1].
__device__ __forceinline__ int z_slice(float v, const FilterParams &p) {
    const float t = fminf(fmaxf(rintf(v * p.zscale), 0.f), (float)(p.zbins - 1));
    return (int)t;
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

// Packed fp32 pairs (Blackwell's two-wide fp32 instructions): each lane of a pair is rounded exactly
// as the scalar instruction would round it.
__device__ __forceinline__ float2 pair(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Compensated (Kahan) accumulation s += x with running error term c, on a pair.
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 x) {
    const float2 y = sub2(x, c);
    const float2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}

// Adds x to the sliding sums s: compensated, or plain (c then stays 0).
__device__ __forceinline__ void sum_add2(float2 &s, float2 &c, int compensated, float2 x) {
    if (compensated) kahan_add2(s, c, x);
    else s = add2(s, x);
}

// A term pair's (cos, sin), (C, S) = ((cos a, cos b), (sin a, sin b)), both angles advanced by the angle
// whose (cos, sin) pair-broadcasts are (cs, ss) (nss = -ss).
__device__ __forceinline__ void rot2(float2 &C, float2 &S, float2 cs, float2 ss, float2 nss) {
    const float2 cn = fma2(S, nss, mul2(C, cs));
    S = fma2(C, ss, mul2(S, cs));
    C = cn;
}

// One tile: output columns [x0, x0 + tw) x rows [y0, y0 + th) of one image,
// cosine terms [g NK, g NK + NK) of p.  All threads of the CTA call it; it
// ends on a barrier, so the shared memory can be reused right after.
// ZB (the 3-D form, Eqs. (35)-(36) with the z axis): only neighbours whose slice lies within p.rz of
// slice zc enter the window sums, and only output pixels of slice zc are stored.  ZB = 1: with weight 1
// (the range box); ZB = 2 (Haar range series): with weight zw[zc - n(y) + p.rz] (zw: shared memory).
// `mode`:
// kModeFinal divides and stores Î; kModePartial stores this group's numerator
// and denominator planes (part); kModeCache / kModeCacheF16 / kModeCacheBF16
// store the window sums of every frequency of the group (part = the cache
// [k][H][W][4], of fp32 / fp16 / bf16).
//
// The NK terms are processed as NK / 2 pairs of consecutive terms with the packed pair instructions:
// pair p holds terms (2p, 2p + 1) of the group in the two lanes of every float2.
// PRE > 0: the pixel and its base rotation are read from the pre-pass buffer `pre` ([H][W] elements of
// PreElem<PRE>) instead of the input and a sincospi per window edge.
template <int NK, int M, bool RING, int ZB = 0, int PRE = 0>
__device__ __forceinline__ void tile_body(const FilterParams &p, const float *__restrict__ in, size_t in_pitch,
                                          float *__restrict__ out, size_t out_pitch, float *__restrict__ part, int H,
                                          int W, int x0, int y0, int tw, int th, int ncols, int g, int mode,
                                          int depth, float *smem, int zc = 0, const float *zw = nullptr,
                                          const void *__restrict__ pre = nullptr) {
    static_assert(NK % 2 == 0, "terms are processed in pairs");
    static_assert(!(ZB && RING), "the 3-D form runs without the ring");
    static_assert(!(PRE && (ZB || RING)), "the pre-pass variants run without the ring and the slice window");
    using PF = typename PreElem<PRE>::T;
    constexpr int NP = NK / 2;        // term pairs per group
    constexpr int NROW = M * NK * 4;  // exchange rows per image row: windows x basis images x terms
    constexpr int NE = 2 * M + 1;     // edges per step: M entering rows, M leaving rows, the output row
    // Exchange [depth][ZC][NRP] floats, column-major so that every row offset is a compile-time constant:
    // column threads store a column, scan lanes walk along rows, output threads read a column.  Row
    // (q * 4 + t) * NK + i holds window q, basis image t (cos I, sin I, cos, sin) of term i, so a term
    // pair is one float2.  NRP is even and NRP / 2 odd: a warp's float2 accesses to consecutive columns,
    // and its lanes' float2 accesses along a column, hit distinct banks.
    constexpr int NRP = NROW + 2;
    constexpr int NP2 = NRP / 2;      // column pitch in float2
    const int ZC = ncols + 2;         // tile column c at index c + 1; columns 0 and ncols + 1 stay 0
    // `depth` exchange buffers: 2 -> the output phase reads the row the scan finished in the same step (two
    // barriers per row); 3 -> it reads the row scanned one step earlier (one barrier per row)
    float *zb0 = smem;
    // [depth][NP][tw] float4: a_k cos, a_k' cos, a_k sin, a_k' sin of a term pair at the output row
    float4 *wb0 = reinterpret_cast<float4 *>(smem + depth * ZC * NRP);
    // RING: per column, the basis inputs of the last D rows, so each row's load and sincospi happen once
    // instead of at every window edge: (v, cos pi t, sin pi t) in ringA, (cos, sin)(pi k0 t) in ringB (only
    // touched, and only allocated, for groups whose first frequency k0 is 2 or more)
    const int D = p.vhi - p.vlo + 2;
    // (with RING the output weights are recomputed from the ring and wb0 is not allocated)
    float4 *ringA = reinterpret_cast<float4 *>(smem + depth * ZC * NRP) + (RING ? 0 : depth * NP * tw);  // [D][ncols]
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

    // this group's terms: k0 .. k0 + NK - 1 (consecutive; the host zero-weights the frequencies it pads with)
    const int k0 = p.k[g * NK];
    float aa[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) aa[i] = p.a[g * NK + i];

    float2 V[NP][4][M];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < M; ++r) V[i][t][r] = make_float2(0.f, 0.f);

    // pair (C, S) of terms (k0, k0 + 1) from the base rotation (c1, s1) and the anchor (c0, s0) = (cos, sin)(pi k0 t),
    // and the pair step (cos, sin)(2 pi t) broadcast to both lanes
    auto start_pair = [&](float c1, float s1, float c0, float s0, float2 &C, float2 &S, float2 &cs, float2 &ss,
                          float2 &nss) {
        C = make_float2(c0, fmaf(c0, c1, -s0 * s1));
        S = make_float2(s0, fmaf(s0, c1, c0 * s1));
        const float c2 = fmaf(c1, c1, -s1 * s1), s2 = 2.f * c1 * s1;
        cs = pair(c2);
        ss = pair(s2);
        nss = pair(-s2);
    };
    // Row addresses as one 32 x 32 -> 64-bit multiply-add on this column's base address (the launch keeps row
    // pitches below 2^32 bytes; rows are loaded only inside [0, H)).
    const char *col_in = reinterpret_cast<const char *>(in + (colv ? xcol : 0));
    const unsigned in_pb = (unsigned)(in_pitch * sizeof(float));
    const char *col_pre = reinterpret_cast<const char *>(pre) + (PRE && colv ? (size_t)xcol * sizeof(PF) : 0);
    const unsigned pre_pb = (unsigned)((size_t)W * sizeof(PF));
    // pixel (minus i_lo) of this thread's column at image row `row`, 0 outside the image
    auto pixel = [&](int row) -> float {
        return (colv && (unsigned)row < (unsigned)H)
                   ? __ldg(reinterpret_cast<const float *>(col_in + (size_t)(unsigned)row * in_pb)) - p.i_lo
                   : 0.f;
    };
    // what an edge loads one step ahead: the pixel, or (PRE) its pre-pass element (zero outside the image)
    auto edge_load = [&](int row) -> PF {
        if constexpr (PRE == 0) {
            return pixel(row);
        } else {
            PF z;
            if constexpr (PRE == 1) z = make_float4(0.f, 0.f, 0.f, 0.f);
            else z = make_float2(0.f, 0.f);
            return (colv && (unsigned)row < (unsigned)H)
                       ? __ldg(reinterpret_cast<const PF *>(col_pre + (size_t)(unsigned)row * pre_pb))
                       : z;
        }
    };
    // the pixel and the basis of a loaded element: v (0 when !valid), base rotation (c1, s1) and the group's
    // starting value (c0, s0) ((0, 0) when !live)
    auto edge_basis = [&](const PF &e, bool valid, bool live, float &v, float &c1, float &s1, float &c0, float &s0) {
        if constexpr (PRE == 0) {
            v = valid ? e : 0.f;
            basis_start(v, p.inv_p, p.inv_p_lo, k0, live, c1, s1, c0, s0);
        } else {
            pre_basis<PRE>(e, v, c1, s1);
            if (!valid) v = 0.f;
            pre_anchor(v, p.inv_p, p.inv_p_lo, k0, live, c1, s1, c0, s0);
        }
    };

    // window sums at the first output row: every row of the span once
    if (is_col) {
        PF vn = edge_load(y0 + p.vlo);  // the next row's pixel is loaded one iteration ahead
        for (int off = p.vlo; off <= p.vhi; ++off) {
            const int row = y0 + off;
            const PF ve = vn;
            if (off < p.vhi) vn = edge_load(row + 1);
            if (row < 0 || row >= H) continue;
            float v, c1, s1, c0, s0;
            if constexpr (PRE == 0) v = ve;
            bool inz = true;  // 3-D form: the neighbour's slice window (and its weight)
            float wz = 1.f;
            if (ZB) {
                const int dz = zc - z_slice(v, p);
                inz = abs(dz) <= p.rz;
                if (ZB == 2) wz = inz ? zw[dz + p.rz] : 0.f;
            }
            edge_basis(ve, true, colv && inz, v, c1, s1, c0, s0);
            if (ZB == 2) {
                c0 *= wz;
                s0 *= wz;
            }
            if (RING) {
                const int sl = pos_mod(row, D) * ncols + tid;
                ringA[sl] = make_float4(v, c1, s1, 0.f);
                if (k0 >= 2) ringB[sl] = make_float2(c0, s0);
            }
            const float2 v2 = pair(v);
            float2 C, S, cs, ss, nss;
            start_pair(c1, s1, c0, s0, C, S, cs, ss, nss);
            bool in_w[M];
#pragma unroll
            for (int r = 0; r < M; ++r) in_w[r] = off >= p.v0[r] && off <= p.v1[r];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                if (i > 0) rot2(C, S, cs, ss, nss);
                const float2 gi[4] = {mul2(C, v2), mul2(S, v2), C, S};
#pragma unroll
                for (int r = 0; r < M; ++r)
                    if (in_w[r]) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) V[i][t][r] = add2(V[i][t][r], gi[t]);
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
    PF pf[RING ? 1 : NE];
    // ZB: bit d = the output row y - d of this column lies in slice zc (set in the column phase of row y)
    unsigned zrow = 0;
    if constexpr (RING) {
        pf[0] = pixel(y0 + 1 + p.vhi);
    } else {
#pragma unroll
        for (int e = 0; e < NE; ++e)  // at j == 0 only the output edge is live
            if (e == 2 * M) pf[e] = edge_load(y0);
            else pf[e] = PF{};
    }
    for (int j = 0; j < nout + lag; ++j) {
        const int y = y0 + j;
        if (ZB) zrow <<= 1;
        if (is_col && j < nout) {
            PF Ie[NE];
            float vr = 0.f;
            if constexpr (RING) {
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
                    for (int e = 0; e < NE; ++e) pf[e] = edge_load(y + 1 + edge_off(e));
                }
            }
            if (RING && j > 0) {  // the newest row of the span enters the ring
                const int row = y + p.vhi;
                if (row < H) {
                    float a, b, c, s;
                    basis_start(vr, p.inv_p, p.inv_p_lo, k0, colv, a, b, c, s);
                    const int sl = ring_slot(ys, p.vhi, D) * ncols + tid;
                    ringA[sl] = make_float4(vr, a, b, 0.f);
                    if (k0 >= 2) ringB[sl] = make_float2(c, s);
                }
            }
            float2 *zb = reinterpret_cast<float2 *>(zb0 + (mod_depth(j, depth) * ZC + tid + 1) * NRP);
            float4 *wb = wb0 + mod_depth(j, depth) * NP * tw;
            // one edge at a time: its term pairs update the sums of its window (only one edge's state is live)
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                if (RING && e == 2 * M) continue;  // RING: the output phase rebuilds the output row's basis
                if (e == 2 * M && !is_out) continue;  // the output row's weights are only needed by output columns
                const int off = edge_off(e);
                const int row = y + off;
                // at j == 0 the sums already hold row y0: only the output-row edge is live
                const bool valid = colv && row >= 0 && row < H && (j > 0 || e == 2 * M);
                float v, c1, s1, c0, s0;
                if (RING) {
                    // slots of rows outside the image were never written: do not read them
                    const int sl = ring_slot(ys, off, D) * ncols + tid;
                    const float4 A = valid ? ringA[sl] : make_float4(0.f, 1.f, 0.f, 0.f);
                    v = A.x;
                    c1 = A.y;
                    s1 = A.z;
                    if (k0 == 0) {
                        c0 = valid ? 1.f : 0.f;
                        s0 = 0.f;
                    } else if (k0 == 1) {
                        c0 = valid ? A.y : 0.f;
                        s0 = valid ? A.z : 0.f;
                    } else {
                        const float2 B = valid ? ringB[sl] : make_float2(0.f, 0.f);
                        c0 = B.x;
                        s0 = B.y;
                    }
                } else {
                    // the prefetched value is 0 outside the image; `valid` also masks the rows that the
                    // sums already hold at j == 0
                    if constexpr (PRE == 0) v = valid ? Ie[e] : 0.f;
                    bool live = valid;
                    float wz = 1.f;
                    if (ZB) {
                        const int n = z_slice(v, p);
                        if (e < 2 * M) {  // a window edge: the slice window (and the weight of the offset)
                            live = valid && abs(zc - n) <= p.rz;
                            if (ZB == 2) wz = live ? zw[zc - n + p.rz] : 0.f;
                        } else {          // the output row: its own slice
                            zrow |= (valid && n == zc) ? 1u : 0u;
                        }
                    }
                    edge_basis(Ie[e], valid, live, v, c1, s1, c0, s0);
                    if (ZB == 2 && e < 2 * M) {  // the pair starts from the anchor: scaling it scales the edge
                        c0 *= wz;
                        s0 *= wz;
                    }
                }
                float2 C, S, cs, ss, nss;
                start_pair(c1, s1, c0, s0, C, S, cs, ss, nss);
                const int r = e < M ? e : e - M;                          // window of an entering / leaving edge
                const float2 Iv = pair(e >= M && e < 2 * M ? -v : v);    // leaving rows enter with a minus sign
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    if (i > 0) rot2(C, S, cs, ss, nss);
                    if (e < 2 * M) {
                        V[i][0][r] = fma2(C, Iv, V[i][0][r]);
                        V[i][1][r] = fma2(S, Iv, V[i][1][r]);
                        if (e < M) {
                            V[i][2][r] = add2(V[i][2][r], C);
                            V[i][3][r] = add2(V[i][3][r], S);
                        } else {
                            V[i][2][r] = sub2(V[i][2][r], C);
                            V[i][3][r] = sub2(V[i][3][r], S);
                        }
                    } else if (!RING && is_out) {
                        const float2 a2 = make_float2(aa[2 * i], aa[2 * i + 1]);
                        const float2 ca = mul2(a2, C), sa = mul2(a2, S);
                        wb[i * tw + xl] = make_float4(ca.x, ca.y, sa.x, sa.y);
                    }
                }
            }
            // mix per horizontal window and publish
#pragma unroll
            for (int i = 0; i < NP; ++i)
#pragma unroll
                for (int q = 0; q < M; ++q)
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        float2 z = mul2(pair(p.C[0][q]), V[i][t][0]);
#pragma unroll
                        for (int r = 1; r < M; ++r) z = fma2(pair(p.C[r][q]), V[i][t][r], z);
                        zb[(q * 4 + t) * NP + i] = z;
                    }
        } else if (!is_col && j >= 1 && j - 1 < nout) {
            const int st = tid - ncols;
            const int seg = st >> 5, l = st & 31;  // scan warp, lane = row pair
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
        if (is_out && j >= lag && (!ZB || ((zrow >> lag) & 1u))) {
            const int yo = y - lag;
            const int zo = mod_depth(j - lag, depth) * ZC * NP2;
            const float4 *wp = wb0 + mod_depth(j - lag, depth) * NP * tw + xl;
            const int x = x0 + xl;
            const size_t plane = (size_t)H * W, px = (size_t)yo * W + x;
            float2 num2 = make_float2(0.f, 0.f), den2 = make_float2(0.f, 0.f);
            // RING: (cos, sin) of the output row's term pairs from this column's ring entry (row yo is still in
            // the ring: it holds rows y + vlo - 1 .. y + vhi, and lag <= 1 - vlo)
            float2 Co = make_float2(0.f, 0.f), So = Co, cso = Co, sso = Co, nsso = Co;
            if (RING) {
                const int sl = ring_slot(ys, -lag, D) * ncols + tid;
                const float4 A = ringA[sl];
                float c0 = 1.f, s0 = 0.f;
                if (k0 == 1) {
                    c0 = A.y;
                    s0 = A.z;
                } else if (k0 >= 2) {
                    const float2 B = ringB[sl];
                    c0 = B.x;
                    s0 = B.y;
                }
                start_pair(A.y, A.z, c0, s0, Co, So, cso, sso, nsso);
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                float2 F[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    F[t] = zq[0][zo + t * NP + i];
#pragma unroll
                    for (int q = 1; q < M; ++q) F[t] = add2(F[t], zq[q][zo + (q * 4 + t) * NP + i]);
                }
                if (mode >= kModeCache) {
                    // the window sums of frequencies k0 + 2i, k0 + 2i + 1: the cache is [k][pixel][t], the four sums
                    // of a pixel and frequency side by side (one 16-byte fp32 or 8-byte 16-bit load when weighting),
                    // stored as fp32, or rounded once to fp16 / bf16
                    const size_t ia = ((size_t)(k0 + 2 * i) * plane + px) * 4;
                    const size_t ib = ((size_t)(k0 + 2 * i + 1) * plane + px) * 4;
                    if (mode == kModeCache) {
                        *reinterpret_cast<float4 *>(part + ia) = make_float4(F[0].x, F[1].x, F[2].x, F[3].x);
                        *reinterpret_cast<float4 *>(part + ib) = make_float4(F[0].y, F[1].y, F[2].y, F[3].y);
                    } else if (mode == kModeCacheF16) {
                        __half2 *h = reinterpret_cast<__half2 *>(reinterpret_cast<__half *>(part) + ia);
                        h[0] = __floats2half2_rn(F[0].x, F[1].x);
                        h[1] = __floats2half2_rn(F[2].x, F[3].x);
                        h = reinterpret_cast<__half2 *>(reinterpret_cast<__half *>(part) + ib);
                        h[0] = __floats2half2_rn(F[0].y, F[1].y);
                        h[1] = __floats2half2_rn(F[2].y, F[3].y);
                    } else {
                        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(part) + ia);
                        h[0] = __floats2bfloat162_rn(F[0].x, F[1].x);
                        h[1] = __floats2bfloat162_rn(F[2].x, F[3].x);
                        h = reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(part) + ib);
                        h[0] = __floats2bfloat162_rn(F[0].y, F[1].y);
                        h[1] = __floats2bfloat162_rn(F[2].y, F[3].y);
                    }
                    continue;
                }
                float2 wc, ws;
                if (RING) {
                    if (i > 0) rot2(Co, So, cso, sso, nsso);
                    const float2 a2 = make_float2(aa[2 * i], aa[2 * i + 1]);
                    wc = mul2(a2, Co);
                    ws = mul2(a2, So);
                } else {
                    const float4 w = wp[i * tw];
                    wc = make_float2(w.x, w.y);
                    ws = make_float2(w.z, w.w);
                }
                num2 = fma2(wc, F[0], fma2(ws, F[1], num2));
                den2 = fma2(wc, F[2], fma2(ws, F[3], den2));
            }
            const float num = num2.x + num2.y, den = den2.x + den2.y;
            if (mode >= kModeCache) {
            } else if (mode == kModePartial) {
                float *pp = part + (size_t)(2 * g) * plane + px;
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

template <int NK, int M, bool RING, int PRE = 0>
__global__ void __launch_bounds__(512, 1)
bf_fused_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth, int mode,
                const __grid_constant__ FilterParams p, const void *__restrict__ pre) {
    extern __shared__ __align__(16) float smem[];
    tile_body<NK, M, RING, 0, PRE>(p, in, in_pitch, out, out_pitch, part, H, W, blockIdx.x * tw, blockIdx.y * th, tw, th,
                                   ncols, blockIdx.z, mode, depth, smem, 0, nullptr, pre);
}

// The basis pre-pass of the PRE variants: per pixel, v = I - i_lo and the base rotation (cos, sin)(pi v / P) exactly
// as the tile body computes them (basis_start), stored as PreElem<PRE> ([H][W], packed rows).  HBM-bound: 4 bytes
// read and 16 (fp32) or 8 (16-bit) written per pixel.
template <int PRE>
__global__ void __launch_bounds__(256) bf_basis_kernel(const float *__restrict__ in, size_t in_pitch,
                                                       void *__restrict__ pre, int H, int W, float inv_p,
                                                       float inv_p_lo, float i_lo) {
    using PF = typename PreElem<PRE>::T;
    PF *dst = reinterpret_cast<PF *>(pre);
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t y = i / W, x = i - y * W;
        const float v = __ldg(in + y * in_pitch + x) - i_lo;
        float c1, s1, c0, s0;
        basis_start(v, inv_p, inv_p_lo, 0, true, c1, s1, c0, s0);
        if constexpr (PRE == 1) {
            dst[i] = make_float4(v, c1, s1, 0.f);
        } else {
            unsigned u;
            if constexpr (PRE == 2) {
                const __half2 h = __floats2half2_rn(c1, s1);
                u = *reinterpret_cast<const unsigned *>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(c1, s1);
                u = *reinterpret_cast<const unsigned *>(&h);
            }
            dst[i] = make_float2(v, __uint_as_float(u));
        }
    }
}

// Persistent batched form: each CTA repeatedly takes the next work item from
// the cursor (largest items first, as the host ordered them) and runs the
// tile body with that image's parameters staged in shared memory.  The loop is
// bounded by the item count.
template <int NK, int M>
__global__ void __launch_bounds__(512, 1)
bf_batch_kernel(const BatchImage *__restrict__ imgs, const FilterParams *__restrict__ params,
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
                                w.th, ncols, w.g, im.groups > 1 ? kModePartial : kModeFinal, 2, smem);
    }
}


// The 3-D form (Sec. IV-D), persistent: each CTA repeatedly takes the next work item from the cursor
// (counters[1]) and runs the tile body restricted to one slice.  items[0 .. counters[0]) hold (tile, slice)
// for every slice present among a tile's output pixels; item i of term group g is i + g counters[0].  The
// loop is bounded by max_iter.  ZB = 2: the weight table (2 p.rz + 1 floats of zwp) is first copied into
// dynamic shared memory at float offset zw_off, after the tile's exchange.
template <int NK, int M, int ZB>
__device__ __forceinline__ void zslice_body(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out,
                                            size_t out_pitch, float *__restrict__ part, int H, int W, int tw, int th,
                                            int ncols, int depth, int tiles_x, int groups,
                                            const int2 *__restrict__ items, int cap, int *__restrict__ counters,
                                            int max_iter, int zw_off, const FilterParams &p, const ZWeights &zwp) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_item;
    float *zw = smem + zw_off;
    if (ZB == 2) {
        for (int i = threadIdx.x; i < 2 * p.rz + 1; i += blockDim.x) zw[i] = zwp.w[i];
        __syncthreads();
    }
    const int n = min(counters[0], cap);
    const int total = n * groups;
    for (int iter = 0; iter < max_iter; ++iter) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters + 1, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= total) break;
        const int g = it / n;
        const int2 w = items[it - g * n];
        const int ty = w.x / tiles_x, tx = w.x - ty * tiles_x;
        tile_body<NK, M, false, ZB>(p, in, in_pitch, out, out_pitch, part, H, W, tx * tw, ty * th, tw, th, ncols,
                                    g, groups > 1 ? kModePartial : kModeFinal, depth, smem, w.y, zw);
    }
}

#define BF_ZSLICE_PARAMS                                                                                        \
    const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,                  \
        float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth, int tiles_x, int groups, \
        const int2 *__restrict__ items, int cap, int *__restrict__ counters, int max_iter, int zw_off,         \
        const __grid_constant__ FilterParams p, const __grid_constant__ ZWeights zwp
#define BF_ZSLICE_ARGS \
    in, in_pitch, out, out_pitch, part, H, W, tw, th, ncols, depth, tiles_x, groups, items, cap, counters, max_iter, zw_off, p, zwp

template <int NK, int M, int ZB>
__global__ void __launch_bounds__(512, 1) bf_zslice_kernel(BF_ZSLICE_PARAMS) {
    zslice_body<NK, M, ZB>(BF_ZSLICE_ARGS);
}

// Slice kernels for CTAs of at most 256 threads, bounded in registers so that more CTAs fit an SM (the
// general kernel takes 100-128 registers and stops at two): the Haar series' NK = 2 kernel at 64 registers
// (four CTAs), the range box's small classes at 80 (three).  Only classes that fit without spilling more
// than a few bytes are instantiated.
template <int NK, int M, int ZB>
__global__ void __launch_bounds__(256, ZB == 2 ? 4 : 3) bf_zslice_small_kernel(BF_ZSLICE_PARAMS) {
    zslice_body<NK, M, ZB>(BF_ZSLICE_ARGS);
}
constexpr int kZSmallRegs[3] = {0, 80, 64};  // by ZB

// The Haar series' NK = 2 kernel for CTAs of up to 512 threads with the 64-register budget of its 256-thread
// form: two CTAs per SM where shared memory allows, instead of one at 100-128 registers.
template <int NK, int M, int ZB>
__global__ void __launch_bounds__(512, 2) bf_zslice_mid_kernel(BF_ZSLICE_PARAMS) {
    zslice_body<NK, M, ZB>(BF_ZSLICE_ARGS);
}

}  // namespace

// The Haar range series runs one constant cosine term: its slice kernels exist for NK = 2 only.
template <int NK, int M>
constexpr const void *zhaar_kernel() {
    if constexpr (NK == 2) return (const void *)bf_zslice_kernel<2, M, 2>;
    else return nullptr;
}
template <int NK, int M>
constexpr const void *zhaar_small_kernel() {  // more windows than two spill at 64 registers
    if constexpr (NK == 2 && M <= 2) return (const void *)bf_zslice_small_kernel<2, M, 2>;
    else return nullptr;
}
template <int NK, int M>
constexpr const void *zhaar_mid_kernel() {  // the same classes as the 256-thread form
    if constexpr (NK == 2 && M <= 2) return (const void *)bf_zslice_mid_kernel<2, M, 2>;
    else return nullptr;
}
template <int NK, int M>
constexpr const void *zbox_small_kernel() {  // within 8 bytes of spill at 80 registers
    if constexpr ((M <= 2 && NK <= 4) || (M == 3 && NK == 2)) return (const void *)bf_zslice_small_kernel<NK, M, 1>;
    else return nullptr;
}

#define BF_ZCLASS(M, NK)                                                                              \
    {M, NK, (const void *)bf_zslice_kernel<NK, M, 1>, zbox_small_kernel<NK, M>(), zhaar_kernel<NK, M>(), \
     zhaar_small_kernel<NK, M>(), zhaar_mid_kernel<NK, M>(), kZSmallRegs[1], kZSmallRegs[2]}

#define BF_PRE_CLASS(M, NK)                                                                          \
    {M, NK, {(const void *)bf_fused_kernel<NK, M, false, 1>, (const void *)bf_fused_kernel<NK, M, false, 2>, \
             (const void *)bf_fused_kernel<NK, M, false, 3>}}

#define BF_CLASS(M, NK)                                                                                 \
    {M, NK, {(const void *)bf_fused_kernel<NK, M, false>, (const void *)bf_fused_kernel<NK, M, true>},  \
     (const void *)bf_batch_kernel<NK, M>}

}  // namespace bfi
