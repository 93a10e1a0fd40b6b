// The hybrid layout's kernel: one launch over both kinds of term groups of a gapped selection.  Groups
// 0 .. gp - 1 (grid.z) run the packed-pair tile body on the windows of consecutive frequencies (params pk),
// the groups after them the scalar tile body on the other selected terms (params ps); every group writes its
// partial numerator and denominator planes (the scalar groups' after the packed ones), and a finalize divides.
// One launch keeps the GPU as full as a single-family launch of the same number of groups.
#pragma once

#include "bf_tile.cuh"
#include "bf_tile_scalar.cuh"

namespace bfi {

namespace {

template <int NK, int M, bool RING>
__global__ void __launch_bounds__(512, 1)
bf_hybrid_kernel(const float *__restrict__ in, size_t in_pitch, float *__restrict__ out, size_t out_pitch,
                 float *__restrict__ part, int H, int W, int tw, int th, int ncols, int depth, int gp,
                 const __grid_constant__ FilterParams pk, const __grid_constant__ FilterParams ps) {
    extern __shared__ __align__(16) float smem[];
    const int g = blockIdx.z;  // uniform over the CTA: each CTA runs one tile body, barriers included
    if (g < gp)
        tile_body<NK, M, RING>(pk, in, in_pitch, out, out_pitch, part, H, W, blockIdx.x * tw, blockIdx.y * th, tw, th,
                               ncols, g, kModePartial, depth, smem);
    else
        sc::tile_body<NK, M, RING>(ps, in, in_pitch, out, out_pitch, part + 2 * (size_t)gp * H * W, H, W,
                                   blockIdx.x * tw, blockIdx.y * th, tw, th, ncols, g - gp, true, depth, smem);
}

}  // namespace

#define BF_HYBRID_CLASS(M, NK) \
    {M, NK, {(const void *)bf_hybrid_kernel<NK, M, false>, (const void *)bf_hybrid_kernel<NK, M, true>}}

}  // namespace bfi
