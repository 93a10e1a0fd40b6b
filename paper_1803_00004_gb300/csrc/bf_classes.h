// Kernel class tables of the fused filter: one entry per (windows per axis M, cosine terms per CTA NK),
// filled by the translation units that instantiate the kernels (kernels_*.cu).
#pragma once

namespace bfi {

constexpr int kScanThreads = 64;  // two scan warps per CTA

// Output of a tile: Î (divide and store), a term group's partial numerator / denominator planes, or the
// window sums of each frequency (the pre-computation cache; packed family only).
// The cache modes store the sums as fp32, fp16 or bf16.
constexpr int kModeFinal = 0, kModePartial = 1, kModeCache = 2, kModeCacheF16 = 3, kModeCacheBF16 = 4;

struct KernelClass {
    int m, nk;
    const void *fn[2];  // tile kernels without / with the basis ring
    const void *batch_fn;
};

// Packed-pair family (terms in consecutive pairs; bf_tile.cuh): kernels_m*.cu.
extern const KernelClass kClassesM1[];
extern const KernelClass kClassesM2[];
extern const KernelClass kClassesM3[];
extern const KernelClass kClassesM4to6[];
extern const int kNumClassesM1, kNumClassesM2, kNumClassesM3, kNumClassesM4to6;

// Pre-pass variants of the packed family (no ring; bf_tile.cuh): fn[PRE - 1] reads the basis inputs stored by
// the pre-pass in fp32 (PRE = 1), fp16 (2) or bf16 (3): kernels_p*.cu.
struct PreKernelClass {
    int m, nk;
    const void *fn[3];
};
extern const PreKernelClass kPreClassesM1[];
extern const PreKernelClass kPreClassesM2M3[];
extern const PreKernelClass kPreClassesM4to6[];
extern const int kNumPreClassesM1, kNumPreClassesM2M3, kNumPreClassesM4to6;

// The 3-D form's persistent slice kernels (packed family without the ring; bf_tile.cuh): kernels_z_*.cu.
// box: the range box; haar: the Haar range series' weight table (NK = 2 only).  The *_small kernels are the
// same bounded to CTAs of at most 256 threads and *_regs registers (nullptr where they would spill);
// haar_mid is the Haar kernel for CTAs of up to 512 threads at haar_small_regs registers.
struct ZKernelClass {
    int m, nk;
    const void *box, *box_small, *haar, *haar_small, *haar_mid;
    int box_small_regs, haar_small_regs;
};
extern const ZKernelClass kZClassesM1M2[];
extern const ZKernelClass kZClassesM3to6[];
extern const int kNumZClassesM1M2, kNumZClassesM3to6;

// Hybrid layout (packed groups, then scalar groups, in one launch; bf_tile_hybrid.cuh): kernels_h_*.cu, fn[ring].
struct HybridKernelClass {
    int m, nk;
    const void *fn[2];
};
extern const HybridKernelClass kHybridClassesM1[];
extern const HybridKernelClass kHybridClassesM2[];
extern const int kNumHybridClassesM1, kNumHybridClassesM2;

// Scalar family (any term set; bf_tile_scalar.cuh): kernels_s_*.cu.
extern const KernelClass kScalarClassesM1M2[];
extern const KernelClass kScalarClassesM3to6[];
extern const int kNumScalarClassesM1M2, kNumScalarClassesM3to6;

}  // namespace bfi
