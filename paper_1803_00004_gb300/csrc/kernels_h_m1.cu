// Instantiations of the hybrid layout's kernels for M = 1 (separate translation unit so the kernel classes
// compile in parallel).
#include "bf_tile_hybrid.cuh"

namespace bfi {

const HybridKernelClass kHybridClassesM1[] = {BF_HYBRID_CLASS(1, 16), BF_HYBRID_CLASS(1, 8), BF_HYBRID_CLASS(1, 4),
                                              BF_HYBRID_CLASS(1, 2)};
const int kNumHybridClassesM1 = sizeof(kHybridClassesM1) / sizeof(kHybridClassesM1[0]);

}  // namespace bfi
