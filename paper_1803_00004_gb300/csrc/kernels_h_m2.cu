// Instantiations of the hybrid layout's kernels for M = 2 (separate translation unit so the kernel classes
// compile in parallel).
#include "bf_tile_hybrid.cuh"

namespace bfi {

const HybridKernelClass kHybridClassesM2[] = {BF_HYBRID_CLASS(2, 8), BF_HYBRID_CLASS(2, 4), BF_HYBRID_CLASS(2, 2)};
const int kNumHybridClassesM2 = sizeof(kHybridClassesM2) / sizeof(kHybridClassesM2[0]);

}  // namespace bfi
