// Instantiations of the fused filter kernels for one range of window counts
// (separate translation unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const KernelClass kClassesM2[] = {BF_CLASS(2, 8), BF_CLASS(2, 4), BF_CLASS(2, 2)};
const int kNumClassesM2 = sizeof(kClassesM2) / sizeof(kClassesM2[0]);

}  // namespace bfi
