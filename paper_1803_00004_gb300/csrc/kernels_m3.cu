// Instantiations of the fused filter kernels for one range of window counts
// (separate translation unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const KernelClass kClassesM3[] = {BF_CLASS(3, 4), BF_CLASS(3, 2)};
const int kNumClassesM3 = sizeof(kClassesM3) / sizeof(kClassesM3[0]);

}  // namespace bfi
