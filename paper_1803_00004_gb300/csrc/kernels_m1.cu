// Instantiations of the fused filter kernels for one range of window counts
// (separate translation unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const KernelClass kClassesM1[] = {BF_CLASS(1, 16), BF_CLASS(1, 8), BF_CLASS(1, 4), BF_CLASS(1, 2)};
const int kNumClassesM1 = sizeof(kClassesM1) / sizeof(kClassesM1[0]);

}  // namespace bfi
