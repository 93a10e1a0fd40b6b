// Instantiations of the fused filter kernels for one range of window counts
// (separate translation unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const KernelClass kClassesM4to6[] = {BF_CLASS(4, 2), BF_CLASS(5, 2), BF_CLASS(6, 2)};
const int kNumClassesM4to6 = sizeof(kClassesM4to6) / sizeof(kClassesM4to6[0]);

}  // namespace bfi
