// Instantiations of the scalar-family fused kernels for M = 3 .. 6 (separate translation unit so the
// kernel classes compile in parallel).
#include "bf_tile_scalar.cuh"

namespace bfi {

const KernelClass kScalarClassesM3to6[] = {BF_SCALAR_CLASS(3, 5), BF_SCALAR_CLASS(3, 4), BF_SCALAR_CLASS(3, 2),
                                           BF_SCALAR_CLASS(4, 2), BF_SCALAR_CLASS(5, 1), BF_SCALAR_CLASS(6, 1)};
const int kNumScalarClassesM3to6 = sizeof(kScalarClassesM3to6) / sizeof(kScalarClassesM3to6[0]);

}  // namespace bfi
