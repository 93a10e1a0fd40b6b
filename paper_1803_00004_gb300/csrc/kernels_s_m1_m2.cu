// Instantiations of the scalar-family fused kernels for M = 1, 2 (separate translation unit so the kernel
// classes compile in parallel).
#include "bf_tile_scalar.cuh"

namespace bfi {

const KernelClass kScalarClassesM1M2[] = {BF_SCALAR_CLASS(1, 16), BF_SCALAR_CLASS(1, 8), BF_SCALAR_CLASS(1, 4),
                                          BF_SCALAR_CLASS(1, 2),  BF_SCALAR_CLASS(2, 8), BF_SCALAR_CLASS(2, 4),
                                          BF_SCALAR_CLASS(2, 2)};
const int kNumScalarClassesM1M2 = sizeof(kScalarClassesM1M2) / sizeof(kScalarClassesM1M2[0]);

}  // namespace bfi
