// Instantiations of the 3-D form's slice kernels for one and two windows per axis (separate translation
// unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const ZKernelClass kZClassesM1M2[] = {BF_ZCLASS(1, 16), BF_ZCLASS(1, 8), BF_ZCLASS(1, 4), BF_ZCLASS(1, 2),
                                     BF_ZCLASS(2, 8),  BF_ZCLASS(2, 4), BF_ZCLASS(2, 2)};
const int kNumZClassesM1M2 = sizeof(kZClassesM1M2) / sizeof(kZClassesM1M2[0]);

}  // namespace bfi
