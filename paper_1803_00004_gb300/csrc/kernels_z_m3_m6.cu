// Instantiations of the 3-D form's slice kernels for three to six windows per axis.
#include "bf_tile.cuh"

namespace bfi {

const ZKernelClass kZClassesM3to6[] = {BF_ZCLASS(3, 4), BF_ZCLASS(3, 2), BF_ZCLASS(4, 2), BF_ZCLASS(5, 2),
                                      BF_ZCLASS(6, 2)};
const int kNumZClassesM3to6 = sizeof(kZClassesM3to6) / sizeof(kZClassesM3to6[0]);

}  // namespace bfi
