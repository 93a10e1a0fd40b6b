// Instantiations of the fused filter's pre-pass variants (basis inputs read from the pre-pass buffer in fp32,
// fp16 or bf16) for one window count (separate translation unit so the kernel classes compile in parallel).
#include "bf_tile.cuh"

namespace bfi {

const PreKernelClass kPreClassesM1[] = {BF_PRE_CLASS(1, 16), BF_PRE_CLASS(1, 8), BF_PRE_CLASS(1, 4),
                                        BF_PRE_CLASS(1, 2)};
const int kNumPreClassesM1 = sizeof(kPreClassesM1) / sizeof(kPreClassesM1[0]);

}  // namespace bfi
