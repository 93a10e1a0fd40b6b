// Instantiations of the fused filter's pre-pass variants (basis inputs read from the pre-pass buffer in fp32,
// fp16 or bf16) for two and three windows per axis (separate translation unit so the kernel classes compile in
// parallel).
#include "bf_tile.cuh"

namespace bfi {

const PreKernelClass kPreClassesM2M3[] = {BF_PRE_CLASS(2, 8), BF_PRE_CLASS(2, 4), BF_PRE_CLASS(2, 2), BF_PRE_CLASS(3, 4),
                                          BF_PRE_CLASS(3, 2)};
const int kNumPreClassesM2M3 = sizeof(kPreClassesM2M3) / sizeof(kPreClassesM2M3[0]);

}  // namespace bfi
