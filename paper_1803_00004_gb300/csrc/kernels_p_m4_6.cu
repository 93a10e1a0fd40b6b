// Instantiations of the fused filter's pre-pass variants (basis inputs read from the pre-pass buffer in fp32,
// fp16 or bf16) for four to six windows per axis (separate translation unit so the kernel classes compile in
// parallel).
#include "bf_tile.cuh"

namespace bfi {

const PreKernelClass kPreClassesM4to6[] = {BF_PRE_CLASS(4, 2), BF_PRE_CLASS(5, 2), BF_PRE_CLASS(6, 2)};
const int kNumPreClassesM4to6 = sizeof(kPreClassesM4to6) / sizeof(kPreClassesM4to6[0]);

}  // namespace bfi
