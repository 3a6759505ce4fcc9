// Fast-path apply kernels for 2n = 512 = 32 x 16 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(512, 32, 16)
}  // namespace vie
