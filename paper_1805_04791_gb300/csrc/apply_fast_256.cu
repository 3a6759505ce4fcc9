// Fast-path apply kernels for 2n = 256 = 16 x 16 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(256, 16, 16)
}  // namespace vie
