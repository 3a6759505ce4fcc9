// Fast-path apply kernels for 2n = 192 = 24 x 8 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(192, 24, 8)
}  // namespace vie
