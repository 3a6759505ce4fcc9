// Fast-path apply kernels for 2n = 128 = 16 x 8 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(128, 16, 8)
}  // namespace vie
