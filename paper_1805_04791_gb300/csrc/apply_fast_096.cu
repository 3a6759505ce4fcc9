// Fast-path apply kernels for 2n = 96 = 12 x 8 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(96, 12, 8)
}  // namespace vie
