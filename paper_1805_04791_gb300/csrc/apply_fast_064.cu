// Fast-path apply kernels for 2n = 64 = 8 x 8 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(64, 8, 8)
}  // namespace vie
