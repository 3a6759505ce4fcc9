// Fast-path apply kernels for 2n = 384 = 24 x 16 (see apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
VIE_FAST_DEFINE(384, 24, 16)
}  // namespace vie
