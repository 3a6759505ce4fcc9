// Double-word (VIE_DF64) fast path for 2n = 256 = 16 x 16 (see fast_pass_dw in apply_fast.cuh).
#include "apply_fast.cuh"

namespace vie {
vie_status fast_pass_dw_256(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                            int wid, void* A, void* B, int C, cudaStream_t st, bool* used) {
  return fast_pass_dw<16, 16>(pass, P, K, in, out, nrhs, wid, (cdf*)A, (cdf*)B, C, st, used);
}
}  // namespace vie
