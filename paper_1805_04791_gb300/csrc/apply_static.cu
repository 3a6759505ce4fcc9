// vie_apply_static: the operator apply with its scratch in a fixed device
// array instead of memory the library allocates.
//
// Some callers cannot let a library allocate device memory at the point where
// they apply the operator: solvers embedded in frameworks that own the whole
// device memory through their own arena or pool (a cudaMalloc there fails, or
// takes memory the arena has promised elsewhere), and latency-bound loops that
// may not take the device-wide synchronisation a cudaMalloc/cudaFree can cause
// or the risk of an out-of-memory failure in the middle of a run.  For them
// the five passes of the apply use the file-scope array below as their padded
// intermediates.  The array is a fixed kStaticScratchBytes per device and
// stays resident, for every GPU that loads the library, until the process
// exits.
#include <algorithm>
#include <mutex>
#include <string>

#include "vie_internal.h"

namespace vie {

static const size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static const int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mutex;

// Device address of the array on the current device (looked up once per device).
static vie_status scratch_address(void** out) {
  int dev = 0;
  VIE_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("vie_apply_static: device index out of range");
    return VIE_EINVAL;
  }
  std::lock_guard<std::mutex> g(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return VIE_OK;
}

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_apply_static(vie_problem* P, const void* x, void* y, int precision, int nrhs,
                                       void* stream) {
  if (!P || !x || !y || nrhs < 1 || (precision != VIE_FP64 && precision != VIE_FP32)) {
    set_error("vie_apply_static: bad argument");
    return VIE_EINVAL;
  }
  const size_t vb = grid_vec_bytes(P, P->ncomp, nrhs, precision == VIE_FP32 ? sizeof(float2) : sizeof(double2));
  if (ranges_overlap(x, vb, y, vb)) {
    set_error("vie_apply_static: x and y must not overlap");
    return VIE_EINVAL;
  }
  const KernelSet& K = P->kapply;
  const int C = std::max(cin_of(K.mode), cout_of(K.mode));
  const size_t need = apply_workspace_bytes(P->n, P->nk, C, nrhs, precision);
  if (need > kStaticScratchBytes) {
    set_error("vie_apply_static: this grid size, component count, precision and nrhs need " +
              std::to_string(need) + " bytes of scratch; the static array holds " +
              std::to_string(kStaticScratchBytes));
    return VIE_EINVAL;
  }
  // the z-pass schedule must already be chosen (by this handle, or for this
  // shape by any handle of the process): choosing it would time candidates
  // with events and launch them on the scratch
  if (!p3_schedule_ready(P, K, precision)) {
    set_error("vie_apply_static: call vie_tune (or vie_apply once) for this precision and grid size first");
    return VIE_EINVAL;
  }
  void* scratch = nullptr;
  vie_status s = scratch_address(&scratch);
  if (s != VIE_OK) return s;
  // Run the ordinary pipeline on the static array: the workspace record of the
  // handle points at the array for the duration of the call, and since the
  // array is large enough the pipeline never reallocates it.
  const Workspace saved = P->ws;
  P->ws.buf = scratch;
  P->ws.bytes = kStaticScratchBytes;
  s = run_apply(P, K, x, y, precision, nrhs, true, (cudaStream_t)stream);
  P->ws = saved;
  return s;
}
