// Internal state of a problem handle and host-side helpers shared by the
// translation units of the library.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vie.h"
#include "vie_fft.cuh"

namespace vie {

// Symbols of the discrete kernels (Fourier multipliers of the truncated
// Green's function): 1, i k_a, -k_a k_b.
enum Sym { SYM_1 = 0, SYM_DX, SYM_DY, SYM_DZ, SYM_XX, SYM_YY, SYM_ZZ, SYM_XY, SYM_XZ, SYM_YZ, SYM_COUNT };

// Which kernel-array set a convolution pass uses (how the k-space mixing works).
enum KMode {
  KM_SYM3 = 0,     // 3 -> 3, symmetric 3x3 (6 arrays: xx yy zz xy xz yz)
  KM_MAXWELL6 = 1, // 6 -> 6: [Q J + P x M ; Q M - P x J] (6 Q arrays + 3 P arrays)
  KM_DIV = 2,      // 3 -> 1: sum_a G_a J_a (3 arrays)
  KM_EMRED = 3,    // 3 -> 6: [Q J ; -P x J] (6 Q arrays + 3 P arrays)
};

// Per-array parity on the (2n)^3 grid: bit a set = odd under k_a -> -k_a (a = 0 x, 1 y, 2 z).
// Order of the arrays in a set: Q (xx yy zz xy xz yz) then P (x y z).
__host__ __device__ __forceinline__ int sym_parity(int a) {
  switch (a) {
    case 3: return 1 | 2;
    case 4: return 1 | 4;
    case 5: return 2 | 4;
    case 6: return 1;
    case 7: return 2;
    case 8: return 4;
    default: return 0;
  }
}

struct KernelSet {
  int mode = 0;
  int narr = 0;                 // 3, 6 or 9
  double2* oct64 = nullptr;     // [narr][(n+1)^3] FP64
  float2* oct32 = nullptr;      // [narr][(n+1)^3] FP32
  cdf* octdf = nullptr;         // [narr][(n+1)^3] double-word (built on first VIE_DF64 apply)
};

struct Workspace {
  void* buf = nullptr;
  size_t bytes = 0;
};

// Optional per-kernel event timing of the apply pipeline (vie_profile_*).
static const int kProfSlots = 5;
struct Profiler {
  bool on = false;
  int cap = 0;
  int count = 0;
  std::vector<cudaEvent_t> ev;  // (kProfSlots + 1) events per recorded apply
};

}  // namespace vie

struct vie_problem {
  int kind = 0;
  int n = 0;
  int ncomp = 3;   // unknown components: 3, or 6 for Maxwell with mu
  int has_mu = 0;
  double lo = 0, hi = 0, D = 0, h = 0, L = 0, omega = 0;
  int device = 0;
  cudaStream_t stream = nullptr;  // home stream: memory is freed stream-ordered on it at destroy
  // Convolution grid: M = 2 nk points per axis.  nk = n when 2n factors into
  // the codelet radices 2, 3, 5, 7, 11, else the smallest such nk > n: a
  // circular convolution of length M >= 2n - 1 equals the zero-padded linear
  // one on the n^3 output nodes, so the apply never needs Bluestein lines.
  int nk = 0;
  vie::FftPlan planM;        // length-M line DFT (direct)
  double2* tw64 = nullptr;   // its line table: exp(-2 pi i j / M), j < M
  float2* tw32 = nullptr;
  double2* He64 = nullptr;   // [6][n^3] symmetric H_eps (xx yy zz xy xz yz)
  float2* He32 = nullptr;
  double2* Hm64 = nullptr;   // [6][n^3] H_mu (Maxwell with mu)
  float2* Hm32 = nullptr;
  vie::cdf* twdf = nullptr;  // double-word copies of tw64, He64, Hm64 (first VIE_DF64 apply)
  vie::cdf* Hedf = nullptr;
  vie::cdf* Hmdf = nullptr;
  double2* sym_oct = nullptr;  // [SYM_COUNT][(n+1)^3] raw symbol kernels DFT_{2n}, FP64
  unsigned sym_mask = 0;       // symbols computed so far
  vie::KernelSet kapply;     // operator kernels (with I/2, 2H sign and 1/(2n)^3 folded in)
  vie::KernelSet keval;      // scattered-field kernels
  vie::Workspace ws;         // padded intermediates
  vie::Workspace ks;         // Krylov workspace
  vie::Profiler prof;
  int p3_variant[3][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};  // tuned z-pass variant per (precision, mode)
  int* dflag = nullptr;      // device error flag (NaN, bad input)
  double t_precompute = 0;   // wall seconds of the set-up in vie_problem_create
  double opnorm = 0;         // upper bound of ||A||_2 of the operator (set-up)
  // device-resident GMRES: pinned host copies of the per-member Arnoldi state
  // (one slot per step in flight) and the events that mark each copy complete
  void* arn_host = nullptr;
  size_t arn_host_bytes = 0;
  cudaEvent_t arn_ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // single right-hand-side GMRES steps replayed as CUDA graphs (one per step
  // index), valid while every pointer and size baked into them is unchanged
  cudaStream_t cap_stream = nullptr;  // non-blocking stream the graphs are captured on and run on
  cudaEvent_t cap_ev[2] = {nullptr, nullptr};
  std::vector<long long> graph_key;
  std::vector<cudaGraphExec_t> graph_exec;
  int graph_cycles = 0;  // cycles run with graph_key (graphs are built from the second on)
};

namespace vie {

void set_error(const std::string& msg);
// Stream-ordered device allocation (no device-wide synchronisation, so
// concurrent problems on other streams keep running).
cudaError_t dalloc(void** p, size_t bytes, cudaStream_t st);
void dfree(void* p, cudaStream_t st);
vie_status cuda_fail(cudaError_t e, const char* what);
// Whether the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb);
// Bytes of nrhs vectors of c components on the problem's grid, elem bytes per value.
size_t grid_vec_bytes(const vie_problem* P, int c, int nrhs, size_t elem);

#define VIE_CK(call)                                               \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess) return ::vie::cuda_fail(_e, #call);     \
  } while (0)

// precompute.cu
vie_status build_medium(vie_problem* P, const void* eps, const void* mu, cudaStream_t st);
vie_status build_kernels(vie_problem* P, cudaStream_t st);
vie_status build_eval_kernels(vie_problem* P, cudaStream_t st);
vie_status make_line_table(const FftPlan& pl, double2** t64, float2** t32, cudaStream_t st);
// Double-word copies of the twiddles, medium tensors and apply kernels (idempotent).
vie_status build_df(vie_problem* P, cudaStream_t st);

// apply.cu
// Convolution pipeline: out = epilogue(K * pad(in)).  prec: vie_precision.
// in/out layout [nrhs][c][n][n][n] complex.  with_identity 1: out = in + H u;
// 2: out = H u (the operator minus the identity); 0: out = u (u = the
// convolution).
vie_status run_apply(vie_problem* P, const KernelSet& K, const void* in, void* out, int prec, int nrhs,
                     int with_identity, cudaStream_t st);
size_t apply_workspace_bytes(int n, int nk, int c, int nrhs, int prec);
// Kernel half-size nk of an n-point grid (the convolution grid is 2 nk).
int conv_half(int n);
// Grow the padded-intermediate workspace for an apply of K at this precision and
// nrhs (stream-ordered on st); afterwards run_apply does not allocate.
vie_status ensure_apply_workspace(vie_problem* P, const KernelSet& K, int prec, int nrhs, cudaStream_t st);
// Pick (by timing, unless VIE_TUNE=0) the z-pass variant for (prec, K.mode); returns it in *variant.
vie_status tune_apply(vie_problem* P, const KernelSet& K, int prec, int* variant, cudaStream_t st);
// Whether run_apply at this precision can start without choosing a z-pass
// schedule (no tuning launches, no timing events): the shape runs the generic
// kernels or one fixed schedule, the handle holds its choice, a variant is
// forced (VIE_P3_VARIANT), or the process-wide cache has this shape's choice,
// which is then copied into the handle.
bool p3_schedule_ready(vie_problem* P, const KernelSet& K, int prec);

// krylov.cu
vie_status run_solve(vie_problem* P, const void* rhs, void* J, const vie_solve_opts* opt, vie_solve_info* info,
                     cudaStream_t st);
vie_status run_rhs(vie_problem* P, const double* d, const double* p, int nrhs, void* out, cudaStream_t st);

// Allow a kernel the device's full opt-in dynamic shared memory.  The attribute
// is process-wide per kernel: setting it to each launch's own size would race
// between threads launching the same kernel with different sizes (one lowers
// the limit under the other's launch), so it is always set to the same maximum.
inline int smem_optin_bytes() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = b > 0 ? b : 48 * 1024;
  }
  return v;
}
// Whether (current device, kernel) has had its attributes set (first call: no),
// and marking it done; thread-safe (capi.cu).
bool kernel_configured(const void* kernel);
void kernel_mark_configured(const void* kernel);
// The attribute is set once per device and kernel: a driver call at every
// launch costs microseconds of host time, which small grids (launch-bound
// solver loops) pay on every apply.
template <typename K>
inline cudaError_t allow_smem(K* kernel, bool max_carveout = false) {
  if (kernel_configured((const void*)kernel)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_bytes());
  if (e == cudaSuccess && max_carveout)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) kernel_mark_configured((const void*)kernel);
  return e;
}

inline int cin_of(int mode) { return mode == KM_MAXWELL6 ? 6 : 3; }
inline int cout_of(int mode) { return mode == KM_SYM3 ? 3 : (mode == KM_DIV ? 1 : 6); }

}  // namespace vie
