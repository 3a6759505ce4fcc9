// extern "C" entry points of include/vie.h: argument checks, handle life
// cycle and dispatch to the set-up, apply and solver translation units.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <string>

#include "vie_internal.h"

namespace vie {

static thread_local std::string g_last_error;

static std::mutex g_cfg_mutex;
static std::set<std::pair<int, const void*>> g_cfg_done;

bool kernel_configured(const void* kernel) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(g_cfg_mutex);
  return g_cfg_done.count({dev, kernel}) != 0;
}

void kernel_mark_configured(const void* kernel) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(g_cfg_mutex);
  g_cfg_done.insert({dev, kernel});
}

void set_error(const std::string& msg) { g_last_error = msg; }

cudaError_t dalloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  return cudaMallocAsync(p, bytes, st);
}

void dfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

vie_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? VIE_ENOMEM : VIE_ECUDA;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

size_t grid_vec_bytes(const vie_problem* P, int c, int nrhs, size_t elem) {
  return elem * (size_t)nrhs * (size_t)c * (size_t)P->n * (size_t)P->n * (size_t)P->n;
}

// Grid sizes: any n in [4, 512].  2n and 3n that factor into the codelet
// radices (2, 3, 5, 7, 11) take direct transforms, others Bluestein's; at
// n = 512 the set-up holds about 100 GB on the device, and an allocation that
// fails returns VIE_ENOMEM.
static bool valid_size(int n) { return n >= 4 && n <= 512; }

int conv_half(int n) {
  for (int m = n;; ++m) {
    int r = m;
    for (int p : {2, 3, 5, 7, 11})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

static void free_set(KernelSet& k, cudaStream_t st) {
  dfree(k.oct64, st);
  dfree(k.oct32, st);
  dfree(k.octdf, st);
  k.oct64 = nullptr;
  k.oct32 = nullptr;
  k.octdf = nullptr;
}

static void free_problem(vie_problem* P) {
  if (!P) return;
  cudaStream_t st = P->stream;
  void* ptrs[] = {P->tw64, P->tw32, P->He64, P->He32, P->Hm64, P->Hm32, P->twdf, P->Hedf, P->Hmdf,
                  P->sym_oct, P->ws.buf, P->ks.buf, P->dflag};
  for (void* q : ptrs) dfree(q, st);
  free_set(P->kapply, st);
  free_set(P->keval, st);
  cudaStreamSynchronize(st);
  for (cudaEvent_t e : P->prof.ev) cudaEventDestroy(e);
  for (cudaEvent_t e : P->arn_ev)
    if (e) cudaEventDestroy(e);
  if (P->arn_host) cudaFreeHost(P->arn_host);
  for (cudaGraphExec_t g : P->graph_exec)
    if (g) cudaGraphExecDestroy(g);
  for (cudaEvent_t e : P->cap_ev)
    if (e) cudaEventDestroy(e);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  delete P;
}

}  // namespace vie

using namespace vie;

extern "C" {

const char* vie_last_error(void) { return g_last_error.c_str(); }

vie_status vie_problem_create(int kind, int n, double lo, double hi, double omega, const void* eps, const void* mu,
                              void* stream, vie_problem** out) {
  g_last_error.clear();
  if (!out) {
    set_error("out is NULL");
    return VIE_EINVAL;
  }
  *out = nullptr;
  if (kind < VIE_LAPLACE || kind > VIE_MAXWELL) {
    set_error("unknown kind");
    return VIE_EINVAL;
  }
  if (!valid_size(n)) {
    set_error("n must be in [4, 512]");
    return VIE_EINVAL;
  }
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi)) {
    set_error("box must satisfy lo < hi");
    return VIE_EINVAL;
  }
  if (!(omega >= 0.0) || !std::isfinite(omega)) {
    set_error("omega must be finite and >= 0");
    return VIE_EINVAL;
  }
  if (kind != VIE_LAPLACE && omega == 0.0) {
    set_error("Helmholtz/Maxwell need omega > 0 (use a tiny omega for the quasi-static limit)");
    return VIE_EINVAL;
  }
  if (!eps) {
    set_error("eps is NULL");
    return VIE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const auto t_start = std::chrono::steady_clock::now();
  vie_problem* P = new vie_problem();
  P->kind = kind;
  P->n = n;
  P->has_mu = (kind == VIE_MAXWELL && mu != nullptr) ? 1 : 0;
  P->ncomp = P->has_mu ? 6 : 3;
  P->lo = lo;
  P->hi = hi;
  P->D = hi - lo;
  P->h = P->D / n;
  P->L = std::sqrt(3.0) * P->D;
  P->omega = kind == VIE_LAPLACE ? 0.0 : omega;
  cudaGetDevice(&P->device);
  P->stream = st;
  P->nk = conv_half(n);
  if (!make_line_plan(2 * P->nk, &P->planM) || P->planM.Q != P->planM.M) {
    delete P;
    set_error("bad FFT size");
    return VIE_EINVAL;
  }
  vie_status s = VIE_OK;
  cudaError_t e = dalloc((void**)&P->dflag, sizeof(int) * 4, st);
  if (e != cudaSuccess) s = cuda_fail(e, "cudaMalloc(flag)");
  if (s == VIE_OK) s = make_line_table(P->planM, &P->tw64, &P->tw32, st);
  if (s == VIE_OK) s = build_medium(P, eps, mu, st);
  if (s == VIE_OK) s = build_kernels(P, st);
  if (s == VIE_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "vie_problem_create");
  }
  if (s != VIE_OK) {
    free_problem(P);
    return s;
  }
  P->t_precompute = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  *out = P;
  return VIE_OK;
}

int vie_problem_ncomp(const vie_problem* P) { return P ? P->ncomp : 0; }

vie_status vie_apply(vie_problem* P, const void* x, void* y, int precision, int nrhs, void* stream) {
  if (!P || !x || !y || nrhs < 1 || (precision != VIE_FP64 && precision != VIE_FP32 && precision != VIE_DF64)) {
    set_error("vie_apply: bad argument");
    return VIE_EINVAL;
  }
  const size_t vb = grid_vec_bytes(P, P->ncomp, nrhs, precision == VIE_FP32 ? sizeof(float2) : sizeof(double2));
  if (ranges_overlap(x, vb, y, vb)) {
    set_error("vie_apply: x and y must not overlap");
    return VIE_EINVAL;
  }
  return run_apply(P, P->kapply, x, y, precision, nrhs, true, (cudaStream_t)stream);
}

vie_status vie_rhs_plane_wave(vie_problem* P, const double* d, const double* p, int nrhs, void* rhs_out,
                              void* stream) {
  if (!P || !d || !rhs_out || nrhs < 1 || (P->kind == VIE_MAXWELL && !p)) {
    set_error("vie_rhs_plane_wave: bad argument");
    return VIE_EINVAL;
  }
  // a plane wave needs a unit propagation direction (|d| fixes the wavenumber w |d|)
  // and, for Maxwell, a transverse polarisation (d . p = 0, else E_in is not a
  // solution of the free-space equations); Laplace's d is the field E0 itself
  for (int r = 0; r < nrhs && P->kind != VIE_LAPLACE; ++r) {
    const double* dr = d + 3 * (size_t)r;
    const double dn = std::sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
    if (!(std::fabs(dn - 1.0) <= 1e-8)) {
      set_error("vie_rhs_plane_wave: d must be a unit vector");
      return VIE_EINVAL;
    }
    if (P->kind == VIE_MAXWELL) {
      const double* pr = p + 3 * (size_t)r;
      const double pn = std::sqrt(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
      const double dp = dr[0] * pr[0] + dr[1] * pr[1] + dr[2] * pr[2];
      if (!std::isfinite(pn) || !(std::fabs(dp) <= 1e-8 * pn)) {
        set_error("vie_rhs_plane_wave: p must be finite and perpendicular to d");
        return VIE_EINVAL;
      }
    }
  }
  return run_rhs(P, d, p, nrhs, rhs_out, (cudaStream_t)stream);
}

vie_status vie_solve(vie_problem* P, const void* rhs, void* J, const vie_solve_opts* opt, vie_solve_info* info,
                     void* stream) {
  if (!P || !rhs || !J || !opt || opt->nrhs < 1 || opt->restart < 1 || opt->restart > 200 || !(opt->tol > 0) ||
      opt->max_inner < 1 || opt->max_outer < 0 ||
      (opt->mode == VIE_SOLVE_MIXED && !(opt->inner_tol > 0 && opt->inner_tol < 1)) ||
      (opt->mode != VIE_SOLVE_FP64 && opt->mode != VIE_SOLVE_MIXED && opt->mode != VIE_SOLVE_BICGSTAB) ||
      (opt->check_fp64 != 0 && opt->check_fp64 != 1)) {
    set_error("vie_solve: bad argument");
    return VIE_EINVAL;
  }
  const size_t vb = grid_vec_bytes(P, P->ncomp, opt->nrhs, sizeof(double2));
  if (ranges_overlap(rhs, vb, J, vb)) {
    set_error("vie_solve: rhs and J must not overlap");
    return VIE_EINVAL;
  }
  return run_solve(P, rhs, J, opt, info, (cudaStream_t)stream);
}

vie_status vie_eval_scattered(vie_problem* P, const void* J, void* field_out, int nrhs, void* stream) {
  if (!P || !J || !field_out || nrhs < 1) {
    set_error("vie_eval_scattered: bad argument");
    return VIE_EINVAL;
  }
  if (ranges_overlap(J, grid_vec_bytes(P, P->ncomp, nrhs, sizeof(double2)), field_out,
                     grid_vec_bytes(P, P->kind == VIE_MAXWELL ? 6 : 1, nrhs, sizeof(double2)))) {
    set_error("vie_eval_scattered: J and field_out must not overlap");
    return VIE_EINVAL;
  }
  vie_status s = build_eval_kernels(P, (cudaStream_t)stream);
  if (s != VIE_OK) return s;
  return run_apply(P, P->keval, J, field_out, VIE_FP64, nrhs, false, (cudaStream_t)stream);
}

size_t vie_problem_bytes(int kind, int n, int nrhs, int restart, int has_mu) {
  if (n < 1 || nrhs < 1 || restart < 1) return 0;
  const size_t N = (size_t)n * n * n;
  const size_t nk = (size_t)conv_half(n);
  const size_t O3 = (nk + 1) * (nk + 1) * (nk + 1);
  const int c = (kind == VIE_MAXWELL && has_mu) ? 6 : 3;
  const int nsym = kind == VIE_MAXWELL ? 10 : 9;
  size_t held = 144 * N * (has_mu ? 2 : 1);  // H: 6 entries, FP64 + FP32
  held += 16 * O3 * nsym;                    // raw symbol octants
  held += 24 * O3 * 18;                      // apply + eval kernel sets, FP64 + FP32
  held += 96 * N * (has_mu ? 2 : 1) + 16 * O3 * (kind == VIE_MAXWELL ? 9 : 6);  // double-word copies (mixed solve)
  // set-up peak: oversampled (3n)^3 and convolution-grid (2nk)^3 FP64 transform buffers
  const size_t setup = held + 16 * (27 * N + 8 * nk * nk * nk);
  // steady state: FP64 apply workspace, mixed-precision Krylov group
  size_t steady = held + apply_workspace_bytes(n, (int)nk, c, nrhs, VIE_FP64);
  steady += (size_t)nrhs * c * N * (8 * (size_t)(restart + 1) + 16 * 2 + 8);
  return setup > steady ? setup : steady;
}

vie_status vie_tune(vie_problem* P, int precision, int* variant, void* stream) {
  if (!P || !variant || (precision != VIE_FP64 && precision != VIE_FP32 && precision != VIE_DF64)) {
    set_error("vie_tune: bad argument");
    return VIE_EINVAL;
  }
  return tune_apply(P, P->kapply, precision, variant, (cudaStream_t)stream);
}

vie_status vie_profile_begin(vie_problem* P, int cap) {
  if (!P || cap < 1 || cap > 100000) {
    set_error("vie_profile_begin: bad argument");
    return VIE_EINVAL;
  }
  Profiler& pf = P->prof;
  const size_t need = (size_t)cap * (kProfSlots + 1);
  while (pf.ev.size() < need) {
    cudaEvent_t e;
    VIE_CK(cudaEventCreate(&e));
    pf.ev.push_back(e);
  }
  pf.on = true;
  pf.cap = cap;
  pf.count = 0;
  return VIE_OK;
}

vie_status vie_profile_end(vie_problem* P, double* ms, int nslots, int* count) {
  if (!P || !ms || nslots < 0) {
    set_error("vie_profile_end: bad argument");
    return VIE_EINVAL;
  }
  Profiler& pf = P->prof;
  VIE_CK(cudaDeviceSynchronize());
  for (int k = 0; k < nslots; ++k) ms[k] = 0.0;
  for (int a = 0; a < pf.count; ++a) {
    cudaEvent_t* ev = &pf.ev[(size_t)a * (kProfSlots + 1)];
    for (int k = 0; k < kProfSlots && k < nslots; ++k) {
      float t = 0.f;
      VIE_CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      ms[k] += t;
    }
  }
  if (count) *count = pf.count;
  pf.on = false;
  pf.count = 0;
  return VIE_OK;
}

vie_status vie_problem_destroy(vie_problem* P) {
  free_problem(P);
  return VIE_OK;
}

}  // extern "C"
