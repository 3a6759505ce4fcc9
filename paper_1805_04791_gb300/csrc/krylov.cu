// Right-hand sides and the GMRES solve of (I + B + K) J = b.
//
// Sec. 1 and Sec. 6 name GMRES (and Bi-CGStab, used in Sec. 5) as the
// iterative solvers for these second-kind equations.  Two modes:
//  * FP64: restarted GMRES(m) on the FP64 apply, FP64 everywhere.
//  * mixed: FP64 iterative refinement r = b - A x (FP64 apply), inner GMRES(m)
//    on the FP32 apply with an FP32 Krylov basis; Hessenberg matrix, Givens
//    rotations, least squares and the iterate x in FP64.
// Arnoldi: classical Gram-Schmidt, one device reduction per step (inner
// products and |w|^2 in one pass, the update and |w'|^2 in a second), and a
// second Gram-Schmidt pass only when the first removed more than 3/4 of the
// norm.  Reductions use a fixed order (reruns are bit-identical); per-thread
// partial sums are FP64 for an FP64 basis and FP32 for an FP32 basis, the
// cross-thread sums always FP64.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "vie_internal.h"

namespace vie {

typedef std::complex<double> cd;

// ---------------------------------------------------------------- RHS
__global__ void k_rhs(const double2* __restrict__ He, const double2* __restrict__ Hm, int kind, int has_mu, int n,
                      double lo, double h, double w, double3 d, double3 p, double2* __restrict__ out, int c) {
  const long long N = (long long)n * n * n;
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < N;
       pt += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(pt % n), iy = (int)((pt / n) % n), iz = (int)(pt / ((long long)n * n));
    const double x = lo + (ix + 0.5) * h, y = lo + (iy + 0.5) * h, z = lo + (iz + 0.5) * h;
    double2 g[3];
    double2 gm[3];
    double sc = 2.0;
    if (kind == VIE_LAPLACE) {
      // grad phi_in = -E0
      g[0] = make_double2(-d.x, 0);
      g[1] = make_double2(-d.y, 0);
      g[2] = make_double2(-d.z, 0);
    } else {
      double s, cph;
      sincos(w * (d.x * x + d.y * y + d.z * z), &s, &cph);
      const double2 ph = make_double2(cph, s);
      if (kind == VIE_HELMHOLTZ) {
        // grad phi_in = i w d e^{i w d.x}; 2 H_{eps^-1} = -2 H_eps
        const double2 iwph = make_double2(-w * ph.y, w * ph.x);
        g[0] = d.x * iwph;
        g[1] = d.y * iwph;
        g[2] = d.z * iwph;
        sc = -2.0;
      } else {
        g[0] = p.x * ph;
        g[1] = p.y * ph;
        g[2] = p.z * ph;
        const double3 q = make_double3(d.y * p.z - d.z * p.y, d.z * p.x - d.x * p.z, d.x * p.y - d.y * p.x);
        gm[0] = q.x * ph;
        gm[1] = q.y * ph;
        gm[2] = q.z * ph;
      }
    }
    for (int blk = 0; blk < c / 3; ++blk) {
      const double2* H = blk == 0 ? He : Hm;
      const double2* v = blk == 0 ? g : gm;
      const double2 hxx = H[pt], hyy = H[N + pt], hzz = H[2 * N + pt];
      const double2 hxy = H[3 * N + pt], hxz = H[4 * N + pt], hyz = H[5 * N + pt];
      double2 o0 = cmul(hxx, v[0]) + cmul(hxy, v[1]) + cmul(hxz, v[2]);
      double2 o1 = cmul(hxy, v[0]) + cmul(hyy, v[1]) + cmul(hyz, v[2]);
      double2 o2 = cmul(hxz, v[0]) + cmul(hyz, v[1]) + cmul(hzz, v[2]);
      out[(3 * blk + 0) * N + pt] = sc * o0;
      out[(3 * blk + 1) * N + pt] = sc * o1;
      out[(3 * blk + 2) * N + pt] = sc * o2;
    }
  }
}

vie_status run_rhs(vie_problem* P, const double* d, const double* p, int nrhs, void* out, cudaStream_t st) {
  const long long N = (long long)P->n * P->n * P->n;
  for (int r = 0; r < nrhs; ++r) {
    double3 dd = make_double3(d[3 * r], d[3 * r + 1], d[3 * r + 2]);
    double3 pp = p ? make_double3(p[3 * r], p[3 * r + 1], p[3 * r + 2]) : make_double3(0, 0, 0);
    const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
    k_rhs<<<blocks, 256, 0, st>>>(P->He64, P->Hm64, P->kind, P->has_mu, P->n, P->lo, P->h, P->omega, dd, pp,
                                  (double2*)out + (long long)r * P->ncomp * N, P->ncomp);
    VIE_CK(cudaGetLastError());
  }
  return VIE_OK;
}

// ------------------------------------------------------------ vector ops
static const int kRedBlocks = 304;  // 2 x 152 SMs
static const int kRedThreads = 256;
static const int kDotChunk = 8;

template <typename V>
__device__ __forceinline__ double2 to_d(V a) {
  return make_double2((double)a.x, (double)a.y);
}

// Per-thread accumulation type: FP64 for an FP64 basis; FP32 for an FP32
// basis (each thread sums only ~L / 77824 terms in FP32 before the FP64
// cross-thread reduction -- far below the inner tolerance of the FP32 solve,
// and it keeps the FP32 Arnoldi process off GB300's slow FP64 pipes).
template <typename TB> struct Acc;
template <> struct Acc<double2> { typedef double T; typedef double2 V; };
template <> struct Acc<float2> { typedef float T; typedef float2 V; };

// partial[i * G + block] = sum over this block's elements of conj(V_i) w, i < k;
// if with_self, slot k also gets conj(w) w.
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const TB* __restrict__ Vb, long long ldv, int k,
                                                          const TB* __restrict__ w, long long L, double2* partial,
                                                          int with_self) {
  typedef typename Acc<TB>::T AT;
  __shared__ double2 red[kRedThreads / 32][kDotChunk];
  const int G = gridDim.x;
  const int ktot = k + (with_self ? 1 : 0);
  for (int i0 = 0; i0 < ktot; i0 += kDotChunk) {
    const int cnt = min(kDotChunk, ktot - i0);
    AT ar[kDotChunk], ai[kDotChunk];
#pragma unroll
    for (int t = 0; t < kDotChunk; ++t) ar[t] = ai[t] = (AT)0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)G * blockDim.x) {
      const TB we = w[e];
#pragma unroll
      for (int t = 0; t < kDotChunk; ++t)
        if (t < cnt) {
          const int i = i0 + t;
          const TB v = (i < k) ? Vb[(long long)i * ldv + e] : we;
          ar[t] += v.x * we.x + v.y * we.y;
          ai[t] += v.x * we.y - v.y * we.x;
        }
    }
#pragma unroll
    for (int t = 0; t < kDotChunk; ++t) {
      double2 a = make_double2((double)ar[t], (double)ai[t]);
      for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, off);
        a.y += __shfl_down_sync(0xffffffffu, a.y, off);
      }
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][t] = a;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double2 sm = make_double2(0, 0);
      for (int wgi = 0; wgi < kRedThreads / 32; ++wgi) sm = sm + red[wgi][threadIdx.x];
      partial[(long long)(i0 + threadIdx.x) * G + blockIdx.x] = sm;
    }
    __syncthreads();
  }
}

__global__ void k_reduce_partials(const double2* __restrict__ partial, int k, int G, double2* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= k) return;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < G; b += blockDim.x) s = s + partial[(long long)i * G + b];
  __shared__ double2 red[32];
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, off);
    s.y += __shfl_down_sync(0xffffffffu, s.y, off);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0, 0);
    for (int j = 0; j < (int)(blockDim.x + 31) / 32; ++j) t = t + red[j];
    out[i] = t;
  }
}

// w -= sum_i coef[i] V_i (coef on the device); if norm_partial, also the
// block partial sums of |w|^2 after the update (slot blockIdx.x).
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_axpy_norm(TB* __restrict__ w, const TB* __restrict__ Vb, long long ldv,
                                                           int k, const double2* __restrict__ coef, long long L,
                                                           double2* norm_partial) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cs[256];
  __shared__ double red[kRedThreads / 32];
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) {
    cs[i].x = (AT)coef[i].x;
    cs[i].y = (AT)coef[i].y;
  }
  __syncthreads();
  AT nn = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    TB acc = w[e];
    for (int i = 0; i < k; ++i) {
      const TB v = Vb[(long long)i * ldv + e];
      const typename Acc<TB>::V c = cs[i];
      acc.x -= c.x * v.x - c.y * v.y;
      acc.y -= c.x * v.y + c.y * v.x;
    }
    w[e] = acc;
    nn += acc.x * acc.x + acc.y * acc.y;
  }
  if (norm_partial) {
    double d = (double)nn;
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int j = 0; j < kRedThreads / 32; ++j) t += red[j];
      norm_partial[blockIdx.x] = make_double2(t, 0.0);
    }
  }
}

// x += sum_i coef[i] V_i with x FP64 and V of type TB (products in TB's precision).
template <typename TB>
__global__ void k_update(double2* __restrict__ x, const TB* __restrict__ Vb, long long ldv, int k,
                         const double2* __restrict__ coef, long long L) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cs[256];
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) {
    cs[i].x = (AT)coef[i].x;
    cs[i].y = (AT)coef[i].y;
  }
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    AT ax = 0, ay = 0;
    for (int i = 0; i < k; ++i) {
      const TB v = Vb[(long long)i * ldv + e];
      ax += cs[i].x * v.x - cs[i].y * v.y;
      ay += cs[i].x * v.y + cs[i].y * v.x;
    }
    x[e].x += (double)ax;
    x[e].y += (double)ay;
  }
}

// dst = scale * src (types may differ)
template <typename TD, typename TS>
__global__ void k_scale(TD* __restrict__ dst, const TS* __restrict__ src, double scale, long long L) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    dst[e].x = scale * (double)src[e].x;
    dst[e].y = scale * (double)src[e].y;
  }
}

// r = b - r
__global__ void k_bminus(double2* __restrict__ r, const double2* __restrict__ b, long long L) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - r[e];
}

static int ew_blocks(long long L) { return (int)std::min<long long>((L + 255) / 256, 152LL * 8); }

struct KrylovBufs {
  double2* partial = nullptr;  // [(m+2) * G]
  double2* hdev = nullptr;     // [2 (m+3)]
  double2* r = nullptr;        // FP64 residual / work
  double2* w64 = nullptr;      // FP64 Arnoldi vector
  float2* w32 = nullptr;       // FP32 Arnoldi vector
  void* V = nullptr;           // basis (m+1) x L, FP64 or FP32
};

// h[0..k-1] = V^H w (+ slot k = |w|^2 if with_self), left on the device in kb.hdev + off.
template <typename TB>
static vie_status dots_dev(const TB* V, long long L, int k, const TB* w, bool with_self, KrylovBufs& kb, int off,
                           cudaStream_t st) {
  const int kt = k + (with_self ? 1 : 0);
  k_multidot<TB><<<kRedBlocks, kRedThreads, 0, st>>>(V, L, k, w, L, kb.partial, with_self ? 1 : 0);
  VIE_CK(cudaGetLastError());
  k_reduce_partials<<<kt, 256, 0, st>>>(kb.partial, kt, kRedBlocks, kb.hdev + off);
  VIE_CK(cudaGetLastError());
  return VIE_OK;
}

// w -= V h (h at kb.hdev + hoff on the device); |w|^2 to kb.hdev + noff.
template <typename TB>
static vie_status axpy_norm_dev(TB* w, const TB* V, long long L, int k, KrylovBufs& kb, int hoff, int noff,
                                cudaStream_t st) {
  k_axpy_norm<TB><<<kRedBlocks, kRedThreads, 0, st>>>(w, V, L, k, kb.hdev + hoff, L, kb.partial);
  VIE_CK(cudaGetLastError());
  k_reduce_partials<<<1, 256, 0, st>>>(kb.partial, 1, kRedBlocks, kb.hdev + noff);
  VIE_CK(cudaGetLastError());
  return VIE_OK;
}

static vie_status norm2(const double2* v, long long L, KrylovBufs& kb, double* out, cudaStream_t st) {
  vie_status s = dots_dev<double2>(v, L, 1, v, false, kb, 0, st);
  if (s != VIE_OK) return s;
  double2 h;
  VIE_CK(cudaMemcpyAsync(&h, kb.hdev, sizeof(double2), cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  *out = std::sqrt(std::max(0.0, h.x));
  return VIE_OK;
}

// One GMRES(m) cycle on the operator applied in the precision of TB (basis
// type TB).  Arnoldi by classical Gram-Schmidt with one device-resident
// reduction per step and a second pass only when the projection removed
// more than 3/4 of the norm (Kahan-Parlett "twice is enough").
//   rhs r (FP64, norm beta); result x (FP64) += V y.
template <typename TB>
static vie_status gmres_cycle(vie_problem* P, const double2* r, double beta, double2* x, int m, double stop_abs,
                              KrylovBufs& kb, int* steps, double* est, int* applies, cudaStream_t st) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  TB* V = (TB*)kb.V;
  TB* w = (TB*)(sizeof(TB) == sizeof(double2) ? (void*)kb.w64 : (void*)kb.w32);
  const int prec = sizeof(TB) == sizeof(double2) ? VIE_FP64 : VIE_FP32;
  k_scale<TB, double2><<<ew_blocks(L), 256, 0, st>>>(V, r, 1.0 / beta, L);
  VIE_CK(cudaGetLastError());
  std::vector<cd> Hm((size_t)(m + 1) * m, cd(0, 0)), cs(m), sn(m), g(m + 1, cd(0, 0));
  g[0] = beta;
  int j = 0;
  std::vector<double2> hb(2 * (m + 3));
  *est = beta;
  const int H2 = m + 3;  // offset of the second-pass coefficients in hdev
  for (; j < m; ++j) {
    vie_status s = run_apply(P, P->kapply, V + (long long)j * L, w, prec, 1, true, st);
    if (s != VIE_OK) return s;
    ++*applies;
    s = dots_dev<TB>(V, L, j + 1, w, true, kb, 0, st);  // h, |w|^2 at slot j+1
    if (s != VIE_OK) return s;
    s = axpy_norm_dev<TB>(w, V, L, j + 1, kb, 0, j + 2, st);  // |w'|^2 at slot j+2
    if (s != VIE_OK) return s;
    VIE_CK(cudaMemcpyAsync(hb.data(), kb.hdev, sizeof(double2) * (j + 3), cudaMemcpyDeviceToHost, st));
    VIE_CK(cudaStreamSynchronize(st));
    std::vector<cd> h(j + 1);
    for (int i = 0; i <= j; ++i) h[i] = cd(hb[i].x, hb[i].y);
    const double w0 = hb[j + 1].x;
    double wn2 = hb[j + 2].x;
    if (wn2 < 0.0625 * w0) {
      // second Gram-Schmidt pass
      s = dots_dev<TB>(V, L, j + 1, w, false, kb, H2, st);
      if (s != VIE_OK) return s;
      s = axpy_norm_dev<TB>(w, V, L, j + 1, kb, H2, H2 + j + 1, st);
      if (s != VIE_OK) return s;
      VIE_CK(cudaMemcpyAsync(hb.data() + H2, kb.hdev + H2, sizeof(double2) * (j + 2), cudaMemcpyDeviceToHost, st));
      VIE_CK(cudaStreamSynchronize(st));
      for (int i = 0; i <= j; ++i) h[i] += cd(hb[H2 + i].x, hb[H2 + i].y);
      wn2 = hb[H2 + j + 1].x;
    }
    const double hn = std::sqrt(std::max(0.0, wn2));
    if (!std::isfinite(hn) || !std::isfinite(w0)) {
      set_error("non-finite value in the Arnoldi process");
      return VIE_ENAN;
    }
    for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = h[i];
    Hm[(size_t)(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
      const cd a = Hm[(size_t)i * m + j], bb = Hm[(size_t)(i + 1) * m + j];
      Hm[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
      Hm[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
    }
    const cd a = Hm[(size_t)j * m + j], bb = Hm[(size_t)(j + 1) * m + j];
    const double den = std::sqrt(std::norm(a) + std::norm(bb));
    cs[j] = den > 0 ? a / den : cd(1, 0);
    sn[j] = den > 0 ? bb / den : cd(0, 0);
    Hm[(size_t)j * m + j] = std::conj(cs[j]) * a + std::conj(sn[j]) * bb;
    Hm[(size_t)(j + 1) * m + j] = 0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = std::conj(cs[j]) * g[j];
    *est = std::abs(g[j + 1]);
    if (*est <= stop_abs || hn == 0.0 || j + 1 == m) {
      ++j;
      break;
    }
    k_scale<TB, TB><<<ew_blocks(L), 256, 0, st>>>(V + (long long)(j + 1) * L, w, 1.0 / hn, L);
    VIE_CK(cudaGetLastError());
  }
  // back substitution R y = g
  std::vector<cd> y(j);
  for (int i = j - 1; i >= 0; --i) {
    cd acc = g[i];
    for (int q = i + 1; q < j; ++q) acc -= Hm[(size_t)i * m + q] * y[q];
    y[i] = acc / Hm[(size_t)i * m + i];
  }
  VIE_CK(cudaMemcpyAsync(kb.hdev, y.data(), sizeof(double2) * j, cudaMemcpyHostToDevice, st));
  k_update<TB><<<ew_blocks(L), 256, 0, st>>>(x, V, L, j, kb.hdev, L);
  VIE_CK(cudaGetLastError());
  VIE_CK(cudaStreamSynchronize(st));  // y is a host temporary
  *steps = j;
  return VIE_OK;
}

static vie_status ensure_krylov(vie_problem* P, int m, bool mixed, KrylovBufs& kb) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  const size_t need = sizeof(double2) * ((size_t)(m + 2) * kRedBlocks + 2 * (m + 3)) + sizeof(double2) * 2 * L +
                      sizeof(float2) * L + esz * (size_t)(m + 1) * L + 4096;
  if (P->ks.bytes < need) {
    if (P->ks.buf) {
      cudaDeviceSynchronize();
      cudaFree(P->ks.buf);
      P->ks.buf = nullptr;
      P->ks.bytes = 0;
    }
    if (cudaMalloc(&P->ks.buf, need) != cudaSuccess) {
      set_error("out of device memory for the Krylov basis");
      return VIE_ENOMEM;
    }
    P->ks.bytes = need;
  }
  char* p = (char*)P->ks.buf;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) & ~(size_t)255;
    return (void*)q;
  };
  kb.partial = (double2*)take(sizeof(double2) * (size_t)(m + 2) * kRedBlocks);
  kb.hdev = (double2*)take(sizeof(double2) * 2 * (m + 3));
  kb.r = (double2*)take(sizeof(double2) * L);
  kb.w64 = (double2*)take(sizeof(double2) * L);
  kb.w32 = (float2*)take(sizeof(float2) * L);
  kb.V = take(esz * (size_t)(m + 1) * L);
  return VIE_OK;
}

vie_status run_solve(vie_problem* P, const void* rhs, void* Jv, const vie_solve_opts* opt, vie_solve_info* info,
                     cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const int m = opt->restart;
  const bool mixed = opt->mode == VIE_SOLVE_MIXED;
  KrylovBufs kb;
  vie_status s = ensure_krylov(P, m, mixed, kb);
  if (s != VIE_OK) return s;
  vie_solve_info inf{};
  vie_status final_status = VIE_OK;
  double worst = 0.0;
  for (int rr = 0; rr < opt->nrhs; ++rr) {
    const double2* b = (const double2*)rhs + rr * L;
    double2* x = (double2*)Jv + rr * L;
    double nb = 0.0, nx = 0.0;
    s = norm2(b, L, kb, &nb, st);
    if (s != VIE_OK) return s;
    s = norm2(x, L, kb, &nx, st);
    if (s != VIE_OK) return s;
    if (!(nb > 0.0) || !std::isfinite(nb)) {
      if (nb == 0.0) {
        VIE_CK(cudaMemsetAsync(x, 0, sizeof(double2) * L, st));
        continue;
      }
      set_error("non-finite right-hand side");
      return VIE_ENAN;
    }
    double rel = 1.0;
    bool conv = false;
    int total_inner = 0;
    const int max_outer = mixed ? opt->max_outer : std::max(1, opt->max_outer);
    for (int outer = 0; outer <= max_outer; ++outer) {
      // FP64 residual r = b - A x (r = b for a zero initial guess)
      double beta = 0.0;
      if (outer == 0 && nx == 0.0) {
        VIE_CK(cudaMemcpyAsync(kb.r, b, sizeof(double2) * L, cudaMemcpyDeviceToDevice, st));
        beta = nb;
      } else {
        s = run_apply(P, P->kapply, x, kb.r, VIE_FP64, 1, true, st);
        if (s != VIE_OK) return s;
        ++inf.applies_fp64;
        k_bminus<<<ew_blocks(L), 256, 0, st>>>(kb.r, b, L);
        VIE_CK(cudaGetLastError());
        s = norm2(kb.r, L, kb, &beta, st);
        if (s != VIE_OK) return s;
      }
      if (!std::isfinite(beta)) {
        set_error("non-finite residual");
        return VIE_ENAN;
      }
      rel = beta / nb;
      if (rel <= opt->tol) {
        conv = true;
        break;
      }
      if (outer == max_outer || total_inner >= opt->max_inner) break;
      int steps = 0;
      double est = 0.0;
      int ap = 0;
      const int mm = std::min(m, opt->max_inner - total_inner);
      if (mixed) {
        s = gmres_cycle<float2>(P, kb.r, beta, x, mm, opt->inner_tol * beta, kb, &steps, &est, &ap, st);
        inf.applies_fp32 += ap;
      } else {
        s = gmres_cycle<double2>(P, kb.r, beta, x, mm, 0.5 * opt->tol * nb, kb, &steps, &est, &ap, st);
        inf.applies_fp64 += ap;
      }
      if (s != VIE_OK) return s;
      total_inner += steps;
      ++inf.outer_iters;
    }
    inf.inner_iters += total_inner;
    worst = std::max(worst, rel);
    if (!conv) final_status = VIE_ENOCONV;
  }
  VIE_CK(cudaStreamSynchronize(st));
  inf.rel_residual = worst;
  inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (final_status == VIE_ENOCONV) set_error("GMRES did not reach the tolerance within the iteration limits");
  return final_status;
}

}  // namespace vie
