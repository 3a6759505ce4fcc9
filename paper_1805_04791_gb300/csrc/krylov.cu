// Right-hand sides and the GMRES solve of (I + B + K) J = b.
//
// Sec. 1 and Sec. 6 name GMRES (and Bi-CGStab, used in Sec. 5) as the
// iterative solvers for these second-kind equations.  Three modes:
//  * FP64: restarted GMRES(m) on the FP64 apply, FP64 everywhere.
//  * mixed: iterative refinement r = b - A x computed to FP64 accuracy (the
//    double-word apply; VIE_RESIDUAL_FP64=1 takes the native FP64 apply),
//    inner GMRES(m) on the FP32 apply with an FP32 Krylov basis; Hessenberg
//    matrix, Givens rotations, least squares and the iterate x in FP64.
//  * Bi-CGStab (the solver of Sec. 5) on the FP64 apply.
// Arnoldi: classical Gram-Schmidt, one device reduction per step (inner
// products and |w|^2 in one pass, the update and |w'|^2 in a second), and a
// second Gram-Schmidt pass only when the first removed more than 3/4 of the
// norm.  Reductions use a fixed order (reruns are bit-identical); per-thread
// and warp sums are in the basis precision (FP64 or FP32), the cross-warp and
// cross-block sums FP64.
#include <cstdlib>
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
// Right-hand sides are solved in lockstep groups of nb: every Arnoldi step is
// one batched operator apply over the group and one batched reduction, with a
// single device-to-host copy of all the group's Hessenberg columns.  Device
// layout of a group: vectors [r][L] (r < nb); Krylov basis [i][r][L].
static const int kRedBlocks = 608;  // 4 x 152 SMs: the most blocks a reduction uses
static const int kRedThreads = 256;
// A sum of squares clamped at zero (rounding can leave it slightly negative),
// with NaN kept: std::max(0.0, NaN) returns 0.0, which would turn a NaN
// residual into a converged one and hide it from the non-finite checks.
static inline double nonneg(double v) { return v < 0.0 ? 0.0 : v; }

static const int kDotChunk = 8;
// Blocks of a reduction over L elements: at least 8 elements per thread, so a
// short vector does not pay for hundreds of idle blocks' reduction trees.
static int red_blocks(long long L) {
  const long long b = (L + 8LL * kRedThreads - 1) / (8LL * kRedThreads);
  return (int)std::max<long long>(1, std::min<long long>(b, kRedBlocks));
}

// Per-thread accumulation type: FP64 for an FP64 basis; FP32 for an FP32
// basis (each thread sums only ~L / 77824 terms in FP32 before the FP64
// cross-thread reduction -- far below the inner tolerance of the FP32 solve,
// and it keeps the FP32 Arnoldi process off GB300's slow FP64 pipes).
template <typename TB> struct Acc;
template <> struct Acc<double2> { typedef double T; typedef double2 V; };
template <> struct Acc<float2> { typedef float T; typedef float2 V; };

// partial[(r * ldp + i) * G + block] = block's share of conj(V_i[r]) w[r], i < k;
// with_self: slot k gets conj(w[r]) w[r].  grid = (G, nb).
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const TB* __restrict__ V, long long ldi, int k,
                                                          const TB* __restrict__ w, long long L, double2* partial,
                                                          int ldp, int with_self) {
  typedef typename Acc<TB>::T AT;
  __shared__ double2 red[kRedThreads / 32][kDotChunk];
  const int G = gridDim.x, r = blockIdx.y;
  const TB* Vr = V + (long long)r * L;
  const TB* wr = w + (long long)r * L;
  const int ktot = k + (with_self ? 1 : 0);
  for (int i0 = 0; i0 < ktot; i0 += kDotChunk) {
    const int cnt = min(kDotChunk, ktot - i0);
    AT ar[kDotChunk], ai[kDotChunk];
#pragma unroll
    for (int t = 0; t < kDotChunk; ++t) ar[t] = ai[t] = (AT)0;
    const long long stride = (long long)G * blockDim.x;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // two elements per iteration: twice the loads in flight per thread
    for (; e + stride < L; e += 2 * stride) {
      const TB wa = wr[e], wb = wr[e + stride];
#pragma unroll
      for (int t = 0; t < kDotChunk; ++t)
        if (t < cnt) {
          const int i = i0 + t;
          const TB va = (i < k) ? Vr[(long long)i * ldi + e] : wa;
          const TB vb = (i < k) ? Vr[(long long)i * ldi + e + stride] : wb;
          ar[t] += va.x * wa.x + va.y * wa.y + vb.x * wb.x + vb.y * wb.y;
          ai[t] += va.x * wa.y - va.y * wa.x + vb.x * wb.y - vb.y * wb.x;
        }
    }
    for (; e < L; e += stride) {
      const TB we = wr[e];
#pragma unroll
      for (int t = 0; t < kDotChunk; ++t)
        if (t < cnt) {
          const int i = i0 + t;
          const TB v = (i < k) ? Vr[(long long)i * ldi + e] : we;
          ar[t] += v.x * we.x + v.y * we.y;
          ai[t] += v.x * we.y - v.y * we.x;
        }
    }
    // warp sums in the accumulation type, for the slots in use only (cnt is
    // block-uniform); the cross-warp and cross-block sums are FP64
#pragma unroll
    for (int t = 0; t < kDotChunk; ++t)
      if (t < cnt) {
        AT ax = ar[t], ay = ai[t];
        for (int off = 16; off > 0; off >>= 1) {
          ax += __shfl_down_sync(0xffffffffu, ax, off);
          ay += __shfl_down_sync(0xffffffffu, ay, off);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][t] = make_double2((double)ax, (double)ay);
      }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double2 sm = make_double2(0, 0);
      for (int wgi = 0; wgi < kRedThreads / 32; ++wgi) sm = sm + red[wgi][threadIdx.x];
      partial[((long long)r * ldp + i0 + threadIdx.x) * G + blockIdx.x] = sm;
    }
    __syncthreads();
  }
}

// out[r * ldo + i] = sum_b partial[(r * ldp + i) * G + b], grid = (k, nb).
__global__ void k_reduce_partials(const double2* __restrict__ partial, int k, int G, int ldp,
                                  double2* __restrict__ out, int ldo) {
  const int i = blockIdx.x, r = blockIdx.y;
  if (i >= k) return;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < G; b += blockDim.x) s = s + partial[((long long)r * ldp + i) * G + b];
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
    out[(long long)r * ldo + i] = t;
  }
}

// w[r] -= sum_i coef[r * ldc + i] V_i[r]; block partial sums of |w[r]|^2 to
// partial[r * ldp * G + block].  grid = (G, nb).
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_axpy_norm(TB* __restrict__ w, const TB* __restrict__ V, long long ldi,
                                                           int k, const double2* __restrict__ coef, int ldc,
                                                           long long L, double2* partial, int ldp) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cs[256];
  __shared__ double red[kRedThreads / 32];
  const int r = blockIdx.y;
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) {
    cs[i].x = (AT)coef[(long long)r * ldc + i].x;
    cs[i].y = (AT)coef[(long long)r * ldc + i].y;
  }
  __syncthreads();
  TB* wr = w + (long long)r * L;
  const TB* Vr = V + (long long)r * L;
  AT nn = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    TB acc = wr[e];
    AT sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
    int i = 0;
    for (; i + 4 <= k; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const TB v = Vr[(long long)(i + u) * ldi + e];
        const typename Acc<TB>::V c = cs[i + u];
        sx[u] += c.x * v.x - c.y * v.y;
        sy[u] += c.x * v.y + c.y * v.x;
      }
    }
    for (; i < k; ++i) {
      const TB v = Vr[(long long)i * ldi + e];
      const typename Acc<TB>::V c = cs[i];
      sx[0] += c.x * v.x - c.y * v.y;
      sy[0] += c.x * v.y + c.y * v.x;
    }
    acc.x -= (sx[0] + sx[1]) + (sx[2] + sx[3]);
    acc.y -= (sy[0] + sy[1]) + (sy[2] + sy[3]);
    wr[e] = acc;
    nn += acc.x * acc.x + acc.y * acc.y;
  }
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int j = 0; j < kRedThreads / 32; ++j) t += red[j];
    partial[(long long)r * ldp * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
  }
}

// x[r] += sum_i coef[r * ldc + i] V_i[r]  (x FP64, products in TB's precision).  grid = (blocks, nb).
template <typename TB>
__global__ void k_update(double2* __restrict__ x, const TB* __restrict__ V, long long ldi, int k,
                         const double2* __restrict__ coef, int ldc, long long L) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cs[256];
  const int r = blockIdx.y;
  for (int i = threadIdx.x; i < k && i < 256; i += blockDim.x) {
    cs[i].x = (AT)coef[(long long)r * ldc + i].x;
    cs[i].y = (AT)coef[(long long)r * ldc + i].y;
  }
  __syncthreads();
  double2* xr = x + (long long)r * L;
  const TB* Vr = V + (long long)r * L;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    AT ax = 0, ay = 0;
    for (int i = 0; i < k; ++i) {
      const TB v = Vr[(long long)i * ldi + e];
      ax += cs[i].x * v.x - cs[i].y * v.y;
      ay += cs[i].x * v.y + cs[i].y * v.x;
    }
    xr[e].x += (double)ax;
    xr[e].y += (double)ay;
  }
}

// dst[r] = scale[r] * src[r].  grid = (blocks, nb).  FP32 -> FP32 scales in
// FP32 (FP64 conversions run on GB300's slow FP64 pipe); FP64 -> FP32 rounds
// the FP64 product once.
template <typename TD, typename TS>
__global__ void k_scale(TD* __restrict__ dst, const TS* __restrict__ src, const double* __restrict__ scale,
                        long long L) {
  const int r = blockIdx.y;
  TD* d = dst + (long long)r * L;
  const TS* s = src + (long long)r * L;
  if constexpr (sizeof(TD) == sizeof(float2) && sizeof(TS) == sizeof(float2)) {
    const float sc = (float)scale[r];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L;
         e += (long long)gridDim.x * blockDim.x) {
      const TS v = s[e];
      d[e].x = sc * v.x;
      d[e].y = sc * v.y;
    }
  } else {
    const double sc = scale[r];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L;
         e += (long long)gridDim.x * blockDim.x) {
      const TS v = s[e];
      d[e].x = sc * (double)v.x;
      d[e].y = sc * (double)v.y;
    }
  }
}

// r = b - r
__global__ void k_bminus(double2* __restrict__ r, const double2* __restrict__ b, long long L) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - r[e];
}

static int ew_blocks(long long L) { return (int)std::min<long long>((L + 255) / 256, 152LL * 16); }

struct Group {
  int nb = 1;
  int m = 1;
  long long L = 0;
  double2* partial = nullptr;  // [nb][m+3][G]
  double2* hdev = nullptr;     // [nb][HS]
  double* sdev = nullptr;      // [nb] scales
  double2* r = nullptr;        // [nb][L] FP64
  double2* w64 = nullptr;      // [nb][L]
  float2* w32 = nullptr;       // [nb][L]
  void* V = nullptr;           // [m+1][nb][L]
  int HS = 0;                  // stride of hdev per rhs
};

static int ldp_of(const Group& g) { return g.m + 3; }

// norms of nb vectors [r][L] (FP64) -> host
static vie_status norms_host(const double2* v, Group& g, std::vector<double>& out, cudaStream_t st) {
  const int G = red_blocks(g.L);
  k_multidot<double2><<<dim3(G, g.nb), kRedThreads, 0, st>>>(v, 0, 0, v, g.L, g.partial, ldp_of(g), 1);
  VIE_CK(cudaGetLastError());
  k_reduce_partials<<<dim3(1, g.nb), 256, 0, st>>>(g.partial, 1, G, ldp_of(g), g.hdev, g.HS);
  VIE_CK(cudaGetLastError());
  std::vector<double2> h((size_t)g.nb * g.HS);
  VIE_CK(cudaMemcpyAsync(h.data(), g.hdev, sizeof(double2) * g.nb * g.HS, cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  out.resize(g.nb);
  for (int r = 0; r < g.nb; ++r) out[r] = std::sqrt(nonneg(h[(size_t)r * g.HS].x));
  return VIE_OK;
}

// One GMRES(m) cycle for the whole group on the operator applied in the
// precision of TB (basis type TB).  Arnoldi: classical Gram-Schmidt, one
// device reduction per step (inner products and |w|^2 in one pass, the update
// and |w'|^2 in a second), a second Gram-Schmidt pass when the first removed
// more than 3/4 of some member's norm (Kahan-Parlett "twice is enough").
//   r (FP64 residuals, norms beta[r]); x (FP64) += V y.  Members with
//   beta = 0 ride along with zero vectors.  Returns steps per member.
template <typename TB>
static vie_status gmres_cycle(vie_problem* P, Group& g, const std::vector<double>& beta, double2* x,
                              const std::vector<double>& stop_abs, std::vector<int>& steps, int* applies,
                              cudaStream_t st) {
  const long long L = g.L;
  const int nb = g.nb, m = g.m, HS = g.HS, ldp = ldp_of(g);
  const long long ldi = (long long)nb * L;
  TB* V = (TB*)g.V;
  TB* w = (TB*)(sizeof(TB) == sizeof(double2) ? (void*)g.w64 : (void*)g.w32);
  const int prec = sizeof(TB) == sizeof(double2) ? VIE_FP64 : VIE_FP32;
  const int G = red_blocks(L);
  const dim3 ewg(ew_blocks(L), nb), redg(G, nb);
  std::vector<double> sc(nb);
  for (int r = 0; r < nb; ++r) sc[r] = beta[r] > 0 ? 1.0 / beta[r] : 0.0;
  VIE_CK(cudaMemcpyAsync(g.sdev, sc.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
  k_scale<TB, double2><<<ewg, 256, 0, st>>>(V, g.r, g.sdev, L);
  VIE_CK(cudaGetLastError());
  std::vector<cd> Hm((size_t)nb * (m + 1) * m, cd(0, 0)), cs((size_t)nb * m), sn((size_t)nb * m),
      gg((size_t)nb * (m + 1), cd(0, 0));
  std::vector<char> done(nb, 0);
  steps.assign(nb, 0);
  int active = 0;
  for (int r = 0; r < nb; ++r) {
    gg[(size_t)r * (m + 1)] = beta[r];
    if (beta[r] <= stop_abs[r] || beta[r] == 0.0) done[r] = 1;
    else ++active;
  }
  std::vector<double2> hb((size_t)nb * HS);
  const int H2 = m + 3;  // second-pass slot offset inside a member's hdev row
  for (int j = 0; j < m && active > 0; ++j) {
    vie_status s = run_apply(P, P->kapply, V + (long long)j * ldi, w, prec, nb, true, st);
    if (s != VIE_OK) return s;
    *applies += active;
    k_multidot<TB><<<redg, kRedThreads, 0, st>>>(V, ldi, j + 1, w, L, g.partial, ldp, 1);
    VIE_CK(cudaGetLastError());
    k_reduce_partials<<<dim3(j + 2, nb), 256, 0, st>>>(g.partial, j + 2, G, ldp, g.hdev, HS);
    VIE_CK(cudaGetLastError());
    k_axpy_norm<TB><<<redg, kRedThreads, 0, st>>>(w, V, ldi, j + 1, g.hdev, HS, L, g.partial, ldp);
    VIE_CK(cudaGetLastError());
    k_reduce_partials<<<dim3(1, nb), 256, 0, st>>>(g.partial, 1, G, ldp, g.hdev + (j + 2), HS);
    VIE_CK(cudaGetLastError());
    VIE_CK(cudaMemcpyAsync(hb.data(), g.hdev, sizeof(double2) * nb * HS, cudaMemcpyDeviceToHost, st));
    VIE_CK(cudaStreamSynchronize(st));
    bool reorth = false;
    for (int r = 0; r < nb; ++r)
      if (!done[r] && hb[(size_t)r * HS + j + 2].x < 0.0625 * hb[(size_t)r * HS + j + 1].x) reorth = true;
    if (reorth) {
      k_multidot<TB><<<redg, kRedThreads, 0, st>>>(V, ldi, j + 1, w, L, g.partial, ldp, 0);
      VIE_CK(cudaGetLastError());
      k_reduce_partials<<<dim3(j + 1, nb), 256, 0, st>>>(g.partial, j + 1, G, ldp, g.hdev + H2, HS);
      VIE_CK(cudaGetLastError());
      k_axpy_norm<TB><<<redg, kRedThreads, 0, st>>>(w, V, ldi, j + 1, g.hdev + H2, HS, L, g.partial, ldp);
      VIE_CK(cudaGetLastError());
      k_reduce_partials<<<dim3(1, nb), 256, 0, st>>>(g.partial, 1, G, ldp, g.hdev + H2 + j + 1, HS);
      VIE_CK(cudaGetLastError());
      VIE_CK(cudaMemcpyAsync(hb.data(), g.hdev, sizeof(double2) * nb * HS, cudaMemcpyDeviceToHost, st));
      VIE_CK(cudaStreamSynchronize(st));
    }
    for (int r = 0; r < nb; ++r) {
      sc[r] = 0.0;
      if (done[r]) continue;
      const double2* hr = &hb[(size_t)r * HS];
      const double w0 = hr[j + 1].x;
      double wn2 = reorth ? hr[H2 + j + 1].x : hr[j + 2].x;
      const double hn = std::sqrt(nonneg(wn2));
      if (!std::isfinite(hn) || !std::isfinite(w0)) {
        set_error("non-finite value in the Arnoldi process");
        return VIE_ENAN;
      }
      cd* H = &Hm[(size_t)r * (m + 1) * m];
      cd* c_ = &cs[(size_t)r * m];
      cd* s_ = &sn[(size_t)r * m];
      cd* g_ = &gg[(size_t)r * (m + 1)];
      for (int i = 0; i <= j; ++i) {
        cd h(hr[i].x, hr[i].y);
        if (reorth) h += cd(hr[H2 + i].x, hr[H2 + i].y);
        H[(size_t)i * m + j] = h;
      }
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const cd a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = std::conj(c_[i]) * a + std::conj(s_[i]) * bb;
        H[(size_t)(i + 1) * m + j] = -s_[i] * a + c_[i] * bb;
      }
      const cd a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double den = std::sqrt(std::norm(a) + std::norm(bb));
      c_[j] = den > 0 ? a / den : cd(1, 0);
      s_[j] = den > 0 ? bb / den : cd(0, 0);
      H[(size_t)j * m + j] = std::conj(c_[j]) * a + std::conj(s_[j]) * bb;
      H[(size_t)(j + 1) * m + j] = 0;
      g_[j + 1] = -s_[j] * g_[j];
      g_[j] = std::conj(c_[j]) * g_[j];
      steps[r] = j + 1;
      if (std::abs(g_[j + 1]) <= stop_abs[r] || hn == 0.0) {
        done[r] = 1;
        --active;
      } else {
        sc[r] = 1.0 / hn;
      }
    }
    if (j + 1 < m && active > 0) {
      VIE_CK(cudaMemcpyAsync(g.sdev, sc.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
      k_scale<TB, TB><<<ewg, 256, 0, st>>>(V + (long long)(j + 1) * ldi, w, g.sdev, L);
      VIE_CK(cudaGetLastError());
    }
  }
  // back substitution R y = g per member; coefficients to the device, x += V y
  int kmax = 0;
  for (int r = 0; r < nb; ++r) kmax = std::max(kmax, steps[r]);
  if (kmax == 0) return VIE_OK;
  std::vector<cd> y((size_t)nb * HS, cd(0, 0));
  for (int r = 0; r < nb; ++r) {
    const int jr = steps[r];
    const cd* H = &Hm[(size_t)r * (m + 1) * m];
    const cd* g_ = &gg[(size_t)r * (m + 1)];
    cd* yr = &y[(size_t)r * HS];
    for (int i = jr - 1; i >= 0; --i) {
      cd acc = g_[i];
      for (int q = i + 1; q < jr; ++q) acc -= H[(size_t)i * m + q] * yr[q];
      yr[i] = acc / H[(size_t)i * m + i];
    }
  }
  VIE_CK(cudaMemcpyAsync(g.hdev, y.data(), sizeof(double2) * nb * HS, cudaMemcpyHostToDevice, st));
  k_update<TB><<<ewg, 256, 0, st>>>(x, V, ldi, kmax, g.hdev, HS, L);
  VIE_CK(cudaGetLastError());
  VIE_CK(cudaStreamSynchronize(st));  // y is a host temporary
  return VIE_OK;
}

// Bytes of Krylov workspace per right-hand side.
static size_t group_bytes_per_rhs(long long L, int m, bool mixed) {
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  return esz * (size_t)(m + 1) * L + sizeof(double2) * 2 * L + sizeof(float2) * L +
         sizeof(double2) * ((size_t)(m + 3) * kRedBlocks + 2 * (m + 4)) + 64;
}

static vie_status ensure_group(vie_problem* P, int m, bool mixed, int nb, Group& g, cudaStream_t st) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const size_t need = group_bytes_per_rhs(L, m, mixed) * nb + 16 * 4096;
  if (P->ks.bytes < need) {
    dfree(P->ks.buf, st);
    P->ks.buf = nullptr;
    P->ks.bytes = 0;
    if (dalloc(&P->ks.buf, need, st) != cudaSuccess) {
      cudaGetLastError();
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
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  g.nb = nb;
  g.m = m;
  g.L = L;
  g.HS = 2 * (m + 4);
  g.partial = (double2*)take(sizeof(double2) * (size_t)nb * (m + 3) * kRedBlocks);
  g.hdev = (double2*)take(sizeof(double2) * (size_t)nb * g.HS);
  g.sdev = (double*)take(sizeof(double) * nb);
  g.r = (double2*)take(sizeof(double2) * (size_t)nb * L);
  g.w64 = (double2*)take(sizeof(double2) * (size_t)nb * L);
  g.w32 = (float2*)take(sizeof(float2) * (size_t)nb * L);
  g.V = take(esz * (size_t)(m + 1) * nb * L);
  return VIE_OK;
}

// Lockstep group size: every right-hand side at once if the Krylov basis and
// the batched FP64 apply workspace fit in 80% of free device memory.
static int pick_group(vie_problem* P, int nrhs, int m, bool mixed) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) return 1;
  freeb += P->ks.bytes + P->ws.bytes;  // our own workspaces are reusable
  const size_t per = group_bytes_per_rhs(L, m, mixed) +
                     apply_workspace_bytes(P->n, std::max(cin_of(P->kapply.mode), cout_of(P->kapply.mode)), 1,
                                           VIE_FP64);
  long long nb = (long long)(0.8 * (double)freeb / (double)per);
  const char* cap = getenv("VIE_GROUP_MAX");
  if (cap) nb = std::min<long long>(nb, atoi(cap));
  return (int)std::max<long long>(1, std::min<long long>(nb, std::min(nrhs, 64)));
}

// ------------------------------------------------------------ Bi-CGStab
// Unpreconditioned Bi-CGStab (van der Vorst 1992), the solver the paper's
// experiments use (Sec. 5), on the FP64 apply; two operator applies per
// iteration.  Reductions: up to four inner products conj(a_i) b_i per pass.
struct Dots4 {
  const double2* a[4];
  const double2* b[4];
  int k;
};

__global__ void __launch_bounds__(kRedThreads) k_dots4(Dots4 d, long long L, double2* partial) {
  __shared__ double2 red[kRedThreads / 32][4];
  double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < d.k) {
        const double2 x = d.a[t][e], y = d.b[t][e];
        ar[t] += x.x * y.x + x.y * y.y;
        ai[t] += x.x * y.y - x.y * y.x;
      }
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < d.k) {  // block-uniform
      double2 a = make_double2(ar[t], ai[t]);
      for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, off);
        a.y += __shfl_down_sync(0xffffffffu, a.y, off);
      }
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][t] = a;
    }
  __syncthreads();
  if (threadIdx.x < d.k) {
    double2 sm = make_double2(0, 0);
    for (int w = 0; w < kRedThreads / 32; ++w) sm = sm + red[w][threadIdx.x];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = sm;
  }
}

// y = a0 x0 + a1 x1 + a2 x2 (x_i may be null; y may alias x0)
__global__ void k_lincomb(double2* y, const double2* x0, double2 a0, const double2* x1, double2 a1, const double2* x2,
                          double2 a2, long long L) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x) {
    double2 v = make_double2(0, 0);
    if (x0) v = v + cmul(a0, x0[e]);
    if (x1) v = v + cmul(a1, x1[e]);
    if (x2) v = v + cmul(a2, x2[e]);
    y[e] = v;
  }
}

static vie_status dots_host(Dots4 d, long long L, double2* partial, double2* dev, std::vector<cd>& out,
                            cudaStream_t st) {
  const int G = red_blocks(L);
  k_dots4<<<G, kRedThreads, 0, st>>>(d, L, partial);
  VIE_CK(cudaGetLastError());
  k_reduce_partials<<<dim3(d.k, 1), 256, 0, st>>>(partial, d.k, G, 0, dev, 0);
  VIE_CK(cudaGetLastError());
  double2 h[4];
  VIE_CK(cudaMemcpyAsync(h, dev, sizeof(double2) * d.k, cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  out.resize(d.k);
  for (int i = 0; i < d.k; ++i) out[i] = cd(h[i].x, h[i].y);
  return VIE_OK;
}

static vie_status run_bicgstab(vie_problem* P, const void* rhs, void* Jv, const vie_solve_opts* opt,
                               vie_solve_info* inf, double* worst, bool* all_conv, cudaStream_t st) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const size_t need = sizeof(double2) * (6 * L + (size_t)4 * kRedBlocks + 8) + 8 * 256;
  if (P->ks.bytes < need) {
    dfree(P->ks.buf, st);
    P->ks.buf = nullptr;
    P->ks.bytes = 0;
    if (dalloc(&P->ks.buf, need, st) != cudaSuccess) {
      cudaGetLastError();
      set_error("out of device memory for the Bi-CGStab vectors");
      return VIE_ENOMEM;
    }
    P->ks.bytes = need;
  }
  double2* base = (double2*)P->ks.buf;
  double2 *r = base, *rh = base + L, *p = base + 2 * L, *v = base + 3 * L, *sv = base + 4 * L, *tv = base + 5 * L;
  double2* partial = base + 6 * L;
  double2* dev = partial + 4 * kRedBlocks;
  const int eb = ew_blocks(L);
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  auto C = [](cd z) { return make_double2(z.real(), z.imag()); };
  *all_conv = true;
  for (int rr = 0; rr < opt->nrhs; ++rr) {
    const double2* b = (const double2*)rhs + rr * L;
    double2* x = (double2*)Jv + rr * L;
    std::vector<cd> d;
    Dots4 q{{b, x, nullptr, nullptr}, {b, x, nullptr, nullptr}, 2};
    vie_status s = dots_host(q, L, partial, dev, d, st);
    if (s != VIE_OK) return s;
    const double nb = std::sqrt(nonneg(d[0].real())), nx = std::sqrt(nonneg(d[1].real()));
    if (!std::isfinite(nb)) {
      set_error("non-finite right-hand side");
      return VIE_ENAN;
    }
    if (nb == 0.0) {
      VIE_CK(cudaMemsetAsync(x, 0, sizeof(double2) * L, st));
      continue;
    }
    if (nx == 0.0) {
      VIE_CK(cudaMemcpyAsync(r, b, sizeof(double2) * L, cudaMemcpyDeviceToDevice, st));
    } else {
      s = run_apply(P, P->kapply, x, r, VIE_FP64, 1, true, st);
      if (s != VIE_OK) return s;
      ++inf->applies_fp64;
      k_bminus<<<eb, 256, 0, st>>>(r, b, L);
    }
    VIE_CK(cudaMemcpyAsync(rh, r, sizeof(double2) * L, cudaMemcpyDeviceToDevice, st));
    VIE_CK(cudaMemsetAsync(p, 0, sizeof(double2) * L, st));
    VIE_CK(cudaMemsetAsync(v, 0, sizeof(double2) * L, st));
    cd rho = 1, alpha = 1, omega = 1;
    double rel = 1.0;
    bool conv = false;
    for (int it = 0; it < opt->max_inner; ++it) {
      q = Dots4{{rh, r, nullptr, nullptr}, {r, r, nullptr, nullptr}, 2};
      s = dots_host(q, L, partial, dev, d, st);
      if (s != VIE_OK) return s;
      rel = std::sqrt(nonneg(d[1].real())) / nb;
      if (!std::isfinite(rel)) {
        set_error("non-finite residual");
        return VIE_ENAN;
      }
      if (rel <= opt->tol) {
        conv = true;
        break;
      }
      const cd rho_new = d[0];
      const cd beta = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
      // p = r + beta (p - omega v)
      k_lincomb<<<eb, 256, 0, st>>>(p, r, one, p, C(beta), v, C(-beta * omega), L);
      s = run_apply(P, P->kapply, p, v, VIE_FP64, 1, true, st);
      if (s != VIE_OK) return s;
      ++inf->applies_fp64;
      q = Dots4{{rh, nullptr, nullptr, nullptr}, {v, nullptr, nullptr, nullptr}, 1};
      s = dots_host(q, L, partial, dev, d, st);
      if (s != VIE_OK) return s;
      alpha = rho / d[0];
      k_lincomb<<<eb, 256, 0, st>>>(sv, r, one, v, C(-alpha), nullptr, zero, L);
      q = Dots4{{sv, nullptr, nullptr, nullptr}, {sv, nullptr, nullptr, nullptr}, 1};
      s = dots_host(q, L, partial, dev, d, st);
      if (s != VIE_OK) return s;
      if (std::sqrt(nonneg(d[0].real())) / nb <= opt->tol) {
        k_lincomb<<<eb, 256, 0, st>>>(x, x, one, p, C(alpha), nullptr, zero, L);
        rel = std::sqrt(nonneg(d[0].real())) / nb;
        conv = true;
        ++inf->inner_iters;
        break;
      }
      s = run_apply(P, P->kapply, sv, tv, VIE_FP64, 1, true, st);
      if (s != VIE_OK) return s;
      ++inf->applies_fp64;
      q = Dots4{{tv, tv, nullptr, nullptr}, {sv, tv, nullptr, nullptr}, 2};
      s = dots_host(q, L, partial, dev, d, st);
      if (s != VIE_OK) return s;
      omega = d[0] / d[1];
      k_lincomb<<<eb, 256, 0, st>>>(x, x, one, p, C(alpha), sv, C(omega), L);
      k_lincomb<<<eb, 256, 0, st>>>(r, sv, one, tv, C(-omega), nullptr, zero, L);
      VIE_CK(cudaGetLastError());
      ++inf->inner_iters;
    }
    *worst = std::max(*worst, rel);
    if (!conv) *all_conv = false;
  }
  return VIE_OK;
}

// ||b - A x|| / ||b|| of one right-hand side with the native FP64 apply (the
// optional final check of vie_solve_opts.check_fp64).  Its scratch is its own
// stream-ordered allocation, so the solver's workspaces are left alone.
static vie_status fp64_residual(vie_problem* P, const double2* b, const double2* x, long long L, cudaStream_t st,
                                double* rel) {
  const int G = red_blocks(L);
  void* buf = nullptr;
  const size_t rbytes = ((sizeof(double2) * (size_t)L + 255) / 256) * 256;
  VIE_CK(dalloc(&buf, rbytes + sizeof(double2) * (2 * (size_t)G + 4), st));
  double2* r = (double2*)buf;
  double2* partial = (double2*)((char*)buf + rbytes);
  double2* out = partial + 2 * G;
  vie_status s = run_apply(P, P->kapply, x, r, VIE_FP64, 1, true, st);
  double2 h[2] = {make_double2(0, 0), make_double2(0, 0)};
  if (s == VIE_OK) {
    k_bminus<<<ew_blocks(L), 256, 0, st>>>(r, b, L);
    k_multidot<double2><<<dim3(G, 1), kRedThreads, 0, st>>>(r, 0, 0, r, L, partial, 2, 1);
    k_reduce_partials<<<dim3(1, 1), 256, 0, st>>>(partial, 1, G, 2, out, 2);
    k_multidot<double2><<<dim3(G, 1), kRedThreads, 0, st>>>(b, 0, 0, b, L, partial, 2, 1);
    k_reduce_partials<<<dim3(1, 1), 256, 0, st>>>(partial, 1, G, 2, out + 1, 2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "fp64 residual check");
  }
  dfree(buf, st);
  if (s != VIE_OK) return s;
  const double nb = std::sqrt(nonneg(h[1].x));
  *rel = nb > 0 ? std::sqrt(nonneg(h[0].x)) / nb : 0.0;
  return VIE_OK;
}

static vie_status check_fp64_all(vie_problem* P, const void* rhs, const void* Jv, int nrhs, cudaStream_t st,
                                 double* worst) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  *worst = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    double rel = 0.0;
    vie_status s = fp64_residual(P, (const double2*)rhs + (long long)r * L, (const double2*)Jv + (long long)r * L,
                                 L, st, &rel);
    if (s != VIE_OK) return s;
    if (!(rel <= *worst)) *worst = rel;  // keeps NaN
  }
  return VIE_OK;
}

static bool residual_fp64() {
  const char* e = getenv("VIE_RESIDUAL_FP64");
  return e && e[0] == '1';
}

vie_status run_solve(vie_problem* P, const void* rhs, void* Jv, const vie_solve_opts* opt, vie_solve_info* info,
                     cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const int m = opt->restart;
  const bool mixed = opt->mode == VIE_SOLVE_MIXED;
  vie_solve_info inf{};
  inf.t_precompute = P->t_precompute;
  inf.rel_residual_fp64 = -1.0;
  vie_status final_status = VIE_OK;
  double worst = 0.0;
  if (opt->mode == VIE_SOLVE_BICGSTAB) {
    bool all = true;
    vie_status s = run_bicgstab(P, rhs, Jv, opt, &inf, &worst, &all, st);
    if (s != VIE_OK) return s;
    VIE_CK(cudaStreamSynchronize(st));
    inf.rel_residual = worst;
    if (opt->check_fp64) {
      s = check_fp64_all(P, rhs, Jv, opt->nrhs, st, &inf.rel_residual_fp64);
      if (s != VIE_OK) return s;
    }
    inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    if (!all) {
      set_error("Bi-CGStab did not reach the tolerance within max_inner iterations");
      return VIE_ENOCONV;
    }
    return VIE_OK;
  }
  const int gsz = pick_group(P, opt->nrhs, m, mixed);
  for (int r0 = 0; r0 < opt->nrhs; r0 += gsz) {
    const int nb = std::min(gsz, opt->nrhs - r0);
    Group g;
    vie_status s = ensure_group(P, m, mixed, nb, g, st);
    if (s != VIE_OK) return s;
    const double2* b = (const double2*)rhs + (long long)r0 * L;
    double2* x = (double2*)Jv + (long long)r0 * L;
    std::vector<double> nbv, nxv, beta(nb), rel(nb, 1.0);
    s = norms_host(b, g, nbv, st);
    if (s != VIE_OK) return s;
    s = norms_host(x, g, nxv, st);
    if (s != VIE_OK) return s;
    bool x_zero = true;
    for (int r = 0; r < nb; ++r) {
      if (!std::isfinite(nbv[r])) {
        set_error("non-finite right-hand side");
        return VIE_ENAN;
      }
      if (nbv[r] == 0.0 && nxv[r] != 0.0) {
        // b = 0 has the unique solution J = 0
        VIE_CK(cudaMemsetAsync(x + (long long)r * L, 0, sizeof(double2) * L, st));
        nxv[r] = 0.0;
      }
      if (nxv[r] != 0.0) x_zero = false;
    }
    std::vector<char> conv(nb, 0);
    int total_inner = 0;
    const int max_outer = mixed ? opt->max_outer : std::max(1, opt->max_outer);
    for (int outer = 0; outer <= max_outer; ++outer) {
      // FP64 residuals r = b - A x (r = b for zero initial guesses)
      if (outer == 0 && x_zero) {
        VIE_CK(cudaMemcpyAsync(g.r, b, sizeof(double2) * nb * L, cudaMemcpyDeviceToDevice, st));
        beta = nbv;
      } else {
        // mixed: the residual in double-word arithmetic (FP64 accuracy, FP32
        // pipes); VIE_RESIDUAL_FP64=1 takes the native FP64 apply instead
        s = run_apply(P, P->kapply, x, g.r, (mixed && !residual_fp64()) ? VIE_DF64 : VIE_FP64, nb, true, st);
        if (s != VIE_OK) return s;
        inf.applies_fp64 += nb;
        k_bminus<<<ew_blocks(L * nb), 256, 0, st>>>(g.r, b, L * nb);
        VIE_CK(cudaGetLastError());
        s = norms_host(g.r, g, beta, st);
        if (s != VIE_OK) return s;
      }
      bool all = true;
      std::vector<double> stop(nb), bx(nb);
      for (int r = 0; r < nb; ++r) {
        if (!std::isfinite(beta[r])) {
          set_error("non-finite residual");
          return VIE_ENAN;
        }
        rel[r] = nbv[r] > 0 ? beta[r] / nbv[r] : 0.0;
        conv[r] = rel[r] <= opt->tol;
        if (!conv[r]) all = false;
        // converged members ride along with zero vectors
        bx[r] = conv[r] ? 0.0 : beta[r];
        // mixed: an inner solve need not go below what the overall target
        // requires; the 0.25 leaves room for the FP32 operator's own error
        stop[r] = mixed ? std::max(opt->inner_tol * beta[r], 0.25 * opt->tol * nbv[r]) : 0.5 * opt->tol * nbv[r];
      }
      if (all || outer == max_outer || total_inner >= opt->max_inner) break;
      std::vector<int> steps;
      int ap = 0;
      g.m = std::min(m, opt->max_inner - total_inner);
      if (mixed) {
        s = gmres_cycle<float2>(P, g, bx, x, stop, steps, &ap, st);
        inf.applies_fp32 += ap;
      } else {
        s = gmres_cycle<double2>(P, g, bx, x, stop, steps, &ap, st);
        inf.applies_fp64 += ap;
      }
      g.m = m;
      if (s != VIE_OK) return s;
      int smax = 0;
      for (int r = 0; r < nb; ++r) {
        smax = std::max(smax, steps[r]);
        inf.inner_iters += steps[r];
      }
      total_inner += smax;
      ++inf.outer_iters;
    }
    for (int r = 0; r < nb; ++r) {
      worst = std::max(worst, rel[r]);
      if (!conv[r]) final_status = VIE_ENOCONV;
    }
  }
  VIE_CK(cudaStreamSynchronize(st));
  inf.rel_residual = worst;
  if (opt->check_fp64) {
    vie_status s = check_fp64_all(P, rhs, Jv, opt->nrhs, st, &inf.rel_residual_fp64);
    if (s != VIE_OK) return s;
  }
  inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (final_status == VIE_ENOCONV) set_error("GMRES did not reach the tolerance within the iteration limits");
  return final_status;
}

}  // namespace vie
