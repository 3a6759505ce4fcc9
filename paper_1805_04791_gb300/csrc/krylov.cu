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
__host__ __device__ static inline double nonneg(double v) { return v < 0.0 ? 0.0 : v; }

static const int kDotChunk = 8;
static const int kArnSlots = 8;  // pinned state copies in flight (steps)
static const int kArnLag = 2;    // steps the host may issue past the state it has read
static_assert(kArnSlots == (int)(sizeof(((vie_problem*)nullptr)->arn_ev) / sizeof(cudaEvent_t)), "event slots");
static_assert(kArnSlots > kArnLag + 1, "a slot is not reused while the host may still read it");
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
// r -= y (y the FP32 apply of a refinement correction)
__global__ void k_rminus32(double2* __restrict__ r, const float2* __restrict__ y, long long L) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = y[i];
    r[i].x -= (double)v.x;
    r[i].y -= (double)v.y;
  }
}

__global__ void k_bminus(double2* __restrict__ r, const double2* __restrict__ b, long long L) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - r[e];
}

static int ew_blocks(long long L) { return (int)std::min<long long>((L + 255) / 256, 152LL * 16); }

// ------------------------------------------------ device-resident Arnoldi
// A GMRES(m) cycle runs without a host round trip per step.  The basis is kept
// unnormalised: slot i holds W_i with V_i = s_i W_i (s_i FP64, on the device),
// so the apply of step j writes A W_j straight into slot j + 1 and no scaling
// pass is needed.  Per step and group (lockstep right-hand sides, grid.y = member):
//   apply        slot j+1 = A W_j
//   k_arn_dots   (pass 0)  h_i = s_i s_j <W_i, A W_j>, |w|^2 = s_j^2 |A W_j|^2
//   k_arn_axpy   (pass 0)  W_{j+1} -= sum_i (h_i s_i / s_j) W_i and |w'|^2; the
//                          last block either asks for a second pass (|w'|^2 <
//                          |w|^2 / 16, Kahan-Parlett "twice is enough") or
//                          finalises the step
//   k_arn_dots / k_arn_axpy (pass 1)  the second classical Gram-Schmidt pass;
//                          their blocks return at entry unless it was asked for
// Finalising (one thread) applies the earlier Givens rotations to the new
// Hessenberg column, forms the next rotation, updates the residual estimate
// |g_{j+1}|, sets s_{j+1} = s_j / h_{j+1,j}, and marks the member done when the
// tolerance is reached, on breakdown (h_{j+1,j} = 0) or on a non-finite value.
// Blocks of a member that is done return at entry.  Reductions finish in the
// last block: each block stores its partial sums, fences, and counts itself in
// with an atomic; the block that completes the count reads every partial
// (bypassing L1), and resets the counter for the next kernel.
struct ArnState {
  int done;      // converged, breakdown, or non-finite
  int steps;     // completed Arnoldi steps of this cycle
  int reorth;    // the current step needs the second Gram-Schmidt pass
  int nan;       // a non-finite value was met
  double gabs;   // |g_steps|: the GMRES residual estimate
  double stop;   // absolute stopping threshold of the cycle
  double wn2;    // |w|^2 of the current step before projection
  double beta;   // initial residual norm of the cycle
  double ynorm;  // |y| of the cycle's least-squares solution: the norm of its correction
};

__host__ __device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double dnorm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 dscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// Device-side arrays of one group's Arnoldi state (carved from the Krylov workspace).
struct ArnLayout {
  int m = 0;
  int shift = 0;               // the basis spans (A - I) v: add 1 to each h_jj
  ArnState* st = nullptr;      // [nb]
  double* sc = nullptr;        // [nb][m + 2] basis scale factors s_i
  double2* R = nullptr;        // [nb][m][m + 1] rotated Hessenberg columns (upper triangle)
  double2* cs = nullptr;       // [nb][m]
  double2* sn = nullptr;       // [nb][m]
  double2* gv = nullptr;       // [nb][m + 1] rotated right-hand side of the least squares
  double2* hcol = nullptr;     // [nb][2][m + 2] coefficients of passes 0 and 1
  double2* coef = nullptr;     // [nb][m] update coefficients y_i s_i
  double2* partial = nullptr;  // [nb][m + 3][G] block partial sums
  unsigned* cnt = nullptr;     // [nb] last-block counters
};

// Whether this block completes the member's reduction (call after storing partials).
__device__ __forceinline__ bool arn_last_block(unsigned* cnt) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// Sum over blocks of partial[(r ldp + i) G + b] for i < k, one warp per i; the sum
// of slot i replaces its block-0 entry (the only reader of slot i is this warp).
__device__ __forceinline__ void arn_reduce(double2* partial, int r, int ldp, int G, int k) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < k; i += nw) {
    double2* p = partial + ((long long)r * ldp + i) * G;
    double2 sm = make_double2(0, 0);
    for (int b = lane; b < G; b += 32) sm = sm + __ldcg(p + b);
    for (int off = 16; off > 0; off >>= 1) {
      sm.x += __shfl_down_sync(0xffffffffu, sm.x, off);
      sm.y += __shfl_down_sync(0xffffffffu, sm.y, off);
    }
    __syncwarp();
    if (lane == 0) p[0] = sm;
  }
  __syncthreads();
}

// Basis values moved per 16-byte access: two FP32 complex or one FP64 complex.
template <typename TB> struct Pack;
template <> struct Pack<float2> {
  static constexpr int W = 2;
  typedef float4 P;
  static __device__ __forceinline__ float2 get(const float4& p, int q) {
    return q == 0 ? make_float2(p.x, p.y) : make_float2(p.z, p.w);
  }
  static __device__ __forceinline__ void put(float4& p, int q, float2 v) {
    if (q == 0) { p.x = v.x; p.y = v.y; } else { p.z = v.x; p.w = v.y; }
  }
};
template <> struct Pack<double2> {
  static constexpr int W = 1;
  typedef double2 P;
  static __device__ __forceinline__ double2 get(const double2& p, int) { return p; }
  static __device__ __forceinline__ void put(double2& p, int, double2 v) { p = v; }
};

// Pass p: block partials of <W_i, W_{j+1}>, i <= j (pass 0 also |W_{j+1}|^2); the last
// block stores h_i = s_i s_j <W_i, W_{j+1}> and (pass 0) |w|^2 = s_j^2 |W_{j+1}|^2.
// Vectors are read in 16-byte packs, two packs in flight per thread; ldi and L
// are multiples of the pack width except for an odd tail handled element-wise.
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_arn_dots(const TB* __restrict__ V, long long ldi, int j, long long L,
                                                          ArnLayout A, int pass) {
  typedef typename Acc<TB>::T AT;
  typedef Pack<TB> PK;
  typedef typename PK::P P;
  constexpr int W = PK::W;
  __shared__ double2 red[kRedThreads / 32][kDotChunk];
  const int r = blockIdx.y, G = gridDim.x, m = A.m, ldp = m + 3;
  ArnState* S = A.st + r;
  if (S->done || (pass == 1 && !S->reorth)) return;  // block-uniform
  const TB* Vr = V + (long long)r * L;
  const TB* wr = V + (long long)(j + 1) * ldi + (long long)r * L;
  const int k = j + 1, ktot = k + (pass == 0 ? 1 : 0);
  // packs when every vector start is pack-aligned (ldi, L multiples of W), else element-wise
  const bool packed = (W > 1) && (ldi % W == 0) && (L % W == 0);
  const long long NP = packed ? L / W : 0;  // packs per vector
  const long long stride = (long long)G * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int i0 = 0; i0 < ktot; i0 += kDotChunk) {
    const int cnt = min(kDotChunk, ktot - i0);
    AT ar[kDotChunk], ai[kDotChunk];
#pragma unroll
    for (int t = 0; t < kDotChunk; ++t) ar[t] = ai[t] = (AT)0;
    auto acc1 = [&](int t, TB v, TB we) {
      ar[t] += v.x * we.x + v.y * we.y;
      ai[t] += v.x * we.y - v.y * we.x;
    };
    if (packed) {
      const P* wp = (const P*)wr;
      long long e = tid;
      for (; e + stride < NP; e += 2 * stride) {
        const P wa = wp[e], wb = wp[e + stride];
#pragma unroll
        for (int t = 0; t < kDotChunk; ++t)
          if (t < cnt) {
            const int i = i0 + t;
            const P va = (i < k) ? ((const P*)(Vr + (long long)i * ldi))[e] : wa;
            const P vb = (i < k) ? ((const P*)(Vr + (long long)i * ldi))[e + stride] : wb;
#pragma unroll
            for (int q = 0; q < W; ++q) {
              acc1(t, PK::get(va, q), PK::get(wa, q));
              acc1(t, PK::get(vb, q), PK::get(wb, q));
            }
          }
      }
      for (; e < NP; e += stride) {
        const P wa = wp[e];
#pragma unroll
        for (int t = 0; t < kDotChunk; ++t)
          if (t < cnt) {
            const int i = i0 + t;
            const P va = (i < k) ? ((const P*)(Vr + (long long)i * ldi))[e] : wa;
#pragma unroll
            for (int q = 0; q < W; ++q) acc1(t, PK::get(va, q), PK::get(wa, q));
          }
      }
    } else {
      for (long long e = tid; e < L; e += stride) {
        const TB we = wr[e];
#pragma unroll
        for (int t = 0; t < kDotChunk; ++t)
          if (t < cnt) {
            const int i = i0 + t;
            acc1(t, (i < k) ? Vr[(long long)i * ldi + e] : we, we);
          }
      }
    }
    // warp sums in the accumulation type (slots in use only), cross-warp in FP64
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
      for (int w = 0; w < kRedThreads / 32; ++w) sm = sm + red[w][threadIdx.x];
      A.partial[((long long)r * ldp + i0 + threadIdx.x) * G + blockIdx.x] = sm;
    }
    __syncthreads();
  }
  if (!arn_last_block(A.cnt + r)) return;
  arn_reduce(A.partial, r, ldp, G, ktot);
  if (threadIdx.x == 0) A.cnt[r] = 0;
  const double* sc = A.sc + (long long)r * (m + 2);
  double2* h = A.hcol + ((long long)r * 2 + pass) * (m + 2);
  const double sj = sc[j + 1];  // scale of W_{j+1} as currently stored
  for (int i = threadIdx.x; i < ktot; i += blockDim.x) {
    const double2 raw = A.partial[((long long)r * ldp + i) * G];
    if (i < k) h[i] = dscale(sc[i] * sj, raw);
    else S->wn2 = sj * sj * raw.x;
  }
}

// Finalise step j of member r (called by the whole block, thread 0 does the
// serial part): Hessenberg column h (i <= j) and h_{j+1,j} = hn; rotations,
// residual estimate, next scale, done flag.  The column and the earlier
// rotations are staged in shared memory by all threads first, so that the
// serial rotation chain runs on shared memory instead of making a dependent
// global-memory round trip per rotation.
static const int kMaxRestart = 200;
__device__ void arn_finalize(ArnLayout& A, int r, int j, const double2* h0, const double2* h1, double hn) {
  __shared__ double2 col[kMaxRestart + 1], csh[kMaxRestart], snh[kMaxRestart];
  __shared__ int bad;
  const int m = A.m;
  ArnState* S = A.st + r;
  double2* Rc = A.R + ((long long)r * m + j) * (m + 1);
  double2* cs = A.cs + (long long)r * m;
  double2* sn = A.sn + (long long)r * m;
  double2* g = A.gv + (long long)r * (m + 1);
  double* sc = A.sc + (long long)r * (m + 2);
  if (threadIdx.x == 0) bad = !(isfinite(hn) && isfinite(S->wn2));
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double2 v = h0[i];
    if (h1) v = v + h1[i];
    if (A.shift && i == j) v.x += 1.0;  // h(A) = h(A - I) + I
    if (!(isfinite(v.x) && isfinite(v.y))) bad = 1;
    col[i] = v;
    if (i < j) {
      csh[i] = cs[i];
      snh[i] = sn[i];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (bad) {
    S->nan = 1;
    S->done = 1;
    return;
  }
  // earlier rotations G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]] on rows i, i+1
  double2 a = col[0];
  for (int i = 0; i < j; ++i) {
    const double2 b = col[i + 1];
    col[i] = cmul(dconj(csh[i]), a) + cmul(dconj(snh[i]), b);
    a = cmul(csh[i], b) - cmul(snh[i], a);
  }
  const double den = sqrt(dnorm2(a) + hn * hn);
  const double id = den > 0 ? 1.0 / den : 0.0;
  const double2 c = den > 0 ? dscale(id, a) : make_double2(1, 0);
  const double2 sv = make_double2(hn * id, 0);
  col[j] = cmul(dconj(c), a) + dscale(hn, dconj(sv));
  for (int i = 0; i <= j; ++i) Rc[i] = col[i];
  cs[j] = c;
  sn[j] = sv;
  const double2 gj = g[j];
  const double2 gn = dscale(-1.0, cmul(sv, gj));
  g[j + 1] = gn;
  g[j] = cmul(dconj(c), gj);
  S->steps = j + 1;
  S->gabs = sqrt(dnorm2(gn));
  S->reorth = 0;
  if (S->gabs <= S->stop || hn == 0.0) {
    S->done = 1;
  } else {
    sc[j + 1] /= hn;
    if (j + 1 < m) sc[j + 2] = sc[j + 1];  // W_{j+2} = A W_{j+1} starts at the scale of W_{j+1}
  }
}

// Pass p: W_{j+1} -= sum_{i <= j} (h_i s_i / s_{j+1}) W_i and block partials of
// |W_{j+1}|^2; the last block decides on the second pass (pass 0) or finalises
// the step.  s_{j+1} is the scale W_{j+1} is stored at (v = s W at unit norm).
// Pass 0 also multiplies W_{j+1} by the power of two c that brings its stored
// norm into [1/2, 1) before the projection (known from the pass-0 dots), and
// divides s_{j+1} by c: a power of two leaves every mantissa as it was, and the
// stored basis stays near unit norm.  Without it each stored vector would be
// about h_{j+1,j} times the previous one, which overflows the FP32 basis within
// a cycle when the operator norm is large (tens, at high frequency).
template <typename TB>
__global__ void __launch_bounds__(kRedThreads) k_arn_axpy(TB* __restrict__ V, long long ldi, int j, long long L,
                                                          ArnLayout A, int pass) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cf[256];
  __shared__ double red[kRedThreads / 32];
  const int r = blockIdx.y, G = gridDim.x, m = A.m, ldp = m + 3;
  ArnState* S = A.st + r;
  if (S->done || (pass == 1 && !S->reorth)) return;  // block-uniform
  double* sc = A.sc + (long long)r * (m + 2);
  const double2* h = A.hcol + ((long long)r * 2 + pass) * (m + 2);
  const int k = j + 1;
  const double u = sc[j + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double f = sc[i] / u;
    cf[i].x = (AT)(h[i].x * f);
    cf[i].y = (AT)(h[i].y * f);
  }
  // c = 2^-E with |W_{j+1}| = f 2^E, f in [1/2, 1) (|W_{j+1}|^2 = wn2 / u^2), E clamped
  // so that c stays a normal FP32 number
  int E = 0;
  if (pass == 0) {
    const double rawn = sqrt(S->wn2) / u;
    if (rawn > 0.0 && isfinite(rawn)) frexp(rawn, &E);
    E = E < -100 ? -100 : (E > 100 ? 100 : E);
  }
  const AT cscale = (AT)ldexp(1.0, -E);
  __syncthreads();
  const TB* Vr = V + (long long)r * L;
  TB* wr = V + (long long)(j + 1) * ldi + (long long)r * L;
  AT nn = 0;
  typedef Pack<TB> PK;
  typedef typename PK::P P;
  constexpr int W = PK::W;
  const bool packed = (W > 1) && (ldi % W == 0) && (L % W == 0);
  const long long NPK = packed ? L / W : L;  // units (packs or elements) per vector
  const long long stride = (long long)G * blockDim.x;
  // one unit: W elements of W_{j+1} at unit e, minus the projection, and its |.|^2
  auto unit = [&](long long e) {
    TB acc[W];
    P pw;
    if (packed) {
      pw = ((const P*)wr)[e];
#pragma unroll
      for (int q = 0; q < W; ++q) acc[q] = PK::get(pw, q);
    } else {
      acc[0] = wr[e];
    }
    AT sx[W][4], sy[W][4];
#pragma unroll
    for (int q = 0; q < W; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) sx[q][u] = sy[q][u] = 0;
    int i = 0;
    for (; i + 4 <= k; i += 4) {  // four basis loads in flight
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const typename Acc<TB>::V c = cf[i + u];
        if (packed) {
          const P pv = ((const P*)(Vr + (long long)(i + u) * ldi))[e];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            const TB v = PK::get(pv, q);
            sx[q][u] += c.x * v.x - c.y * v.y;
            sy[q][u] += c.x * v.y + c.y * v.x;
          }
        } else {
          const TB v = Vr[(long long)(i + u) * ldi + e];
          sx[0][u] += c.x * v.x - c.y * v.y;
          sy[0][u] += c.x * v.y + c.y * v.x;
        }
      }
    }
    for (; i < k; ++i) {
      const typename Acc<TB>::V c = cf[i];
      if (packed) {
        const P pv = ((const P*)(Vr + (long long)i * ldi))[e];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          const TB v = PK::get(pv, q);
          sx[q][0] += c.x * v.x - c.y * v.y;
          sy[q][0] += c.x * v.y + c.y * v.x;
        }
      } else {
        const TB v = Vr[(long long)i * ldi + e];
        sx[0][0] += c.x * v.x - c.y * v.y;
        sy[0][0] += c.x * v.y + c.y * v.x;
      }
    }
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (q == 0 || packed) {
        acc[q].x -= (sx[q][0] + sx[q][1]) + (sx[q][2] + sx[q][3]);
        acc[q].y -= (sy[q][0] + sy[q][1]) + (sy[q][2] + sy[q][3]);
        if (E != 0) {  // block-uniform
          acc[q].x *= cscale;
          acc[q].y *= cscale;
        }
        nn += acc[q].x * acc[q].x + acc[q].y * acc[q].y;
      }
    if (packed) {
#pragma unroll
      for (int q = 0; q < W; ++q) PK::put(pw, q, acc[q]);
      ((P*)wr)[e] = pw;
    } else {
      wr[e] = acc[0];
    }
  };
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NPK; e += stride) unit(e);
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += red[w];
    A.partial[((long long)r * ldp + m + 2) * G + blockIdx.x] = make_double2(t, 0.0);
  }
  if (!arn_last_block(A.cnt + r)) return;
  __shared__ double nw2s;
  __shared__ int fin;
  if (threadIdx.x < 32) {
    double t = 0;
    for (int b = threadIdx.x; b < G; b += 32) t += __ldcg(&A.partial[((long long)r * ldp + m + 2) * G + b]).x;
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) {
      A.cnt[r] = 0;
      const double us = ldexp(u, E);  // scale of the stored W_{j+1}: u / c
      sc[j + 1] = us;
      const double nw2 = nonneg(us * us * t);  // |w'|^2 at true scale
      nw2s = nw2;
      fin = 1;
      if (pass == 0 && nw2 < 0.0625 * S->wn2) {
        S->reorth = 1;  // the second pass finalises
        fin = 0;
      }
    }
  }
  __syncthreads();
  if (fin) {
    const double2* h0 = A.hcol + (long long)r * 2 * (m + 2);
    arn_finalize(A, r, j, h0, pass == 1 ? h0 + (m + 2) : nullptr, sqrt(nw2s));
  }
}

// Start of a cycle: state of member r from its residual norm beta and threshold.
__global__ void k_arn_init(ArnLayout A, const double* __restrict__ init, int nb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  const int m = A.m;
  const double beta = init[2 * r], stop = init[2 * r + 1];
  ArnState* S = A.st + r;
  S->done = (beta <= stop || beta == 0.0) ? 1 : 0;
  S->steps = 0;
  S->reorth = 0;
  S->nan = isfinite(beta) ? 0 : 1;
  S->gabs = beta;
  S->stop = stop;
  S->wn2 = 0.0;
  S->beta = beta;
  A.sc[(long long)r * (m + 2)] = 1.0;      // W_0: the normalised residual
  A.sc[(long long)r * (m + 2) + 1] = 1.0;  // W_1 = A W_0 before its projection
  double2* g = A.gv + (long long)r * (m + 1);
  g[0] = make_double2(beta, 0.0);
  A.cnt[r] = 0;
}

// End of a cycle: back substitution R y = g (k = steps) and coef_i = y_i s_i,
// one block per member: column by column from the last, the block subtracts
// R_{i'i} y_i from every earlier row in parallel.  |y| is the norm of the
// cycle's correction sum_i y_i v_i (orthonormal v_i, to the basis precision's
// orthogonality).
__global__ void k_arn_solve(ArnLayout A, int nb) {
  const int r = blockIdx.x;
  if (r >= nb) return;
  const int m = A.m, k = A.st[r].steps;
  __shared__ double2 y[kMaxRestart];
  __shared__ double red[32];
  const double2* g = A.gv + (long long)r * (m + 1);
  const double* sc = A.sc + (long long)r * (m + 2);
  for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = g[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double2* Ri = A.R + ((long long)r * m + i) * (m + 1);  // column i, rows <= i
    const double2 d = Ri[i];
    const double2 yi = dscale(1.0 / dnorm2(d), cmul(y[i], dconj(d)));
    __syncthreads();  // every thread has read y[i]
    for (int q = threadIdx.x; q < i; q += blockDim.x) y[q] = y[q] - cmul(Ri[q], yi);
    if (threadIdx.x == 0) y[i] = yi;
    __syncthreads();
  }
  double yn = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    yn += dnorm2(y[i]);
    A.coef[(long long)r * m + i] = dscale(sc[i], y[i]);
  }
  for (int off = 16; off > 0; off >>= 1) yn += __shfl_down_sync(0xffffffffu, yn, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = yn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    A.st[r].ynorm = sqrt(t);
  }
}

// x[r] += d[r] = sum_{i < steps[r]} coef[r][i] W_i[r]  (x FP64, products in TB's
// precision); d is also stored to dout[r] when dout is given (a basis slot the
// sum does not read).  grid = (blocks, nb).
template <typename TB>
__global__ void k_arn_update(double2* __restrict__ x, const TB* __restrict__ V, long long ldi, ArnLayout A,
                             long long L, TB* __restrict__ dout) {
  typedef typename Acc<TB>::T AT;
  __shared__ typename Acc<TB>::V cs[256];
  const int r = blockIdx.y, m = A.m;
  const int k = min(A.st[r].steps, 256);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    cs[i].x = (AT)A.coef[(long long)r * m + i].x;
    cs[i].y = (AT)A.coef[(long long)r * m + i].y;
  }
  __syncthreads();
  if (k == 0) {  // no correction: d = 0
    if (dout)
      for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L; e += (long long)gridDim.x * blockDim.x)
        dout[(long long)r * L + e] = TB{};
    return;
  }
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
    if (dout) {
      TB d;
      d.x = ax;
      d.y = ay;
      dout[(long long)r * L + e] = d;
    }
  }
}

struct Group {
  int nb = 1;
  int m = 1;
  long long L = 0;
  double2* partial = nullptr;  // [nb][m+3][G] (norms of the outer loop)
  double2* hdev = nullptr;     // [nb][HS]
  double2* r = nullptr;        // [nb][L] FP64
  void* V = nullptr;           // [m+1][nb][L] unnormalised basis W_i
  int HS = 0;                  // stride of hdev per rhs
  ArnLayout A;
  double* init = nullptr;      // [nb][2] device: beta, stop per member
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

// norms of two sets of nb vectors with one host synchronisation
static vie_status norms2_host(const double2* v, const double2* w, Group& g, std::vector<double>& ov,
                              std::vector<double>& ow, cudaStream_t st) {
  const int G = red_blocks(g.L);
  k_multidot<double2><<<dim3(G, g.nb), kRedThreads, 0, st>>>(v, 0, 0, v, g.L, g.partial, ldp_of(g), 1);
  k_multidot<double2><<<dim3(G, g.nb), kRedThreads, 0, st>>>(w, 0, 0, w, g.L, g.partial + G, ldp_of(g), 1);
  VIE_CK(cudaGetLastError());
  k_reduce_partials<<<dim3(1, g.nb), 256, 0, st>>>(g.partial, 1, G, ldp_of(g), g.hdev, g.HS);
  k_reduce_partials<<<dim3(1, g.nb), 256, 0, st>>>(g.partial + G, 1, G, ldp_of(g), g.hdev + 1, g.HS);
  VIE_CK(cudaGetLastError());
  std::vector<double2> h((size_t)g.nb * g.HS);
  VIE_CK(cudaMemcpyAsync(h.data(), g.hdev, sizeof(double2) * g.nb * g.HS, cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  ov.resize(g.nb);
  ow.resize(g.nb);
  for (int r = 0; r < g.nb; ++r) {
    ov[r] = std::sqrt(nonneg(h[(size_t)r * g.HS].x));
    ow[r] = std::sqrt(nonneg(h[(size_t)r * g.HS + 1].x));
  }
  return VIE_OK;
}

// CUDA graphs for single right-hand-side GMRES steps (VIE_GRAPHS=0 turns them off).
static bool graphs_enabled() {
  const char* e = getenv("VIE_GRAPHS");
  return !(e && e[0] == '0');
}

// Arnoldi on A - I (the apply's epilogue writes H u instead of x + H u): the
// same Krylov space as A's, with h_jj(A) = h_jj(A - I) + 1 added in the
// finalisation.  For these second-kind operators A v = v + (A - I) v is
// dominated by v, so projecting v out of A v cancels most of its norm and
// forces the second Gram-Schmidt pass; (A - I) v carries no such component.
// VIE_ARNOLDI_SHIFT=0 orthogonalises A v itself.
static bool arnoldi_shift() {
  const char* e = getenv("VIE_ARNOLDI_SHIFT");
  return !(e && e[0] == '0');
}

// Pinned host mirror of the group's per-member state, one slot per step in flight.
static vie_status ensure_mirror(vie_problem* P, int nb) {
  const size_t need = sizeof(ArnState) * (size_t)nb * kArnSlots;
  if (P->arn_host_bytes < need) {
    if (P->arn_host) cudaFreeHost(P->arn_host);
    P->arn_host = nullptr;
    P->arn_host_bytes = 0;
    VIE_CK(cudaMallocHost(&P->arn_host, need));
    P->arn_host_bytes = need;
  }
  for (int i = 0; i < kArnSlots; ++i)
    if (!P->arn_ev[i]) VIE_CK(cudaEventCreateWithFlags(&P->arn_ev[i], cudaEventDisableTiming));
  return VIE_OK;
}

// One GMRES(m) cycle for the whole group on the operator applied in the
// precision of TB (basis type TB), device-resident (see above).  r holds the
// FP64 residuals with norms beta[r]; x (FP64) += V y.  Members with beta = 0 or
// beta <= stop are done from the start.  Returns the steps of each member.
template <typename TB>
static vie_status gmres_cycle(vie_problem* P, Group& g, const std::vector<double>& beta, double2* x,
                              const std::vector<double>& stop_abs, std::vector<int>& steps, int* applies,
                              cudaStream_t st, TB* dout = nullptr, std::vector<double>* dnorm = nullptr) {
  const long long L = g.L;
  const int nb = g.nb, m = g.m;
  const long long ldi = (long long)nb * L;
  TB* V = (TB*)g.V;
  const int prec = sizeof(TB) == sizeof(double2) ? VIE_FP64 : VIE_FP32;
  // Arnoldi kernels: up to one 16-byte pack per thread (at most kRedBlocks blocks),
  // so that short vectors still put enough warps on every SM to hide latency;
  // their reductions finish in the last block, whatever the block count
  const long long packs = (L + 1) / 2;
  const int G = (int)std::max<long long>(1, std::min<long long>((packs + kRedThreads - 1) / kRedThreads, kRedBlocks));
  const dim3 ewg(ew_blocks(L), nb), redg(G, nb);
  vie_status s = ensure_mirror(P, nb);
  if (s != VIE_OK) return s;
  ArnState* mirror = (ArnState*)P->arn_host;
  ArnLayout A = g.A;
  A.shift = arnoldi_shift() ? 1 : 0;
  A.m = m;
  // W_0 = r / beta (s_0 = 1), and the cycle's initial state
  std::vector<double> sc(nb), init(2 * (size_t)nb);
  int active = 0;
  for (int r = 0; r < nb; ++r) {
    sc[r] = beta[r] > 0 ? 1.0 / beta[r] : 0.0;
    init[2 * r] = beta[r];
    init[2 * r + 1] = stop_abs[r];
    if (!(beta[r] <= stop_abs[r] || beta[r] == 0.0)) ++active;
  }
  VIE_CK(cudaMemcpyAsync(g.hdev, sc.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
  VIE_CK(cudaMemcpyAsync(g.init, init.data(), sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, st));
  k_scale<TB, double2><<<ewg, 256, 0, st>>>(V, g.r, (const double*)g.hdev, L);
  VIE_CK(cudaGetLastError());
  k_arn_init<<<(nb + 63) / 64, 64, 0, st>>>(A, g.init, nb);
  VIE_CK(cudaGetLastError());
  // (copies from pageable memory have left sc and init by the time they return)
  steps.assign(nb, 0);
  if (active == 0) return VIE_OK;
  // The host runs at most kArnLag steps ahead of the state it has read; when the
  // residual estimates predict convergence within that lag it waits for the
  // latest step instead, so few steps are issued after every member is done.
  std::vector<ArnState> cur, prev;  // the latest state read, and the one before it
  auto all_done = [&](const std::vector<ArnState>& ms) {
    for (int r = 0; r < nb; ++r)
      if (!ms[r].done) return false;
    return true;
  };
  auto near_done = [&]() {
    if (cur.empty() || prev.empty()) return false;
    for (int r = 0; r < nb; ++r) {
      if (cur[r].done) continue;
      const int ds = cur[r].steps - prev[r].steps;
      if (ds <= 0 || !(prev[r].gabs > 0) || !(cur[r].gabs > 0)) return true;
      const double rate = std::pow(cur[r].gabs / prev[r].gabs, 1.0 / ds);
      if (!(rate < 1.0)) return true;
      const double need = std::log(cur[r].stop / cur[r].gabs) / std::log(rate);
      if (need <= kArnLag + 1) return true;
    }
    return false;
  };
  // One step: the apply (on contiguous runs of members not yet seen as done when
  // `compact`; members that finished within the last kArnLag steps still ride
  // along, harmlessly), both Gram-Schmidt passes, and the state copy + event.
  auto enqueue_step = [&](int j, cudaStream_t ss, bool compact, bool capturing) -> vie_status {
    for (int r0 = 0; r0 < nb;) {
      if (compact && !cur.empty() && cur[r0].done) {
        ++r0;
        continue;
      }
      int r1 = r0 + 1;
      while (r1 < nb && !(compact && !cur.empty() && cur[r1].done)) ++r1;
      vie_status e = run_apply(P, P->kapply, V + (long long)j * ldi + (long long)r0 * L,
                               V + (long long)(j + 1) * ldi + (long long)r0 * L, prec, r1 - r0, A.shift ? 2 : 1, ss);
      if (e != VIE_OK) return e;
      r0 = r1;
    }
    for (int pass = 0; pass < 2; ++pass) {
      k_arn_dots<TB><<<redg, kRedThreads, 0, ss>>>(V, ldi, j, L, A, pass);
      VIE_CK(cudaGetLastError());
      k_arn_axpy<TB><<<redg, kRedThreads, 0, ss>>>(V, ldi, j, L, A, pass);
      VIE_CK(cudaGetLastError());
    }
    VIE_CK(cudaMemcpyAsync(mirror + (size_t)(j % kArnSlots) * nb, A.st, sizeof(ArnState) * nb,
                           cudaMemcpyDeviceToHost, ss));
    // inside a stream capture the record must be External to become an event-record
    // node of the graph (a plain one only expresses a dependency within the capture)
    if (capturing) VIE_CK(cudaEventRecordWithFlags(P->arn_ev[j % kArnSlots], ss, cudaEventRecordExternal));
    else VIE_CK(cudaEventRecord(P->arn_ev[j % kArnSlots], ss));
    return VIE_OK;
  };
  // Single right-hand sides replay each step as a CUDA graph (one per step index,
  // captured the first time it is needed from the second cycle with the same
  // layout on), which removes the per-kernel launch costs that dominate small
  // grids.  Everything a graph bakes in is part of the key.
  bool use_graphs = false;
  if (nb == 1 && !P->prof.on && graphs_enabled() && p3_schedule_ready(P, P->kapply, prec)) {
    s = ensure_apply_workspace(P, P->kapply, prec, nb, st);
    if (s != VIE_OK) return s;
    const std::vector<long long> key = {prec, nb, m, G, L, (long long)(uintptr_t)V, (long long)(uintptr_t)A.st,
                                        (long long)(uintptr_t)A.partial, (long long)(uintptr_t)mirror,
                                        (long long)(uintptr_t)P->ws.buf, (long long)P->ws.bytes,
                                        P->p3_variant[prec][P->kapply.mode], A.shift};
    if (key != P->graph_key) {
      for (cudaGraphExec_t ge : P->graph_exec)
        if (ge) cudaGraphExecDestroy(ge);
      P->graph_exec.clear();
      P->graph_key = key;
      P->graph_cycles = 0;
    }
    if (P->graph_cycles >= 1) {
      if (!P->cap_stream) VIE_CK(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
      for (cudaEvent_t& e : P->cap_ev)
        if (!e) VIE_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      use_graphs = true;
    }
    ++P->graph_cycles;
  }
  cudaStream_t ss = st;
  if (use_graphs) {  // the steps run on the capture stream, after everything enqueued on st
    ss = P->cap_stream;
    VIE_CK(cudaEventRecord(P->cap_ev[0], st));
    VIE_CK(cudaStreamWaitEvent(ss, P->cap_ev[0], 0));
    if ((int)P->graph_exec.size() < m) P->graph_exec.resize(m, nullptr);
  }
  int read_step = -1;
  for (int j = 0; j < m; ++j) {
    // read back the state of step j - kArnLag, or of step j - 1 near convergence
    int want = near_done() ? j - 1 : j - kArnLag;
    if (want > read_step) {
      VIE_CK(cudaEventSynchronize(P->arn_ev[want % kArnSlots]));
      const ArnState* ms = mirror + (size_t)(want % kArnSlots) * nb;
      prev.swap(cur);
      cur.assign(ms, ms + nb);
      read_step = want;
      if (all_done(cur)) break;
    }
    if (!use_graphs) {
      s = enqueue_step(j, ss, true, false);
      if (s != VIE_OK) return s;
      continue;
    }
    if (!P->graph_exec[j]) {
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(ss, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const vie_status es = enqueue_step(j, ss, false, true);
        const cudaError_t ee = cudaStreamEndCapture(ss, &graph);
        cudaGraphExec_t ge = nullptr;
        if (es == VIE_OK && ee == cudaSuccess && graph && cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess)
          P->graph_exec[j] = ge;
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();  // a failed capture leaves the step to direct launches
    }
    if (P->graph_exec[j]) {
      VIE_CK(cudaGraphLaunch(P->graph_exec[j], ss));
    } else {
      s = enqueue_step(j, ss, false, false);
      if (s != VIE_OK) return s;
    }
  }
  if (use_graphs) {
    VIE_CK(cudaEventRecord(P->cap_ev[1], ss));
    VIE_CK(cudaStreamWaitEvent(st, P->cap_ev[1], 0));
  }
  // back substitution and x += V y on the device; the final state to the host
  k_arn_solve<<<nb, 128, 0, st>>>(A, nb);
  VIE_CK(cudaGetLastError());
  k_arn_update<TB><<<ewg, 256, 0, st>>>(x, V, ldi, A, L, dout);
  VIE_CK(cudaGetLastError());
  std::vector<ArnState> fin(nb);
  VIE_CK(cudaMemcpyAsync(fin.data(), A.st, sizeof(ArnState) * nb, cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < nb; ++r) {
    if (fin[r].nan) {
      set_error("non-finite value in the Arnoldi process");
      return VIE_ENAN;
    }
    steps[r] = fin[r].steps;
    *applies += fin[r].steps;
  }
  if (dnorm) {
    dnorm->resize(nb);
    for (int r = 0; r < nb; ++r) (*dnorm)[r] = fin[r].steps > 0 ? fin[r].ynorm : 0.0;
  }
  return VIE_OK;
}

// Bytes of Krylov workspace per right-hand side.
static size_t group_bytes_per_rhs(long long L, int m, bool mixed) {
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  const size_t arn = sizeof(ArnState) + sizeof(double) * (m + 2) + sizeof(double2) * ((size_t)m * (m + 1) + 2 * m +
                     (m + 1) + 2 * (m + 2) + m) + sizeof(unsigned) + 2 * sizeof(double);
  return esz * (size_t)(m + 1) * L + sizeof(double2) * L + sizeof(double2) * ((size_t)(m + 3) * kRedBlocks +
         2 * (m + 4)) + arn + 16 * 256;
}

static vie_status ensure_group(vie_problem* P, int m, bool mixed, int nb, Group& g, cudaStream_t st) {
  const long long L = (long long)P->ncomp * P->n * P->n * P->n;
  const size_t need = group_bytes_per_rhs(L, m, mixed) * nb + 32 * 4096;
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
  g.init = (double*)take(sizeof(double) * 2 * (size_t)nb);
  g.A.m = m;
  g.A.st = (ArnState*)take(sizeof(ArnState) * (size_t)nb);
  g.A.sc = (double*)take(sizeof(double) * (size_t)nb * (m + 2));
  g.A.R = (double2*)take(sizeof(double2) * (size_t)nb * m * (m + 1));
  g.A.cs = (double2*)take(sizeof(double2) * (size_t)nb * m);
  g.A.sn = (double2*)take(sizeof(double2) * (size_t)nb * m);
  g.A.gv = (double2*)take(sizeof(double2) * (size_t)nb * (m + 1));
  g.A.hcol = (double2*)take(sizeof(double2) * (size_t)nb * 2 * (m + 2));
  g.A.coef = (double2*)take(sizeof(double2) * (size_t)nb * m);
  g.A.partial = g.partial;
  g.A.cnt = (unsigned*)take(sizeof(unsigned) * (size_t)nb);
  g.r = (double2*)take(sizeof(double2) * (size_t)nb * L);
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
                     apply_workspace_bytes(P->n, P->nk, std::max(cin_of(P->kapply.mode), cout_of(P->kapply.mode)), 1,
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
static bool residual_update_allowed() {
  const char* e = getenv("VIE_RESIDUAL_UPDATE");
  return !(e && e[0] == '0');
}

// Bound on |A_32 d - A d| for the FP32 apply of d (u = 2^-24): the normwise
// error bound of a radix-2 FFT with precomputed twiddles, log2(N) eta with
// eta = mu + gamma_4 (sqrt 2 + mu) ~ 6.7 u per level (Higham, Accuracy and
// Stability of Numerical Algorithms, 2nd ed., Sec. 24.1), for the forward and
// the inverse transform of the convolution (14 u log2(M^3)), plus 4 u for the
// rounding of d, the kernel values, the mixing and the epilogue; scaled by
// the set-up's bound ||A|| <= opnorm.
static double fp32_apply_error(const vie_problem* P, double dn) {
  const double u = 5.9604644775390625e-8;
  const double M = 2.0 * P->nk;
  return (14.0 * u * 3.0 * std::log2(M) + 4.0 * u) * P->opnorm * dn * 1.01;
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
    s = norms2_host(b, x, g, nbv, nxv, st);
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
    // mixed: after a small correction d the residual is updated as r -= A_32 d
    // (an FP32 apply) instead of recomputed as b - A x (a double-word apply),
    // when the bound on the FP32 apply's error is at most 0.7 of the tolerance
    // (the inner solve stops at 0.25 of it); err holds the accumulated bound,
    // and convergence is judged on |r| + err.
    std::vector<double> err(nb, 0.0), dn(nb, 0.0);
    bool update_next = false;
    const int max_outer = mixed ? opt->max_outer : std::max(1, opt->max_outer);
    for (int outer = 0; outer <= max_outer; ++outer) {
      // FP64 residuals r = b - A x (r = b for zero initial guesses)
      if (outer == 0 && x_zero) {
        VIE_CK(cudaMemcpyAsync(g.r, b, sizeof(double2) * nb * L, cudaMemcpyDeviceToDevice, st));
        beta = nbv;
      } else if (update_next) {
        // d is in basis slot m (FP32); its apply goes to slot 0
        float2* Vb = (float2*)g.V;
        const long long ldi = (long long)nb * L;
        s = run_apply(P, P->kapply, Vb + (long long)m * ldi, Vb, VIE_FP32, nb, true, st);
        if (s != VIE_OK) return s;
        inf.applies_fp32 += nb;
        k_rminus32<<<ew_blocks(L * nb), 256, 0, st>>>(g.r, Vb, L * nb);
        VIE_CK(cudaGetLastError());
        s = norms_host(g.r, g, beta, st);
        if (s != VIE_OK) return s;
        for (int r = 0; r < nb; ++r) err[r] += fp32_apply_error(P, dn[r]);
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
        std::fill(err.begin(), err.end(), 0.0);
      }
      bool all = true;
      std::vector<double> stop(nb), bx(nb);
      for (int r = 0; r < nb; ++r) {
        if (!std::isfinite(beta[r])) {
          set_error("non-finite residual");
          return VIE_ENAN;
        }
        rel[r] = nbv[r] > 0 ? (beta[r] + err[r]) / nbv[r] : 0.0;
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
        const bool upd = residual_update_allowed() && !residual_fp64();
        // slot m: the last basis vector, which the update of x does not read
        float2* dslot = upd ? (float2*)g.V + (long long)m * nb * L : nullptr;
        s = gmres_cycle<float2>(P, g, bx, x, stop, steps, &ap, st, dslot, upd ? &dn : nullptr);
        inf.applies_fp32 += ap;
        // update the next residual if every member's bound stays within 0.7 of the tolerance
        update_next = upd && s == VIE_OK;
        for (int r = 0; r < nb && update_next; ++r)
          if (err[r] + fp32_apply_error(P, dn[r]) > 0.7 * opt->tol * nbv[r]) update_next = false;
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
