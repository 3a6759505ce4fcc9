// The operator apply (I + B + K) x of Eqs. (eq:intLap), (eq:intH), (eq:intM),
// and the scattered-field evaluation, as a pruned zero-padded 3D convolution
// (Sec. 5: the truncated kernel transform applied with the FFT).
//
// Five passes over HBM, all shared-memory tiled with mixed-radix Stockham
// FFTs (vie_fft.cuh):
//   P1  x-lines: zero-pad n -> 2n, forward FFT          x [c][n][n][n]    -> A [c][n][n][2n]
//   P2  y-lines: zero-pad, forward FFT                   A                 -> B [c][n][2n][2n]
//   P3  z-pencils of all components: zero-pad, forward FFT, per-k kernel
//       mixing (3x3 symmetric, 6x6 Maxwell, divergence or E/H), inverse
//       FFT, keep z < n                                  B                 -> B (in place)
//   P4  y-lines: inverse FFT, keep y < n                 B                 -> A
//   P5  x-lines of all components: inverse FFT, keep x < n, epilogue
//       y = x + H u (u the convolution; H per node, 3x3 symmetric)  A      -> y
// The padded z-planes z >= n are never stored (their input is zero and their
// output is discarded).  The kernel arrays are octants of the (2n)^3 DFT with
// the identity part of T, the sign and factor 2 of B, and the 1/(2n)^3 of the
// inverse DFT folded in.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "vie_fft2.cuh"
#include "vie_internal.h"

namespace vie {

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double2* K(const KernelSet& k) { return k.oct64; }
  static const double2* H(const double2* h64, const float2*) { return h64; }
  static const double2* tw(const vie_problem* P) { return P->tw64; }
};
template <> struct Prec<float> {
  static const float2* K(const KernelSet& k) { return k.oct32; }
  static const float2* H(const double2*, const float2* h32) { return h32; }
  static const float2* tw(const vie_problem* P) { return P->tw32; }
};

template <typename V>
__device__ __forceinline__ void load_tw(V* tw, const V* __restrict__ twg, int M) {
  for (int j = flat_tid(); j < M; j += flat_nthreads()) tw[j] = twg[j];
}

// ---------------------------------------------------------------- P1
template <typename T>
__global__ void k_p1(const typename CT<T>::V* __restrict__ x, typename CT<T>::V* __restrict__ A, int n, FftPlan pl,
                     const typename CT<T>::V* __restrict__ twg, int nl, int C) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, LS = M + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + M;
  V* b1 = b0 + nl * LS;
  load_tw(tw, twg, M);
  const long long N = (long long)n * n * n;
  const int c = blockIdx.y, b = blockIdx.z, nc = gridDim.y;
  const V* src = x + ((long long)b * nc + c) * N;
  V* dst = A + ((long long)b * C + c) * ((long long)n * n * M);
  const int r0 = blockIdx.x * nl;
  const int rows = n * n;
  for (int l = threadIdx.y; l < nl; l += blockDim.y) {
    const int r = r0 + l;
    for (int j = threadIdx.x; j < M; j += blockDim.x)
      b0[l * LS + j] = (j < n && r < rows) ? src[(long long)r * n + j] : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* res = tile_fft<-1, T>(b0, b1, pl, tw, nl, LS);
  for (int l = threadIdx.y; l < nl; l += blockDim.y) {
    const int r = r0 + l;
    if (r >= rows) continue;
    for (int j = threadIdx.x; j < M; j += blockDim.x) dst[(long long)r * M + j] = res[l * LS + j];
  }
}

// ---------------------------------------------------------------- P2 / P4
// Lines along y.  FWD: in = A [bc][z][y<n][kx], out = B [bc][z][ky][kx].
//                 INV: in = B, out = A (keep y < n).
template <typename T, int S>
__global__ void k_py(const typename CT<T>::V* __restrict__ in, typename CT<T>::V* __restrict__ out, int n,
                     FftPlan pl, const typename CT<T>::V* __restrict__ twg, int nl, int C, int ncomp) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, LS = M + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + M;
  V* b1 = b0 + nl * LS;
  load_tw(tw, twg, M);
  const int kx0 = blockIdx.x * nl, z = blockIdx.y;
  const int bc = blockIdx.z;  // rhs * ncomp + comp
  const int b = bc / ncomp, c = bc - b * ncomp;
  const long long plane = ((long long)b * C + c) * n + z;  // index of the (bc, z) slab
  const int nin = (S < 0) ? n : M;                          // input rows
  const int nout = (S < 0) ? M : n;                         // output rows
  const V* src = in + plane * (long long)nin * M;
  V* dst = out + plane * (long long)nout * M;
  const int tid = flat_tid(), nt = flat_nthreads();
  for (int idx = tid; idx < nl * M; idx += nt) {
    const int j = idx / nl, l = idx - j * nl;
    b0[l * LS + j] = (j < nin) ? src[(long long)j * M + kx0 + l] : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* res = tile_fft<S, T>(b0, b1, pl, tw, nl, LS);
  for (int idx = tid; idx < nl * nout; idx += nt) {
    const int j = idx / nl, l = idx - j * nl;
    dst[(long long)j * M + kx0 + l] = res[l * LS + j];
  }
}

// ---------------------------------------------------------------- P3
template <typename V>
__device__ __forceinline__ V kval(const V* __restrict__ K, int a, long long O3, int O, int par, int kz, int ky,
                                  int kx, int n) {
  const int M = 2 * n;
  int sgn = 1;
  int oz = kz, oy = ky, ox = kx;
  if (kz > n) { oz = M - kz; if (par & 4) sgn = -sgn; }
  if (ky > n) { oy = M - ky; if (par & 2) sgn = -sgn; }
  if (kx > n) { ox = M - kx; if (par & 1) sgn = -sgn; }
  V v = K[a * O3 + ((long long)oz * O + oy) * O + ox];
  if (sgn < 0) { v.x = -v.x; v.y = -v.y; }
  return v;
}

template <typename T>
__global__ void k_p3(typename CT<T>::V* __restrict__ B, int n, FftPlan pl, const typename CT<T>::V* __restrict__ twg,
                     int nl, int C, const typename CT<T>::V* __restrict__ K, int mode) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, LS = M + 1;
  const int cin = (mode == KM_MAXWELL6) ? 6 : 3;
  const int cout = (mode == KM_SYM3) ? 3 : (mode == KM_DIV ? 1 : 6);
  const int cmax = cin > cout ? cin : cout;
  V* tw = (V*)smraw;
  V* b0 = tw + M;
  V* b1 = b0 + cmax * nl * LS;
  load_tw(tw, twg, M);
  const int kx0 = blockIdx.x * nl, ky = blockIdx.y, b = blockIdx.z;
  const long long zs = (long long)M * M;           // z stride within a component
  const long long cs = (long long)n * zs;          // component stride
  V* base = B + (long long)b * C * cs + (long long)ky * M + kx0;
  const int tid = flat_tid(), nt = flat_nthreads();
  // load: line (c, l) holds z in [0, M)
  for (int idx = tid; idx < cin * nl * M; idx += nt) {
    const int l = idx % nl;
    const int t = idx / nl;
    const int z = t % M, c = t / M;
    b0[(c * nl + l) * LS + z] = (z < n) ? base[c * cs + z * zs + l] : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* fw = tile_fft<-1, T>(b0, b1, pl, tw, cin * nl, LS);
  V* ob = (fw == b0) ? b1 : b0;
  // per-k mixing
  const int O = n + 1;
  const long long O3 = (long long)O * O * O;
  for (int idx = tid; idx < nl * M; idx += nt) {
    const int l = idx % nl, kz = idx / nl;
    const int kx = kx0 + l;
    V u[6];
    for (int c = 0; c < cin; ++c) u[c] = fw[(c * nl + l) * LS + kz];
    V o[6];
    if (mode == KM_DIV) {
      V acc = CT<T>::make(0, 0);
      for (int a = 0; a < 3; ++a) acc = acc + cmul(kval(K, a, O3, O, sym_parity(6 + a), kz, ky, kx, n), u[a]);
      o[0] = acc;
    } else {
      V q[6];
      for (int a = 0; a < 6; ++a) q[a] = kval(K, a, O3, O, sym_parity(a), kz, ky, kx, n);
      // symmetric 3x3: [xx xy xz; xy yy yz; xz yz zz]
      const V qxx = q[0], qyy = q[1], qzz = q[2], qxy = q[3], qxz = q[4], qyz = q[5];
      o[0] = cmul(qxx, u[0]) + cmul(qxy, u[1]) + cmul(qxz, u[2]);
      o[1] = cmul(qxy, u[0]) + cmul(qyy, u[1]) + cmul(qyz, u[2]);
      o[2] = cmul(qxz, u[0]) + cmul(qyz, u[1]) + cmul(qzz, u[2]);
      if (mode == KM_MAXWELL6 || mode == KM_EMRED) {
        V p[3];
        for (int a = 0; a < 3; ++a) p[a] = kval(K, 6 + a, O3, O, sym_parity(6 + a), kz, ky, kx, n);
        // P x J
        const V pxj0 = cmul(p[1], u[2]) - cmul(p[2], u[1]);
        const V pxj1 = cmul(p[2], u[0]) - cmul(p[0], u[2]);
        const V pxj2 = cmul(p[0], u[1]) - cmul(p[1], u[0]);
        if (mode == KM_EMRED) {
          o[3] = CT<T>::make(-pxj0.x, -pxj0.y);
          o[4] = CT<T>::make(-pxj1.x, -pxj1.y);
          o[5] = CT<T>::make(-pxj2.x, -pxj2.y);
        } else {
          // u[3..5] = M: Q M - P x J ; and add P x M to the J rows
          o[3] = cmul(qxx, u[3]) + cmul(qxy, u[4]) + cmul(qxz, u[5]) - pxj0;
          o[4] = cmul(qxy, u[3]) + cmul(qyy, u[4]) + cmul(qyz, u[5]) - pxj1;
          o[5] = cmul(qxz, u[3]) + cmul(qyz, u[4]) + cmul(qzz, u[5]) - pxj2;
          o[0] = o[0] + (cmul(p[1], u[5]) - cmul(p[2], u[4]));
          o[1] = o[1] + (cmul(p[2], u[3]) - cmul(p[0], u[5]));
          o[2] = o[2] + (cmul(p[0], u[4]) - cmul(p[1], u[3]));
        }
      }
    }
    for (int c = 0; c < cout; ++c) ob[(c * nl + l) * LS + kz] = o[c];
  }
  __syncthreads();
  V* iv = tile_fft<+1, T>(ob, fw, pl, tw, cout * nl, LS);
  for (int idx = tid; idx < cout * nl * n; idx += nt) {
    const int l = idx % nl;
    const int t = idx / nl;
    const int z = t % n, c = t / n;
    base[c * cs + z * zs + l] = iv[(c * nl + l) * LS + z];
  }
}

// ---------------------------------------------------------------- P5
template <typename T>
__global__ void k_p5(const typename CT<T>::V* __restrict__ A, const typename CT<T>::V* __restrict__ xin,
                     typename CT<T>::V* __restrict__ y, int n, FftPlan pl, const typename CT<T>::V* __restrict__ twg,
                     int nr, int C, int cout, const typename CT<T>::V* __restrict__ He,
                     const typename CT<T>::V* __restrict__ Hm, int with_identity) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, LS = M + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + M;
  V* b1 = b0 + cout * nr * LS;
  load_tw(tw, twg, M);
  const int r0 = blockIdx.x * nr, b = blockIdx.y;
  const int rows = n * n;
  const long long N = (long long)n * n * n;
  const long long cs = (long long)rows * M;
  const V* src = A + (long long)b * C * cs;
  for (int line = threadIdx.y; line < cout * nr; line += blockDim.y) {
    const int c = line / nr, r = r0 + line - (line / nr) * nr;
    for (int j = threadIdx.x; j < M; j += blockDim.x)
      b0[line * LS + j] = (r < rows) ? src[c * cs + (long long)r * M + j] : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* res = tile_fft<+1, T>(b0, b1, pl, tw, cout * nr, LS);
  const int tid = flat_tid(), nt = flat_nthreads();
  for (int idx = tid; idx < nr * n; idx += nt) {
    const int r = idx / n, xx = idx - r * n;
    const int row = r0 + r;
    if (row >= rows) continue;
    const long long pt = (long long)row * n + xx;
    V u[6];
    for (int c = 0; c < cout; ++c) u[c] = res[(c * nr + r) * LS + xx];
    if (with_identity) {
      for (int blk = 0; blk < cout / 3; ++blk) {
        const V* H = blk == 0 ? He : Hm;
        const V hxx = H[0 * N + pt], hyy = H[1 * N + pt], hzz = H[2 * N + pt];
        const V hxy = H[3 * N + pt], hxz = H[4 * N + pt], hyz = H[5 * N + pt];
        const V* xi = xin + ((long long)b * cout + 3 * blk) * N + pt;
        V* yo = y + ((long long)b * cout + 3 * blk) * N + pt;
        const V a0 = u[3 * blk], a1 = u[3 * blk + 1], a2 = u[3 * blk + 2];
        yo[0] = xi[0] + cmul(hxx, a0) + cmul(hxy, a1) + cmul(hxz, a2);
        yo[N] = xi[N] + cmul(hxy, a0) + cmul(hyy, a1) + cmul(hyz, a2);
        yo[2 * N] = xi[2 * N] + cmul(hxz, a0) + cmul(hyz, a1) + cmul(hzz, a2);
      }
    } else {
      for (int c = 0; c < cout; ++c) y[((long long)b * cout + c) * N + pt] = u[c];
    }
  }
}

// ------------------------------------------------ register-resident fast path
// For 2n = R1 * R2 in {64, 128, 256, 512} every line is transformed by R2
// threads with one shared-memory transpose per direction (vie_fft2.cuh).
// Thread layouts: "row" passes (x-lines, contiguous) put the R2 threads of a
// line on consecutive lanes; "column" passes (y- and z-lines, one line per
// kx) put consecutive kx on consecutive lanes.  Every global access is a
// full 128-byte (FP32) or 256-byte (FP64) segment per half-warp.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) f_p1(const typename CT<T>::V* __restrict__ x, typename CT<T>::V* __restrict__ A,
                                            int n, int C, const typename CT<T>::V* __restrict__ twg) {
  typedef Fft2<T, R1, R2> F;
  typedef typename CT<T>::V V;
  constexpr int M = F::M, L = 256 / R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  load_tw(tw, twg, M);
  const int t = threadIdx.x % R2, l = threadIdx.x / R2;
  const int rows = n * n;
  const int row = blockIdx.x * L + l;
  const bool ok = row < rows;
  const int c = blockIdx.y, b = blockIdx.z, nc = gridDim.y;
  const V* src = x + ((long long)b * nc + c) * ((long long)rows * n) + (long long)row * n;
  V u[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) u[n1] = (n1 < R1 / 2 && ok) ? src[R2 * n1 + t] : CT<T>::make(0, 0);
  __syncthreads();
  V* s = sm + l * F::LS;
  F::template fwd1<true>(u, t, s, tw);
  __syncthreads();
  V X[F::J][R2];
  F::fwd2(X, t, s);
  if (!ok) return;
  V* dst = A + ((long long)b * C + c) * ((long long)rows * M) + (long long)row * M;
#pragma unroll
  for (int j = 0; j < F::J; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) dst[t + R2 * j + R1 * k2] = X[j][k2];
}

// y-lines.  S < 0: A [bc][z][y<n][kx] -> B [bc][z][ky][kx];  S > 0: B -> A (keep y < n).
template <typename T, int R1, int R2, int S>
__global__ void __launch_bounds__(256) f_py(const typename CT<T>::V* __restrict__ in, typename CT<T>::V* __restrict__ out,
                                            int n, int C, int ncomp, const typename CT<T>::V* __restrict__ twg) {
  typedef Fft2<T, R1, R2> F;
  typedef typename CT<T>::V V;
  constexpr int M = F::M, L = 256 / R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  load_tw(tw, twg, M);
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  const int kx = blockIdx.x * L + l, z = blockIdx.y;
  const int bc = blockIdx.z;
  const int b = bc / ncomp, c = bc - b * ncomp;
  const long long plane = ((long long)b * C + c) * n + z;
  V* s = sm + l * F::LS;
  __syncthreads();
  if (S < 0) {
    const V* src = in + plane * (long long)n * M + kx;
    V u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) u[n1] = (n1 < R1 / 2) ? src[(long long)(R2 * n1 + t) * M] : CT<T>::make(0, 0);
    F::template fwd1<true>(u, t, s, tw);
    __syncthreads();
    V X[F::J][R2];
    F::fwd2(X, t, s);
    V* dst = out + plane * (long long)M * M + kx;
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) dst[(long long)(t + R2 * j + R1 * k2) * M] = X[j][k2];
  } else {
    const V* src = in + plane * (long long)M * M + kx;
    V X[F::J][R2];
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) X[j][k2] = src[(long long)(t + R2 * j + R1 * k2) * M];
    F::invA(X, t, s, tw);
    __syncthreads();
    V u[R1];
    F::template invB<true>(u, t, s);
    V* dst = out + plane * (long long)n * M + kx;
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) dst[(long long)(R2 * n1 + t) * M] = u[n1];
  }
}

// z-pencils, one component per thread group: CTA = NP pencils (consecutive
// kx) x CMAX components x R2 threads.  Each group transforms its component
// of its pencil (pruned forward FFT), parks the spectrum in shared memory,
// then each output group forms its component of the kernel product from the
// three (or six) input spectra and runs the pruned inverse FFT.  Keeping one
// component per thread holds registers near 64, so 2 CTAs (24 warps) fit an
// SM.  CTA order pairs mirror pencils (ky, M - ky) x (kx tile, mirrored tile)
// so the four CTAs reading the same kernel octant entries share them in L2.
template <int MODE> struct ModeDim;
template <> struct ModeDim<KM_SYM3> { static constexpr int CI = 3, CO = 3, NT = 3; };
template <> struct ModeDim<KM_MAXWELL6> { static constexpr int CI = 6, CO = 6, NT = 5; };
template <> struct ModeDim<KM_DIV> { static constexpr int CI = 3, CO = 1, NT = 3; };
template <> struct ModeDim<KM_EMRED> { static constexpr int CI = 3, CO = 6, NT = 3; };

// Entry i of output row c: input component b, kernel array a, sign sg.
template <int MODE>
__device__ __forceinline__ int mix_terms(int c, int* b, int* a, int* sg) {
  // symmetric 3x3 index of (p, q)
  auto qi = [](int p, int q) { return p == q ? p : (p + q == 1 ? 3 : (p + q == 2 ? 4 : 5)); };
  int nt = 0;
  if (MODE == KM_DIV) {
    for (int q = 0; q < 3; ++q) { b[nt] = q; a[nt] = q; sg[nt] = 1; ++nt; }
    return nt;
  }
  const int r = c % 3;
  const bool lower = c >= 3;  // M rows (MAXWELL6) or H rows (EMRED)
  if (!(MODE == KM_EMRED && lower)) {
    const int off = (MODE == KM_MAXWELL6 && lower) ? 3 : 0;
    for (int q = 0; q < 3; ++q) { b[nt] = off + q; a[nt] = qi(r, q); sg[nt] = 1; ++nt; }
  }
  if (MODE == KM_MAXWELL6 || (MODE == KM_EMRED && lower)) {
    // J rows: + (P x M)_r ; M rows / H rows: - (P x J)_r ;  (P x v)_r = eps_{r p q} P_p v_q
    const int voff = (MODE == KM_MAXWELL6 && !lower) ? 3 : 0;
    const int s0 = (MODE == KM_MAXWELL6 && !lower) ? 1 : -1;
    const int p1 = (r + 1) % 3, p2 = (r + 2) % 3;
    // eps_{r p1 p2} = +1: term +P_p1 v_p2 ; term -P_p2 v_p1
    b[nt] = voff + p2; a[nt] = 6 + p1; sg[nt] = s0; ++nt;
    b[nt] = voff + p1; a[nt] = 6 + p2; sg[nt] = -s0; ++nt;
  }
  return nt;
}

template <typename T, int R1, int R2, int MODE, int NP>
__global__ void __launch_bounds__(NP * R2 * (ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO))
f_p3b(typename CT<T>::V* __restrict__ B, int n, int C, const typename CT<T>::V* __restrict__ K,
      const typename CT<T>::V* __restrict__ twg) {
  typedef Fft2<T, R1, R2> F;
  typedef typename CT<T>::V V;
  constexpr int CI = ModeDim<MODE>::CI, CO = ModeDim<MODE>::CO, NT = ModeDim<MODE>::NT;
  constexpr int CMAX = CI > CO ? CI : CO;
  constexpr int M = F::M, NTX = M / NP, NTHR = NP * R2 * CMAX;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  const int v = blockIdx.x & 3, g = blockIdx.x >> 2;
  const int kyp = g / (NTX / 2), txp = g - kyp * (NTX / 2);
  if ((v & 1) && (kyp == 0 || kyp == M / 2)) return;  // self-mirrored rows
  const int ky = (v & 1) ? M - kyp : kyp;
  const int tile = (v & 2) ? NTX - 1 - txp : txp;
  for (int j = threadIdx.x; j < M; j += NTHR) tw[j] = twg[j];
  const int l = threadIdx.x % NP, t = (threadIdx.x / NP) % R2, c = threadIdx.x / (NP * R2);
  const int kx = tile * NP + l;
  const int b0 = blockIdx.y;
  const long long zs = (long long)M * M, cs = (long long)n * zs;
  V* colbase = B + (long long)b0 * C * cs + (long long)ky * M + kx;
  V* s = sm + (c * NP + l) * F::LS;
  // pruned forward FFT of component c
  V X[F::J][R2];
  if (c < CI) {
    V u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1)
      u[n1] = (n1 < R1 / 2) ? colbase[c * cs + (long long)(R2 * n1 + t) * zs] : CT<T>::make(0, 0);
    __syncthreads();
    F::template fwd1<true>(u, t, s, tw);
  } else {
    __syncthreads();
  }
  __syncthreads();
  if (c < CI) F::fwd2(X, t, s);
  __syncthreads();
  if (c < CI) {
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) s[t + R2 * j + R1 * k2] = X[j][k2];
  }
  __syncthreads();
  // kernel mixing for output component c
  if (c < CO) {
    int tb[NT], ta[NT], tsg[NT];
    const int ntm = mix_terms<MODE>(c, tb, ta, tsg);
    const int O = n + 1;
    const long long O3 = (long long)O * O * O;
    const bool fy = ky > n, fx = kx > n;
    const int oy = fy ? M - ky : ky, ox = fx ? M - kx : kx;
    const long long rowoff = (long long)oy * O + ox;
    bool neg0[NT], zodd[NT];
    const V* kp[NT];
    const V* xs[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      if (i >= ntm) break;
      const int par = sym_parity(MODE == KM_DIV ? 6 + ta[i] : ta[i]);  // divergence kernels are i k_a (odd)
      neg0[i] = (((par & 2) && fy) != ((par & 1) && fx)) != (tsg[i] < 0);
      zodd[i] = (par & 4) != 0;
      kp[i] = K + ta[i] * O3 + rowoff;
      xs[i] = sm + (tb[i] * NP + l) * F::LS;
    }
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int k = t + R2 * j + R1 * k2;
        const bool fz = k > n;
        const long long zoff = (long long)(fz ? M - k : k) * O * O;
        V acc = CT<T>::make(0, 0);
#pragma unroll
        for (int i = 0; i < NT; ++i) {
          if (i >= ntm) break;
          V kv = kp[i][zoff];
          if (neg0[i] != (zodd[i] && fz)) { kv.x = -kv.x; kv.y = -kv.y; }
          acc = acc + cmul(kv, xs[i][k]);
        }
        X[j][k2] = acc;
      }
  }
  __syncthreads();
  if (c < CO) F::invA(X, t, s, tw);
  __syncthreads();
  if (c < CO) {
    V u[R1];
    F::template invB<true>(u, t, s);
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) colbase[c * cs + (long long)(R2 * n1 + t) * zs] = u[n1];
  }
}

// z-pencils, mirror-group variant.  One CTA owns the (up to) four pencil
// tiles that read the same kernel octant entries -- (ky, M-ky) x (kx tile,
// mirrored kx tile) -- stages those entries once in shared memory ([narr]
// [n+1 octant z][NP+1 octant x]) and then transforms the tiles one after the
// other.  Kernel reads drop from ~12 L2 reads per octant value to ~1, and the
// mixing reads only shared memory.  The line pitch of the transpose buffers
// is chosen so that 8 pencils x 2 threads (FP32) or 8 pencils (FP64) hit
// distinct banks.
template <int MODE, int NP, int R2>
struct P3cThreads {
  static constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
  static constexpr int N = NP * R2 * CMAX;
  static constexpr int MINB = N <= 384 ? 2 : 1;
};

template <typename T, int R1, int R2, int MODE, int NP>
__global__ void __launch_bounds__(P3cThreads<MODE, NP, R2>::N, P3cThreads<MODE, NP, R2>::MINB)
f_p3c(typename CT<T>::V* __restrict__ B, int n, int C, const typename CT<T>::V* __restrict__ K,
      const typename CT<T>::V* __restrict__ twg) {
  typedef Fft2<T, R1, R2> F;
  typedef typename CT<T>::V V;
  constexpr int CI = ModeDim<MODE>::CI, CO = ModeDim<MODE>::CO, NT = ModeDim<MODE>::NT;
  constexpr int CMAX = CI > CO ? CI : CO;
  constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
  constexpr int M = F::M, NTX = M / NP, NTHR = NP * R2 * CMAX;
  constexpr int LS = (sizeof(V) == 8) ? ((F::LS0 + 13) / 16) * 16 + 2 : (F::LS0 | 1);
  constexpr int QW = NP + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  V* slab = sm + CMAX * NP * LS;
  const int kyp = blockIdx.x / (NTX / 2), txp = blockIdx.x - (blockIdx.x / (NTX / 2)) * (NTX / 2);
  const int O = n + 1;
  const long long O3 = (long long)O * O * O;
  for (int j = threadIdx.x; j < M; j += NTHR) tw[j] = twg[j];
  {
    const int tot = NARR * O * QW;
    const V* src = K + ((long long)kyp) * O + NP * txp;
    for (int idx = threadIdx.x; idx < tot; idx += NTHR) {
      const int q = idx % QW, r = idx / QW;
      const int oz = r % O, a = r / O;
      slab[idx] = src[a * O3 + (long long)oz * O * O + q];
    }
  }
  const int l = threadIdx.x % NP, t = (threadIdx.x / NP) % R2, c = threadIdx.x / (NP * R2);
  const int b0 = blockIdx.y;
  const long long zs = (long long)M * M, cs = (long long)n * zs;
  V* s = sm + (c * NP + l) * LS;
  // mixing terms of this thread's output component (fixed for the CTA)
  int tb[NT], ta[NT], tsg[NT];
  const int ntm = (c < CO) ? mix_terms<MODE>(c, tb, ta, tsg) : 0;
  const bool self_y = (kyp == 0 || kyp == M / 2);
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    if ((v & 1) && self_y) continue;  // block-uniform
    const int ky = (v & 1) ? M - kyp : kyp;
    const int tile = (v & 2) ? NTX - 1 - txp : txp;
    const int kx = tile * NP + l;
    V* colbase = B + (long long)b0 * C * cs + (long long)ky * M + kx;
    V X[F::J][R2];
    V u[R1];
    if (c < CI) {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1)
        u[n1] = (n1 < R1 / 2) ? colbase[c * cs + (long long)(R2 * n1 + t) * zs] : CT<T>::make(0, 0);
    }
    __syncthreads();  // previous tile's readers of s are done; slab and tw are visible
    if (c < CI) F::template fwd1<true>(u, t, s, tw);
    __syncthreads();
    if (c < CI) F::fwd2(X, t, s);
    __syncthreads();
    if (c < CI) {
#pragma unroll
      for (int j = 0; j < F::J; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) s[t + R2 * j + R1 * k2] = X[j][k2];
    }
    __syncthreads();
    if (c < CO) {
      const bool fy = ky > n, fx = kx > n;
      const int q = (fx ? M - kx : kx) - NP * txp;
      // per term: kernel pointer, input spectrum, and the sign for kz <= n / kz > n
      T sg0[NT], sg1[NT];
      const V* kp[NT];
      const V* xs[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        if (i >= ntm) break;
        const int par = sym_parity(MODE == KM_DIV ? 6 + ta[i] : ta[i]);
        const bool neg0 = (((par & 2) && fy) != ((par & 1) && fx)) != (tsg[i] < 0);
        sg0[i] = neg0 ? (T)-1 : (T)1;
        sg1[i] = (neg0 != ((par & 4) != 0)) ? (T)-1 : (T)1;
        kp[i] = slab + ta[i] * O * QW + q;
        xs[i] = sm + (tb[i] * NP + l) * LS;
      }
#pragma unroll
      for (int j = 0; j < F::J; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int k = t + R2 * j + R1 * k2;
          // k < n for k2 < R2/2 and k > n for k2 > R2/2 (k = R1 k2 + [0, R1)); only k2 = R2/2 depends on t, j
          const bool fz = (k2 < R2 / 2) ? false : ((k2 > R2 / 2) ? true : (k > n));
          const int zoff = (fz ? M - k : k) * QW;
          T ax = 0, ay = 0;
#pragma unroll
          for (int i = 0; i < NT; ++i) {
            if (i >= ntm) break;
            const V kv = kp[i][zoff];
            const V xv = xs[i][k];
            const T sgn = fz ? sg1[i] : sg0[i];
            const T px = kv.x * xv.x - kv.y * xv.y;
            const T py = kv.x * xv.y + kv.y * xv.x;
            ax = fma(sgn, px, ax);
            ay = fma(sgn, py, ay);
          }
          X[j][k2] = CT<T>::make(ax, ay);
        }
    }
    __syncthreads();
    if (c < CO) F::invA(X, t, s, tw);
    __syncthreads();
    if (c < CO) {
      F::template invB<true>(u, t, s);
#pragma unroll
      for (int n1 = 0; n1 < R1 / 2; ++n1) colbase[c * cs + (long long)(R2 * n1 + t) * zs] = u[n1];
    }
  }
}

// x-lines of all components: inverse, keep x < n, epilogue y = x + H u (or
// y = u).  CO = 3 (one H block) or 6 ([J; M] with H_eps and H_mu, or [E; H]).
template <typename T, int R1, int R2, int CO>
__global__ void __launch_bounds__(256) f_p5(const typename CT<T>::V* __restrict__ A,
                                            const typename CT<T>::V* __restrict__ xin, typename CT<T>::V* __restrict__ y,
                                            int n, int C, int cout, const typename CT<T>::V* __restrict__ He,
                                            const typename CT<T>::V* __restrict__ Hm, int with_identity,
                                            const typename CT<T>::V* __restrict__ twg) {
  typedef Fft2<T, R1, R2> F;
  typedef typename CT<T>::V V;
  constexpr int M = F::M, L = 256 / R2, H2 = R1 / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  load_tw(tw, twg, M);
  const int t = threadIdx.x % R2, l = threadIdx.x / R2;
  const int rows = n * n;
  const int row = blockIdx.x * L + l;
  const bool ok = row < rows;
  const int b = blockIdx.y;
  const long long N = (long long)rows * n;
  const long long cs = (long long)rows * M;
  V* s = sm + l * F::LS;
  V uo[CO][H2];
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CO; ++c) {
    if (c >= cout) break;
    const V* src = A + ((long long)b * C + c) * cs + (long long)row * M;
    V X[F::J][R2];
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) X[j][k2] = ok ? src[t + R2 * j + R1 * k2] : CT<T>::make(0, 0);
    F::invA(X, t, s, tw);
    __syncthreads();
    V u[R1];
    F::template invB<true>(u, t, s);
#pragma unroll
    for (int n1 = 0; n1 < H2; ++n1) uo[c][n1] = u[n1];
    __syncthreads();
  }
  if (!ok) return;
#pragma unroll
  for (int n1 = 0; n1 < H2; ++n1) {
    const long long pt = (long long)row * n + R2 * n1 + t;
    if (with_identity) {
#pragma unroll
      for (int blk = 0; blk < CO / 3; ++blk) {
        const V* H = blk == 0 ? He : Hm;
        const V hxx = H[pt], hyy = H[N + pt], hzz = H[2 * N + pt];
        const V hxy = H[3 * N + pt], hxz = H[4 * N + pt], hyz = H[5 * N + pt];
        const V* xi = xin + ((long long)b * CO + 3 * blk) * N + pt;
        V* yo = y + ((long long)b * CO + 3 * blk) * N + pt;
        const V a0 = uo[3 * blk][n1], a1 = uo[3 * blk + 1][n1], a2 = uo[3 * blk + 2][n1];
        yo[0] = xi[0] + cmul(hxx, a0) + cmul(hxy, a1) + cmul(hxz, a2);
        yo[N] = xi[N] + cmul(hxy, a0) + cmul(hyy, a1) + cmul(hyz, a2);
        yo[2 * N] = xi[2 * N] + cmul(hxz, a0) + cmul(hyz, a1) + cmul(hzz, a2);
      }
    } else {
#pragma unroll
      for (int c = 0; c < CO; ++c)
        if (c < cout) y[((long long)b * cout + c) * N + pt] = uo[c][n1];
    }
  }
}

// ---------------------------------------------------------------- host
static int pow2_divisor(int M, int target) {
  int nl = target;
  while (nl > 1 && M % nl != 0) nl >>= 1;
  return nl;
}

static dim3 line_block(int M) {
  int tx = 1;
  while (tx * 16 < M && tx < 32) tx <<= 1;
  return dim3(tx, 256 / tx);
}

size_t apply_workspace_bytes(int n, int c, int nrhs, int prec) {
  const size_t esz = prec == VIE_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t M = 2 * (size_t)n;
  return esz * (size_t)nrhs * c * ((size_t)n * n * M + (size_t)n * M * M);
}

// Fast-path launches for 2n = R1 R2; returns false if a pass must use the generic kernels.
template <typename T, int R1, int R2>
struct FastPath {
  typedef typename CT<T>::V V;
  static constexpr int M = R1 * R2, L = 256 / R2;
  static size_t smem() { return sizeof(V) * (M + L * Fft2<T, R1, R2>::LS); }
  static vie_status p1(const V* x, V* A, int n, int C, int cin, int nrhs, const V* tw, cudaStream_t st) {
    VIE_CK(cudaFuncSetAttribute(f_p1<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()));
    f_p1<T, R1, R2><<<dim3((n * n + L - 1) / L, cin, nrhs), 256, smem(), st>>>(x, A, n, C, tw);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
  template <int S>
  static vie_status py(const V* in, V* out, int n, int C, int nc, int nrhs, const V* tw, cudaStream_t st) {
    VIE_CK(cudaFuncSetAttribute(f_py<T, R1, R2, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()));
    f_py<T, R1, R2, S><<<dim3(M / L, n, nrhs * nc), 256, smem(), st>>>(in, out, n, C, nc, tw);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
  template <int MODE, int NP>
  static vie_status p3b(V* B, int n, int C, const V* K, int nrhs, const V* tw, cudaStream_t st) {
    constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
    constexpr int NTX = M / NP;
    const size_t sm = sizeof(V) * (M + (size_t)CMAX * NP * Fft2<T, R1, R2>::LS);
    VIE_CK(cudaFuncSetAttribute(f_p3b<T, R1, R2, MODE, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    f_p3b<T, R1, R2, MODE, NP><<<dim3((M / 2 + 1) * (NTX / 2) * 4, nrhs), NP * R2 * CMAX, sm, st>>>(B, n, C, K, tw);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
  template <int MODE, int NP>
  static vie_status p3c(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    typedef Fft2<T, R1, R2> F;
    constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
    constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
    constexpr int LS = (sizeof(V) == 8) ? ((F::LS0 + 13) / 16) * 16 + 2 : (F::LS0 | 1);
    constexpr int NTX = M / NP;
    constexpr int NTHR = P3cThreads<MODE, NP, R2>::N;
    const size_t sm = sizeof(V) * (M + (size_t)CMAX * NP * LS + (size_t)NARR * (n + 1) * (NP + 1));
    const size_t cap = P3cThreads<MODE, NP, R2>::MINB == 2 ? 112 * 1024 : 224 * 1024;
    *done = false;
    if constexpr (NTHR > 1024 || NTX < 2) {
      return VIE_OK;  // shape not expressible: not instantiated
    } else {
      if (sm > cap) return VIE_OK;
      VIE_CK(cudaFuncSetAttribute(f_p3c<T, R1, R2, MODE, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      f_p3c<T, R1, R2, MODE, NP><<<dim3((M / 2 + 1) * (NTX / 2), nrhs), NTHR, sm, st>>>(B, n, C, K, tw);
      VIE_CK(cudaGetLastError());
      *done = true;
      return VIE_OK;
    }
  }
  template <int MODE, int NP>
  static vie_status p3b_ok(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
    *done = false;
    if constexpr (NP * R2 * CMAX > 1024 || M / NP < 2) {
      return VIE_OK;
    } else {
      vie_status e = p3b<MODE, NP>(B, n, C, K, nrhs, tw, st);
      *done = (e == VIE_OK);
      return e;
    }
  }
  template <int MODE>
  static vie_status p3_mode(int variant, V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done,
                            cudaStream_t st) {
    switch (variant) {
      case 0: return p3c<MODE, 8>(B, n, C, K, nrhs, tw, done, st);
      case 1: return p3c<MODE, 16>(B, n, C, K, nrhs, tw, done, st);
      case 2: return p3c<MODE, 4>(B, n, C, K, nrhs, tw, done, st);
      case 3: return p3b_ok<MODE, 8>(B, n, C, K, nrhs, tw, done, st);
      default: return p3b_ok<MODE, 4>(B, n, C, K, nrhs, tw, done, st);
    }
  }
  // Run P3 variant `variant` (0..kP3Variants-1); *done = false if it does not apply to this shape.
  static vie_status p3v(int variant, V* B, int n, int C, const V* K, int mode, int nrhs, const V* tw, bool* done,
                        cudaStream_t st) {
    switch (mode) {
      case KM_SYM3: return p3_mode<KM_SYM3>(variant, B, n, C, K, nrhs, tw, done, st);
      case KM_DIV: return p3_mode<KM_DIV>(variant, B, n, C, K, nrhs, tw, done, st);
      case KM_EMRED: return p3_mode<KM_EMRED>(variant, B, n, C, K, nrhs, tw, done, st);
      default: return p3_mode<KM_MAXWELL6>(variant, B, n, C, K, nrhs, tw, done, st);
    }
  }
  static vie_status p5(const V* A, const V* xin, V* y, int n, int C, int cout, const V* He, const V* Hm, bool wid,
                       int nrhs, const V* tw, cudaStream_t st) {
    const dim3 grid((n * n + L - 1) / L, nrhs);
    if (cout <= 3) {
      VIE_CK(cudaFuncSetAttribute(f_p5<T, R1, R2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()));
      f_p5<T, R1, R2, 3><<<grid, 256, smem(), st>>>(A, xin, y, n, C, cout, He, Hm, wid ? 1 : 0, tw);
    } else {
      VIE_CK(cudaFuncSetAttribute(f_p5<T, R1, R2, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()));
      f_p5<T, R1, R2, 6><<<grid, 256, smem(), st>>>(A, xin, y, n, C, cout, He, Hm, wid ? 1 : 0, tw);
    }
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
};

// Which passes may take the register-resident path.
struct FastSel {
  bool p1 = false, py = false, p3 = false, p5 = false;
};

static FastSel fast_select(int M, int mode, bool with_identity) {
  FastSel f;
  if (M != 64 && M != 128 && M != 256 && M != 512) return f;
  if (getenv("VIE_GENERIC_FFT")) return f;
  const int cin = cin_of(mode), cout = cout_of(mode);
  f.p1 = true;
  f.py = true;
  f.p3 = true;
  f.p5 = (cout <= 3 || cout == 6) && (!with_identity || cout == cin);
  return f;
}

template <typename T, int R1, int R2>
static vie_status fast_pass(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                            bool with_identity, typename CT<T>::V* A, typename CT<T>::V* B, int C, cudaStream_t st) {
  typedef FastPath<T, R1, R2> FP;
  typedef typename CT<T>::V V;
  const int n = P->n;
  const V* tw = Prec<T>::tw(P);
  const int cin = cin_of(K.mode), cout = cout_of(K.mode);
  switch (pass) {
    case 1: return FP::p1((const V*)in, A, n, C, cin, nrhs, tw, st);
    case 2: return FP::template py<-1>(A, B, n, C, cin, nrhs, tw, st);
    case 3: {
      bool done = false;
      vie_status e = FP::p3v(P->p3_variant[sizeof(T) == 8 ? 0 : 1][K.mode], B, n, C, Prec<T>::K(K), K.mode, nrhs,
                             tw, &done, st);
      if (e == VIE_OK && !done) {
        set_error("selected z-pass variant does not apply to this shape");
        return VIE_EINVAL;
      }
      return e;
    }
    case 4: return FP::template py<+1>(B, A, n, C, cout, nrhs, tw, st);
    default:
      return FP::p5(A, (const V*)in, (V*)out, n, C, cout, Prec<T>::H(P->He64, P->He32),
                    P->has_mu ? Prec<T>::H(P->Hm64, P->Hm32) : nullptr, with_identity, nrhs, tw, st);
  }
}

template <typename T>
static vie_status fast_dispatch(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                                bool with_identity, typename CT<T>::V* A, typename CT<T>::V* B, int C,
                                cudaStream_t st) {
  switch (2 * P->n) {
    case 64: return fast_pass<T, 8, 8>(pass, P, K, in, out, nrhs, with_identity, A, B, C, st);
    case 128: return fast_pass<T, 16, 8>(pass, P, K, in, out, nrhs, with_identity, A, B, C, st);
    case 256: return fast_pass<T, 16, 16>(pass, P, K, in, out, nrhs, with_identity, A, B, C, st);
    default: return fast_pass<T, 32, 16>(pass, P, K, in, out, nrhs, with_identity, A, B, C, st);
  }
}

// Autotuner for the z pass: every applicable variant (mirror-group CTAs with
// 8, 16 or 4 pencils, or one tile per CTA with 8 or 4 pencils) is launched once
// to warm up and then timed over 3 launches with CUDA events on the buffer B
// (whose contents are scratch at this point); the fastest is kept for the
// problem's (precision, mode).  VIE_TUNE=0 takes the first applicable variant;
// VIE_P3_VARIANT=k forces variant k.
static const int kP3Variants = 5;

static std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
static std::map<long long, int>& tune_cache() {
  static std::map<long long, int> c;
  return c;
}

template <typename T, int R1, int R2>
static vie_status tune_p3(vie_problem* P, const KernelSet& K, typename CT<T>::V* B, int C, cudaStream_t st,
                          int* best) {
  typedef FastPath<T, R1, R2> FP;
  const typename CT<T>::V* tw = Prec<T>::tw(P);
  const char* force = getenv("VIE_P3_VARIANT");
  const char* tune = getenv("VIE_TUNE");
  const bool timed = !(tune && tune[0] == '0');
  *best = -1;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  VIE_CK(cudaEventCreate(&e0));
  VIE_CK(cudaEventCreate(&e1));
  for (int v = 0; v < kP3Variants; ++v) {
    if (force && atoi(force) != v) continue;
    bool done = false;
    vie_status s = FP::p3v(v, B, P->n, C, Prec<T>::K(K), K.mode, 1, tw, &done, st);
    if (s != VIE_OK) return s;
    if (!done) continue;
    if (!timed || force) {
      *best = v;
      break;
    }
    VIE_CK(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) FP::p3v(v, B, P->n, C, Prec<T>::K(K), K.mode, 1, tw, &done, st);
    VIE_CK(cudaEventRecord(e1, st));
    VIE_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    VIE_CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      *best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*best < 0) {
    set_error("no z-pass variant applies to this shape");
    return VIE_EINVAL;
  }
  return VIE_OK;
}

template <typename T>
static vie_status tune_dispatch(vie_problem* P, const KernelSet& K, typename CT<T>::V* B, int C, cudaStream_t st,
                                int* best) {
  switch (2 * P->n) {
    case 64: return tune_p3<T, 8, 8>(P, K, B, C, st, best);
    case 128: return tune_p3<T, 16, 8>(P, K, B, C, st, best);
    case 256: return tune_p3<T, 16, 16>(P, K, B, C, st, best);
    default: return tune_p3<T, 32, 16>(P, K, B, C, st, best);
  }
}

template <typename T>
static vie_status run_apply_t(vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                              bool with_identity, cudaStream_t st) {
  typedef typename CT<T>::V V;
  const int n = P->n, M = 2 * n;
  const int cin = cin_of(K.mode), cout = cout_of(K.mode);
  const int C = std::max(cin, cout);
  const size_t need = apply_workspace_bytes(n, C, nrhs, sizeof(T) == 8 ? VIE_FP64 : VIE_FP32);
  if (P->ws.bytes < need) {
    dfree(P->ws.buf, st);  // stream-ordered: earlier work on st completes first
    P->ws.buf = nullptr;
    P->ws.bytes = 0;
    cudaError_t e = dalloc(&P->ws.buf, need, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("out of device memory for the apply workspace");
      return VIE_ENOMEM;
    }
    P->ws.bytes = need;
  }
  V* A = (V*)P->ws.buf;
  V* B = A + (size_t)nrhs * C * n * n * M;
  const V* tw = Prec<T>::tw(P);
  const V* Kp = Prec<T>::K(K);
  const FftPlan& pl = P->plan2n;
  const dim3 blk = line_block(M);
  const size_t vs = sizeof(V);
  Profiler& pf = P->prof;
  const bool rec = pf.on && pf.count < pf.cap;
  cudaEvent_t* ev = rec ? &pf.ev[(size_t)pf.count * (kProfSlots + 1)] : nullptr;
  if (rec) {
    VIE_CK(cudaEventRecord(ev[0], st));
    ++pf.count;
  }

  const FastSel fs = fast_select(M, K.mode, with_identity);
  int& p3v = P->p3_variant[sizeof(T) == 8 ? 0 : 1][K.mode];
  if (fs.p3 && p3v < 0) {
    // one decision per (n, precision, mode) per process: every problem of a
    // shape then runs the same arithmetic (bitwise-reproducible results)
    const long long key = ((long long)P->n * 2 + (sizeof(T) == 8 ? 0 : 1)) * 8 + K.mode;
    {
      std::lock_guard<std::mutex> g(tune_mutex());
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) p3v = it->second;
    }
    if (p3v < 0) {
      vie_status e = tune_dispatch<T>(P, K, B, C, st, &p3v);
      if (e != VIE_OK) return e;
      std::lock_guard<std::mutex> g(tune_mutex());
      tune_cache().emplace(key, p3v);
      p3v = tune_cache()[key];
    }
  }
  // P1
  if (fs.p1) {
    vie_status e = fast_dispatch<T>(1, P, K, in, out, nrhs, with_identity, A, B, C, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[1], st));
  } else {
    const int nl = (int)blk.y;
    const size_t smem = vs * (M + 2 * nl * (M + 1));
    VIE_CK(cudaFuncSetAttribute(k_p1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((n * n + nl - 1) / nl, cin, nrhs);
    k_p1<T><<<grid, blk, smem, st>>>((const V*)in, A, n, pl, tw, nl, C);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[1], st));
  }
  const int nly = pow2_divisor(M, sizeof(T) == 8 ? 8 : 16);
  const size_t smem_y = vs * (M + 2 * nly * (M + 1));
  // P2
  if (fs.py) {
    vie_status e = fast_dispatch<T>(2, P, K, in, out, nrhs, with_identity, A, B, C, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[2], st));
  } else {
    VIE_CK(cudaFuncSetAttribute(k_py<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y));
    dim3 grid(M / nly, n, nrhs * cin);
    k_py<T, -1><<<grid, blk, smem_y, st>>>(A, B, n, pl, tw, nly, C, cin);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[2], st));
  }
  // P3
  if (fs.p3) {
    vie_status e = fast_dispatch<T>(3, P, K, in, out, nrhs, with_identity, A, B, C, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[3], st));
  } else {
    int nl = pow2_divisor(M, 8);
    while (nl > 1 && vs * (M + 2 * C * nl * (M + 1)) > 200 * 1024) nl >>= 1;
    const size_t smem = vs * (M + 2 * C * nl * (M + 1));
    VIE_CK(cudaFuncSetAttribute(k_p3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(M / nl, M, nrhs);
    k_p3<T><<<grid, blk, smem, st>>>(B, n, pl, tw, nl, C, Kp, K.mode);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[3], st));
  }
  // P4
  if (fs.py) {
    vie_status e = fast_dispatch<T>(4, P, K, in, out, nrhs, with_identity, A, B, C, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[4], st));
  } else {
    VIE_CK(cudaFuncSetAttribute(k_py<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y));
    dim3 grid(M / nly, n, nrhs * cout);
    k_py<T, +1><<<grid, blk, smem_y, st>>>(B, A, n, pl, tw, nly, C, cout);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[4], st));
  }
  // P5
  if (fs.p5) {
    vie_status e = fast_dispatch<T>(5, P, K, in, out, nrhs, with_identity, A, B, C, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[5], st));
  } else {
    int nr = 4;
    while (nr > 1 && vs * (M + 2 * cout * nr * (M + 1)) > 200 * 1024) nr >>= 1;
    const size_t smem = vs * (M + 2 * cout * nr * (M + 1));
    VIE_CK(cudaFuncSetAttribute(k_p5<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((n * n + nr - 1) / nr, nrhs);
    const V* He = Prec<T>::H(P->He64, P->He32);
    const V* Hm = P->has_mu ? Prec<T>::H(P->Hm64, P->Hm32) : nullptr;
    k_p5<T><<<grid, blk, smem, st>>>(A, (const V*)in, (V*)out, n, pl, tw, nr, C, cout, He, Hm,
                                     with_identity ? 1 : 0);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[5], st));
  }
  return VIE_OK;
}

vie_status tune_apply(vie_problem* P, const KernelSet& K, int prec, int* variant, cudaStream_t st) {
  const int M = 2 * P->n;
  if (!fast_select(M, K.mode, true).p3) {
    *variant = -1;
    return VIE_OK;
  }
  int& v = P->p3_variant[prec == VIE_FP64 ? 0 : 1][K.mode];
  v = -1;
  {
    std::lock_guard<std::mutex> g(tune_mutex());
    tune_cache().erase(((long long)P->n * 2 + (prec == VIE_FP64 ? 0 : 1)) * 8 + K.mode);
  }
  // an apply of a zero vector allocates the workspace and tunes on its first call
  const long long L = (long long)cin_of(K.mode) * P->n * P->n * P->n;
  void *x = nullptr, *y = nullptr;
  const size_t esz = prec == VIE_FP64 ? sizeof(double2) : sizeof(float2);
  VIE_CK(dalloc(&x, esz * L, st));
  VIE_CK(dalloc(&y, esz * (size_t)cout_of(K.mode) * P->n * P->n * P->n, st));
  VIE_CK(cudaMemsetAsync(x, 0, esz * L, st));
  vie_status s = run_apply(P, K, x, y, prec, 1, K.mode == KM_SYM3 || K.mode == KM_MAXWELL6, st);
  dfree(x, st);
  dfree(y, st);
  cudaStreamSynchronize(st);
  *variant = v;
  return s;
}

vie_status run_apply(vie_problem* P, const KernelSet& K, const void* in, void* out, int prec, int nrhs,
                     bool with_identity, cudaStream_t st) {
  if (prec == VIE_FP64) return run_apply_t<double>(P, K, in, out, nrhs, with_identity, st);
  return run_apply_t<float>(P, K, in, out, nrhs, with_identity, st);
}

}  // namespace vie
