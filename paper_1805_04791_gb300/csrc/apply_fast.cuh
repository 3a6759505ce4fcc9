// Register-resident fast path of the operator apply for 2n = R1 R2 in
// {64, 96, 128, 192, 256, 384, 512}: the kernels, their launchers and the
// z-pass autotuner, as templates.  Each size is instantiated in its own
// translation unit (apply_fast_<2n>.cu) so the library builds in parallel.
#pragma once

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "vie_fft2.cuh"
#include "vie_internal.h"

namespace vie {

// Per compute type: its precision id (vie_precision) and the device tables it uses.
template <typename T> struct Prec;
template <> struct Prec<double> {
  static constexpr int id = VIE_FP64;
  static const double2* K(const KernelSet& k) { return k.oct64; }
  static const double2* He(const vie_problem* P) { return P->He64; }
  static const double2* Hm(const vie_problem* P) { return P->Hm64; }
  static const double2* tw(const vie_problem* P) { return P->tw64; }
};
template <> struct Prec<float> {
  static constexpr int id = VIE_FP32;
  static const float2* K(const KernelSet& k) { return k.oct32; }
  static const float2* He(const vie_problem* P) { return P->He32; }
  static const float2* Hm(const vie_problem* P) { return P->Hm32; }
  static const float2* tw(const vie_problem* P) { return P->tw32; }
};
template <> struct Prec<df> {
  static constexpr int id = VIE_DF64;
  static const cdf* K(const KernelSet& k) { return k.octdf; }
  static const cdf* He(const vie_problem* P) { return P->Hedf; }
  static const cdf* Hm(const vie_problem* P) { return P->Hmdf; }
  static const cdf* tw(const vie_problem* P) { return P->twdf; }
};

template <typename V>
__device__ __forceinline__ void load_tw(V* tw, const V* __restrict__ twg, int M) {
  for (int j = flat_tid(); j < M; j += flat_nthreads()) tw[j] = twg[j];
}

// Asynchronous global -> shared copy (cp.async, sm_80+): BYTES in {4, 8, 16},
// both addresses aligned to BYTES.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stage the kernel octant entries of a mirror group in shared memory as
// slab[a][oz][q] (a < narr arrays, oz <= n, q < QW) from src[a O^3 + oz O^2 + q],
// all copies in flight at once; the caller waits (cp_async_wait_all, then a
// barrier) before reading the slab, and can do other work meanwhile.
template <int QW, typename E>
__device__ __forceinline__ void slab_async(E* slab, const E* src, int narr, int O, long long O3, int tid, int nthr) {
  for (int a = 0; a < narr; ++a) {
    const E* sa = src + a * O3;
    E* da = slab + a * O * QW;
    for (int idx = tid; idx < O * QW; idx += nthr) {
      const int oz = idx / QW, q = idx - oz * QW;
      cp_async<sizeof(E)>(da + idx, sa + (long long)oz * O * O + q);
    }
  }
  cp_async_commit();
}

// ------------------------------------------------ register-resident fast path
// For 2n = R1 * R2 in {64, 96, 128, 192, 256, 384, 512} every line is transformed by R2
// threads with one shared-memory transpose per direction (vie_fft2.cuh).
// Thread layouts: "row" passes (x-lines, contiguous) put the R2 threads of a
// line on consecutive lanes; "column" passes (y- and z-lines, one line per
// kx) put consecutive kx on consecutive lanes.  Every global access is a
// full 128-byte (FP32) or 256-byte (FP64) segment per half-warp.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) f_p1(const typename IOT<T>::E* __restrict__ x, typename CT<T>::V* __restrict__ A,
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
  const typename IOT<T>::E* src = x + ((long long)b * nc + c) * ((long long)rows * n) + (long long)row * n;
  V u[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) u[n1] = (n1 < R1 / 2 && ok) ? to_v<T>(src[R2 * n1 + t]) : CT<T>::make(0, 0);
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
    if (F::row(t, j))
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
      if (F::row(t, j))
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) dst[(long long)(t + R2 * j + R1 * k2) * M] = X[j][k2];
  } else {
    const V* src = in + plane * (long long)M * M + kx;
    V X[F::J][R2];
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2)
        X[j][k2] = F::row(t, j) ? src[(long long)(t + R2 * j + R1 * k2) * M] : CT<T>::make(0, 0);
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
// component per thread holds registers near 80 (2n = 256: 2 CTAs, 24 warps,
// per SM).  CTA order pairs mirror pencils (ky, M - ky) x (kx tile, mirrored tile)
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
      if (F::row(t, j))
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
      if (F::row(t, j))
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
          if (neg0[i] != (zodd[i] && fz)) kv = vneg(kv);
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
template <typename T, int R1, int R2, int MODE, int NP>
struct P3cThreads {
  static constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
  static constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
  static constexpr int N = NP * R2 * CMAX;
  static constexpr int M = R1 * R2;
  static constexpr int ESZ = (int)sizeof(typename CT<T>::V);
  static constexpr int LS0 = Fft2<T, R1, R2>::LS0;
  static constexpr int LS = (ESZ == 8) ? ((LS0 + 13) / 16) * 16 + 2 : (LS0 | 1);
  // shared memory of a CTA (2n fixes n, hence the slab extent): two CTAs per
  // SM (and registers capped for them) only where two fit
  static constexpr long long SMEM = (long long)ESZ * (M + (long long)CMAX * NP * LS + (long long)NARR * (M / 2 + 1) * (NP + 1));
  static constexpr int MINB = (N <= 384 && SMEM <= 112 * 1024) ? 2 : 1;
};

template <typename T, int R1, int R2, int MODE, int NP>
__global__ void __launch_bounds__(P3cThreads<T, R1, R2, MODE, NP>::N, P3cThreads<T, R1, R2, MODE, NP>::MINB)
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
  // kernel slab copies in flight while tile 0 runs its forward transform
  slab_async<QW>(slab, K + ((long long)kyp) * O + NP * txp, NARR, O, O3, threadIdx.x, NTHR);
  for (int j = threadIdx.x; j < M; j += NTHR) tw[j] = twg[j];
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
        if (F::row(t, j))
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) s[t + R2 * j + R1 * k2] = X[j][k2];
    }
    cp_async_wait_all();  // the kernel slab (no-op after the first tile)
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
        if (F::row(t, j))
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int k = t + R2 * j + R1 * k2;
          // k < n for k2 < R2/2 and k > n for k2 > R2/2 (k = R1 k2 + [0, R1)); only k2 = R2/2 depends on t, j
          const bool fz = (k2 < R2 / 2) ? false : ((k2 > R2 / 2) ? true : (k > n));
          const int zoff = (fz ? M - k : k) * QW;
          V acc = CT<T>::make(0, 0);
#pragma unroll
          for (int i = 0; i < NT; ++i) {
            if (i >= ntm) break;
            const V kv = kp[i][zoff];
            const V xv = xs[i][k];
            acc = cfma(fz ? sg1[i] : sg0[i], cmul(kv, xv), acc);
          }
          X[j][k2] = acc;
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

// z-pencils, lane-pair variant (FP32 only).  Same mirror-group CTA and
// kernel slab as f_p3c, but every thread carries two neighbouring pencils
// (kx, kx + 1) of its component as the two lanes of f32x2 values: the FFT
// codelets, the twiddle multiplies and the kernel mixing run as packed
// instructions for both pencils at once, and every shared-memory transfer of
// the transposes moves 16 bytes (both pencils' complex values).  The twiddle
// table is stored lane-broadcast ({wr, wr}, {wi, wi}).
template <int MODE, int NP, int R2>
struct P3pThreads {
  static constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
  static constexpr int N = (NP / 2) * R2 * CMAX;
  static constexpr int MINB = N <= 192 ? 2 : 1;
};

template <int R1, int R2, int MODE, int NP>
__global__ void __launch_bounds__(P3pThreads<MODE, NP, R2>::N, P3pThreads<MODE, NP, R2>::MINB)
f_p3p(float2* __restrict__ B, int n, int C, const float2* __restrict__ K, const float2* __restrict__ twg) {
  typedef f32x2 T;
  typedef c32x2 V;
  typedef Fft2<T, R1, R2> F;
  constexpr int CI = ModeDim<MODE>::CI, CO = ModeDim<MODE>::CO, NT = ModeDim<MODE>::NT;
  constexpr int CMAX = CI > CO ? CI : CO;
  constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
  constexpr int M = F::M, NTX = M / NP, NQ = NP / 2, NTHR = NQ * R2 * CMAX;
  constexpr int LS = ((F::LS0 + 13) / 16) * 16 + 2;  // 16-byte elements: LS = 2 mod 16
  constexpr int QW = NP + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  float2* slab = (float2*)(sm + CMAX * NQ * LS);
  const int kyp = blockIdx.x / (NTX / 2), txp = blockIdx.x - (blockIdx.x / (NTX / 2)) * (NTX / 2);
  const int O = n + 1;
  const long long O3 = (long long)O * O * O;
  // kernel slab copies in flight while tile 0 runs its forward transform
  slab_async<QW>(slab, K + ((long long)kyp) * O + NP * txp, NARR, O, O3, threadIdx.x, NTHR);
  for (int j = threadIdx.x; j < M; j += NTHR) {
    const float2 w = twg[j];
    tw[j] = CT<T>::make(T(w.x, w.x), T(w.y, w.y));
  }
  const int l = threadIdx.x % NQ, t = (threadIdx.x / NQ) % R2, c = threadIdx.x / (NQ * R2);
  const int b0 = blockIdx.y;
  const long long zs = (long long)M * M, cs = (long long)n * zs;
  V* s = sm + (c * NQ + l) * LS;
  int tb[NT], ta[NT], tsg[NT];
  const int ntm = (c < CO) ? mix_terms<MODE>(c, tb, ta, tsg) : 0;
  const bool self_y = (kyp == 0 || kyp == M / 2);
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    if ((v & 1) && self_y) continue;  // block-uniform
    const int ky = (v & 1) ? M - kyp : kyp;
    const int tile = (v & 2) ? NTX - 1 - txp : txp;
    const int kx0 = tile * NP + 2 * l;  // lanes: kx0 and kx0 + 1 (kx0 even: 16-byte aligned pairs)
    float2* colbase = B + (long long)b0 * C * cs + (long long)ky * M + kx0;
    V X[F::J][R2];
    V u[R1];
    if (c < CI) {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) {
        if (n1 < R1 / 2) {
          const float4 g = *(const float4*)(colbase + c * cs + (long long)(R2 * n1 + t) * zs);
          u[n1] = CT<T>::make(T(g.x, g.z), T(g.y, g.w));
        } else {
          u[n1] = CT<T>::make(T(0.0), T(0.0));
        }
      }
    }
    __syncthreads();  // previous tile's readers of s are done; slab and tw are visible
    if (c < CI) F::template fwd1<true>(u, t, s, tw);
    __syncthreads();
    if (c < CI) F::fwd2(X, t, s);
    __syncthreads();
    if (c < CI) {
#pragma unroll
      for (int j = 0; j < F::J; ++j)
        if (F::row(t, j))
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) s[t + R2 * j + R1 * k2] = X[j][k2];
    }
    cp_async_wait_all();  // the kernel slab (no-op after the first tile)
    __syncthreads();
    if (c < CO) {
      const bool fy = ky > n;
      const bool fx0 = kx0 > n, fx1 = kx0 + 1 > n;
      const int q0 = (fx0 ? M - kx0 : kx0) - NP * txp, q1 = (fx1 ? M - kx0 - 1 : kx0 + 1) - NP * txp;
      T sg0[NT], sg1[NT];
      const float2* kp[NT];
      const V* xs[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        if (i >= ntm) break;
        const int par = sym_parity(MODE == KM_DIV ? 6 + ta[i] : ta[i]);
        const bool ny = ((par & 2) && fy) != (tsg[i] < 0);
        const bool n0 = ny != ((par & 1) && fx0), n1 = ny != ((par & 1) && fx1);
        const bool oz = (par & 4) != 0;
        sg0[i] = T(n0 ? -1.f : 1.f, n1 ? -1.f : 1.f);
        sg1[i] = T((n0 != oz) ? -1.f : 1.f, (n1 != oz) ? -1.f : 1.f);
        kp[i] = slab + ta[i] * O * QW;
        xs[i] = sm + (tb[i] * NQ + l) * LS;
      }
#pragma unroll
      for (int j = 0; j < F::J; ++j)
        if (F::row(t, j))
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int k = t + R2 * j + R1 * k2;
            const bool fz = (k2 < R2 / 2) ? false : ((k2 > R2 / 2) ? true : (k > n));
            const int zoff = (fz ? M - k : k) * QW;
            T ax(0.0), ay(0.0);
#pragma unroll
            for (int i = 0; i < NT; ++i) {
              if (i >= ntm) break;
              const float2 k0 = kp[i][zoff + q0], k1 = kp[i][zoff + q1];
              const T kr(k0.x, k1.x), ki(k0.y, k1.y);
              const V xv = xs[i][k];
              const T sgn = fz ? sg1[i] : sg0[i];
              const T px = fmadd(kr, xv.x, -(ki * xv.y));
              const T py = fmadd(kr, xv.y, ki * xv.x);
              ax = fmadd(sgn, px, ax);
              ay = fmadd(sgn, py, ay);
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
      for (int n1 = 0; n1 < R1 / 2; ++n1)
        *(float4*)(colbase + c * cs + (long long)(R2 * n1 + t) * zs) =
            make_float4(u[n1].x.a, u[n1].y.a, u[n1].x.b, u[n1].y.b);
    }
  }
}

// z-pencils, component-group variant (FP32 only).  Every thread carries all
// three components of a vector (J, or M for Maxwell) on its pencil: the three
// forward transforms share the twiddles (read once into registers), the kernel
// mixing runs on registers and reads each kernel value of a point once for
// all three outputs, and no spectrum is exchanged through shared memory
// except the other vector's for the Maxwell curl terms (two groups per
// pencil).  Shared-memory traffic per point is about half that of f_p3c.  The
// next tile's inputs are loaded into registers while the current tile runs,
// and the kernel slab is stored [array][x][z] with a row pitch of 2 mod 16
// elements, so the mixing loads of 8 pencils x 2 threads hit distinct banks.
template <int MODE, int NP, int R2>
struct P3tThreads {
  static constexpr int NG = (MODE == KM_MAXWELL6) ? 2 : 1;
  static constexpr int N = NP * R2 * NG;
};

template <int R1, int R2, int MODE, int NP>
__global__ void __launch_bounds__(P3tThreads<MODE, NP, R2>::N)
f_p3t(float2* __restrict__ B, int n, int C, const float2* __restrict__ K, const float2* __restrict__ twg) {
  typedef float T;
  typedef float2 V;
  typedef Fft2<T, R1, R2> F;
  constexpr int NG = P3tThreads<MODE, NP, R2>::NG;
  constexpr int G = 3;                          // components per thread
  constexpr int GO = (MODE == KM_DIV) ? 1 : 3;  // output components per thread
  constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
  constexpr int M = F::M, NTX = M / NP, NTHR = NP * R2 * NG, H = R1 / 2;
  constexpr int NGROUPS = (M / 2 + 1) * (NTX / 2);  // mirror groups
  constexpr int LS = ((F::LS0 + 13) / 16) * 16 + 2;
  constexpr int QW = NP + 1;
  static_assert(MODE == KM_SYM3 || MODE == KM_DIV || MODE == KM_MAXWELL6, "component-group z pass");
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;
  V* sm = tw + M;
  V* slab = sm + NG * G * NP * LS;
  const int O = n + 1, OP = ((O + 13) / 16) * 16 + 2;
  const long long O3 = (long long)O * O * O;
  const int l = threadIdx.x % NP, t = (threadIdx.x / NP) % R2, h = threadIdx.x / (NP * R2);
  const long long zs = (long long)M * M, cs = (long long)n * zs;
  const int b0 = blockIdx.y;
  // The CTA walks mirror groups blockIdx.x, blockIdx.x + gridDim.x, ... (a single
  // group when the grid has one CTA per group).  Group grp = (kyp, txp) owns the tiles
  // (ky, M - ky) x (kx tile, mirrored tile); rows ky = 0 and M/2 mirror onto themselves.
  auto g_kyp = [&](int grp) { return grp / (NTX / 2); };
  auto g_txp = [&](int grp) { return grp - (grp / (NTX / 2)) * (NTX / 2); };
  auto g_self = [&](int grp) {
    const int k = grp / (NTX / 2);
    return k == 0 || k == M / 2;
  };
  auto tile_ky = [&](int grp, int i) {
    const int v = g_self(grp) ? 2 * i : i;
    return (v & 1) ? M - g_kyp(grp) : g_kyp(grp);
  };
  auto tile_kx = [&](int grp, int i) {
    const int v = g_self(grp) ? 2 * i : i;
    return ((v & 2) ? NTX - 1 - g_txp(grp) : g_txp(grp)) * NP + l;
  };
  // kernel slab [a][q][oz] <- K[a][oz][kyp][NP txp + q], copied while other work runs
  auto slab_issue = [&](int grp) {
    const V* src = K + (long long)g_kyp(grp) * O + NP * g_txp(grp);
    for (int a = 0; a < NARR; ++a)
      for (int idx = threadIdx.x; idx < O * QW; idx += NTHR) {
        const int oz = idx / QW, q = idx - oz * QW;
        cp_async<8>(slab + (a * QW + q) * OP + oz, src + a * O3 + (long long)oz * O * O + q);
      }
    cp_async_commit();
  };
  V g[G][H];  // inputs (z < n) of the tile being started, then of the next one
  auto load_inputs = [&](int grp, int i) {
    const V* src =
        B + (long long)b0 * C * cs + (long long)tile_ky(grp, i) * M + tile_kx(grp, i) + (long long)(h * G) * cs;
#pragma unroll
    for (int c = 0; c < G; ++c)
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) g[c][n1] = src[c * cs + (long long)(R2 * n1 + t) * zs];
  };
  int grp = blockIdx.x;
  if (grp >= NGROUPS) return;  // block-uniform
  slab_issue(grp);
  for (int j = threadIdx.x; j < M; j += NTHR) tw[j] = twg[j];
  load_inputs(grp, 0);
  int i = 0;
#pragma unroll 1
  while (true) {
    const int ky = tile_ky(grp, i), kx = tile_kx(grp, i);
    const int txp = g_txp(grp);
    V* colbase = B + (long long)b0 * C * cs + (long long)ky * M + kx;
    V* s0 = sm + ((h * G) * NP + l) * LS;  // this group's transpose lines, component c at s0 + c NP LS
    __syncthreads();                       // previous tile's readers of the transpose lines are done
    {
      V w[R1];
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) w[k1] = tw[t * k1];
#pragma unroll
      for (int c = 0; c < G; ++c) {
        V u[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) u[n1] = (n1 < H) ? g[c][n1] : make_float2(0.f, 0.f);
        F::template fwd1w<true>(u, t, s0 + c * NP * LS, w);
      }
    }
    // the next unit: the next tile of this group, else the first tile of the CTA's next group
    int ngrp = grp, ni = i + 1;
    if (ni >= (g_self(grp) ? 2 : 4)) {
      ngrp = grp + gridDim.x;
      ni = 0;
    }
    const bool more = ngrp < NGROUPS;
    if (more) load_inputs(ngrp, ni);
    __syncthreads();
    V X[G][F::J][R2];
#pragma unroll
    for (int c = 0; c < G; ++c) F::fwd2(X[c], t, s0 + c * NP * LS);
    cp_async_wait_all();  // the kernel slab (no-op after the first tile)
    __syncthreads();      // transpose lines free again; slab visible
    const V* so = sm + (((1 - h) * G) * NP + l) * LS;  // the other group's parked spectra (Maxwell)
    if (NG == 2) {
#pragma unroll
      for (int c = 0; c < G; ++c)
#pragma unroll
        for (int j = 0; j < F::J; ++j)
          if (F::row(t, j))
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) s0[c * NP * LS + t + R2 * j + R1 * k2] = X[c][j][k2];
      __syncthreads();
    }
    {
      const bool fy = ky > n, fx = kx > n;
      const V* kq = slab + ((fx ? M - kx : kx) - NP * txp) * OP;
      T sg0[NARR], sg1[NARR];
#pragma unroll
      for (int a = 0; a < NARR; ++a) {
        const int par = sym_parity(MODE == KM_DIV ? 6 + a : a);
        const bool ng = ((par & 2) && fy) != ((par & 1) && fx);
        sg0[a] = ng ? -1.f : 1.f;
        sg1[a] = (ng != ((par & 4) != 0)) ? -1.f : 1.f;
      }
#pragma unroll
      for (int j = 0; j < F::J; ++j)
        if (F::row(t, j))
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int k = t + R2 * j + R1 * k2;
            const bool fz = (k2 < R2 / 2) ? false : ((k2 > R2 / 2) ? true : (k > n));
            const int zo = fz ? M - k : k;
            V kv[NARR];
#pragma unroll
            for (int a = 0; a < NARR; ++a) {
              kv[a] = kq[a * QW * OP + zo];
              if (sym_parity(MODE == KM_DIV ? 6 + a : a) != 0) kv[a] = (fz ? sg1[a] : sg0[a]) * kv[a];
            }
            const V x0 = X[0][j][k2], x1 = X[1][j][k2], x2 = X[2][j][k2];
            if (MODE == KM_DIV) {
              X[0][j][k2] = cmul(kv[0], x0) + cmul(kv[1], x1) + cmul(kv[2], x2);
            } else {
              // symmetric 3x3: xx yy zz xy xz yz
              V y0 = cmul(kv[0], x0) + cmul(kv[3], x1) + cmul(kv[4], x2);
              V y1 = cmul(kv[3], x0) + cmul(kv[1], x1) + cmul(kv[5], x2);
              V y2 = cmul(kv[4], x0) + cmul(kv[5], x1) + cmul(kv[2], x2);
              if (MODE == KM_MAXWELL6) {
                // J rows + (P x M), M rows - (P x J); P_a = kernel 6 + a, the other vector from shared memory
                const V o0 = so[k], o1 = so[NP * LS + k], o2 = so[2 * NP * LS + k];
                V c0 = cmul(kv[7], o2) - cmul(kv[8], o1);
                V c1 = cmul(kv[8], o0) - cmul(kv[6], o2);
                V c2 = cmul(kv[6], o1) - cmul(kv[7], o0);
                if (h == 0) {
                  y0 = y0 + c0;
                  y1 = y1 + c1;
                  y2 = y2 + c2;
                } else {
                  y0 = y0 - c0;
                  y1 = y1 - c1;
                  y2 = y2 - c2;
                }
              }
              X[0][j][k2] = y0;
              X[1][j][k2] = y1;
              X[2][j][k2] = y2;
            }
          }
    }
    if (NG == 2) __syncthreads();  // the other group has read the parked spectra
#pragma unroll
    for (int c = 0; c < GO; ++c) F::invA(X[c], t, s0 + c * NP * LS, tw);
    __syncthreads();
    // every thread is past this group's mixing: the slab may take the next group's kernel
    if (more && ni == 0) slab_issue(ngrp);
#pragma unroll
    for (int c = 0; c < GO; ++c) {
      V u[R1];
      F::template invB<true>(u, t, s0 + c * NP * LS);
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) colbase[(h * G + c) * cs + (long long)(R2 * n1 + t) * zs] = u[n1];
    }
    if (!more) break;
    grp = ngrp;
    i = ni;
  }
}

// z-pencils, slim component-group variant (FP32; 3x3 symmetric and
// divergence mixing).  Same mirror-group CTA and register layout as f_p3t (each
// thread carries the three components of a vector on its pencil), re-balanced
// for occupancy and for fewer shared-memory instructions:
//  * one transpose line per pencil instead of three: the components go
//    through it one after the other (two barriers per component and
//    direction), so a CTA of NP = 8 pencils at 2n = 256 needs ~75 KB of shared
//    memory and three CTAs share an SM (registers capped for MINB CTAs);
//  * transpose rows have an even pitch, so each thread reads its row back as
//    16-byte pairs (the writes stay 8-byte, column-wise);
//  * the kernel slab is stored [q][z][array]: the 6 (or 3) octant values of a
//    point are adjacent and arrive in three (two) 16-byte loads;
//  * twiddles come from a per-thread table W^{t k1} read as 16-byte pairs;
//  * only the next component's inputs are loaded ahead (16 registers instead
//    of the 48 of a whole next tile);
//  * the kernel mixing runs on packed f32x2 arithmetic with broadcast operands:
//    y += K x as y + K.x (x.x, x.y) + K.y (-x.y, x.x), two packed instructions
//    per complex multiply-add instead of four scalar ones;
//  * the sign of each octant value is fixed per tile in kx and ky and, taking
//    "k >= n" as the mirrored half (odd arrays vanish at k = n), at compile time
//    in kz.
template <int R1, int R2, int MODE, int NP>
struct P3sCfg {
  static constexpr int NARR = (MODE == KM_SYM3) ? 6 : 3;
  static constexpr int NARRP = (NARR + 1) & ~1;  // values per slab point, padded to 16 bytes
  static constexpr int M = R1 * R2;
  static constexpr int PF = R2 + 2, PI = R1 + 2;  // even row pitches: 16-byte row reads
  static constexpr int LS0 = R1 * PF > R2 * PI ? R1 * PF : R2 * PI;
  static constexpr int LS = ((LS0 + 13) / 16) * 16 + 2;  // = 2 mod 16: conflict-free column writes
  static constexpr int QW = NP + 1;
  static constexpr int O = M / 2 + 1;  // octant extent (odd: conflict-free 16-byte slab reads)
  static constexpr int NTHR = NP * R2;
  // W^{t k1} [t][k1] with rows of R1 + 2, and [k1][n2] with rows of R2 + 2 when R1 != R2 (the
  // padding spreads the 16-byte pair reads of different rows over the banks)
  static constexpr int TP1 = R1 + 2, TP2 = R2 + 2;
  static constexpr int NTW = (R1 == R2) ? R2 * TP1 : R2 * TP1 + R1 * TP2;
  static constexpr long long SMEM = 8LL * (NTW + (long long)NP * LS + (long long)QW * O * NARRP);
};

__device__ __forceinline__ float2 bcx2(float2 a) { return make_float2(a.x, a.x); }
__device__ __forceinline__ float2 bcy2(float2 a) { return make_float2(a.y, a.y); }
// i a
__device__ __forceinline__ float2 ipx(float2 a) { return make_float2(-a.y, a.x); }
// a w and a conj(w) as w.x a +- w.y (i a): one packed multiply and one packed FMA
__device__ __forceinline__ float2 pcmul(float2 a, float2 w) {
  return __ffma2_rn(bcy2(w), ipx(a), __fmul2_rn(bcx2(w), a));
}
__device__ __forceinline__ float2 pcmulc(float2 a, float2 w) {
  return __ffma2_rn(make_float2(-w.y, -w.y), ipx(a), __fmul2_rn(bcx2(w), a));
}

template <int R1, int R2, int MODE, int NP, int MINB>
__global__ void __launch_bounds__(NP * R2, MINB)
f_p3s(float2* __restrict__ B, int n, int C, const float2* __restrict__ K, const float2* __restrict__ twg) {
  typedef float T;
  typedef float2 V;
  typedef Fft2<T, R1, R2> F;
  typedef P3sCfg<R1, R2, MODE, NP> Cfg;
  constexpr int G = 3;                          // components per thread
  constexpr int GO = (MODE == KM_DIV) ? 1 : 3;  // output components per thread
  constexpr int NARR = Cfg::NARR, NARRP = Cfg::NARRP;
  constexpr int M = F::M, NTX = M / NP, NTHR = NP * R2, H = R1 / 2;
  constexpr int NGROUPS = (M / 2 + 1) * (NTX / 2);
  constexpr int LS = Cfg::LS, QW = Cfg::QW, PF = Cfg::PF, PI = Cfg::PI;
  // the grid size is fixed by the transform length (n = M / 2): strides and
  // the octant extent are compile-time constants
  constexpr int NN = M / 2, O = Cfg::O;
  constexpr long long O3 = (long long)O * O * O;
  constexpr long long zs = (long long)M * M, cs = (long long)NN * zs;
  static_assert(MODE == KM_SYM3 || MODE == KM_DIV, "slim z pass: 3x3 symmetric or divergence mixing");
  static_assert(R1 % 2 == 0 && R2 % 2 == 0 && (R1 % R2 == 0 || R1 < 2 * R2), "thread layout of Fft2");
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int TP1 = Cfg::TP1, TP2 = Cfg::TP2;
  V* tw1 = (V*)smraw;                             // [t < R2][k1 < R1] = W^{t k1}, row pitch TP1
  V* tw2 = (R1 == R2) ? tw1 : tw1 + R2 * TP1;     // [k1 < R1][n2 < R2] = W^{k1 n2}, row pitch TP2
  V* sm = tw1 + Cfg::NTW;
  V* slab = sm + NP * LS;                     // [q < QW][oz < O][a < NARRP]
  // consecutive lanes hold consecutive pencils (coalesced 64-byte rows of B);
  // a pencil's R2 threads lie in different warps, so its transposes take the
  // CTA barrier (a layout with each pencil's threads in one warp, which needs
  // only warp synchronisation, measured 1.65x slower: 8-byte accesses to 16
  // different z planes per warp instruction)
  const int l = threadIdx.x % NP, t = threadIdx.x / NP;
  auto line_sync = [] { __syncthreads(); };
  const int b0 = blockIdx.y;
  const int grp = blockIdx.x;
  if (grp >= NGROUPS) return;  // block-uniform
  const int kyp = grp / (NTX / 2), txp = grp - (grp / (NTX / 2)) * (NTX / 2);
  const bool self_y = (kyp == 0 || kyp == M / 2);
  {  // kernel slab <- K[a][oz][kyp][NP txp + q], in flight while tile 0 starts
    const V* src = K + (long long)kyp * O + NP * txp;
    for (int a = 0; a < NARR; ++a)
      for (int idx = threadIdx.x; idx < O * QW; idx += NTHR) {
        const int oz = idx / QW, q = idx - oz * QW;
        cp_async<8>(slab + (q * O + oz) * NARRP + a, src + a * O3 + (long long)oz * O * O + q);
      }
    cp_async_commit();
  }
  for (int j = threadIdx.x; j < R2 * R1; j += NTHR) {
    const int r = j / R1, c = j - r * R1;
    tw1[r * TP1 + c] = twg[r * c];
  }
  if (R1 != R2)
    for (int j = threadIdx.x; j < R1 * R2; j += NTHR) {
      const int r = j / R2, c = j - r * R2;
      tw2[r * TP2 + c] = twg[r * c];
    }
  V* s = sm + l * LS;  // this pencil's transpose line
  // inputs (z < n) of one component: the next one is loaded while the current one is transformed
  V g[H];
  auto load_comp = [&](const V* base, int c) {
#pragma unroll
    for (int n1 = 0; n1 < H; ++n1) g[n1] = base[c * cs + (long long)(R2 * n1 + t) * zs];
  };
  auto tile_base = [&](int v) {
    const int ky = (v & 1) ? M - kyp : kyp;
    const int tile = (v & 2) ? NTX - 1 - txp : txp;
    return B + (long long)b0 * C * cs + (long long)ky * M + tile * NP + l;
  };
  load_comp(tile_base(0), 0);
  __syncthreads();  // twiddle tables visible
  const float4* twf = (const float4*)(tw1 + t * TP1);  // W^{t k1}, k1 pairs
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    if ((v & 1) && self_y) continue;  // block-uniform
    const int ky = (v & 1) ? M - kyp : kyp;
    const int tile = (v & 2) ? NTX - 1 - txp : txp;
    const int kx = tile * NP + l;
    V* colbase = B + (long long)b0 * C * cs + (long long)ky * M + kx;
    V X[G][F::J][R2];
    // ---- forward z transforms, one component at a time through the line
#pragma unroll
    for (int c = 0; c < G; ++c) {
      V u[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[n1] = (n1 < H) ? g[n1] : make_float2(0.f, 0.f);
      if (c + 1 < G) load_comp(colbase, c + 1);
      dft_half_in<R1, -1, T>(u);
#pragma unroll
      for (int k2 = 0; k2 < R1 / 2; ++k2) {
        const float4 w = twf[k2];
        if (k2 > 0) u[2 * k2] = cmul(u[2 * k2], make_float2(w.x, w.y));
        u[2 * k2 + 1] = cmul(u[2 * k2 + 1], make_float2(w.z, w.w));
      }
      line_sync();  // earlier readers of the line are done
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) s[k1 * PF + t] = u[k1];
      line_sync();
#pragma unroll
      for (int j = 0; j < F::J; ++j) {
        if (!F::row(t, j)) continue;
        const int k1 = t + R2 * j;
        const float4* row = (const float4*)(s + k1 * PF);
#pragma unroll
        for (int n2 = 0; n2 < R2 / 2; ++n2) {
          const float4 r = row[n2];
          X[c][j][2 * n2] = make_float2(r.x, r.y);
          X[c][j][2 * n2 + 1] = make_float2(r.z, r.w);
        }
        Dft<R2, -1, T>::run(X[c][j]);
      }
    }
    if (v == 0) {           // block-uniform
      cp_async_wait_all();  // the kernel slab
      __syncthreads();      // slab visible to every thread
    }
    line_sync();  // the line is free again
    // ---- the next tile's first component, loaded during the mixing and the inverse
    const int vn = self_y ? (v == 0 ? 2 : 4) : v + 1;  // self-mirrored rows run tiles 0 and 2 only
    if (vn < 4) load_comp(tile_base(vn), 0);
    // ---- kernel mixing on registers
    {
      const bool fy = ky >= NN, fx = kx >= NN;  // tile-uniform
      const V* kq = slab + ((fx ? M - kx : kx) - NP * txp) * O * NARRP;
      float sg0[NARR], sg1[NARR];  // sign of array a for kz < n and kz >= n
#pragma unroll
      for (int a = 0; a < NARR; ++a) {
        const int par = sym_parity(MODE == KM_DIV ? 6 + a : a);
        const bool ng = ((par & 2) && fy) != ((par & 1) && fx);
        sg0[a] = ng ? -1.f : 1.f;
        sg1[a] = (ng != ((par & 4) != 0)) ? -1.f : 1.f;
      }
#pragma unroll
      for (int j = 0; j < F::J; ++j)
        if (F::row(t, j))
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int k = t + R2 * j + R1 * k2;
            const bool fz = k2 >= R2 / 2;  // k >= NN exactly when k2 >= R2/2 (compile time)
            const int zo = fz ? M - k : k;
            const float4* kp = (const float4*)(kq + zo * NARRP);
            V kv[NARRP];
#pragma unroll
            for (int a2 = 0; a2 < NARRP / 2; ++a2) {
              const float4 r = kp[a2];
              kv[2 * a2] = make_float2(r.x, r.y);
              kv[2 * a2 + 1] = make_float2(r.z, r.w);
            }
#pragma unroll
            for (int a = 0; a < NARR; ++a)
              if (sym_parity(MODE == KM_DIV ? 6 + a : a) != 0) kv[a] = (fz ? sg1[a] : sg0[a]) * kv[a];
            const V x0 = X[0][j][k2], x1 = X[1][j][k2], x2 = X[2][j][k2];
            const V p0 = ipx(x0), p1 = ipx(x1), p2 = ipx(x2);
            // y += K x  ==  y + K.x x + K.y (i x), as packed f32x2 products
            auto mac = [](V acc, V kk, V x, V ix) {
              return __ffma2_rn(bcy2(kk), ix, __ffma2_rn(bcx2(kk), x, acc));
            };
            auto mul = [](V kk, V x, V ix) { return __ffma2_rn(bcy2(kk), ix, __fmul2_rn(bcx2(kk), x)); };
            if (MODE == KM_DIV) {
              X[0][j][k2] = mac(mac(mul(kv[0], x0, p0), kv[1], x1, p1), kv[2], x2, p2);
            } else {
              // symmetric 3x3: xx yy zz xy xz yz
              X[0][j][k2] = mac(mac(mul(kv[0], x0, p0), kv[3], x1, p1), kv[4], x2, p2);
              X[1][j][k2] = mac(mac(mul(kv[3], x0, p0), kv[1], x1, p1), kv[5], x2, p2);
              X[2][j][k2] = mac(mac(mul(kv[4], x0, p0), kv[5], x1, p1), kv[2], x2, p2);
            }
          }
    }
    // ---- inverse z transforms, one component at a time through the line
#pragma unroll
    for (int c = 0; c < GO; ++c) {
#pragma unroll
      for (int j = 0; j < F::J; ++j) {
        if (!F::row(t, j)) continue;
        const int k1 = t + R2 * j;
        Dft<R2, +1, T>::run(X[c][j]);
        const float4* wr = (const float4*)(tw2 + k1 * (R1 == R2 ? TP1 : TP2));  // W^{k1 n2}, n2 pairs
#pragma unroll
        for (int n2 = 0; n2 < R2 / 2; ++n2) {
          const float4 w = wr[n2];
          if (n2 > 0) X[c][j][2 * n2] = cmulc(X[c][j][2 * n2], make_float2(w.x, w.y));
          X[c][j][2 * n2 + 1] = cmulc(X[c][j][2 * n2 + 1], make_float2(w.z, w.w));
        }
      }
      if (c > 0) line_sync();  // earlier readers of the line are done
#pragma unroll
      for (int j = 0; j < F::J; ++j) {
        if (!F::row(t, j)) continue;
        const int k1 = t + R2 * j;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) s[n2 * PI + k1] = X[c][j][n2];
      }
      line_sync();
      V u[R1];
      const float4* row = (const float4*)(s + t * PI);
#pragma unroll
      for (int k1 = 0; k1 < R1 / 2; ++k1) {
        const float4 r = row[k1];
        u[2 * k1] = make_float2(r.x, r.y);
        u[2 * k1 + 1] = make_float2(r.z, r.w);
      }
      dft_half_out<R1, +1, T>(u);
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) colbase[c * cs + (long long)(R2 * n1 + t) * zs] = u[n1];
    }
    line_sync();  // the line's last readers are done before the next tile writes it
  }
}

// z pass at 2n = 512 as two 256-point halves on a cluster of two CTAs
// (FP32; 3x3 symmetric, divergence and Maxwell 6x6 mixing).  Only z < n = 256
// of a z-line is nonzero, so with w = exp(-2 pi i / 512) its 512-point
// spectrum splits by the parity r of the frequency,
//   X[2k + r] = sum_{z < 256} (x[z] w^{z r}) W_256^{z k},
// a full 256-point transform of x (r = 0) or of the twisted x[z] w^z (r = 1).
// The kernel mixing is pointwise in k, so each half is mixed on its own, and
// the inverse over all 512 frequencies is the sum of the halves' 256-point
// inverses, the odd one twisted back by w^-z.  CTA r of a cluster owns half r
// of the same pencils: it reads the pencils' inputs (the other CTA's reads of
// the same lines are served by L2), stages the kernel octant entries of
// z-parity r (half the z range of the other mirror-group kernels' slab), and
// after its inverse transforms sends the half of its output that the other
// CTA writes (z >= 128 from r = 0, z < 128 from r = 1) into that CTA's shared
// memory (distributed shared memory; two cluster barriers per tile).  Every
// thread carries three components of a vector (J or M for Maxwell: two thread
// groups, the other vector's spectra parked in shared memory for the curl
// terms) with 16 values each, as the 2n = 256 kernels do.  The twists are
// folded into the radix-16 steps: with z = 16 n1 + t and k = k1 + 16 k2 the
// odd half multiplies its inputs by W_32^{n1} (compile-time constants) before
// the first step, the inter-step twiddles are w^{t (2 k1 + r)}, and the inverse
// mirrors both.
constexpr int oh_pick(int np, int hp) {
  for (int o = 129; o < 145; ++o) {
    const int v = (o * hp) % 8;
    if (np >= 8 ? (v % 2 == 1) : (v == 2 || v == 6)) return o;
  }
  return 129;
}

template <int MODE, int NP>
struct P3hCfg {
  static constexpr int NG = (MODE == KM_MAXWELL6) ? 2 : 1;
  static constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
  static constexpr int NARRP = (NARR + 1) & ~1;  // values per slab point, padded to 16 bytes
  static constexpr int R = 16, M = 512;
  // Line pitch: 8-byte column accesses of the NP pencils x 32/NP threads of a
  // warp fall on distinct bank pairs (at most two lanes per pair) when the
  // pitch is 2 mod 16 for 8 pencils and 8 mod 16 for 4.
  static constexpr int LS = ((R * (R + 1) + 15) / 16) * 16 + (NP >= 8 ? 2 : 8);
  static constexpr int QW = NP + 1;
  // Slab rows of OH >= 129 octant z entries (one parity, oz = 0..256): chosen so
  // that the 16-byte reads of the 8 lanes of a quarter warp (8 pencils, or 4
  // pencils x 2 frequencies) hit 8 distinct bank quads.
  static constexpr int OH = oh_pick(NP, NARRP / 2);
  static constexpr int NTHR = NG * NP * R;
  static constexpr size_t SMEM = 8 * ((size_t)M + (size_t)NG * 3 * NP * LS + (size_t)QW * OH * NARRP);
  // two CTAs per SM where 128 threads and the shared memory allow it
  static constexpr int MINB = (NTHR <= 128 && 2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
// Every thread of both CTAs of the cluster: this thread's shared-memory writes
// (local and remote) are released, the other threads' acquired.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Address of p's counterpart in the shared memory of CTA `rank` of the cluster.
__device__ __forceinline__ unsigned peer_smem(const void* p, unsigned rank) {
  unsigned d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n"
               : "=r"(d)
               : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return d;
}
__device__ __forceinline__ void st_peer(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

template <int MODE, int NP, int MINB, bool PK, bool PS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P3hCfg<MODE, NP>::NTHR, MINB)
f_p3h(float2* __restrict__ B, int C, const float2* __restrict__ K, const float2* __restrict__ twg) {
  typedef float T;
  typedef float2 V;
  typedef P3hCfg<MODE, NP> Cfg;
  constexpr int NG = Cfg::NG, G = 3, GO = (MODE == KM_DIV) ? 1 : 3;
  constexpr int NARR = Cfg::NARR, NARRP = Cfg::NARRP;
  constexpr int R = Cfg::R, M = Cfg::M, NN = M / 2, NTX = M / NP, NTHR = Cfg::NTHR;
  constexpr int NGROUPS = (M / 2 + 1) * (NTX / 2);
  constexpr int LS = Cfg::LS, QW = Cfg::QW, OH = Cfg::OH, PF = R + 1, PI = R + 1;
  constexpr int O = NN + 1;
  constexpr long long O3 = (long long)O * O * O;
  constexpr long long zs = (long long)M * M, cs = (long long)NN * zs;
  static_assert(MODE == KM_SYM3 || MODE == KM_MAXWELL6, "half-spectrum z pass");
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tw = (V*)smraw;                // w^j, j < 512
  V* sm = tw + M;                   // transpose lines [h][c][pencil], LS each
  V* slab = sm + NG * G * NP * LS;  // [q < QW][oz / 2 < OH][a < NARRP], oz of parity r
  const int r = (int)cluster_rank();
  const int l = threadIdx.x % NP, t = (threadIdx.x / NP) % R, h = threadIdx.x / (NP * R);
  const int b0 = blockIdx.y;
  // Both CTAs of a cluster take the same mirror groups: one (PS false), or
  // grp, grp + gstride, ... on a grid of co-resident clusters (PS true).
  const int gstride = PS ? (int)(gridDim.x >> 1) : NGROUPS;
  int grp = blockIdx.x >> 1;
  if (grp >= NGROUPS) return;  // uniform over the cluster
  auto g_kyp = [&](int gr) { return gr / (NTX / 2); };
  auto g_txp = [&](int gr) { return gr - (gr / (NTX / 2)) * (NTX / 2); };
  // kernel slab <- K[a][2 ozh + r][kyp][NP txp + q], in flight while other work runs
  auto slab_issue = [&](int gr) {
    const V* src = K + (long long)g_kyp(gr) * O + NP * g_txp(gr);
    const int ohr = OH - r;  // 2 ozh + r <= n
    for (int a = 0; a < NARR; ++a)
      for (int idx = threadIdx.x; idx < ohr * QW; idx += NTHR) {
        const int ozh = idx / QW, q = idx - ozh * QW;
        cp_async<8>(slab + (q * OH + ozh) * NARRP + a, src + a * O3 + (long long)(2 * ozh + r) * O * O + q);
      }
    cp_async_commit();
  };
  slab_issue(grp);
  for (int j = threadIdx.x; j < M; j += NTHR) tw[j] = twg[j];
  V* s0 = sm + ((h * G) * NP + l) * LS;                    // this group's line of component c: s0 + c NP LS
  const V* so = sm + (((NG - 1 - h) * G) * NP + l) * LS;  // the other vector's lines (Maxwell)
  const unsigned s0_peer = peer_smem(s0, 1u - (unsigned)r);
  V g[R];  // inputs of one component; the next one is loaded while the current one is transformed
  auto load_comp = [&](const V* base, int c) {
#pragma unroll
    for (int n1 = 0; n1 < R; ++n1) g[n1] = base[c * cs + (long long)(R * n1 + t) * zs];
  };
  auto tile_base = [&](int gr, int v) {
    const int ky = (v & 1) ? M - g_kyp(gr) : g_kyp(gr);
    const int tile = (v & 2) ? NTX - 1 - g_txp(gr) : g_txp(gr);
    return B + (long long)b0 * C * cs + (long long)(h * G) * cs + (long long)ky * M + tile * NP + l;
  };
  load_comp(tile_base(grp, 0), 0);
#pragma unroll 1
  for (; grp < NGROUPS; grp += gstride) {
  const int kyp = g_kyp(grp), txp = g_txp(grp);
  const bool self_y = (kyp == 0 || kyp == M / 2);
  const int ngrp = grp + gstride;  // the cluster's next group (PS)
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    if ((v & 1) && self_y) continue;  // uniform over the cluster
    const int ky = (v & 1) ? M - kyp : kyp;
    const int kx = ((v & 2) ? NTX - 1 - txp : txp) * NP + l;
    V* colbase = tile_base(grp, v);
    __syncthreads();  // twiddle table written; the previous tile's readers of the lines are done
    // ---- forward: step 1 of every component into its line, step 2 from the lines
#pragma unroll
    for (int c = 0; c < G; ++c) {
      V u[R];
#pragma unroll
      for (int n1 = 0; n1 < R; ++n1) u[n1] = g[n1];
      if (c + 1 < G) load_comp(colbase, c + 1);
      if (r) {
#pragma unroll
        for (int n1 = 1; n1 < R; ++n1) u[n1] = twc<32, -1, T>(u[n1], n1);
      }
      Dft<R, -1, T>::run(u);
      V* s = s0 + c * NP * LS;
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) s[k1 * PF + t] = PK ? pcmul(u[k1], tw[t * (2 * k1 + r)])
                                                          : cmul(u[k1], tw[t * (2 * k1 + r)]);
    }
    __syncthreads();
    V X[G][R];  // X[c][k2] = spectrum of half r at k = t + 16 k2 (frequency 2k + r)
#pragma unroll
    for (int c = 0; c < G; ++c) {
      const V* s = s0 + c * NP * LS + t * PF;
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) X[c][n2] = s[n2];
      Dft<R, -1, T>::run(X[c]);
    }
    if (v == 0) cp_async_wait_all();  // the kernel slab (block-uniform)
    __syncthreads();                  // lines free again; slab visible
    // the next tile's first component, loaded during the mixing and the inverse
    const int vn = self_y ? (v == 0 ? 2 : 4) : v + 1;
    if (vn < 4) load_comp(tile_base(grp, vn), 0);
    else if (PS && ngrp < NGROUPS) load_comp(tile_base(ngrp, 0), 0);
    if (NG == 2) {  // park the spectra for the other vector's curl terms
#pragma unroll
      for (int c = 0; c < G; ++c)
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) s0[c * NP * LS + t + R * k2] = X[c][k2];
      __syncthreads();
    }
    // ---- kernel mixing on registers
    {
      const bool fy = ky > NN, fx = kx > NN;  // tile-uniform
      const V* kq = slab + ((fx ? M - kx : kx) - NP * txp) * OH * NARRP;
      float sg0[NARR], sg1[NARR];  // sign of array a for frequencies below and above n
#pragma unroll
      for (int a = 0; a < NARR; ++a) {
        const int par = sym_parity(MODE == KM_DIV ? 6 + a : a);
        const bool ng = ((par & 2) && fy) != ((par & 1) && fx);
        sg0[a] = ng ? -1.f : 1.f;
        sg1[a] = (ng != ((par & 4) != 0)) ? -1.f : 1.f;
      }
      const float sgc = (h == 0) ? 1.f : -1.f;  // + (P x M) in the J rows, - (P x J) in the M rows
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) {
        // frequency 2 (t + 16 k2) + r is above n exactly when k2 >= 8 (compile time)
        const bool fz = k2 >= R / 2;
        const int ozh = fz ? NN - t - R * k2 - r : t + R * k2;
        const float4* kp = (const float4*)(kq + ozh * NARRP);
        V kv[NARRP];
#pragma unroll
        for (int a2 = 0; a2 < NARRP / 2; ++a2) {
          const float4 q4 = kp[a2];
          kv[2 * a2] = make_float2(q4.x, q4.y);
          kv[2 * a2 + 1] = make_float2(q4.z, q4.w);
        }
#pragma unroll
        for (int a = 0; a < NARR; ++a)
          if (sym_parity(MODE == KM_DIV ? 6 + a : a) != 0) kv[a] = (fz ? sg1[a] : sg0[a]) * kv[a];
        const V x0 = X[0][k2], x1 = X[1][k2], x2 = X[2][k2];
        if (PK) {
          // y += K x as y + K.x x + K.y (i x) on packed f32x2 instructions with
          // broadcast operands; the J/M sign of the curl terms is in sgc
          const V p0 = ipx(x0), p1 = ipx(x1), p2 = ipx(x2);
          auto mac = [](V acc, V kk, V x, V ix) {
            return __ffma2_rn(bcy2(kk), ix, __ffma2_rn(bcx2(kk), x, acc));
          };
          auto mul = [](V kk, V x, V ix) { return __ffma2_rn(bcy2(kk), ix, __fmul2_rn(bcx2(kk), x)); };
          V y0 = mac(mac(mul(kv[0], x0, p0), kv[3], x1, p1), kv[4], x2, p2);
          V y1 = mac(mac(mul(kv[3], x0, p0), kv[1], x1, p1), kv[5], x2, p2);
          V y2 = mac(mac(mul(kv[4], x0, p0), kv[5], x1, p1), kv[2], x2, p2);
          if (MODE == KM_MAXWELL6) {
            const int k = t + R * k2;
            const V o0 = so[k], o1 = so[NP * LS + k], o2 = so[2 * NP * LS + k];
            const V q0 = ipx(o0), q1 = ipx(o1), q2 = ipx(o2);
            const V c6 = sgc * kv[6], c7 = sgc * kv[7], c8 = sgc * kv[8];
            const V n6 = -sgc * kv[6], n7 = -sgc * kv[7], n8 = -sgc * kv[8];
            // J rows + (P x M), M rows - (P x J)
            y0 = mac(mac(y0, c7, o2, q2), n8, o1, q1);
            y1 = mac(mac(y1, c8, o0, q0), n6, o2, q2);
            y2 = mac(mac(y2, c6, o1, q1), n7, o0, q0);
          }
          X[0][k2] = y0;
          X[1][k2] = y1;
          X[2][k2] = y2;
        } else {
          // symmetric 3x3: xx yy zz xy xz yz
          V y0 = cmul(kv[0], x0) + cmul(kv[3], x1) + cmul(kv[4], x2);
          V y1 = cmul(kv[3], x0) + cmul(kv[1], x1) + cmul(kv[5], x2);
          V y2 = cmul(kv[4], x0) + cmul(kv[5], x1) + cmul(kv[2], x2);
          if (MODE == KM_MAXWELL6) {
            // J rows + (P x M), M rows - (P x J); P_a = kernel 6 + a
            const int k = t + R * k2;
            const V o0 = so[k], o1 = so[NP * LS + k], o2 = so[2 * NP * LS + k];
            const V c0 = cmul(kv[7], o2) - cmul(kv[8], o1);
            const V c1 = cmul(kv[8], o0) - cmul(kv[6], o2);
            const V c2 = cmul(kv[6], o1) - cmul(kv[7], o0);
            if (h == 0) {
              y0 = y0 + c0;
              y1 = y1 + c1;
              y2 = y2 + c2;
            } else {
              y0 = y0 - c0;
              y1 = y1 - c1;
              y2 = y2 - c2;
            }
          }
          X[0][k2] = y0;
          X[1][k2] = y1;
          X[2][k2] = y2;
        }
      }
    }
    if (NG == 2) __syncthreads();  // the other group has read the parked spectra
    // ---- inverse: step A of every output component into its line
#pragma unroll
    for (int c = 0; c < GO; ++c) {
      Dft<R, +1, T>::run(X[c]);
      V* s = s0 + c * NP * LS;
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) s[n2 * PI + t] = PK ? pcmulc(X[c][n2], tw[n2 * (2 * t + r)])
                                                          : cmulc(X[c][n2], tw[n2 * (2 * t + r)]);
    }
    __syncthreads();
    // every thread is past the group's last mixing: the slab may take the next group's kernel
    if (PS && vn >= 4 && ngrp < NGROUPS) slab_issue(ngrp);
    // ---- step B; this CTA keeps outputs z = 16 n1 + t with n1 in [8 r, 8 r + 8)
    V keep[GO][R / 2], send[GO][R / 2];
#pragma unroll
    for (int c = 0; c < GO; ++c) {
      V u[R];
      const V* s = s0 + c * NP * LS + t * PI;
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) u[k1] = s[k1];
      Dft<R, +1, T>::run(u);
      if (r) {
#pragma unroll
        for (int n1 = 1; n1 < R; ++n1) u[n1] = twc<32, +1, T>(u[n1], n1);
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
          keep[c][m] = u[R / 2 + m];
          send[c][m] = u[m];
        }
      } else {
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
          keep[c][m] = u[m];
          send[c][m] = u[R / 2 + m];
        }
      }
    }
    cluster_barrier();  // both CTAs are done reading their lines
#pragma unroll
    for (int c = 0; c < GO; ++c)
#pragma unroll
      for (int m = 0; m < R / 2; ++m)
        st_peer(s0_peer + 8u * (unsigned)(c * NP * LS + m * R + t), send[c][m]);
    cluster_barrier();  // the other CTA's half has arrived
#pragma unroll
    for (int c = 0; c < GO; ++c)
#pragma unroll
      for (int m = 0; m < R / 2; ++m) {
        const V y = keep[c][m] + s0[c * NP * LS + m * R + t];
        colbase[c * cs + (long long)(R * (R / 2 * r + m) + t) * zs] = y;
      }
  }
  }
}

// x-lines of all components: inverse, keep x < n, epilogue y = x + H u
// (with_identity 1), y = H u (2: the operator minus the identity) or y = u (0).  CO = 3 (one H block) or 6 ([J; M] with H_eps and H_mu, or [E; H]).
template <typename T, int R1, int R2, int CO>
__global__ void __launch_bounds__(256) f_p5(const typename CT<T>::V* __restrict__ A,
                                            const typename IOT<T>::E* __restrict__ xin, typename IOT<T>::E* __restrict__ y,
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
  // component c + 1's row is loaded while component c is transformed
  V X[F::J][R2], Xn[F::J][R2];
  auto load_row = [&](int c, V (*D)[R2]) {
    const V* src = A + ((long long)b * C + c) * cs + (long long)row * M;
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) D[j][k2] = (ok && F::row(t, j)) ? src[t + R2 * j + R1 * k2] : CT<T>::make(0, 0);
  };
  load_row(0, X);
#pragma unroll
  for (int c = 0; c < CO; ++c) {
    if (c >= cout) break;
    if (c + 1 < CO && c + 1 < cout) load_row(c + 1, Xn);
    F::invA(X, t, s, tw);
    __syncthreads();
    V u[R1];
    F::template invB<true>(u, t, s);
#pragma unroll
    for (int n1 = 0; n1 < H2; ++n1) uo[c][n1] = u[n1];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < F::J; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) X[j][k2] = Xn[j][k2];
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
        const typename IOT<T>::E* xi = xin + ((long long)b * CO + 3 * blk) * N + pt;
        typename IOT<T>::E* yo = y + ((long long)b * CO + 3 * blk) * N + pt;
        const V a0 = uo[3 * blk][n1], a1 = uo[3 * blk + 1][n1], a2 = uo[3 * blk + 2][n1];
        if (with_identity == 1) {
          yo[0] = from_v<T>(to_v<T>(xi[0]) + cmul(hxx, a0) + cmul(hxy, a1) + cmul(hxz, a2));
          yo[N] = from_v<T>(to_v<T>(xi[N]) + cmul(hxy, a0) + cmul(hyy, a1) + cmul(hyz, a2));
          yo[2 * N] = from_v<T>(to_v<T>(xi[2 * N]) + cmul(hxz, a0) + cmul(hyz, a1) + cmul(hzz, a2));
        } else {  // 2: H u alone
          yo[0] = from_v<T>(cmul(hxx, a0) + cmul(hxy, a1) + cmul(hxz, a2));
          yo[N] = from_v<T>(cmul(hxy, a0) + cmul(hyy, a1) + cmul(hyz, a2));
          yo[2 * N] = from_v<T>(cmul(hxz, a0) + cmul(hyz, a1) + cmul(hzz, a2));
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < CO; ++c)
        if (c < cout) y[((long long)b * cout + c) * N + pt] = from_v<T>(uo[c][n1]);
    }
  }
}

inline size_t smem_optin() { return (size_t)smem_optin_bytes(); }

// Fast-path launches for 2n = R1 R2; returns false if a pass must use the generic kernels.
template <typename T, int R1, int R2>
struct FastPath {
  typedef typename CT<T>::V V;
  typedef Fft2<f32x2, R1, R2> F2;
  static constexpr int M = R1 * R2, L = 256 / R2;
  static size_t smem() { return sizeof(V) * (M + L * Fft2<T, R1, R2>::LS); }
  typedef typename IOT<T>::E E;
  static vie_status p1(const E* x, V* A, int n, int C, int cin, int nrhs, const V* tw, cudaStream_t st) {
    VIE_CK(allow_smem(f_p1<T, R1, R2>));
    f_p1<T, R1, R2><<<dim3((n * n + L - 1) / L, cin, nrhs), 256, smem(), st>>>(x, A, n, C, tw);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
  template <int S>
  static vie_status py(const V* in, V* out, int n, int C, int nc, int nrhs, const V* tw, cudaStream_t st) {
    VIE_CK(allow_smem(f_py<T, R1, R2, S>));
    f_py<T, R1, R2, S><<<dim3(M / L, n, nrhs * nc), 256, smem(), st>>>(in, out, n, C, nc, tw);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
  template <int MODE, int NP>
  static vie_status p3b(V* B, int n, int C, const V* K, int nrhs, const V* tw, cudaStream_t st) {
    constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
    constexpr int NTX = M / NP;
    const size_t sm = sizeof(V) * (M + (size_t)CMAX * NP * Fft2<T, R1, R2>::LS);
    if (sm > smem_optin()) {
      set_error("z-pass tile does not fit in shared memory");
      return VIE_EINVAL;
    }
    VIE_CK(allow_smem(f_p3b<T, R1, R2, MODE, NP>));
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
    constexpr int NTHR = P3cThreads<T, R1, R2, MODE, NP>::N;
    const size_t sm = sizeof(V) * (M + (size_t)CMAX * NP * LS + (size_t)NARR * (n + 1) * (NP + 1));
    const size_t cap = 224 * 1024;
    *done = false;
    if constexpr (NTHR > 1024 || NTX < 2) {
      return VIE_OK;  // shape not expressible: not instantiated
    } else {
      if (sm > cap || sm > smem_optin()) return VIE_OK;
      VIE_CK(allow_smem(f_p3c<T, R1, R2, MODE, NP>));
      f_p3c<T, R1, R2, MODE, NP><<<dim3((M / 2 + 1) * (NTX / 2), nrhs), NTHR, sm, st>>>(B, n, C, K, tw);
      VIE_CK(cudaGetLastError());
      *done = true;
      return VIE_OK;
    }
  }
  template <int MODE, int NP>
  static vie_status p3p(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    *done = false;
    if constexpr (sizeof(T) != 4 || NP < 2 || F2::J * R2 > 16 || R1 > 16) {
      return VIE_OK;  // lane pairs are FP32 only; register budget limits the line length
    } else {
      constexpr int CMAX = ModeDim<MODE>::CI > ModeDim<MODE>::CO ? ModeDim<MODE>::CI : ModeDim<MODE>::CO;
      constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
      constexpr int LS = ((F2::LS0 + 13) / 16) * 16 + 2;
      constexpr int NTX = M / NP;
      constexpr int NTHR = P3pThreads<MODE, NP, R2>::N;
      const size_t sm = 16 * (M + (size_t)CMAX * (NP / 2) * LS) + 8 * (size_t)NARR * (n + 1) * (NP + 1);
      const size_t cap = P3pThreads<MODE, NP, R2>::MINB == 2 ? 112 * 1024 : 224 * 1024;
      if constexpr (NTHR > 1024 || NTX < 2) {
        return VIE_OK;
      } else {
        if (sm > cap || sm > smem_optin()) return VIE_OK;
        VIE_CK(allow_smem(f_p3p<R1, R2, MODE, NP>));
        f_p3p<R1, R2, MODE, NP><<<dim3((M / 2 + 1) * (NTX / 2), nrhs), NTHR, sm, st>>>(
            (float2*)B, n, C, (const float2*)K, (const float2*)tw);
        VIE_CK(cudaGetLastError());
        *done = true;
        return VIE_OK;
      }
    }
  }
  template <int MODE, int NP, bool PERSIST = false>
  static vie_status p3t(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    *done = false;
    if constexpr (sizeof(T) != 4 || Fft2<T, R1, R2>::J * R2 > 16 || R1 > 16 ||
                  !(MODE == KM_SYM3 || MODE == KM_DIV || MODE == KM_MAXWELL6)) {
      return VIE_OK;  // FP32 only; three components of a pencil must fit in registers
    } else {
      typedef Fft2<T, R1, R2> F;
      constexpr int NG = P3tThreads<MODE, NP, R2>::NG;
      constexpr int NARR = (MODE == KM_SYM3) ? 6 : (MODE == KM_DIV ? 3 : 9);
      constexpr int LS = ((F::LS0 + 13) / 16) * 16 + 2;
      constexpr int NTX = M / NP;
      constexpr int NTHR = P3tThreads<MODE, NP, R2>::N;
      const int O = n + 1, OP = ((O + 13) / 16) * 16 + 2;
      const size_t sm = sizeof(V) * (M + (size_t)NG * 3 * NP * LS + (size_t)NARR * (NP + 1) * OP);
      if constexpr (NTHR > 1024 || NTX < 2) {
        return VIE_OK;
      } else {
        if (sm > smem_optin()) return VIE_OK;
        VIE_CK(allow_smem(f_p3t<R1, R2, MODE, NP>));
        int groups = (M / 2 + 1) * (NTX / 2);
        if (PERSIST) {  // as many CTAs as fit at once; each walks several mirror groups
          int dev = 0, sms = 0, per = 0;
          VIE_CK(cudaGetDevice(&dev));
          VIE_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
          VIE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f_p3t<R1, R2, MODE, NP>, NTHR, sm));
          if (per < 1) return VIE_OK;
          groups = std::min(groups, sms * per);
        }
        f_p3t<R1, R2, MODE, NP><<<dim3(groups, nrhs), NTHR, sm, st>>>(
            (float2*)B, n, C, (const float2*)K, (const float2*)tw);
        VIE_CK(cudaGetLastError());
        *done = true;
        return VIE_OK;
      }
    }
  }
  template <int MODE, int NP, int MINB>
  static vie_status p3s(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    *done = false;
    if constexpr (sizeof(T) != 4 || Fft2<T, R1, R2>::J * R2 > 16 || R1 > 16 || R2 % 2 != 0 ||
                  !(MODE == KM_SYM3 || MODE == KM_DIV)) {
      return VIE_OK;  // FP32 only; three components of a pencil must fit in registers
    } else {
      typedef P3sCfg<R1, R2, MODE, NP> Cfg;
      constexpr int NTX = M / NP;
      if constexpr (Cfg::NTHR > 1024 || NTX < 2) {
        return VIE_OK;
      } else {
        if (2 * n != M) return VIE_OK;
        const size_t sm = (size_t)Cfg::SMEM;
        if (sm > smem_optin()) return VIE_OK;
        auto kern = f_p3s<R1, R2, MODE, NP, MINB>;
        // the whole unified L1 as shared memory: MINB CTAs of ~75 KB per SM
        VIE_CK(allow_smem(kern, true));
        const int groups = (M / 2 + 1) * (NTX / 2);
        kern<<<dim3(groups, nrhs), Cfg::NTHR, sm, st>>>((float2*)B, n, C, (const float2*)K, (const float2*)tw);
        VIE_CK(cudaGetLastError());
        *done = true;
        return VIE_OK;
      }
    }
  }
  template <int MODE, int NP, bool PK, bool PS = false>
  static vie_status p3h(V* B, int n, int C, const V* K, int nrhs, const V* tw, bool* done, cudaStream_t st) {
    *done = false;
    if constexpr (sizeof(T) != 4 || M != 512 || !(MODE == KM_SYM3 || MODE == KM_MAXWELL6)) {
      return VIE_OK;  // FP32 at 2n = 512, the operator's kernel sets only
    } else {
      typedef P3hCfg<MODE, NP> Cfg;
      if (2 * n != M) return VIE_OK;
      const size_t sm = Cfg::SMEM;
      if (sm > smem_optin()) return VIE_OK;
      auto kern = f_p3h<MODE, NP, Cfg::MINB, PK, PS>;
      VIE_CK(allow_smem(kern, true));
      int groups = (M / 2 + 1) * (M / NP / 2);  // one cluster of two CTAs per mirror group
      if (PS) {  // as many clusters as are co-resident; each walks several mirror groups
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * groups, nrhs);
        cfg.blockDim = dim3(Cfg::NTHR);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = st;
        int nclu = 0;
        if (cudaOccupancyMaxActiveClusters(&nclu, (const void*)kern, &cfg) != cudaSuccess || nclu < 1) {
          (void)cudaGetLastError();
          return VIE_OK;  // not applicable on this device
        }
        groups = std::max(1, std::min(groups, nclu / nrhs));
      }
      kern<<<dim3(2 * groups, nrhs), Cfg::NTHR, sm, st>>>((float2*)B, C, (const float2*)K, (const float2*)tw);
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
      if (sizeof(V) * (M + (size_t)CMAX * NP * Fft2<T, R1, R2>::LS) > smem_optin()) return VIE_OK;
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
      case 4: return p3p<MODE, 8>(B, n, C, K, nrhs, tw, done, st);
      case 5: return p3p<MODE, 16>(B, n, C, K, nrhs, tw, done, st);
      case 6: return p3p<MODE, 4>(B, n, C, K, nrhs, tw, done, st);
      case 7: return p3t<MODE, 8>(B, n, C, K, nrhs, tw, done, st);
      case 8: return p3t<MODE, 4>(B, n, C, K, nrhs, tw, done, st);
      case 9: return p3t<MODE, 16>(B, n, C, K, nrhs, tw, done, st);
      case 10: return p3t<MODE, 8, true>(B, n, C, K, nrhs, tw, done, st);
      case 11: return p3t<MODE, 4, true>(B, n, C, K, nrhs, tw, done, st);
      case 12: return p3s<MODE, 8, 3>(B, n, C, K, nrhs, tw, done, st);
      case 13: return p3s<MODE, 8, 2>(B, n, C, K, nrhs, tw, done, st);
      case 14: return p3s<MODE, 4, 5>(B, n, C, K, nrhs, tw, done, st);
      case 15: return p3h<MODE, 4, false>(B, n, C, K, nrhs, tw, done, st);
      case 16: return p3h<MODE, 8, false>(B, n, C, K, nrhs, tw, done, st);
      case 17: return p3h<MODE, 8, true>(B, n, C, K, nrhs, tw, done, st);
      default: return p3h<MODE, 8, false, true>(B, n, C, K, nrhs, tw, done, st);
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
  static vie_status p5(const V* A, const E* xin, E* y, int n, int C, int cout, const V* He, const V* Hm, int wid,
                       int nrhs, const V* tw, cudaStream_t st) {
    const dim3 grid((n * n + L - 1) / L, nrhs);
    if (cout <= 3) {
      VIE_CK(allow_smem(f_p5<T, R1, R2, 3>));
      f_p5<T, R1, R2, 3><<<grid, 256, smem(), st>>>(A, xin, y, n, C, cout, He, Hm, wid, tw);
    } else {
      VIE_CK(allow_smem(f_p5<T, R1, R2, 6>));
      f_p5<T, R1, R2, 6><<<grid, 256, smem(), st>>>(A, xin, y, n, C, cout, He, Hm, wid, tw);
    }
    VIE_CK(cudaGetLastError());
    return VIE_OK;
  }
};

template <typename T, int R1, int R2>
vie_status fast_pass(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                            int with_identity, typename CT<T>::V* A, typename CT<T>::V* B, int C, cudaStream_t st) {
  typedef FastPath<T, R1, R2> FP;
  typedef typename CT<T>::V V;
  const int n = P->n;
  const V* tw = Prec<T>::tw(P);
  const int cin = cin_of(K.mode), cout = cout_of(K.mode);
  switch (pass) {
    case 1: return FP::p1((const typename IOT<T>::E*)in, A, n, C, cin, nrhs, tw, st);
    case 2: return FP::template py<-1>(A, B, n, C, cin, nrhs, tw, st);
    case 3: {
      bool done = false;
      vie_status e = FP::p3v(P->p3_variant[Prec<T>::id][K.mode], B, n, C, Prec<T>::K(K), K.mode, nrhs,
                             tw, &done, st);
      if (e == VIE_OK && !done) {
        set_error("selected z-pass variant does not apply to this shape");
        return VIE_EINVAL;
      }
      return e;
    }
    case 4: return FP::template py<+1>(B, A, n, C, cout, nrhs, tw, st);
    default:
      return FP::p5(A, (const typename IOT<T>::E*)in, (typename IOT<T>::E*)out, n, C, cout, Prec<T>::He(P),
                    P->has_mu ? Prec<T>::Hm(P) : nullptr, with_identity, nrhs, tw, st);
  }
}

// Autotuner for the z pass: every applicable variant (mirror-group CTAs with
// 8, 16 or 4 pencils, one tile per CTA with 8 pencils, lane-pair
// mirror-group CTAs with 8, 16 or 4 pencils, component-group mirror-group
// CTAs with 8, 4 or 16 pencils, component-group CTAs of 8 or 4 pencils
// sized to the device, each walking several mirror groups, or slim
// component-group CTAs of 8 pencils for three or two CTAs per SM, or of 4
// pencils for five) runs once untimed
// (a pass over all candidates, which also brings the clocks up), then two
// rounds of 3 launches timed with CUDA events on the buffer B (whose contents
// are scratch at this point); each keeps its best round and the fastest is
// kept for the problem's (precision, mode).  VIE_TUNE=0 takes the first
// applicable variant; VIE_P3_VARIANT=k forces variant k.
static const int kP3Variants = 19;
static const int kP3Generic = 99;

template <typename T, int R1, int R2>
vie_status tune_p3(vie_problem* P, const KernelSet& K, typename CT<T>::V* B, int C, cudaStream_t st,
                          int* best) {
  typedef FastPath<T, R1, R2> FP;
  const typename CT<T>::V* tw = Prec<T>::tw(P);
  const char* force = getenv("VIE_P3_VARIANT");
  const char* tune = getenv("VIE_TUNE");
  const bool timed = !(tune && tune[0] == '0');
  *best = -1;
  // applicable variants, each launched once untimed (this also brings the
  // clocks up, so that the first candidates are not timed while they ramp)
  std::vector<int> cand;
  for (int v = 0; v < kP3Variants; ++v) {
    if (force && atoi(force) != v) continue;
    bool done = false;
    vie_status s = FP::p3v(v, B, P->n, C, Prec<T>::K(K), K.mode, 1, tw, &done, st);
    if (s != VIE_OK) return s;
    if (done) cand.push_back(v);
  }
  if (cand.empty()) {
    if (force) {
      set_error("forced z-pass variant does not apply to this shape");
      return VIE_EINVAL;
    }
    *best = kP3Generic;  // no register-resident variant fits: generic kernel
    return VIE_OK;
  }
  if (!timed || force || cand.size() == 1) {
    *best = cand[0];
    return VIE_OK;
  }
  // two rounds of 3 timed launches per candidate; each keeps its best round
  std::vector<float> ms(cand.size(), 1e30f);
  cudaEvent_t e0, e1;
  VIE_CK(cudaEventCreate(&e0));
  VIE_CK(cudaEventCreate(&e1));
  for (int round = 0; round < 2; ++round)
    for (size_t c = 0; c < cand.size(); ++c) {
      bool done = false;
      VIE_CK(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) FP::p3v(cand[c], B, P->n, C, Prec<T>::K(K), K.mode, 1, tw, &done, st);
      VIE_CK(cudaEventRecord(e1, st));
      VIE_CK(cudaEventSynchronize(e1));
      float t = 0.f;
      VIE_CK(cudaEventElapsedTime(&t, e0, e1));
      ms[c] = std::min(ms[c], t);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  size_t b = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (ms[c] < ms[b]) b = c;
  *best = cand[b];
  return VIE_OK;
}

// Double-word (VIE_DF64) fast path: the register-resident P1, P2, P4 and the
// mirror-group z pass for the operator's kernel sets only (3x3 symmetric,
// Maxwell 6x6), one fixed schedule each (8 pencils per tile, 4 for Maxwell),
// no tuning.  Instantiated for 2n = 256 only, in its own translation unit
// (apply_fast_dw_256.cu): the unrolled double-word codelets are long to
// compile, so every other shape and mode keeps the generic kernels.
// *used = false if this (pass, mode) has no double-word fast kernel.
template <int R1, int R2>
vie_status fast_pass_dw(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                        int with_identity, cdf* A, cdf* B, int C, cudaStream_t st, bool* used) {
  typedef FastPath<df, R1, R2> FP;
  const int n = P->n;
  const cdf* tw = Prec<df>::tw(P);
  const int cin = cin_of(K.mode), cout = cout_of(K.mode);
  *used = true;
  switch (pass) {
    case 1: return FP::p1((const double2*)in, A, n, C, cin, nrhs, tw, st);
    case 2: return FP::template py<-1>(A, B, n, C, cin, nrhs, tw, st);
    case 3: {
      bool done = false;
      vie_status e = VIE_OK;
      if (K.mode == KM_SYM3) {
        e = FP::template p3c<KM_SYM3, 8>(B, n, C, Prec<df>::K(K), nrhs, tw, &done, st);
        if (e == VIE_OK && !done) e = FP::template p3c<KM_SYM3, 4>(B, n, C, Prec<df>::K(K), nrhs, tw, &done, st);
      } else if (K.mode == KM_MAXWELL6) {
        e = FP::template p3c<KM_MAXWELL6, 4>(B, n, C, Prec<df>::K(K), nrhs, tw, &done, st);
      }
      if (e == VIE_OK && !done) *used = false;
      return e;
    }
    case 4: return FP::template py<+1>(B, A, n, C, cout, nrhs, tw, st);
    default:
      return FP::p5(A, (const double2*)in, (double2*)out, n, C, cout, Prec<df>::He(P),
                    P->has_mu ? Prec<df>::Hm(P) : nullptr, with_identity, nrhs, tw, st);
  }
}
vie_status fast_pass_dw_256(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                            int wid, void* A, void* B, int C, cudaStream_t st, bool* used);

// Per-size entry points (one translation unit each).
#define VIE_FAST_SIZES(X) X(64, 8, 8) X(96, 12, 8) X(128, 16, 8) X(192, 24, 8) X(256, 16, 16) X(384, 24, 16) X(512, 32, 16)

#define VIE_FAST_DECL(MM, RA, RB)                                                                                   \
  vie_status fast_pass_##MM(bool f64, int pass, vie_problem* P, const KernelSet& K, const void* in, void* out,       \
                            int nrhs, int wid, void* A, void* B, int C, cudaStream_t st);                         \
  vie_status tune_p3_##MM(bool f64, vie_problem* P, const KernelSet& K, void* B, int C, cudaStream_t st, int* best);
VIE_FAST_SIZES(VIE_FAST_DECL)

#define VIE_FAST_DEFINE(MM, RA, RB)                                                                                 \
  vie_status fast_pass_##MM(bool f64, int pass, vie_problem* P, const KernelSet& K, const void* in, void* out,       \
                            int nrhs, int wid, void* A, void* B, int C, cudaStream_t st) {                        \
    return f64 ? fast_pass<double, RA, RB>(pass, P, K, in, out, nrhs, wid, (double2*)A, (double2*)B, C, st)         \
               : fast_pass<float, RA, RB>(pass, P, K, in, out, nrhs, wid, (float2*)A, (float2*)B, C, st);           \
  }                                                                                                                \
  vie_status tune_p3_##MM(bool f64, vie_problem* P, const KernelSet& K, void* B, int C, cudaStream_t st, int* best) { \
    return f64 ? tune_p3<double, RA, RB>(P, K, (double2*)B, C, st, best)                                             \
               : tune_p3<float, RA, RB>(P, K, (float2*)B, C, st, best);                                              \
  }

}  // namespace vie
