// Register-resident two-step FFT of length M = R1 * R2 for lines that are
// processed by T = R2 threads each (thread t owns the k1 rows t + R2 j < R1).
//
//   forward  X[k1 + R1 k2] = sum_{n2} W_R2^{n2 k2} W_M^{n2 k1} sum_{n1} W_R1^{n1 k1} x[R2 n1 + n2]
//   inverse  x[R2 n1 + n2] = sum_{k1} W_R1^{-n1 k1} W_M^{-n2 k1} sum_{k2} W_R2^{-n2 k2} X[k1 + R1 k2]
//
// Step 1 of the forward transform runs in thread n2 (an R1-point DFT on its
// registers), the twiddled result goes through shared memory once, and step 2
// runs ceil(R1/T) R2-point DFTs per thread.  After the forward transform thread
// t holds X[k1 + R1 k2] for k1 = t + T j < R1 and all k2 -- exactly the
// layout the inverse transform starts from, so a pointwise multiply in k-space
// (the kernel mixing of the convolution) needs no data movement.
// Pruning for zero padding: the forward input may be limited to its first
// half (n1 < R1/2) and the inverse output to its first half (n1 < R1/2).
//
// Shared-memory transpose layout per line: rows of R2 + 1 (forward) or R1 + 1
// (inverse) elements and an odd line pitch, so that 16 consecutive lines or
// 16 consecutive rows hit distinct banks for 8-byte and 16-byte elements.
#pragma once

#include "vie_fft.cuh"

namespace vie {

// cos(pi j / 16), j = 0..31
__device__ __forceinline__ double cos_pi16(int j) {
  const double c[32] = {1.0,
                        0.98078528040323044913,
                        0.92387953251128675613,
                        0.83146961230254523708,
                        0.70710678118654752440,
                        0.55557023301960222474,
                        0.38268343236508977173,
                        0.19509032201612826785,
                        0.0,
                        -0.19509032201612826785,
                        -0.38268343236508977173,
                        -0.55557023301960222474,
                        -0.70710678118654752440,
                        -0.83146961230254523708,
                        -0.92387953251128675613,
                        -0.98078528040323044913,
                        -1.0,
                        -0.98078528040323044913,
                        -0.92387953251128675613,
                        -0.83146961230254523708,
                        -0.70710678118654752440,
                        -0.55557023301960222474,
                        -0.38268343236508977173,
                        -0.19509032201612826785,
                        0.0,
                        0.19509032201612826785,
                        0.38268343236508977173,
                        0.55557023301960222474,
                        0.70710678118654752440,
                        0.83146961230254523708,
                        0.92387953251128675613,
                        0.98078528040323044913};
  return c[j & 31];
}

// cos(2 pi j / 24), j = 0..23
__device__ __forceinline__ double cos_2pi24(int j) {
  const double c[24] = {1.0,
                        0.96592582628906828675,
                        0.86602540378443864676,
                        0.70710678118654752440,
                        0.5,
                        0.25881904510252076235,
                        0.0,
                        -0.25881904510252076235,
                        -0.5,
                        -0.70710678118654752440,
                        -0.86602540378443864676,
                        -0.96592582628906828675,
                        -1.0,
                        -0.96592582628906828675,
                        -0.86602540378443864676,
                        -0.70710678118654752440,
                        -0.5,
                        -0.25881904510252076235,
                        0.0,
                        0.25881904510252076235,
                        0.5,
                        0.70710678118654752440,
                        0.86602540378443864676,
                        0.96592582628906828675};
  return c[((j % 24) + 24) % 24];
}

// a * W_R^{S j} with W_R = exp(2 pi i / R) (R divides 32 or 24)
template <int R, int S, typename T>
__device__ __forceinline__ typename CT<T>::V twc(typename CT<T>::V a, int j) {
  double c, s;
  if constexpr (32 % R == 0) {
    const int q = (j * (32 / R)) & 31;  // angle pi q / 16
    // quarter turns are exact swaps and negations (j is a constant in every caller)
    if (q == 8) return mul_si<S>(a);
    if (q == 24) return mul_si<-S>(a);
    c = cos_pi16(q);
    s = S * cos_pi16(q + 24);  // sin(pi q/16) = cos(pi (q - 8)/16)
  } else {
    static_assert(24 % R == 0, "twiddle table covers R | 32 and R | 24");
    const int q = (j * (24 / R)) % 24;  // angle 2 pi q / 24
    if (q == 6) return mul_si<S>(a);
    if (q == 18) return mul_si<-S>(a);
    c = cos_2pi24(q);
    s = S * cos_2pi24(q + 18);  // sin(t) = cos(t - pi/2)
  }
  return rot(a, (T)c, (T)s);
}

// DFT of length P Q on registers by the same two-step split as the line FFT:
// X[k1 + P k2] = sum_{n2} W_Q^{n2 k2} W_{PQ}^{n2 k1} sum_{n1} W_P^{n1 k1} x[Q n1 + n2].
template <int P, int Q, int S, typename T>
struct DftPQ {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    V y[Q][P];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) y[n2][n1] = u[Q * n1 + n2];
      Dft<P, S, T>::run(y[n2]);
#pragma unroll
      for (int k1 = 1; k1 < P; ++k1)
        if (n2 != 0) y[n2][k1] = twc<P * Q, S, T>(y[n2][k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      V z[Q];
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) z[n2] = y[n2][k1];
      Dft<Q, S, T>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) u[k1 + P * k2] = z[k2];
    }
  }
};
template <int S, typename T> struct Dft<6, S, T> : DftPQ<2, 3, S, T> {};
template <int S, typename T> struct Dft<12, S, T> : DftPQ<4, 3, S, T> {};
template <int S, typename T> struct Dft<24, S, T> : DftPQ<8, 3, S, T> {};

template <int S, typename T> struct Dft<32, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    V e[16], o[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      e[r] = u[2 * r];
      o[r] = u[2 * r + 1];
    }
    Dft<16, S, T>::run(e);
    Dft<16, S, T>::run(o);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const V t = (q == 0) ? o[0] : twc<32, S, T>(o[q], q);
      u[q] = e[q] + t;
      u[q + 16] = e[q] - t;
    }
  }
};

// DFT_R of u[0..R/2-1] followed by R/2 zeros (decimation in frequency).
template <int R, int S, typename T>
__device__ __forceinline__ void dft_half_in(typename CT<T>::V* u) {
  typedef typename CT<T>::V V;
  constexpr int H = R / 2;
  V a[H], b[H];
#pragma unroll
  for (int r = 0; r < H; ++r) {
    a[r] = u[r];
    b[r] = (r == 0) ? u[0] : twc<R, S, T>(u[r], r);
  }
  Dft<H, S, T>::run(a);
  Dft<H, S, T>::run(b);
#pragma unroll
  for (int m = 0; m < H; ++m) {
    u[2 * m] = a[m];
    u[2 * m + 1] = b[m];
  }
}

// First R/2 outputs of the DFT_R of u[0..R-1] (decimation in time).
template <int R, int S, typename T>
__device__ __forceinline__ void dft_half_out(typename CT<T>::V* u) {
  typedef typename CT<T>::V V;
  constexpr int H = R / 2;
  V a[H], b[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    a[m] = u[2 * m];
    b[m] = u[2 * m + 1];
  }
  Dft<H, S, T>::run(a);
  Dft<H, S, T>::run(b);
#pragma unroll
  for (int n = 0; n < H; ++n) u[n] = a[n] + ((n == 0) ? b[0] : twc<R, S, T>(b[n], n));
}

template <typename T, int R1, int R2>
struct Fft2 {
  typedef typename CT<T>::V V;
  static constexpr int M = R1 * R2;
  static constexpr int NT = R2;                 // threads per line
  static constexpr int J = (R1 + R2 - 1) / R2;  // k1 rows per thread (k1 = t + R2 j < R1)
  // Does thread t own row j?  Always true when R2 divides R1.
  static __device__ __forceinline__ bool row(int t, int j) { return (R1 % R2 == 0) || (t + R2 * j < R1); }
  static constexpr int PF = R2 + 1;      // forward transpose row pitch
  static constexpr int PI = R1 + 1;      // inverse transpose row pitch
  static constexpr int LS0 = (R1 * PF > R2 * PI ? R1 * PF : R2 * PI);
  static constexpr int LS = (LS0 % 2 == 0) ? LS0 + 1 : LS0;  // odd line pitch

  // Step 1 forward.  u[n1] = x[R2 n1 + t]; HALF: only n1 < R1/2 are nonzero.
  template <bool HALF>
  static __device__ __forceinline__ void fwd1(V* u, int t, V* s, const V* tw) {
    if (HALF) dft_half_in<R1, -1, T>(u);
    else Dft<R1, -1, T>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      V v = u[k1];
      if (k1 != 0) v = cmul(v, tw[t * k1]);
      s[k1 * PF + t] = v;
    }
  }
  // Step 1 forward with the twiddles W_M^{t k1} already in registers (w[k1]).
  template <bool HALF>
  static __device__ __forceinline__ void fwd1w(V* u, int t, V* s, const V* w) {
    if (HALF) dft_half_in<R1, -1, T>(u);
    else Dft<R1, -1, T>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      V v = u[k1];
      if (k1 != 0) v = cmul(v, w[k1]);
      s[k1 * PF + t] = v;
    }
  }
  // Step 2 forward: X[j][k2] = X[k1 = t + R2 j][k2].
  static __device__ __forceinline__ void fwd2(V (*X)[R2], int t, const V* s) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!row(t, j)) continue;
      const int k1 = t + R2 * j;
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) X[j][n2] = s[k1 * PF + n2];
      Dft<R2, -1, T>::run(X[j]);
    }
  }
  // Step A inverse from the forward layout.
  static __device__ __forceinline__ void invA(V (*X)[R2], int t, V* s, const V* tw) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!row(t, j)) continue;
      const int k1 = t + R2 * j;
      Dft<R2, +1, T>::run(X[j]);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        V v = X[j][n2];
        if (n2 != 0 && k1 != 0) v = cmulc(v, tw[n2 * k1]);
        s[n2 * PI + k1] = v;
      }
    }
  }
  // Step B inverse: u[n1] = x[R2 n1 + t]; HALF: only n1 < R1/2 are produced.
  template <bool HALF>
  static __device__ __forceinline__ void invB(V* u, int t, const V* s) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) u[k1] = s[t * PI + k1];
    if (HALF) dft_half_out<R1, +1, T>(u);
    else Dft<R1, +1, T>::run(u);
  }
};

}  // namespace vie
