// Device-side building blocks shared by every kernel of the library:
// complex arithmetic on CUDA vector types, small DFT codelets, and a
// shared-memory mixed-radix (2, 3, 4, 5, 7, 8, 11, 16) Stockham FFT that
// transforms a tile of lines resident in shared memory; line lengths with a
// larger prime factor go through Bluestein's chirp-z algorithm on top of it.
//
// The FFT is the engine of the truncated-kernel method of Sec. 5 (steps a-c:
// truncate the Green's function, transform it, cut off at the grid Nyquist
// frequency); every volume potential is applied as a zero-padded circular
// convolution on a (2n)^3 grid.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace vie {

// ------------------------------------------------------------ complex math
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// FP32 complex add/sub/scale as one packed f32x2 instruction on sm_100+
// (element-wise IEEE round-to-nearest: bit-identical to two scalar ops, half
// the issue slots -- the FFT butterflies are mostly complex adds).  The
// compiler builtins keep the operations visible to register allocation and
// scheduling.
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a + (-1) b: one rounding, same as a - b
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fmul2_rn(make_float2(s, s), a);
#else
  return make_float2(s * a.x, s * a.y);
#endif
}

__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

template <typename T> struct CT;
template <> struct CT<double> {
  typedef double2 V;
  static __host__ __device__ __forceinline__ V make(double a, double b) { return make_double2(a, b); }
};
template <> struct CT<float> {
  typedef float2 V;
  static __host__ __device__ __forceinline__ V make(float a, float b) { return make_float2(a, b); }
};

// ------------------------------------------------ lane pairs: two lines at once
// f32x2 holds the same quantity of two independent transforms (its lanes a
// and b); c32x2 is a complex number whose real and imaginary parts are such
// pairs.  Every arithmetic operation on them is one packed f32x2 instruction
// (sm_100 and later), so a codelet instantiated on f32x2 transforms two lines
// for the instruction count of one, and a multiplication by +-i is a swap of
// register roles rather than arithmetic.  Each lane is rounded exactly as the
// scalar operation would be.
struct __align__(8) f32x2 {
  float a, b;
  f32x2() = default;
  __host__ __device__ constexpr f32x2(float x, float y) : a(x), b(y) {}
  __host__ __device__ constexpr f32x2(double s) : a((float)s), b((float)s) {}  // broadcast
};
struct __align__(16) c32x2 {
  f32x2 x, y;
};
template <> struct CT<f32x2> {
  typedef c32x2 V;
  static __device__ __forceinline__ V make(f32x2 a, f32x2 b) {
    V r;
    r.x = a;
    r.y = b;
    return r;
  }
};
__device__ __forceinline__ float2 f2(f32x2 v) { return make_float2(v.a, v.b); }
__device__ __forceinline__ f32x2 p2(float2 v) { return f32x2(v.x, v.y); }
__device__ __forceinline__ f32x2 operator+(f32x2 x, f32x2 y) { return p2(__fadd2_rn(f2(x), f2(y))); }
// x - y as x + (-1) y: one rounding, identical to a subtraction
__device__ __forceinline__ f32x2 operator-(f32x2 x, f32x2 y) {
  return p2(__ffma2_rn(f2(y), make_float2(-1.f, -1.f), f2(x)));
}
__device__ __forceinline__ f32x2 operator*(f32x2 x, f32x2 y) { return p2(__fmul2_rn(f2(x), f2(y))); }
__device__ __forceinline__ f32x2 operator-(f32x2 x) { return f32x2(-x.a, -x.b); }
__device__ __forceinline__ f32x2& operator+=(f32x2& x, f32x2 y) {
  x = x + y;
  return x;
}
__device__ __forceinline__ c32x2 operator+(c32x2 a, c32x2 b) { return CT<f32x2>::make(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ c32x2 operator-(c32x2 a, c32x2 b) { return CT<f32x2>::make(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ c32x2 operator*(f32x2 s, c32x2 a) { return CT<f32x2>::make(s * a.x, s * a.y); }

// a * b + c with one rounding
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ f32x2 fmadd(f32x2 a, f32x2 b, f32x2 c) { return p2(__ffma2_rn(f2(a), f2(b), f2(c))); }

__device__ __forceinline__ c32x2 cmul(c32x2 a, c32x2 b) {
  return CT<f32x2>::make(fmadd(a.x, b.x, -(a.y * b.y)), fmadd(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ c32x2 cmulc(c32x2 a, c32x2 b) {
  return CT<f32x2>::make(fmadd(a.x, b.x, a.y * b.y), fmadd(a.y, b.x, -(a.x * b.y)));
}

// ------------------------------------------------ double-word arithmetic
// df holds a real number as the unevaluated sum hi + lo of two FP32 values
// with |lo| <= ulp(hi)/2, about 48 significant bits.  The operations are the
// double-word algorithms of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017):
// addition "AccurateDWPlusDW" (relative error <= 3u^2) and multiplication
// "DWTimesDW3" (<= 4u^2, with FMA), built on Knuth's TwoSum, Dekker's
// Fast2Sum and the FMA-exact product, u = 2^-24.  Every step is an explicitly
// rounded intrinsic, so compiler contraction cannot alter the error-free
// transformations.  All of it runs on the FP32 pipes, which on this GPU have
// 64 times the FP64 throughput.
struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
// A complex double-word number is stored as two lane pairs, h = (re.hi, im.hi)
// and l = (re.lo, im.lo), so that the real and imaginary parts go through every
// double-word step together as packed f32x2 instructions (each lane rounded
// exactly as the scalar algorithm would be); multiplication by +-i is a lane
// swap.
struct __align__(16) cdf {
  float2 h, l;
};
template <> struct CT<df> {
  typedef cdf V;
  static __host__ __device__ __forceinline__ V make(df re, df im) {
    V r;
    r.h = make_float2(re.hi, im.hi);
    r.l = make_float2(re.lo, im.lo);
    return r;
  }
};
// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// s + e = a + b exactly when the exponent of a is not below that of b (Fast2Sum)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df x, df y) {
  const df s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl1 = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ df fmadd(df a, df b, df c) { return a * b + c; }

// ---- lane-pair building blocks (two independent double-words per operation)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 bcx(float2 a) { return make_float2(a.x, a.x); }
__device__ __forceinline__ float2 bcy(float2 a) { return make_float2(a.y, a.y); }
// (h, l) <- Fast2Sum(a, b) and TwoSum(a, b), per lane
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& h, float2& l) {
  h = add2(a, b);
  l = sub2(b, sub2(h, a));
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& h, float2& l) {
  h = add2(a, b);
  const float2 bb = sub2(h, a);
  l = add2(sub2(a, sub2(h, bb)), sub2(b, bb));
}
// AccurateDWPlusDW per lane: (xh, xl) + (yh, yl)
__device__ __forceinline__ cdf dw_add2(float2 xh, float2 xl, float2 yh, float2 yl) {
  float2 sh, sl, th, tl, vh, vl;
  two_sum2(xh, yh, sh, sl);
  two_sum2(xl, yl, th, tl);
  fast_two_sum2(sh, add2(sl, th), vh, vl);
  cdf r;
  fast_two_sum2(vh, add2(tl, vl), r.h, r.l);
  return r;
}
// DWTimesDW3 per lane: (xh, xl) (yh, yl)
__device__ __forceinline__ cdf dw_mul2(float2 xh, float2 xl, float2 yh, float2 yl) {
  const float2 ch = mul2(xh, yh);
  const float2 cl1 = fma2(xh, yh, neg2(ch));
  const float2 tl1 = fma2(xh, yl, mul2(xl, yl));
  const float2 cl2 = fma2(xl, yh, tl1);
  cdf r;
  fast_two_sum2(ch, add2(cl1, cl2), r.h, r.l);
  return r;
}
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return dw_add2(a.h, a.l, b.h, b.l); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return dw_add2(a.h, a.l, neg2(b.h), neg2(b.l)); }
__device__ __forceinline__ cdf operator*(df s, cdf a) {
  return dw_mul2(a.h, a.l, make_float2(s.hi, s.hi), make_float2(s.lo, s.lo));
}
// a b = a (bx, bx) + swap(a) (-by, by)
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  const cdf p = dw_mul2(a.h, a.l, bcx(b.h), bcx(b.l));
  const cdf q = dw_mul2(swp(a.h), swp(a.l), make_float2(-b.h.y, b.h.y), make_float2(-b.l.y, b.l.y));
  return p + q;
}
// a conj(b) = a (bx, bx) + swap(a) (by, -by)
__device__ __forceinline__ cdf cmulc(cdf a, cdf b) {
  const cdf p = dw_mul2(a.h, a.l, bcx(b.h), bcx(b.l));
  const cdf q = dw_mul2(swp(a.h), swp(a.l), make_float2(b.h.y, -b.h.y), make_float2(b.l.y, -b.l.y));
  return p + q;
}
// a (c + i s) = a (c, c) + swap(a) (-s, s)
__device__ __forceinline__ cdf rot(cdf a, df c, df s) {
  const cdf p = dw_mul2(a.h, a.l, make_float2(c.hi, c.hi), make_float2(c.lo, c.lo));
  const cdf q = dw_mul2(swp(a.h), swp(a.l), make_float2(-s.hi, s.hi), make_float2(-s.lo, s.lo));
  return p + q;
}
__device__ __forceinline__ cdf cfma(df s, cdf a, cdf c) { return c + s * a; }
__device__ __forceinline__ cdf vneg(cdf a) {
  cdf r;
  r.h = neg2(a.h);
  r.l = neg2(a.l);
  return r;
}
// S i a = swap(a) (-S, S)
template <int S>
__device__ __forceinline__ cdf mul_si(cdf a) {
  cdf r;
  r.h = (S > 0) ? make_float2(-a.h.y, a.h.x) : make_float2(a.h.y, -a.h.x);
  r.l = (S > 0) ? make_float2(-a.l.y, a.l.x) : make_float2(a.l.y, -a.l.x);
  return r;
}
template <int S>
__device__ __forceinline__ cdf addi(cdf a, cdf b) {
  const cdf ib = mul_si<S>(b);
  return dw_add2(a.h, a.l, ib.h, ib.l);
}
template <int S>
__device__ __forceinline__ cdf subi(cdf a, cdf b) { return addi<-S>(a, b); }

// Element type a compute type reads and writes at the operator's interface
// (the FP64 vectors x, y for the double-word path), and the conversions.
template <typename T> struct IOT { typedef typename CT<T>::V E; };
template <> struct IOT<df> { typedef double2 E; };
template <typename T>
__device__ __forceinline__ typename CT<T>::V to_v(typename IOT<T>::E e) { return e; }
template <>
__device__ __forceinline__ cdf to_v<df>(double2 e) { return CT<df>::make(df(e.x), df(e.y)); }
template <typename T>
__device__ __forceinline__ typename IOT<T>::E from_v(typename CT<T>::V v) { return v; }
template <>
__device__ __forceinline__ double2 from_v<df>(cdf v) {
  return make_double2((double)v.h.x + (double)v.l.x, (double)v.h.y + (double)v.l.y);
}

// a * (S i) for S = +1 / -1
template <int S, typename V>
__device__ __forceinline__ V mul_si(V a) {
  V r;
  if (S > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
// a + S i b  and  a - S i b (no negation needed on any element type)
template <int S, typename V>
__device__ __forceinline__ V addi(V a, V b) {
  V r;
  if (S > 0) { r.x = a.x - b.y; r.y = a.y + b.x; } else { r.x = a.x + b.y; r.y = a.y - b.x; }
  return r;
}
template <int S, typename V>
__device__ __forceinline__ V subi(V a, V b) { return addi<-S>(a, b); }
// a (c + i s) for real c, s
template <typename T, typename V>
__device__ __forceinline__ V rot(V a, T c, T s) {
  V r;
  r.x = fmadd(-s, a.y, c * a.x);
  r.y = fmadd(s, a.x, c * a.y);
  return r;
}
// c + s a for real s, and -a (overloaded for the packed double-word complex)
template <typename T, typename V>
__device__ __forceinline__ V cfma(T s, V a, V c) {
  V r;
  r.x = fmadd(s, a.x, c.x);
  r.y = fmadd(s, a.y, c.y);
  return r;
}
template <typename V>
__device__ __forceinline__ V vneg(V a) {
  V r;
  r.x = -a.x;
  r.y = -a.y;
  return r;
}

// ------------------------------------------------------------ codelets
// In-place DFT of length R on registers: U_q = sum_r u_r exp(S 2 pi i r q / R).
template <int R, int S, typename T> struct Dft;

template <int S, typename T> struct Dft<2, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    V t = u[0];
    u[0] = t + u[1];
    u[1] = t - u[1];
  }
};

template <int S, typename T> struct Dft<3, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    const T h3 = (T)0.86602540378443864676;  // sqrt(3)/2
    V t = u[1] + u[2];
    V m = cfma((T)-0.5, t, u[0]);
    V d = h3 * (u[1] - u[2]);
    u[0] = u[0] + t;
    u[1] = addi<S>(m, d);
    u[2] = subi<S>(m, d);
  }
};

template <int S, typename T> struct Dft<4, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    V a0 = u[0] + u[2], a1 = u[0] - u[2];
    V b0 = u[1] + u[3], b1 = u[1] - u[3];
    u[0] = a0 + b0;
    u[2] = a0 - b0;
    u[1] = addi<S>(a1, b1);
    u[3] = subi<S>(a1, b1);
  }
};

template <int S, typename T> struct Dft<8, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    const T r2 = (T)0.70710678118654752440;
    V e[4] = {u[0], u[2], u[4], u[6]};
    V o[4] = {u[1], u[3], u[5], u[7]};
    Dft<4, S, T>::run(e);
    Dft<4, S, T>::run(o);
    // w8^q = exp(S 2 pi i q / 8): w8 = (1 + S i)/sqrt2, w8^2 = S i, w8^3 = S i w8
    V o1 = r2 * addi<S>(o[1], o[1]);
    V o3 = r2 * addi<S>(o[3], o[3]);
    u[0] = e[0] + o[0];
    u[4] = e[0] - o[0];
    u[1] = e[1] + o1;
    u[5] = e[1] - o1;
    u[2] = addi<S>(e[2], o[2]);
    u[6] = subi<S>(e[2], o[2]);
    u[3] = addi<S>(e[3], o3);
    u[7] = subi<S>(e[3], o3);
  }
};

// cos(pi j / 8), j = 0..15
__device__ __forceinline__ double cos_pi8(int j) {
  const double c[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                        0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                        -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                        0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
  return c[j & 15];
}

template <int S, typename T> struct Dft<16, S, T> {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    // r = 4 r1 + r2, q = q1 + 4 q2
    V a[4][4];
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) {
      V t[4] = {u[r2], u[4 + r2], u[8 + r2], u[12 + r2]};
      Dft<4, S, T>::run(t);
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1) {
        const int j = r2 * q1;  // w16^(r2 q1)
        if (j == 0) {
          a[q1][r2] = t[q1];
        } else if (j == 4) {  // w16^4 = S i: a swap, no multiply
          a[q1][r2] = mul_si<S>(t[q1]);
        } else {
          const T c = (T)cos_pi8(j);
          const T s = (T)(S * cos_pi8(j + 12));  // sin(pi j/8) = cos(pi (j - 4)/8) = cos(pi (j+12)/8)
          a[q1][r2] = rot(t[q1], c, s);
        }
      }
    }
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
      Dft<4, S, T>::run(a[q1]);
#pragma unroll
      for (int q2 = 0; q2 < 4; ++q2) u[q1 + 4 * q2] = a[q1][q2];
    }
  }
};

// Odd prime R in {5, 7, 11}: with H = (R - 1)/2 and q = 1..H,
//   A_q = u_0 + sum_{r=1}^{H} (u_r + u_{R-r}) cos(2 pi r q / R)
//   B_q =       sum_{r=1}^{H} (u_r - u_{R-r}) sin(2 pi r q / R)
//   U_q = A_q + S i B_q,  U_{R-q} = A_q - S i B_q,  U_0 = sum_r u_r.
template <int R> struct OddRoots;
template <> struct OddRoots<5> {
  static __device__ __forceinline__ double c(int j) {
    const double t[3] = {1.0, 0.309016994374947424102, -0.809016994374947424102};
    return t[j];
  }
  static __device__ __forceinline__ double s(int j) {
    const double t[3] = {0.0, 0.951056516295153572116, 0.587785252292473129169};
    return t[j];
  }
};
template <> struct OddRoots<7> {
  static __device__ __forceinline__ double c(int j) {
    const double t[4] = {1.0, 0.623489801858733530525, -0.222520933956314404289, -0.900968867902419126236};
    return t[j];
  }
  static __device__ __forceinline__ double s(int j) {
    const double t[4] = {0.0, 0.781831482468029808708, 0.974927912181823607018, 0.433883739117558120476};
    return t[j];
  }
};
template <> struct OddRoots<11> {
  static __device__ __forceinline__ double c(int j) {
    const double t[6] = {1.0, 0.841253532831181168862, 0.415415013001886425529, -0.142314838273285140444,
                         -0.654860733945285064057, -0.95949297361449738989};
    return t[j];
  }
  static __device__ __forceinline__ double s(int j) {
    const double t[6] = {0.0, 0.540640817455597582108, 0.909631995354518371412, 0.989821441880932732376,
                         0.755749574354258283774, 0.281732556841429697711};
    return t[j];
  }
};

template <int R, int S, typename T>
struct DftOdd {
  typedef typename CT<T>::V V;
  static __device__ __forceinline__ void run(V* u) {
    constexpr int H = (R - 1) / 2;
    V a[H + 1], b[H + 1];
    V sum = u[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      a[r] = u[r] + u[R - r];
      b[r] = u[r] - u[R - r];
      sum = sum + a[r];
    }
    const V u0 = u[0];
    u[0] = sum;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      V A = u0, B;
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        int j = (r * q) % R;
        const T cs = (T)OddRoots<R>::c(j <= H ? j : R - j);
        const T sn = (T)((j <= H) ? OddRoots<R>::s(j) : -OddRoots<R>::s(R - j));
        A = cfma(cs, a[r], A);
        B = (r == 1) ? sn * b[r] : cfma(sn, b[r], B);
      }
      u[q] = addi<S>(A, B);
      u[R - q] = subi<S>(A, B);
    }
  }
};
template <int S, typename T> struct Dft<5, S, T> : DftOdd<5, S, T> {};
template <int S, typename T> struct Dft<7, S, T> : DftOdd<7, S, T> {};
template <int S, typename T> struct Dft<11, S, T> : DftOdd<11, S, T> {};

// ------------------------------------------------------------ FFT plan
// A line DFT of length M runs as radix stages of length Q.  Q = M when M
// factors into the codelet radices; otherwise Q is the smallest such length
// with Q >= 2M - 1 and the DFT is Bluestein's chirp-z convolution (line_fft).
struct FftPlan {
  int M;      // transform length
  int Q;      // length of the radix-stage transform (M, or Bluestein's padded length)
  int ns;     // number of stages of the length-Q transform
  int R[8];   // radices, first stage first
};

// Factor Q = 2^a 3^b 5^c 7^d 11^e into radices 16, 8, 4, 2, 3, 5, 7, 11 as a
// direct plan of length M = Q; returns false if Q has other factors.
inline bool make_plan(int Q, FftPlan* pl) {
  pl->M = Q;
  pl->Q = Q;
  pl->ns = 0;
  int m = Q;
  const int rad[8] = {16, 8, 4, 2, 3, 5, 7, 11};
  for (int k = 0; k < 8; ++k)
    while (m % rad[k] == 0 && m > 1) {
      if (pl->ns >= 8) return false;
      pl->R[pl->ns++] = rad[k];
      m /= rad[k];
    }
  return m == 1 && Q >= 2;
}

// Plan of a length-M line DFT for any M >= 2: direct when M is smooth, else
// Bluestein with the smallest smooth Q >= 2M - 1.
inline bool make_line_plan(int M, FftPlan* pl) {
  if (M < 2) return false;
  if (make_plan(M, pl)) return true;
  for (int Q = 2 * M - 1; Q <= 8 * M; ++Q)
    if (make_plan(Q, pl)) {
      pl->M = M;
      return true;
    }
  return false;
}

// Entries of a plan's line table: the Q twiddles exp(-2 pi i j / Q), and for a
// Bluestein plan also the chirps and the transformed chirp kernel.
inline int line_table_len(const FftPlan& pl) { return pl.Q == pl.M ? pl.M : 2 * pl.Q + 2 * pl.M; }

// One Stockham stage of radix R over nl lines of length M stored at stride ls.
// Butterfly i of a line reads in[i + r M/R] (r < R), twiddles by
// exp(S 2 pi i r k / (p R)) with k = i mod p, and writes out[(i - k) R + k + r p].
// tw[j] = exp(-2 pi i j / M).  Thread layout: blockDim = (TX, TY).
template <int R, int S, typename T>
__device__ __forceinline__ void stage(const typename CT<T>::V* __restrict__ in, typename CT<T>::V* __restrict__ out,
                                      int M, int p, const typename CT<T>::V* __restrict__ tw, int nl, int ls) {
  typedef typename CT<T>::V V;
  const int nb = M / R;
  const int step = M / (p * R);
  for (int l = threadIdx.y; l < nl; l += blockDim.y) {
    const V* src = in + l * ls;
    V* dst = out + l * ls;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const int k = i % p;
      V u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = src[i + r * nb];
      if (k != 0) {
        const int st = k * step;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          V w = tw[r * st];
          u[r] = (S < 0) ? cmul(u[r], w) : cmulc(u[r], w);
        }
      }
      Dft<R, S, T>::run(u);
      const int j = (i - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[j + r * p] = u[r];
    }
  }
}

// Length-Q transform (the radix stages of the plan) of nl lines held in buffer
// a (stride ls) in place-of-ping-pong with b.  Must be called by every thread
// of the block after the data is in a and synchronised.  Returns the buffer
// that holds the result (synchronised).
template <int S, typename T>
__device__ typename CT<T>::V* tile_fft(typename CT<T>::V* a, typename CT<T>::V* b, const FftPlan& pl,
                                       const typename CT<T>::V* tw, int nl, int ls) {
  int p = 1;
  for (int s = 0; s < pl.ns; ++s) {
    const int R = pl.R[s];
    switch (R) {
      case 16: stage<16, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 8: stage<8, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 4: stage<4, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 2: stage<2, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 3: stage<3, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 5: stage<5, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      case 7: stage<7, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
      default: stage<11, S, T>(a, b, pl.Q, p, tw, nl, ls); break;
    }
    __syncthreads();
    typename CT<T>::V* t = a;
    a = b;
    b = t;
    p *= R;
  }
  return a;
}

__device__ __forceinline__ int flat_tid() { return threadIdx.y * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int flat_nthreads() { return blockDim.x * blockDim.y; }

// Length-M DFT  X_k = sum_{j<M} x_j exp(S 2 pi i j k / M)  of nl lines whose
// first M entries are in buffer a (stride ls >= Q + 1), ping-pong with b (same
// shape); tw holds the Q twiddles of the plan, bt the rest of its line table.
// Same calling rules and result as tile_fft; the entries k >= M of the result
// lines are scratch.
//
// Bluestein's chirp-z identity: with c_j = exp(S pi i j^2 / M), 2 j k = j^2 +
// k^2 - (k - j)^2 gives X_k = c_k sum_j (x_j c_j) conj(c_{k-j}), a linear
// convolution of length 2M - 1 evaluated as a circular one of length Q:
//   a = (x c, 0, ..., 0),  X = c * F+( F-(a) * H ) on k < M,
// where F-/F+ are the unnormalised length-Q transforms of sign -/+ and
// H = F-(conj c placed at j and Q - j for |j| < M) / Q is tabulated.  The
// chirp angles are reduced exactly (j^2 mod 2M) when the table is made.
// Table bt: c for S = -1 (M entries), c for S = +1 (M), H for S = -1 (Q);
// H for S = +1 is its complex conjugate (the chirp kernel is even).
template <int S, typename T>
__device__ typename CT<T>::V* line_fft(typename CT<T>::V* a, typename CT<T>::V* b, const FftPlan& pl,
                                       const typename CT<T>::V* tw, const typename CT<T>::V* __restrict__ bt, int nl,
                                       int ls) {
  typedef typename CT<T>::V V;
  if (pl.Q == pl.M) return tile_fft<S, T>(a, b, pl, tw, nl, ls);
  const int M = pl.M, Q = pl.Q;
  const V* __restrict__ ch = bt + (S < 0 ? 0 : M);
  const V* __restrict__ hh = bt + 2 * M;
  const int tid = flat_tid(), nt = flat_nthreads();
  for (int idx = tid; idx < nl * Q; idx += nt) {
    const int l = idx / Q, j = idx - l * Q;
    V& v = a[l * ls + j];
    v = (j < M) ? cmul(v, ch[j]) : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* r = tile_fft<-1, T>(a, b, pl, tw, nl, ls);
  for (int idx = tid; idx < nl * Q; idx += nt) {
    const int l = idx / Q, k = idx - l * Q;
    V& v = r[l * ls + k];
    v = (S < 0) ? cmul(v, hh[k]) : cmulc(v, hh[k]);
  }
  __syncthreads();
  r = tile_fft<+1, T>(r, (r == a) ? b : a, pl, tw, nl, ls);
  for (int idx = tid; idx < nl * M; idx += nt) {
    const int l = idx / M, k = idx - l * M;
    V& v = r[l * ls + k];
    v = cmul(v, ch[k]);
  }
  __syncthreads();
  return r;
}

}  // namespace vie
