// Set-up kernels of a problem, on the device, to FP64 accuracy (FP64 arithmetic,
// except the kernel-transform cube FFTs, which run in double-word arithmetic on
// the FP32 pipes unless VIE_SETUP_FP64=1):
//  * H_eps = (eps + I)^-1 (eps - I) per node (Eq. (rhodef), Lemma 1), stored as
//    the 6 entries of the symmetric tensor in FP64 and FP32;
//  * the transform of the truncated Green's function (Sec. 5, steps a-b),
//    tabulated once per distinct integer |m|^2 of the oversampled frequency grid;
//  * the discrete kernels of every Fourier symbol (1, i k_a, -k_a k_b) with the
//    grid Nyquist cutoff (Sec. 5, step c), brought to the (2n)^3 convolution
//    grid and stored as octants (the kernels are even or odd in each axis).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>

#include "vie_internal.h"

namespace vie {

// ---------------------------------------------------------------- twiddles
template <typename V>
__global__ void k_twiddle(V* tw, int M) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  double s, c;
  sincospi(2.0 * (double)j / (double)M, &s, &c);
  tw[j].x = c;
  tw[j].y = -s;
}

// exp(-2 pi i num / den) for 0 <= num < den: the quarter turns are taken out
// in integer arithmetic, the rest is an angle in [0, pi/2).
static void exp_m2pi(long long num, long long den, double* c, double* s) {
  const long long q = (4 * num) / den, rem = 4 * num - q * den;
  const double t = M_PI * (double)rem / (2.0 * (double)den);
  const double c0 = std::cos(t), s0 = std::sin(t);
  double cc, ss;  // cos, sin of the full angle
  switch (q & 3) {
    case 0: cc = c0; ss = s0; break;
    case 1: cc = -s0; ss = c0; break;
    case 2: cc = -c0; ss = -s0; break;
    default: cc = s0; ss = -c0; break;
  }
  *c = cc;
  *s = -ss;
}

// Line table of a plan (line_table_len entries, layout of line_fft): the Q
// twiddles exp(-2 pi i j / Q) on the device; for a Bluestein plan then the
// chirps c-_j = exp(-pi i j^2 / M) and c+_j = conj(c-_j) with j^2 reduced mod
// 2M, and H-_k = (1/Q) sum_{|j|<M} c+_j exp(-2 pi i j k / Q)
//             = (1/Q) (1 + 2 sum_{0<j<M} c+_j cos(2 pi j k / Q)),
// all in FP64 on the host.
vie_status make_line_table(const FftPlan& pl, double2** t64, float2** t32, cudaStream_t st) {
  const int M = pl.M, Q = pl.Q, len = line_table_len(pl);
  VIE_CK(dalloc((void**)t64, sizeof(double2) * len, st));
  VIE_CK(dalloc((void**)t32, sizeof(float2) * len, st));
  k_twiddle<double2><<<(Q + 127) / 128, 128, 0, st>>>(*t64, Q);
  k_twiddle<float2><<<(Q + 127) / 128, 128, 0, st>>>(*t32, Q);
  VIE_CK(cudaGetLastError());
  if (Q == M) return VIE_OK;
  std::vector<double2> h(len - Q);
  std::vector<float2> h32(len - Q);
  for (int j = 0; j < M; ++j) {
    double c, sn;
    exp_m2pi(((long long)j * j) % (2LL * M), 2LL * M, &c, &sn);
    h[j] = make_double2(c, sn);
    h[M + j] = make_double2(c, -sn);
  }
  std::vector<double> cq(Q);
  for (int t = 0; t < Q; ++t) {
    double c, sn;
    exp_m2pi(t, Q, &c, &sn);
    cq[t] = c;
  }
  for (int k = 0; k < Q; ++k) {
    double re = 0.0, im = 0.0;
    int jk = 0;  // j k mod Q
    for (int j = 1; j < M; ++j) {
      jk += k;
      if (jk >= Q) jk -= Q;
      re += h[M + j].x * cq[jk];
      im += h[M + j].y * cq[jk];
    }
    h[2 * M + k] = make_double2((1.0 + 2.0 * re) / Q, 2.0 * im / Q);
  }
  for (size_t i = 0; i < h.size(); ++i) h32[i] = make_float2((float)h[i].x, (float)h[i].y);
  VIE_CK(cudaMemcpyAsync(*t64 + Q, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st));
  VIE_CK(cudaMemcpyAsync(*t32 + Q, h32.data(), sizeof(float2) * h32.size(), cudaMemcpyHostToDevice, st));
  VIE_CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  return VIE_OK;
}

// ------------------------------------------------------------ medium tensor
// H = (A)^-1 (eps - I) = I - 2 A^-1 with A = eps + I, via the adjugate.
__global__ void k_medium(const double2* __restrict__ eps, double2* __restrict__ H64, float2* __restrict__ H32,
                         long long N, int realonly, int* flag) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    double2 a[3][3];
    double mag = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double2 v = eps[(i * 3 + j) * N + p];
        if (realonly) v.y = 0.0;
        a[i][j] = v;
        mag = fmax(mag, fabs(v.x) + fabs(v.y));
      }
    const double tol = 1e-12 * (1.0 + mag);
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (fabs(a[i][j].x - a[j][i].x) + fabs(a[i][j].y - a[j][i].y) > tol) atomicOr(flag, 1);
    for (int i = 0; i < 3; ++i) a[i][i].x += 1.0;
    double2 adj[3][3];
    adj[0][0] = cmul(a[1][1], a[2][2]) - cmul(a[1][2], a[2][1]);
    adj[0][1] = cmul(a[0][2], a[2][1]) - cmul(a[0][1], a[2][2]);
    adj[0][2] = cmul(a[0][1], a[1][2]) - cmul(a[0][2], a[1][1]);
    adj[1][0] = cmul(a[1][2], a[2][0]) - cmul(a[1][0], a[2][2]);
    adj[1][1] = cmul(a[0][0], a[2][2]) - cmul(a[0][2], a[2][0]);
    adj[1][2] = cmul(a[0][2], a[1][0]) - cmul(a[0][0], a[1][2]);
    adj[2][0] = cmul(a[1][0], a[2][1]) - cmul(a[1][1], a[2][0]);
    adj[2][1] = cmul(a[0][1], a[2][0]) - cmul(a[0][0], a[2][1]);
    adj[2][2] = cmul(a[0][0], a[1][1]) - cmul(a[0][1], a[1][0]);
    double2 det = cmul(a[0][0], adj[0][0]) + cmul(a[0][1], adj[1][0]) + cmul(a[0][2], adj[2][0]);
    const double dd = det.x * det.x + det.y * det.y;
    if (!(dd > 0.0) || !isfinite(dd)) {
      atomicOr(flag, 2);
      continue;
    }
    // 1/det = conj(det)/|det|^2
    const double2 inv = make_double2(det.x / dd, -det.y / dd);
    const int ii[6] = {0, 1, 2, 0, 0, 1};
    const int jj[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
      double2 q = cmul(adj[ii[e]][jj[e]], inv);
      double2 h = make_double2(-2.0 * q.x, -2.0 * q.y);
      if (ii[e] == jj[e]) h.x += 1.0;
      H64[e * N + p] = h;
      H32[e * N + p] = make_float2((float)h.x, (float)h.y);
    }
  }
}

vie_status build_medium(vie_problem* P, const void* eps, const void* mu, cudaStream_t st) {
  const long long N = (long long)P->n * P->n * P->n;
  VIE_CK(dalloc((void**)&P->He64, sizeof(double2) * 6 * N, st));
  VIE_CK(dalloc((void**)&P->He32, sizeof(float2) * 6 * N, st));
  VIE_CK(cudaMemsetAsync(P->dflag, 0, sizeof(int), st));
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
  k_medium<<<blocks, 256, 0, st>>>((const double2*)eps, P->He64, P->He32, N, P->kind == VIE_LAPLACE, P->dflag);
  VIE_CK(cudaGetLastError());
  if (P->has_mu) {
    VIE_CK(dalloc((void**)&P->Hm64, sizeof(double2) * 6 * N, st));
    VIE_CK(dalloc((void**)&P->Hm32, sizeof(float2) * 6 * N, st));
    k_medium<<<blocks, 256, 0, st>>>((const double2*)mu, P->Hm64, P->Hm32, N, 0, P->dflag);
    VIE_CK(cudaGetLastError());
  }
  int flag = 0;
  VIE_CK(cudaMemcpyAsync(&flag, P->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  if (flag & 1) {
    set_error("eps/mu must be symmetric at every node");
    return VIE_EINVAL;
  }
  if (flag & 2) {
    set_error("eps + I (or mu + I) is singular or non-finite at some node");
    return VIE_EINVAL;
  }
  return VIE_OK;
}

// ------------------------------------------------ truncated kernel transform
// G^_L(kappa) = (1/kappa) int_0^L sin(kappa r) e^{i w r} dr (Sec. 5, steps a-b),
// evaluated as [E(w + kappa) - E(w - kappa)] / (2 i kappa) with
// E(a) = int_0^L e^{i a r} dr = L e^{i a L/2} sinc(a L/2): no cancellation at
// kappa = w.  kappa = 0: int_0^L r e^{i w r} dr, closed form for wL >= 1/2,
// power series sum_q (i w L)^q L^2 / (q! (q + 2)) below.  On the grids used
// here every other kappa has kappa L >= 2 pi sqrt(3)/3, far from the
// cancellation of the E difference at small kappa L.
__device__ double2 dev_E(double a, double L) {
  const double t = 0.5 * a * L;
  const double sc = (t == 0.0) ? 1.0 : sin(t) / t;
  double s, c;
  sincos(t, &s, &c);
  return make_double2(L * c * sc, L * s * sc);
}

__device__ double2 dev_ghat(double kappa, double w, double L) {
  if (kappa == 0.0) {
    const double wl = w * L;
    if (fabs(wl) < 0.5) {
      double2 acc = make_double2(0.0, 0.0);
      double2 term = make_double2(1.0, 0.0);  // (i w L)^q / q!
      for (int q = 0; q < 40; ++q) {
        const double f = L * L / (double)(q + 2);
        acc = acc + f * term;
        term = cmul(term, make_double2(0.0, wl / (double)(q + 1)));
      }
      return acc;
    }
    double s, c;
    sincos(wl, &s, &c);
    return make_double2((c + s * wl - 1.0) / (w * w), (s - c * wl) / (w * w));
  }
  const double2 d = dev_E(w + kappa, L) - dev_E(w - kappa, L);
  return make_double2(d.y / (2.0 * kappa), -d.x / (2.0 * kappa));
}

__global__ void k_ghat_table(double2* tab, int jmax, double dk, double w, double L) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > jmax) return;
  tab[j] = dev_ghat(dk * sqrt((double)j), w, L);
}

// F(m) = S~(k_m) G^(|k_m|) on the (sn)^3 grid in FFT order.  Even sn: m in
// [-sn/2, sn/2), and on an axis with m_a = -sn/2 (Nyquist) an odd factor k_a is
// replaced by 0 (the mean of its values at -pi/h and +pi/h), an even factor k_a^2
// is kept.  Odd sn (odd n): m in [-(sn-1)/2, (sn-1)/2], no Nyquist entry.  Either
// way |m_a| <= sn/2 (integer division), so m.m <= 3 (sn/2)^2, the table's length.
__global__ void k_build_F(double2* __restrict__ F, const double2* __restrict__ tab, int sn, int sym, double dk) {
  const long long tot = (long long)sn * sn * sn;
  const int hp = (sn + 1) / 2;                // first index of a negative m
  const int nyq = (sn % 2 == 0) ? sn / 2 : -1;  // index of m = -sn/2, if any
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % sn);
    const int iy = (int)((idx / sn) % sn);
    const int iz = (int)(idx / ((long long)sn * sn));
    const int mx = ix < hp ? ix : ix - sn, my = iy < hp ? iy : iy - sn, mz = iz < hp ? iz : iz - sn;
    const long long j = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
    const double2 G = tab[j];
    const double kx = dk * mx, ky = dk * my, kz = dk * mz;
    const double ox = (ix == nyq) ? 0.0 : kx, oy = (iy == nyq) ? 0.0 : ky, oz = (iz == nyq) ? 0.0 : kz;
    double2 v;
    switch (sym) {
      case SYM_1: v = G; break;
      case SYM_DX: v = make_double2(-ox * G.y, ox * G.x); break;
      case SYM_DY: v = make_double2(-oy * G.y, oy * G.x); break;
      case SYM_DZ: v = make_double2(-oz * G.y, oz * G.x); break;
      case SYM_XX: v = (-kx * kx) * G; break;
      case SYM_YY: v = (-ky * ky) * G; break;
      case SYM_ZZ: v = (-kz * kz) * G; break;
      case SYM_XY: v = (-ox * oy) * G; break;
      case SYM_XZ: v = (-ox * oz) * G; break;
      default: v = (-oy * oz) * G; break;
    }
    F[idx] = v;
  }
}

// Generic in-place FFT of a cubic M^3 FP64 array along one axis (0 x, 1 y, 2 z).
template <int S, typename T>
__global__ void k_fft_cube(double2* __restrict__ data, int M, int axis, FftPlan pl,
                           const typename CT<T>::V* __restrict__ twg, int nl) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Q = pl.Q, LS = Q + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + Q;
  V* b1 = b0 + nl * LS;
  const int tid = flat_tid(), nt = flat_nthreads();
  for (int j = tid; j < Q; j += nt) tw[j] = twg[j];
  const long long MM = (long long)M * M;
  // address of element j of tile line l
  auto addr = [&](int l, int j) -> long long {
    if (axis == 0) return ((long long)blockIdx.x * nl + l) * M + j;
    if (axis == 1) return (long long)blockIdx.y * MM + (long long)j * M + (long long)blockIdx.x * nl + l;
    return (long long)j * MM + (long long)blockIdx.y * M + (long long)blockIdx.x * nl + l;
  };
  for (int idx = tid; idx < nl * M; idx += nt) {
    int l, j;
    if (axis == 0) { l = idx / M; j = idx - l * M; } else { j = idx / nl; l = idx - j * nl; }
    b0[l * LS + j] = to_v<T>(data[addr(l, j)]);
  }
  __syncthreads();
  V* r = line_fft<S, T>(b0, b1, pl, tw, twg + Q, nl, LS);
  for (int idx = tid; idx < nl * M; idx += nt) {
    int l, j;
    if (axis == 0) { l = idx / M; j = idx - l * M; } else { j = idx / nl; l = idx - j * nl; }
    data[addr(l, j)] = from_v<T>(r[l * LS + j]);
  }
}

// Lines per tile: a power of two dividing M, with the tile within 200 KB.
static int pick_nl(const FftPlan& pl, size_t vs) {
  int nl = 8;
  while (nl > 1 && (pl.M % nl != 0 || vs * (pl.Q + 2 * (size_t)nl * (pl.Q + 1)) > 200 * 1024)) nl >>= 1;
  return nl;
}

// In-place 3D DFT of an FP64 cube, lines along each axis in turn; arithmetic in
// T (FP64, or double-word on the FP32 pipes), one block row per tile line.
template <int S, typename T>
static vie_status fft_cube(double2* data, int M, const FftPlan& pl, const typename CT<T>::V* tw, cudaStream_t st) {
  const size_t vs = sizeof(typename CT<T>::V);
  const int nl = pick_nl(pl, vs);
  const size_t smem = vs * (pl.Q + 2 * nl * (pl.Q + 1));
  if (smem > (size_t)smem_optin_bytes()) {
    set_error("set-up transform line too long for shared memory");
    return VIE_EINVAL;
  }
  VIE_CK(allow_smem(k_fft_cube<S, T>));
  // threads per line: M/16 up to 32 for direct plans; a long Bluestein line
  // (one to four per tile) one per 16 elements of Q, up to 128, and at most
  // 256 threads per block
  int tx = std::max(1, std::min(32, M / 16));
  if (pl.Q != pl.M) {
    tx = 32;
    while (tx * 16 < pl.Q && tx < 128 && 2 * tx * nl <= 256) tx <<= 1;
  }
  const dim3 blk(tx, nl);
  for (int axis = 0; axis < 3; ++axis) {
    dim3 grid = axis == 0 ? dim3((unsigned)((long long)M * M / nl), 1) : dim3(M / nl, M);
    k_fft_cube<S, T><<<grid, blk, smem, st>>>(data, M, axis, pl, tw, nl);
    VIE_CK(cudaGetLastError());
  }
  return VIE_OK;
}

// e[M^3] (M = 2 nk >= 2n) from the inverse-transformed F[(sn)^3]: offsets d in
// [-(n-1), n-1] at index d mod M, indices n..M-n left zero; scale folds the
// 1/(sn)^3 of the inverse DFT.
__global__ void k_embed(const double2* __restrict__ F, double2* __restrict__ e, int n, int nk, int sn, double scale) {
  const int M = 2 * nk;
  const long long tot = (long long)M * M * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(idx % M), ey = (int)((idx / M) % M), ez = (int)(idx / ((long long)M * M));
    if ((ex >= n && ex <= M - n) || (ey >= n && ey <= M - n) || (ez >= n && ez <= M - n)) {
      e[idx] = make_double2(0.0, 0.0);
      continue;
    }
    const int sx = ex < n ? ex : ex - M + sn;
    const int sy = ey < n ? ey : ey - M + sn;
    const int sz = ez < n ? ez : ez - M + sn;
    e[idx] = scale * F[((long long)sz * sn + sy) * sn + sx];
  }
}

__global__ void k_octant(const double2* __restrict__ E, double2* __restrict__ oct, int nk) {
  const int M = 2 * nk, O = nk + 1;
  const long long tot = (long long)O * O * O;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ox = (int)(idx % O), oy = (int)((idx / O) % O), oz = (int)(idx / ((long long)O * O));
    oct[idx] = E[((long long)oz * M + oy) * M + ox];
  }
}

// Combine raw symbol octants into the kernel arrays of one pass.
//   coef layout per output array a: up to 2 terms (sym index, complex factor).
struct CombineDesc {
  int narr;
  int sym[9][2];
  double2 fac[9][2];
};

__global__ void k_combine(const double2* __restrict__ sym_oct, double2* __restrict__ out64, float2* __restrict__ out32,
                          long long O3, CombineDesc cd, double diag_add_scale, int diag_mask) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < O3;
       idx += (long long)gridDim.x * blockDim.x) {
    for (int a = 0; a < cd.narr; ++a) {
      double2 v = make_double2(0.0, 0.0);
      for (int t = 0; t < 2; ++t) {
        const int s = cd.sym[a][t];
        if (s < 0) continue;
        v = v + cmul(cd.fac[a][t], sym_oct[(long long)s * O3 + idx]);
      }
      if (diag_mask & (1 << a)) v.x += diag_add_scale;
      out64[a * O3 + idx] = v;
      out32[a * O3 + idx] = make_float2((float)v.x, (float)v.y);
    }
  }
}

static vie_status combine(vie_problem* P, KernelSet& K, int mode, const CombineDesc& cd, double diag_add,
                          int diag_mask, cudaStream_t st) {
  const long long O = P->nk + 1, O3 = O * O * O;
  K.mode = mode;
  K.narr = cd.narr;
  VIE_CK(dalloc((void**)&K.oct64, sizeof(double2) * cd.narr * O3, st));
  VIE_CK(dalloc((void**)&K.oct32, sizeof(float2) * cd.narr * O3, st));
  const int blocks = (int)std::min<long long>((O3 + 255) / 256, 152LL * 16);
  k_combine<<<blocks, 256, 0, st>>>(P->sym_oct, K.oct64, K.oct32, O3, cd, diag_add, diag_mask);
  VIE_CK(cudaGetLastError());
  return VIE_OK;
}

// Compute the raw octant kernels of the symbols in `mask` (bit = Sym) that are
// not computed yet.
static vie_status to_df(const double2* src, cdf** dst, long long count, cudaStream_t st);

static vie_status compute_symbols(vie_problem* P, unsigned mask, cudaStream_t st) {
  mask &= ~P->sym_mask;
  if (!mask) return VIE_OK;
  const int n = P->n, sn = 3 * n, M = 2 * P->nk;
  const double dk = 2.0 * M_PI / (3.0 * P->D);
  const int jmax = 3 * (sn / 2) * (sn / 2);
  const double w = P->kind == VIE_LAPLACE ? 0.0 : P->omega;
  double2* tab = nullptr;
  double2 *F = nullptr, *E = nullptr, *tw_sn = nullptr;
  float2* tw_sn32 = nullptr;
  FftPlan plsn;
  if (!make_line_plan(sn, &plsn)) {
    set_error("bad oversampled grid size");
    return VIE_EINVAL;
  }
  const long long O = P->nk + 1;
  const long long S3 = (long long)sn * sn * sn, M3 = (long long)M * M * M, O3 = O * O * O;
  if (!P->sym_oct) VIE_CK(dalloc((void**)&P->sym_oct, sizeof(double2) * SYM_COUNT * O3, st));
  VIE_CK(dalloc((void**)&tab, sizeof(double2) * (jmax + 1), st));
  k_ghat_table<<<(jmax + 256) / 256, 256, 0, st>>>(tab, jmax, dk, w, P->L);
  VIE_CK(cudaGetLastError());
  VIE_CK(dalloc((void**)&F, sizeof(double2) * S3, st));
  VIE_CK(dalloc((void**)&E, sizeof(double2) * M3, st));
  vie_status s = make_line_table(plsn, &tw_sn, &tw_sn32, st);
  if (s != VIE_OK) return s;
  // the kernel-transform FFTs run in double-word arithmetic (FP64 accuracy on
  // the FP32 pipes); VIE_SETUP_FP64=1 keeps them in native FP64
  const char* e64 = getenv("VIE_SETUP_FP64");
  const bool dw = !(e64 && e64[0] == '1');
  cdf *tw_sndf = nullptr, *tw_2ndf = nullptr;
  if (dw) {
    s = to_df(tw_sn, &tw_sndf, line_table_len(plsn), st);
    if (s == VIE_OK) s = to_df(P->tw64, &tw_2ndf, line_table_len(P->planM), st);
    if (s != VIE_OK) return s;
  }
  const int gb = 152 * 16;
  for (int sym = 0; sym < SYM_COUNT; ++sym) {
    if (!(mask & (1u << sym))) continue;
    k_build_F<<<gb, 256, 0, st>>>(F, tab, sn, sym, dk);
    VIE_CK(cudaGetLastError());
    s = dw ? fft_cube<+1, df>(F, sn, plsn, tw_sndf, st) : fft_cube<+1, double>(F, sn, plsn, tw_sn, st);
    if (s != VIE_OK) return s;
    k_embed<<<gb, 256, 0, st>>>(F, E, n, P->nk, sn, 1.0 / (double)S3);
    VIE_CK(cudaGetLastError());
    s = dw ? fft_cube<-1, df>(E, M, P->planM, tw_2ndf, st) : fft_cube<-1, double>(E, M, P->planM, P->tw64, st);
    if (s != VIE_OK) return s;
    k_octant<<<gb, 256, 0, st>>>(E, P->sym_oct + (long long)sym * O3, P->nk);
    VIE_CK(cudaGetLastError());
  }
  dfree(F, st);
  dfree(E, st);
  dfree(tab, st);
  dfree(tw_sn, st);
  dfree(tw_sn32, st);
  dfree(tw_sndf, st);
  dfree(tw_2ndf, st);
  P->sym_mask |= mask;
  return VIE_OK;
}

static const unsigned kQmask = (1u << SYM_XX) | (1u << SYM_YY) | (1u << SYM_ZZ) | (1u << SYM_XY) | (1u << SYM_XZ) |
                               (1u << SYM_YZ);
static const unsigned kDmask = (1u << SYM_DX) | (1u << SYM_DY) | (1u << SYM_DZ);

// Kernel sets: `which` 0 = operator apply, 1 = scattered field.
static vie_status combine_sets(vie_problem* P, int which, cudaStream_t st);

// ------------------------------------------------ operator norm bound
__device__ __forceinline__ double dnorm2c(double2 a) { return a.x * a.x + a.y * a.y; }

// max over points of the Frobenius norm of a symmetric 3x3 tensor field stored
// as 6 arrays (xx yy zz xy xz yz) of stride S, with 3 more arrays (a curl
// symbol p: the 6x6 Maxwell kernel [[Q, p x], [-p x, Q]]) when np == 3, into
// *out as the bit pattern of a non-negative double (ordered like the double).
__global__ void k_fro_max(const double2* __restrict__ a, long long S, int np, unsigned long long* out) {
  double mx = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
    double f = 0.0;
    for (int e = 0; e < 6; ++e) f += (e < 3 ? 1.0 : 2.0) * dnorm2c(a[e * S + i]);
    if (np == 3) {
      double p = 0.0;
      for (int e = 6; e < 9; ++e) p += dnorm2c(a[e * S + i]);
      f = 2.0 * f + 4.0 * p;
    }
    mx = fmax(mx, f);
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sqrt(mx)));
}

// Upper bound of ||A||_2 = ||I + H conv||_2 <= 1 + max ||H||_F max_k ||K^(k)||_F with
// the kernel's eigenvalues M^3 K_stored (the 1/M^3 of the inverse DFT is folded
// into the stored octants).  Used to bound the error of an FP32 apply.
static vie_status op_norm_bound(vie_problem* P, cudaStream_t st) {
  unsigned long long* d = nullptr;
  VIE_CK(dalloc((void**)&d, 3 * sizeof(unsigned long long), st));
  VIE_CK(cudaMemsetAsync(d, 0, 3 * sizeof(unsigned long long), st));
  const long long O = P->nk + 1, O3 = O * O * O, N = (long long)P->n * P->n * P->n;
  const int np = P->kapply.mode == KM_MAXWELL6 ? 3 : 0;
  k_fro_max<<<152 * 4, 256, 0, st>>>(P->kapply.oct64, O3, np, d);
  k_fro_max<<<152 * 4, 256, 0, st>>>(P->He64, N, 0, d + 1);
  if (P->Hm64) k_fro_max<<<152 * 4, 256, 0, st>>>(P->Hm64, N, 0, d + 2);
  VIE_CK(cudaGetLastError());
  unsigned long long h[3];
  VIE_CK(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
  VIE_CK(cudaStreamSynchronize(st));
  dfree(d, st);
  double v[3];
  for (int i = 0; i < 3; ++i) memcpy(&v[i], &h[i], sizeof(double));
  const double M = 2.0 * P->nk;
  P->opnorm = 1.0 + std::max(v[1], v[2]) * v[0] * M * M * M;
  return VIE_OK;
}

vie_status build_kernels(vie_problem* P, cudaStream_t st) {
  // the operator needs -k_a k_b (and, for Maxwell, 1; with mu also the curl
  // symbols i k_a); the symbols only the scattered field needs are built on
  // its first use
  unsigned mask = kQmask;
  if (P->kind == VIE_MAXWELL) mask |= (1u << SYM_1) | (P->has_mu ? kDmask : 0u);
  vie_status s = compute_symbols(P, mask, st);
  if (s != VIE_OK) return s;
  s = combine_sets(P, 0, st);
  if (s != VIE_OK) return s;
  return op_norm_bound(P, st);
}

vie_status build_eval_kernels(vie_problem* P, cudaStream_t st) {
  if (P->keval.oct64) return VIE_OK;
  const unsigned mask = P->kind == VIE_MAXWELL ? (kQmask | kDmask | (1u << SYM_1)) : kDmask;
  vie_status s = compute_symbols(P, mask, st);
  if (s != VIE_OK) return s;
  return combine_sets(P, 1, st);
}

static vie_status combine_sets(vie_problem* P, int which, cudaStream_t st) {
  const int M = 2 * P->nk;
  const long long M3 = (long long)M * M * M;
  const double w = P->kind == VIE_LAPLACE ? 0.0 : P->omega;
  vie_status s = VIE_OK;
  // Fold constants: apply kernels give u with y = x + H u; the 1/(2n)^3 of the
  // inverse DFT is folded in too.
  const double nrm = 1.0 / (double)M3;
  const int Q[6] = {SYM_XX, SYM_YY, SYM_ZZ, SYM_XY, SYM_XZ, SYM_YZ};
  const int Dd[3] = {SYM_DX, SYM_DY, SYM_DZ};
  CombineDesc ca{}, ce{};
  for (int a = 0; a < 9; ++a)
    for (int t = 0; t < 2; ++t) {
      ca.sym[a][t] = -1;
      ce.sym[a][t] = -1;
      ca.fac[a][t] = make_double2(0, 0);
      ce.fac[a][t] = make_double2(0, 0);
    }
  const double w2 = w * w;
  if (P->kind == VIE_LAPLACE || P->kind == VIE_HELMHOLTZ) {
    // Laplace  (Eq. (eq:intLap)):  u = -2 T_0 x  (y = x + H_eps u)
    // Helmholtz (Eq. (eq:intH), H_{eps^-1} = -H_eps): u = +2 T_w x
    const double sg = P->kind == VIE_LAPLACE ? -2.0 : 2.0;
    ca.narr = 6;
    for (int a = 0; a < 6; ++a) {
      ca.sym[a][0] = Q[a];
      ca.fac[a][0] = make_double2(sg * nrm, 0);
    }
    if (which == 0) {
      s = combine(P, P->kapply, KM_SYM3, ca, sg * 0.5 * nrm, 0x7, st);
      if (s != VIE_OK) return s;
    }
    // phi_sc = div V J
    ce.narr = 3;
    for (int a = 0; a < 3; ++a) {
      ce.sym[a][0] = Dd[a];
      ce.fac[a][0] = make_double2(nrm, 0);
    }
    if (which == 1) {
      s = combine(P, P->keval, KM_DIV, ce, 0.0, 0, st);
      if (s != VIE_OK) return s;
    }
  } else {
    // Maxwell (Eq. (eq:intM)): u_J = Q' J + P' x M, u_M = Q' M - P' x J with
    // Q' = -2 (K + I/2 + w^2 V), P'_a = -2 i w K_{i k_a}.
    ca.narr = P->has_mu ? 9 : 6;
    for (int a = 0; a < 6; ++a) {
      ca.sym[a][0] = Q[a];
      ca.fac[a][0] = make_double2(-2.0 * nrm, 0);
      if (a < 3) {
        ca.sym[a][1] = SYM_1;
        ca.fac[a][1] = make_double2(-2.0 * w2 * nrm, 0);
      }
    }
    for (int a = 0; a < 3; ++a) {
      ca.sym[6 + a][0] = Dd[a];
      ca.fac[6 + a][0] = make_double2(0, -2.0 * w * nrm);
    }
    if (which == 0) {
      s = combine(P, P->kapply, P->has_mu ? KM_MAXWELL6 : KM_SYM3, ca, -nrm, 0x7, st);
      if (s != VIE_OK) return s;
    }
    // E_sc = Q'' J + P'' x M, H_sc = Q'' M - P'' x J; Q'' = K + w^2 V, P''_a = i w K_{i k_a}
    ce.narr = 9;
    for (int a = 0; a < 6; ++a) {
      ce.sym[a][0] = Q[a];
      ce.fac[a][0] = make_double2(nrm, 0);
      if (a < 3) {
        ce.sym[a][1] = SYM_1;
        ce.fac[a][1] = make_double2(w2 * nrm, 0);
      }
    }
    for (int a = 0; a < 3; ++a) {
      ce.sym[6 + a][0] = Dd[a];
      ce.fac[6 + a][0] = make_double2(0, w * nrm);
    }
    if (which == 1) {
      s = combine(P, P->keval, P->has_mu ? KM_MAXWELL6 : KM_EMRED, ce, 0.0, 0, st);
      if (s != VIE_OK) return s;
    }
  }
  VIE_CK(cudaStreamSynchronize(st));
  return VIE_OK;
}

// ------------------------------------------------------------ double-word copies
// v -> (hi, lo) with hi = fl32(v), lo = fl32(v - hi): the double-word value
// equals v to about 2^-48 relative.
__global__ void k_to_df(const double2* __restrict__ src, cdf* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = CT<df>::make(df(v.x), df(v.y));
  }
}

static vie_status to_df(const double2* src, cdf** dst, long long count, cudaStream_t st) {
  VIE_CK(dalloc((void**)dst, sizeof(cdf) * (size_t)count, st));
  const long long blocks = std::min<long long>((count + 255) / 256, 4096);
  k_to_df<<<(unsigned)blocks, 256, 0, st>>>(src, *dst, count);
  VIE_CK(cudaGetLastError());
  return VIE_OK;
}

vie_status build_df(vie_problem* P, cudaStream_t st) {
  if (P->kapply.octdf) return VIE_OK;
  const long long N = (long long)P->n * P->n * P->n;
  const long long O3 = (long long)(P->nk + 1) * (P->nk + 1) * (P->nk + 1);
  vie_status s = VIE_OK;
  if (!P->twdf) s = to_df(P->tw64, &P->twdf, line_table_len(P->planM), st);
  if (s == VIE_OK && !P->Hedf) s = to_df(P->He64, &P->Hedf, 6 * N, st);
  if (s == VIE_OK && P->Hm64 && !P->Hmdf) s = to_df(P->Hm64, &P->Hmdf, 6 * N, st);
  if (s == VIE_OK) s = to_df(P->kapply.oct64, &P->kapply.octdf, (long long)P->kapply.narr * O3, st);
  return s;
}

}  // namespace vie
