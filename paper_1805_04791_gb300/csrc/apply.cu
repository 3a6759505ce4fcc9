// The operator apply (I + B + K) x of Eqs. (eq:intLap), (eq:intH), (eq:intM),
// and the scattered-field evaluation, as a pruned zero-padded 3D convolution
// (Sec. 5: the truncated kernel transform applied with the FFT).
//
// The convolution grid has M = 2 nk points per axis: nk = n when 2n factors
// into the codelet radices 2, 3, 5, 7, 11, else the smallest such nk > n (a
// circular convolution of length M >= 2n - 1 equals the zero-padded linear one
// on the n^3 output nodes; n = 326, 2n = 4 x 163, runs on M = 660).
// Five passes over HBM.  For M = 2n in {64, 96, 128, 192, 256, 384, 512} they
// are the register-resident kernels of apply_fast.cuh (chosen here, with the
// z-pass autotuner); every other grid, and the double-word passes without a
// fast kernel, run the shared-memory Stockham kernels of this file
// (vie_fft.cuh):
//   P1  x-lines: zero-pad n -> M, forward FFT           x [c][n][n][n]    -> A [c][n][n][M]
//   P2  y-lines: zero-pad, forward FFT                   A                 -> B [c][n][M][M]
//   P3  z-pencils of all components: zero-pad, forward FFT, per-k kernel
//       mixing (3x3 symmetric, 6x6 Maxwell, divergence or E/H), inverse
//       FFT, keep z < n                                  B                 -> B (in place)
//   P4  y-lines: inverse FFT, keep y < n                 B                 -> A
//   P5  x-lines of all components: inverse FFT, keep x < n, epilogue
//       y = x + H u (u the convolution; H per node, 3x3 symmetric)  A      -> y
// The padded z-planes z >= n are never stored (their input is zero and their
// output is discarded).  The kernel arrays are octants (nk + 1)^3 of the M^3
// DFT with the identity part of T, the sign and factor 2 of B, and the 1/M^3
// of the inverse DFT folded in.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "apply_fast.cuh"

namespace vie {
// Generic kernels (any line plan): shared-memory Stockham passes with the
// twiddle table staged in shared memory (line_fft, vie_fft.cuh; the apply's
// plans are direct, Bluestein's algorithm is taken by the set-up's 3n lines).
// Tile lines have the plan's inner length Q (= M for a direct plan) plus one.
// ---------------------------------------------------------------- P1
template <typename T>
__global__ void k_p1(const typename IOT<T>::E* __restrict__ x, typename CT<T>::V* __restrict__ A, int n, FftPlan pl,
                     const typename CT<T>::V* __restrict__ twg, int nl, int C) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, Q = pl.Q, LS = Q + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + Q;
  V* b1 = b0 + nl * LS;
  load_tw(tw, twg, Q);
  const long long N = (long long)n * n * n;
  const int c = blockIdx.y, b = blockIdx.z, nc = gridDim.y;
  const typename IOT<T>::E* src = x + ((long long)b * nc + c) * N;
  V* dst = A + ((long long)b * C + c) * ((long long)n * n * M);
  const int r0 = blockIdx.x * nl;
  const int rows = n * n;
  for (int l = threadIdx.y; l < nl; l += blockDim.y) {
    const int r = r0 + l;
    for (int j = threadIdx.x; j < M; j += blockDim.x)
      b0[l * LS + j] = (j < n && r < rows) ? to_v<T>(src[(long long)r * n + j]) : CT<T>::make(0, 0);
  }
  __syncthreads();
  V* res = line_fft<-1, T>(b0, b1, pl, tw, twg + Q, nl, LS);
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
  const int M = pl.M, Q = pl.Q, LS = Q + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + Q;
  V* b1 = b0 + nl * LS;
  load_tw(tw, twg, Q);
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
  V* res = line_fft<S, T>(b0, b1, pl, tw, twg + Q, nl, LS);
  for (int idx = tid; idx < nl * nout; idx += nt) {
    const int j = idx / nl, l = idx - j * nl;
    dst[(long long)j * M + kx0 + l] = res[l * LS + j];
  }
}

// ---------------------------------------------------------------- P3
// Kernel value at (kz, ky, kx) of the M = 2 nk grid from its octant (nk + 1)^3.
template <typename V>
__device__ __forceinline__ V kval(const V* __restrict__ K, int a, long long O3, int O, int par, int kz, int ky,
                                  int kx, int nk) {
  const int M = 2 * nk;
  int sgn = 1;
  int oz = kz, oy = ky, ox = kx;
  if (kz > nk) { oz = M - kz; if (par & 4) sgn = -sgn; }
  if (ky > nk) { oy = M - ky; if (par & 2) sgn = -sgn; }
  if (kx > nk) { ox = M - kx; if (par & 1) sgn = -sgn; }
  V v = K[a * O3 + ((long long)oz * O + oy) * O + ox];
  return (sgn < 0) ? vneg(v) : v;
}

template <typename T>
__global__ void k_p3(typename CT<T>::V* __restrict__ B, int n, FftPlan pl, const typename CT<T>::V* __restrict__ twg,
                     int nl, int C, const typename CT<T>::V* __restrict__ K, int mode) {
  const int nk = pl.M / 2;  // kernel half-size: the octants are (nk + 1)^3
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, Q = pl.Q, LS = Q + 1;
  const int cin = (mode == KM_MAXWELL6) ? 6 : 3;
  const int cout = (mode == KM_SYM3) ? 3 : (mode == KM_DIV ? 1 : 6);
  const int cmax = cin > cout ? cin : cout;
  V* tw = (V*)smraw;
  V* b0 = tw + Q;
  V* b1 = b0 + cmax * nl * LS;
  load_tw(tw, twg, Q);
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
  V* fw = line_fft<-1, T>(b0, b1, pl, tw, twg + Q, cin * nl, LS);
  V* ob = (fw == b0) ? b1 : b0;
  // per-k mixing
  const int O = nk + 1;
  const long long O3 = (long long)O * O * O;
  for (int idx = tid; idx < nl * M; idx += nt) {
    const int l = idx % nl, kz = idx / nl;
    const int kx = kx0 + l;
    V u[6];
    for (int c = 0; c < cin; ++c) u[c] = fw[(c * nl + l) * LS + kz];
    V o[6];
    if (mode == KM_DIV) {
      V acc = CT<T>::make(0, 0);
      for (int a = 0; a < 3; ++a) acc = acc + cmul(kval(K, a, O3, O, sym_parity(6 + a), kz, ky, kx, nk), u[a]);
      o[0] = acc;
    } else {
      V q[6];
      for (int a = 0; a < 6; ++a) q[a] = kval(K, a, O3, O, sym_parity(a), kz, ky, kx, nk);
      // symmetric 3x3: [xx xy xz; xy yy yz; xz yz zz]
      const V qxx = q[0], qyy = q[1], qzz = q[2], qxy = q[3], qxz = q[4], qyz = q[5];
      o[0] = cmul(qxx, u[0]) + cmul(qxy, u[1]) + cmul(qxz, u[2]);
      o[1] = cmul(qxy, u[0]) + cmul(qyy, u[1]) + cmul(qyz, u[2]);
      o[2] = cmul(qxz, u[0]) + cmul(qyz, u[1]) + cmul(qzz, u[2]);
      if (mode == KM_MAXWELL6 || mode == KM_EMRED) {
        V p[3];
        for (int a = 0; a < 3; ++a) p[a] = kval(K, 6 + a, O3, O, sym_parity(6 + a), kz, ky, kx, nk);
        // P x J
        const V pxj0 = cmul(p[1], u[2]) - cmul(p[2], u[1]);
        const V pxj1 = cmul(p[2], u[0]) - cmul(p[0], u[2]);
        const V pxj2 = cmul(p[0], u[1]) - cmul(p[1], u[0]);
        if (mode == KM_EMRED) {
          o[3] = vneg(pxj0);
          o[4] = vneg(pxj1);
          o[5] = vneg(pxj2);
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
  V* iv = line_fft<+1, T>(ob, fw, pl, tw, twg + Q, cout * nl, LS);
  for (int idx = tid; idx < cout * nl * n; idx += nt) {
    const int l = idx % nl;
    const int t = idx / nl;
    const int z = t % n, c = t / n;
    base[c * cs + z * zs + l] = iv[(c * nl + l) * LS + z];
  }
}

// ---------------------------------------------------------------- P5
template <typename T>
__global__ void k_p5(const typename CT<T>::V* __restrict__ A, const typename IOT<T>::E* __restrict__ xin,
                     typename IOT<T>::E* __restrict__ y, int n, FftPlan pl, const typename CT<T>::V* __restrict__ twg,
                     int nr, int C, int cout, const typename CT<T>::V* __restrict__ He,
                     const typename CT<T>::V* __restrict__ Hm, int with_identity) {
  typedef typename CT<T>::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = pl.M, Q = pl.Q, LS = Q + 1;
  V* tw = (V*)smraw;
  V* b0 = tw + Q;
  V* b1 = b0 + cout * nr * LS;
  load_tw(tw, twg, Q);
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
  V* res = line_fft<+1, T>(b0, b1, pl, tw, twg + Q, cout * nr, LS);
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
        const typename IOT<T>::E* xi = xin + ((long long)b * cout + 3 * blk) * N + pt;
        typename IOT<T>::E* yo = y + ((long long)b * cout + 3 * blk) * N + pt;
        const V a0 = u[3 * blk], a1 = u[3 * blk + 1], a2 = u[3 * blk + 2];
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
      for (int c = 0; c < cout; ++c) y[((long long)b * cout + c) * N + pt] = from_v<T>(u[c]);
    }
  }
}

// ---------------------------------------------------------------- host
static int pow2_divisor(int M, int target) {
  int nl = target;
  while (nl > 1 && M % nl != 0) nl >>= 1;
  return nl;
}

// Threads per tile line: one per 16 elements of the length-Q transform, a power
// of two up to 128 (32 for every Q <= 512; the long Bluestein lines take more,
// since only one or two of them fit in a tile).
static dim3 line_block(const FftPlan& pl) {
  int tx = 1;
  while (tx * 16 < pl.Q && tx < 128) tx <<= 1;
  return dim3(tx, 256 / tx);
}

// Shared memory of a generic pass over `lines` tile lines: staged twiddles and
// two ping-pong buffers.
static size_t tile_smem(const FftPlan& pl, size_t vs, int lines) {
  return vs * ((size_t)pl.Q + 2 * (size_t)lines * (pl.Q + 1));
}

// Lines per CTA of a one-component generic pass: as many as a 256-thread block
// holds (one thread row per line), with the tile kept near 72 KB of shared
// memory so that three CTAs share an SM also for 16-byte elements.
static int lines_for(const FftPlan& pl, size_t vs) {
  const int cap = 256 / (int)line_block(pl).x;
  int nl = pow2_divisor(pl.M, cap);
  while (nl > 1 && tile_smem(pl, vs, nl) > 72 * 1024) nl >>= 1;
  return nl;
}
// Block of a generic pass over `lines` lines: no thread row left idle.
static dim3 block_for(const FftPlan& pl, int lines) {
  const dim3 b = line_block(pl);
  return dim3(b.x, std::max(1, std::min((int)b.y, lines)));
}

// The generic passes need C tile lines in shared memory at the least (the z
// pass holds every component of a pencil); long Bluestein lines with six
// components at 16 bytes per element do not fit and the apply is refused
// before anything is launched.
static vie_status check_tiles(const FftPlan& pl, size_t vs, int C) {
  if (tile_smem(pl, vs, C) <= (size_t)smem_optin_bytes()) return VIE_OK;
  set_error("grid too large for the generic kernels at this precision and component count (shared memory)");
  return VIE_EINVAL;
}

size_t apply_workspace_bytes(int n, int nk, int c, int nrhs, int prec) {
  const size_t esz = prec == VIE_FP32 ? sizeof(float2) : sizeof(double2);  // double-word complex is 16 bytes too
  const size_t M = 2 * (size_t)nk;
  return esz * (size_t)nrhs * c * ((size_t)n * n * M + (size_t)n * M * M);
}

// Which passes may take the register-resident path.
struct FastSel {
  bool p1 = false, py = false, p3 = false, p5 = false;
};

// Grid length of the register-resident kernels, which take n = M/2 data points
// per line: 2n when the convolution grid is 2n, else 0 (no fast kernels).
static int fast_grid(const vie_problem* P) { return P->nk == P->n ? 2 * P->n : 0; }

static FastSel fast_select(int M, int mode, int with_identity) {
  FastSel f;
  if (M != 64 && M != 96 && M != 128 && M != 192 && M != 256 && M != 384 && M != 512) return f;
  if (getenv("VIE_GENERIC_FFT")) return f;
  const int cin = cin_of(mode), cout = cout_of(mode);
  f.p1 = true;
  f.py = true;
  f.p3 = true;
  f.p5 = (cout <= 3 || cout == 6) && (!with_identity || cout == cin);
  return f;
}

static std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
static std::map<long long, int>& tune_cache() {
  static std::map<long long, int> c;
  return c;
}
// Key of the process-wide z-pass choice: one per (n, precision, kernel mode).
static long long tune_key(const vie_problem* P, int prec, int mode) { return ((long long)P->n * 4 + prec) * 8 + mode; }

bool p3_schedule_ready(vie_problem* P, const KernelSet& K, int prec) {
  if (prec == VIE_DF64) return true;                       // one fixed schedule
  if (!fast_select(fast_grid(P), K.mode, true).p3) return true;  // generic kernels
  int& v = P->p3_variant[prec][K.mode];
  if (v >= 0) return true;
  if (getenv("VIE_P3_VARIANT")) return true;  // a forced variant is launched untimed
  std::lock_guard<std::mutex> g(tune_mutex());
  auto it = tune_cache().find(tune_key(P, prec, K.mode));
  if (it == tune_cache().end()) return false;
  v = it->second;
  return true;
}


static vie_status fast_dispatch(int pass, vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                                int with_identity, void* A, void* B, int C, int prec, cudaStream_t st,
                                bool* used = nullptr) {
  if (prec == VIE_DF64) {
    bool u = true;
    vie_status e = (2 * P->n == 256) ? fast_pass_dw_256(pass, P, K, in, out, nrhs, with_identity, A, B, C, st, &u)
                                     : VIE_EINVAL;
    if (used) *used = u;
    if (e == VIE_EINVAL) set_error("no double-word fast path for this size");
    return e;
  }
  switch (2 * P->n) {
#define VIE_CASE(MM, RA, RB) \
  case MM: return fast_pass_##MM(prec == VIE_FP64, pass, P, K, in, out, nrhs, with_identity, A, B, C, st);
    VIE_FAST_SIZES(VIE_CASE)
#undef VIE_CASE
    default: set_error("no fast path for this size"); return VIE_EINVAL;
  }
}

static vie_status tune_dispatch(vie_problem* P, const KernelSet& K, void* B, int C, int prec, cudaStream_t st,
                                int* best) {
  switch (2 * P->n) {
#define VIE_CASE(MM, RA, RB) \
  case MM: return tune_p3_##MM(prec == VIE_FP64, P, K, B, C, st, best);
    VIE_FAST_SIZES(VIE_CASE)
#undef VIE_CASE
    default: set_error("no fast path for this size"); return VIE_EINVAL;
  }
}

vie_status ensure_apply_workspace(vie_problem* P, const KernelSet& K, int prec, int nrhs, cudaStream_t st) {
  const int C = std::max(cin_of(K.mode), cout_of(K.mode));
  const size_t need = apply_workspace_bytes(P->n, P->nk, C, nrhs, prec);
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
  return VIE_OK;
}

template <typename T>
static vie_status run_apply_t(vie_problem* P, const KernelSet& K, const void* in, void* out, int nrhs,
                              int with_identity, cudaStream_t st) {
  typedef typename CT<T>::V V;
  const int n = P->n, M = 2 * P->nk;
  const int cin = cin_of(K.mode), cout = cout_of(K.mode);
  const int C = std::max(cin, cout);
  {
    vie_status e = ensure_apply_workspace(P, K, Prec<T>::id, nrhs, st);
    if (e != VIE_OK) return e;
  }
  V* A = (V*)P->ws.buf;
  V* B = A + (size_t)nrhs * C * n * n * M;
  const V* tw = Prec<T>::tw(P);
  const V* Kp = Prec<T>::K(K);
  const FftPlan& pl = P->planM;
  const size_t vs = sizeof(V);
  {
    vie_status e = check_tiles(pl, vs, C);
    if (e != VIE_OK) return e;
  }
  Profiler& pf = P->prof;
  const bool rec = pf.on && pf.count < pf.cap;
  cudaEvent_t* ev = rec ? &pf.ev[(size_t)pf.count * (kProfSlots + 1)] : nullptr;
  if (rec) {
    VIE_CK(cudaEventRecord(ev[0], st));
    ++pf.count;
  }

  // double-word arithmetic runs on the generic kernels only: its fully
  // unrolled register-resident variants take far too long to compile
  FastSel fs = fast_select(fast_grid(P), K.mode, with_identity);
  if (Prec<T>::id == VIE_DF64) {
    // double-word fast kernels exist for 2n = 256 and the operator's kernel sets
    // only; its register-resident P5 (254 registers, one CTA per SM) is slower
    // than the generic one, which it keeps
    if (!(M == 256 && fs.p1 && (K.mode == KM_SYM3 || K.mode == KM_MAXWELL6))) fs = FastSel();
    fs.p5 = false;
  }
  int& p3v = P->p3_variant[Prec<T>::id][K.mode];
  if (fs.p3 && p3v < 0 && Prec<T>::id != VIE_DF64) {  // the double-word z pass has one fixed schedule
    // one decision per (n, precision, mode) per process: every problem of a
    // shape then runs the same arithmetic (bitwise-reproducible results).  A
    // variant forced with VIE_P3_VARIANT bypasses the cache both ways.
    const long long key = tune_key(P, Prec<T>::id, K.mode);
    const bool forced = getenv("VIE_P3_VARIANT") != nullptr;
    if (!forced) {
      std::lock_guard<std::mutex> g(tune_mutex());
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) p3v = it->second;
    }
    if (p3v < 0) {
      vie_status e = tune_dispatch(P, K, B, C, Prec<T>::id, st, &p3v);
      if (e != VIE_OK) return e;
      if (!forced) {
        std::lock_guard<std::mutex> g(tune_mutex());
        tune_cache().emplace(key, p3v);
        p3v = tune_cache()[key];
      }
    }
  }
  if (p3v == kP3Generic) fs.p3 = false;
  // P1
  if (fs.p1) {
    vie_status e = fast_dispatch(1, P, K, in, out, nrhs, with_identity, A, B, C, Prec<T>::id, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[1], st));
  } else {
    const int nl = lines_for(pl, vs);
    const size_t smem = tile_smem(pl, vs, nl);
    VIE_CK(allow_smem(k_p1<T>));
    dim3 grid((n * n + nl - 1) / nl, cin, nrhs);
    k_p1<T><<<grid, block_for(pl, nl), smem, st>>>((const typename IOT<T>::E*)in, A, n, pl, tw, nl, C);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[1], st));
  }
  const int nly = lines_for(pl, vs);
  const size_t smem_y = tile_smem(pl, vs, nly);
  // P2
  if (fs.py) {
    vie_status e = fast_dispatch(2, P, K, in, out, nrhs, with_identity, A, B, C, Prec<T>::id, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[2], st));
  } else {
    VIE_CK(allow_smem(k_py<T, -1>));
    dim3 grid(M / nly, n, nrhs * cin);
    k_py<T, -1><<<grid, block_for(pl, nly), smem_y, st>>>(A, B, n, pl, tw, nly, C, cin);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[2], st));
  }
  // P3
  if (fs.p3) {
    bool used = true;
    vie_status e = fast_dispatch(3, P, K, in, out, nrhs, with_identity, A, B, C, Prec<T>::id, st, &used);
    if (e != VIE_OK) return e;
    if (!used) fs.p3 = false;  // no fast z pass fits this shape: the generic one below
    else if (rec) VIE_CK(cudaEventRecord(ev[3], st));
  }
  if (!fs.p3) {
    int nl = pow2_divisor(M, 8);
    // two CTAs per SM: the z pass is compute bound and needs the warps
    while (nl > 1 && tile_smem(pl, vs, C * nl) > 110 * 1024) nl >>= 1;
    const size_t smem = tile_smem(pl, vs, C * nl);
    VIE_CK(allow_smem(k_p3<T>));
    dim3 grid(M / nl, M, nrhs);
    k_p3<T><<<grid, block_for(pl, C * nl), smem, st>>>(B, n, pl, tw, nl, C, Kp, K.mode);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[3], st));
  }
  // P4
  if (fs.py) {
    vie_status e = fast_dispatch(4, P, K, in, out, nrhs, with_identity, A, B, C, Prec<T>::id, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[4], st));
  } else {
    VIE_CK(allow_smem(k_py<T, +1>));
    dim3 grid(M / nly, n, nrhs * cout);
    k_py<T, +1><<<grid, block_for(pl, nly), smem_y, st>>>(B, A, n, pl, tw, nly, C, cout);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[4], st));
  }
  // P5
  if (fs.p5) {
    vie_status e = fast_dispatch(5, P, K, in, out, nrhs, with_identity, A, B, C, Prec<T>::id, st);
    if (e != VIE_OK) return e;
    if (rec) VIE_CK(cudaEventRecord(ev[5], st));
  } else {
    int nr = 4;
    while (nr > 1 && tile_smem(pl, vs, cout * nr) > 200 * 1024) nr >>= 1;
    const size_t smem = tile_smem(pl, vs, cout * nr);
    VIE_CK(allow_smem(k_p5<T>));
    dim3 grid((n * n + nr - 1) / nr, nrhs);
    const V* He = Prec<T>::He(P);
    const V* Hm = P->has_mu ? Prec<T>::Hm(P) : nullptr;
    k_p5<T><<<grid, block_for(pl, cout * nr), smem, st>>>(A, (const typename IOT<T>::E*)in, (typename IOT<T>::E*)out, n, pl, tw, nr, C,
                                     cout, He, Hm,
                                     with_identity);
    VIE_CK(cudaGetLastError());
    if (rec) VIE_CK(cudaEventRecord(ev[5], st));
  }
  return VIE_OK;
}

vie_status tune_apply(vie_problem* P, const KernelSet& K, int prec, int* variant, cudaStream_t st) {
  if (prec == VIE_DF64 || !fast_select(fast_grid(P), K.mode, true).p3) {  // generic kernels: nothing to tune
    *variant = -1;
    return VIE_OK;
  }
  int& v = P->p3_variant[prec][K.mode];
  v = -1;
  {
    std::lock_guard<std::mutex> g(tune_mutex());
    tune_cache().erase(tune_key(P, prec, K.mode));
  }
  // an apply of a zero vector allocates the workspace and tunes on its first call
  const long long L = (long long)cin_of(K.mode) * P->n * P->n * P->n;
  void *x = nullptr, *y = nullptr;
  const size_t esz = prec == VIE_FP32 ? sizeof(float2) : sizeof(double2);
  VIE_CK(dalloc(&x, esz * L, st));
  VIE_CK(dalloc(&y, esz * (size_t)cout_of(K.mode) * P->n * P->n * P->n, st));
  VIE_CK(cudaMemsetAsync(x, 0, esz * L, st));
  vie_status s = run_apply(P, K, x, y, prec, 1, K.mode == KM_SYM3 || K.mode == KM_MAXWELL6, st);
  dfree(x, st);
  dfree(y, st);
  cudaStreamSynchronize(st);
  *variant = (v == kP3Generic) ? -1 : v;
  return s;
}

vie_status run_apply(vie_problem* P, const KernelSet& K, const void* in, void* out, int prec, int nrhs,
                     int with_identity, cudaStream_t st) {
  if (prec == VIE_FP64) return run_apply_t<double>(P, K, in, out, nrhs, with_identity, st);
  if (prec == VIE_DF64) {
    // double-word tables exist for the operator kernels only
    if (&K != &P->kapply) {
      set_error("double-word arithmetic is available for the operator apply only");
      return VIE_EINVAL;
    }
    vie_status s = build_df(P, st);
    if (s != VIE_OK) return s;
    return run_apply_t<df>(P, K, in, out, nrhs, with_identity, st);
  }
  return run_apply_t<float>(P, K, in, out, nrhs, with_identity, st);
}

}  // namespace vie
