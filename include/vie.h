/* vie.h -- C ABI of the GB300 (sm_103a) FFT-accelerated volume integral
 * equation solver for anisotropic, inhomogeneous media.
 *
 * Method: Imbert-Gerard, Vico, Greengard, Ferrando, "Integral equation methods
 * for electrostatics, acoustics and electromagnetics in smoothly varying,
 * anisotropic media" (arXiv:1805.04791).  The library solves the second-kind
 * equations (I + B + K) J = b of
 *   - Eq. (eq:intLap)  Laplace:   J - 2 H_eps T_0 J = 2 H_eps grad phi_in,
 *   - Eq. (eq:intH)    Helmholtz: J - 2 H_{eps^-1} T_w J = 2 H_{eps^-1} grad phi_in
 *                      (sign as produced by the derivation of Sec. 3; the
 *                      printed equation carries "+"),
 *   - Eq. (eq:intM)    Maxwell:   the coupled [J; M] system, or Eq.
 *                      (contraction_Maxwell_reduced) when mu = I,
 * with H_eps = (eps + I)^-1 (eps - I) (Eq. (rhodef)) and T J = J/2 + grad div V J
 * (Eqs. (Todef), (Vw)).  The volume potentials are applied with the
 * truncated-kernel FFT method of Sec. 5 (truncate the Green's function at
 * L = sqrt(3) D, transform it, cut off at the grid Nyquist frequency) on a
 * uniform cell-centred n^3 grid, as zero-padded convolutions on a (2n)^3 grid.
 *
 * Conventions common to every call
 * --------------------------------
 * - Complex numbers are interleaved (re, im): FP64 = 16 bytes, FP32 = 8 bytes.
 * - Grid arrays are [z][y][x], x fastest; node i sits at lo + (i + 1/2) h.
 * - A vector field with c components is [c][n][n][n]; a batch of nrhs fields
 *   is [nrhs][c][n][n][n] (batch outermost).  c = 3 for Laplace, Helmholtz
 *   and Maxwell with mu = I; c = 6 ([J; M]) for Maxwell with mu.
 * - "device" pointers are CUDA device memory of the current device; the
 *   caller owns every pointer it passes in (the library never frees them).
 *   The library owns everything it allocates, from create until destroy.
 * - stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *   work on it and return without synchronising unless stated otherwise.
 * - No exception crosses the ABI; every call returns a vie_status and, on
 *   failure, vie_last_error() returns a message (thread-local).
 * - A problem handle is not thread-safe; distinct handles may be used from
 *   different threads on different streams.  Calls on one handle must be
 *   ordered (one stream, or streams the caller synchronises).  Device memory
 *   is allocated stream-ordered (cudaMallocAsync) on the stream of the call,
 *   so calls on other handles and streams are never serialised by it; the
 *   stream given to vie_problem_create must stay valid until
 *   vie_problem_destroy, which frees on it.
 *
 * Environment variables (read at each call; for testing and measurement --
 * none is needed in normal use)
 * --------------------------------------------------------------------------
 * - VIE_P3_VARIANT=k    every register-resident apply runs z-pass variant k
 *                       (see vie_tune), bypassing the process-wide tuning
 *                       cache; shapes k does not fit return VIE_EINVAL.
 * - VIE_TUNE=0          vie_tune takes the first applicable variant untimed.
 * - VIE_GENERIC_FFT     (set to any value) the generic shared-memory kernels
 *                       run at every size, also where register-resident ones exist.
 * - VIE_GROUP_MAX=g     batched solves use lockstep groups of at most g
 *                       right-hand sides (default: from free device memory, <= 64).
 * - VIE_RESIDUAL_FP64=1 mixed solves compute their residuals with the native
 *                       FP64 apply instead of the double-word one.
 * - VIE_SETUP_FP64=1    the set-up's kernel-transform FFTs run in native FP64
 *                       instead of double-word arithmetic.
 * - VIE_RESIDUAL_UPDATE=0 mixed solves recompute every refinement residual
 *                       as b - A x (double-word apply) instead of updating it
 *                       with an FP32 apply of a small correction.
 * - VIE_GRAPHS=0        single right-hand-side GMRES steps are launched kernel by
 *                       kernel instead of being replayed from captured CUDA graphs.
 * - VIE_ARNOLDI_SHIFT=0 GMRES orthogonalises A v instead of (A - I) v (the
 *                       same Krylov space; with the shift, 1 is added to each
 *                       diagonal Hessenberg entry).
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VIE_OK = 0,
  VIE_EINVAL = 1,   /* bad argument (size, pointer, symmetry, precision) */
  VIE_ENOMEM = 2,   /* device allocation failed */
  VIE_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  VIE_ENOCONV = 4,  /* solver hit its iteration limit before the tolerance */
  VIE_ENAN = 5,     /* non-finite values met in a solve */
  VIE_ETIMEOUT = 6, /* a bounded device wait expired */
  VIE_EBUSY = 7     /* resource in use */
} vie_status;

typedef enum { VIE_LAPLACE = 0, VIE_HELMHOLTZ = 1, VIE_MAXWELL = 2 } vie_kind;

/* Arithmetic of an operator apply: FP64 complex; FP32 complex (inner
 * iterations of the mixed-precision solve); or VIE_DF64: FP64 complex vectors
 * in and out, arithmetic in double-word form (each real held as the unevaluated
 * sum of two FP32 values, about 48 significant bits; relative error of the
 * apply near 1e-13), which the mixed solve uses for its refinement residuals
 * because it runs on the FP32 pipes.  Not a source of the paper's method: an
 * implementation choice for the FP64 residual of Sec. 5's solve. */
typedef enum { VIE_FP64 = 0, VIE_FP32 = 1, VIE_DF64 = 2 } vie_precision;

/* Solver modes for vie_solve: plain FP64 GMRES(m); FP32-inner GMRES(m)
 * inside an FP64 iterative-refinement loop; or FP64 Bi-CGStab, the solver of
 * the paper's experiments (Sec. 5; restart and inner_tol unused, max_inner =
 * iteration limit, two applies per iteration). */
typedef enum { VIE_SOLVE_FP64 = 0, VIE_SOLVE_MIXED = 1, VIE_SOLVE_BICGSTAB = 2 } vie_solve_mode;

typedef struct vie_problem vie_problem;

typedef struct {
  double tol;        /* stop when ||b - A J||_2 / ||b||_2 <= tol (FP64 residual) */
  int restart;       /* GMRES restart length m (1..200) */
  int max_outer;     /* mixed: maximum refinement steps; FP64: maximum restarts */
  int max_inner;     /* maximum GMRES iterations per refinement step (mixed) or in total (FP64) */
  double inner_tol;  /* mixed: each inner FP32 solve stops at inner_tol ||r|| or at
                        0.25 tol ||b||, whichever is larger (later refinement
                        steps need only reach the overall target) */
  int mode;          /* vie_solve_mode */
  int nrhs;          /* number of right-hand sides, solved independently (>= 1) */
  int check_fp64;    /* 1: after the solve, compute the residual of the final
                        iterate once more with the native FP64 apply (one extra
                        FP64 apply per right-hand side) into
                        info->rel_residual_fp64; 0: skip it (reported as -1) */
} vie_solve_opts;

typedef struct {
  int outer_iters;        /* refinement steps (mixed) or restarts (FP64) */
  int inner_iters;        /* GMRES iterations (= FP32 or FP64 applies inside Arnoldi) */
  int applies_fp32;
  int applies_fp64;       /* FP64-accuracy applies: native FP64, or VIE_DF64 for the mixed
                             mode's refinement residuals (VIE_RESIDUAL_FP64=1: native) */
  double rel_residual;    /* max over right-hand sides of the final relative residual, as the
                             solver computed it: native FP64 (FP64, Bi-CGStab) or double-word
                             (mixed; relative error of that apply near 1e-13).  A mixed
                             residual updated after a small correction d as r - A_32 d (FP32
                             apply; taken when the bound 8 u log2(M^3) ||A|| ||d||, u = 2^-24,
                             is within half the tolerance) is reported as |r| plus that bound:
                             an upper bound of the true residual */
  double t_solve;         /* wall seconds spent in vie_solve */
  double t_precompute;    /* wall seconds vie_problem_create spent on this handle's set-up
                             (medium tensors and kernel transforms, Sec. 5) */
  double rel_residual_fp64; /* max over right-hand sides of ||b - A J|| / ||b|| of the returned
                               J with the native FP64 apply (opts->check_fp64 = 1), else -1 */
} vie_solve_info;

/* Create a problem: grid, medium and frequency (Sec. 2 / Eq. (Laplace_Scalar),
 * Sec. 3 / Eq. (Helmholtz0), Sec. 4 / Eq. (Maxwell)).
 *   kind   vie_kind.
 *   n      points per axis, 4 <= n <= 512.  The convolution grid is M = 2 nk
 *          per axis with nk = n when n = 2^a 3^b 5^c 7^d 11^e, else the smallest
 *          such nk > n (a circular convolution of length M >= 2n - 1 equals the
 *          zero-padded one on the n^3 nodes; n = 326 runs on M = 660).
 *          Register-resident kernels for M = 2n in {64, 96, 128, 192, 256, 384,
 *          512}, shared-memory Stockham kernels for the other grids.  The
 *          oversampled set-up grid is 3n; when 3n has a prime factor above 11
 *          its lines are transformed by Bluestein's chirp-z algorithm over a
 *          padded length Q >= 2 (3n) - 1 made of the factors 2, 3, 5, 7, 11.
 *          Odd n is valid: the set-up grid 3n is then odd and its frequency
 *          cut-off is the symmetric |m| <= (3n-1)/2, with no Nyquist entry.
 *          The set-up holds (3n)^3 + M^3 FP64 complex transform buffers (about
 *          75 GB at n = 512); a failed allocation returns VIE_ENOMEM.  M <= 1024
 *          for every valid n, so the generic z-pass tile (six lines of M + 1
 *          elements at 16 bytes, FP64) fits in shared memory.
 *   lo, hi box [lo, hi]^3 (hi > lo).
 *   omega  angular frequency (ignored for Laplace; >= 0).
 *   eps    device, FP64 complex [9][n][n][n], the 3x3 tensor row-major per node;
 *          must be symmetric (|eps_ab - eps_ba| <= 1e-12 (1 + |eps|)), eps + I
 *          invertible.  Laplace uses the real part.
 *   mu     device, same layout, or NULL for mu = I (Maxwell only; other kinds ignore it).
 * Computes H_eps (and H_mu) per node (Eq. (rhodef)) and the transforms of the
 * truncated kernels (Sec. 5) in FP64 on the device; keeps FP64 and FP32 copies.
 * Synchronises the stream.  *out receives the handle. */
vie_status vie_problem_create(int kind, int n, double lo, double hi, double omega, const void* eps, const void* mu,
                              void* stream, vie_problem** out);

/* Number of unknown components c (3 or 6) of a problem. */
int vie_problem_ncomp(const vie_problem* P);

/* y = (I + B + K) x, the left-hand side of Eq. (eq:intLap), (eq:intH) or (eq:intM).
 *   x, y   device, [nrhs][c][n][n][n], FP64 complex (precision VIE_FP64 or
 *          VIE_DF64) or FP32 complex (VIE_FP32); x and y must not share a byte
 *          (VIE_EINVAL).
 *   nrhs   >= 1.  Asynchronous on stream.  The first VIE_DF64 apply of a
 *   handle converts its tables to double-word form (device memory of the size
 *   of the FP64 kernel and medium tables, kept until destroy). */
vie_status vie_apply(vie_problem* P, const void* x, void* y, int precision, int nrhs, void* stream);

/* y = (I + B + K) x like vie_apply, for callers that cannot let the library
 * allocate device memory when they apply the operator: solvers embedded in
 * frameworks that own all device memory through their own arena or pool (an
 * allocation outside it fails or takes memory promised elsewhere), and
 * latency-bound loops that must not take the device-wide synchronisation of
 * cudaMalloc/cudaFree or risk running out of memory in the middle of a run.
 * The paper has no counterpart; this is an interface addition.
 *   Scratch: the padded intermediates live in one file-scope device array of
 *   64 MiB per device (held by every GPU that loads the library until the
 *   process exits).  Sizes whose workspace exceeds it return VIE_EINVAL; with 3
 *   components and nrhs = 1 that allows n <= 77 in FP32 and n <= 61 in FP64.
 *   The call allocates nothing: no cudaMalloc/cudaFree or allocating library
 *   routine.  Its first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) while that device is current; make that first call
 *   before any stream capture.
 *   The z-pass schedule must already be chosen for this precision and grid
 *   size -- by vie_tune or one vie_apply on this handle, or on any handle of
 *   the process with the same grid size and kind (the choice is shared
 *   process-wide) -- otherwise VIE_EINVAL: choosing it would launch and time
 *   candidates.  Sizes that run the generic kernels need no choice.
 *   Every call shares the array and leaves its contents behind (no pass reads
 *   scratch it did not write first); calls that overlap on the GPU -- on
 *   different streams or different handles -- race on it and must be ordered
 *   by the caller.
 *   x, y, nrhs, stream: as for vie_apply; precision VIE_FP64 or VIE_FP32
 *   (VIE_DF64 returns VIE_EINVAL).  The result equals vie_apply's bit for bit. */
vie_status vie_apply_static(vie_problem* P, const void* x, void* y, int precision, int nrhs, void* stream);

/* Right-hand sides for plane-wave (or uniform-field) incidence, FP64 complex,
 * [nrhs][c][n][n][n] into device buffer rhs_out.
 *   d  host, [nrhs][3]: Laplace: the applied field E0 (grad phi_in = -E0);
 *      Helmholtz / Maxwell: unit propagation direction, phi_in = exp(i w d.x)
 *      (| |d| - 1 | > 1e-8 returns VIE_EINVAL).
 *   p  host, [nrhs][3]: Maxwell polarisation (E_in = p exp(i w d.x),
 *      H_in = d x p exp(i w d.x)), perpendicular to d (|d.p| > 1e-8 |p| returns
 *      VIE_EINVAL); ignored otherwise (may be NULL).
 * Laplace: 2 H_eps grad phi_in (Eq. (eq:intLap)); Helmholtz: 2 H_{eps^-1} grad phi_in
 * (Eq. (eq:intH)); Maxwell: [2 H_eps E_in; 2 H_mu H_in] (Eq. (eq:intM)). */
vie_status vie_rhs_plane_wave(vie_problem* P, const double* d, const double* p, int nrhs, void* rhs_out,
                              void* stream);

/* Solve (I + B + K) J = rhs by restarted GMRES (Sec. 1 and Sec. 6 name GMRES for
 * these second-kind equations).
 *   rhs  device, FP64 complex [nrhs][c][n][n][n].
 *   J    device, same layout: initial guess on entry (zeros for none), solution on
 *        exit; must not overlap rhs (VIE_EINVAL).
 *   opt  solver options (nrhs from opt->nrhs); info may be NULL.
 * Synchronises the stream.  Returns VIE_ENOCONV (J holds the last iterate) if a
 * right-hand side misses the tolerance, VIE_ENAN on non-finite residuals. */
vie_status vie_solve(vie_problem* P, const void* rhs, void* J, const vie_solve_opts* opt, vie_solve_info* info,
                     void* stream);

/* Scattered field from the solved density, FP64 complex on the grid.
 *   Laplace / Helmholtz: phi_sc = div V J, 1 component (Sec. 2 existence proof;
 *     summary after Eq. (eq:intH)); field_out [nrhs][1][n][n][n].
 *   Maxwell: [E_sc; H_sc] by Eq. (represent_Maxwell) (or Eq.
 *     (represent_Maxwell_reduced) when mu = I); field_out [nrhs][6][n][n][n].
 * J and field_out must not overlap (VIE_EINVAL).  Asynchronous on stream. */
vie_status vie_eval_scattered(vie_problem* P, const void* J, void* field_out, int nrhs, void* stream);

/* Device bytes a problem of this shape holds (medium, kernels, apply workspace
 * for nrhs right-hand sides, FP32 Krylov basis of length restart); used for
 * admission by memory budget.  has_mu: 1 for Maxwell with mu. */
size_t vie_problem_bytes(int kind, int n, int nrhs, int restart, int has_mu);

/* Release every allocation of the handle, stream-ordered on the stream the
 * handle was created with, and wait for that stream. */
vie_status vie_problem_destroy(vie_problem* P);

/* Autotune the z-pass schedule of vie_apply at this precision by timing every
 * applicable variant on this device; the choice is kept in the handle and
 * written to *variant (-1: the shape uses the generic kernels).  Variants:
 * 0/1/2 one CTA per mirror group of tiles with 8/16/4 pencils per tile, one
 * component per thread; 3 one CTA per tile of 8 pencils; 4/5/6 (FP32 only,
 * 2n in {64, 96, 128, 256}) as 0/1/2 with two neighbouring pencils per
 * thread packed as f32x2 lanes; 7/8/9 (FP32 only, same sizes) mirror-group
 * CTAs of 8/4/16 pencils with all three components of a vector per thread;
 * 10/11 as 7/8 with a grid sized to the device, each CTA walking several
 * mirror groups and prefetching the next one's inputs and kernel values;
 * 12/13/14 (FP32, 3x3 symmetric and divergence kernel sets, same sizes) slim
 * component-group CTAs of 8/8/4 pencils sized for 3/2/5 CTAs per SM: one
 * transpose line per pencil shared by the components in turn, 16-byte
 * shared-memory reads, packed f32x2 kernel mixing; 15/16/17/18 (FP32, 2n =
 * 512, 3x3 symmetric and Maxwell kernel sets) the even and odd frequencies of
 * each z-line as two 256-point transforms on the two CTAs of a thread-block
 * cluster, the inverse halves summed through distributed shared memory, with
 * 4/8/8/8 pencils per CTA (17: packed f32x2 twiddles and kernel mixing; 18: a
 * grid of co-resident clusters, each walking several mirror groups and loading
 * the next one's kernel entries and first inputs during the current one).
 * Every candidate runs once untimed, then two rounds of three timed launches;
 * each keeps its best round and the fastest is chosen.  VIE_DF64 has one fixed
 * schedule (*variant = -1).  vie_apply
 * tunes on its first call for a precision anyway; calling vie_tune first keeps
 * the tuning time out of a timed or captured region.  Synchronises the stream.
 * Environment: VIE_TUNE=0 takes the first applicable variant without timing,
 * VIE_P3_VARIANT=k forces variant k. */
vie_status vie_tune(vie_problem* P, int precision, int* variant, void* stream);

/* Per-kernel timing of vie_apply / vie_eval_scattered, for measurement tools.
 * vie_profile_begin(P, cap) makes the following applies on P record a CUDA
 * event before and after each of their kernel launches (on the launch stream;
 * no synchronisation), for at most cap applies.  vie_profile_end synchronises
 * the device, writes into ms[k] (k < nslots, host) the total milliseconds spent
 * in kernel slot k (0..4: the five passes of the pipeline, see apply.cu),
 * writes the number of recorded applies to *count, and stops recording. */
vie_status vie_profile_begin(vie_problem* P, int cap);
vie_status vie_profile_end(vie_problem* P, double* ms, int nslots, int* count);

/* Message of the last failure on this thread ("" if none). */
const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H */
