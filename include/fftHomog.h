/*
 * fftHomog.h -- C ABI of the GB300 Basic-Scheme solver for FFT-based
 * homogenisation on anisotropic patterns.
 *
 * Method: Bergmann & Merkert, "FFT-based homogenization on periodic
 * anisotropic translation invariant spaces", arXiv 1701.04685.  The library
 * solves Eq. (pde_coefficients) of Thm. pde_discretization,
 *
 *     E_y + Gamma^p_y (C(y) - C0) : (E_y + eps0) = 0,      y in P(M),
 *
 * by the fixed-point iteration of Sec. 4 (Moulinec & Suquet), with the pattern
 * DFT of Eq. (Fouriermatrix) evaluated as a d-dimensional FFT on the
 * Smith-normal-form grid of M and the periodised Green operator Gamma^p of
 * Def. gamma_tilde_fourier tabulated once in FP64.
 *
 * Conventions used by every entry point:
 *  - Tensors are in Mandel form: a symmetric strain/stress is a vector of
 *    n_v = 3 (d = 2: 11, 22, sqrt2*12) or n_v = 6 (d = 3: 11, 22, 33, sqrt2*23,
 *    sqrt2*13, sqrt2*12) reals; a stiffness is a symmetric n_v x n_v matrix,
 *    row-major.  The Frobenius product of Sec. 3.1 is the Euclidean product.
 *  - Pattern points are stored in "storage order": row-major over the
 *    non-trivial Smith-normal-form axes (the largest axis contiguous).
 *    fh_pattern_points() gives each stored point's coordinates y.
 *  - Host pointers are plain CPU memory.  Arguments documented as "host or
 *    device" may be either; the library asks the CUDA runtime which one.
 *  - Every call returns an fh_status; nothing aborts, traps or exits.  On an
 *    error the thread-local message of fh_last_error() says what failed.
 *  - A solver belongs to one CUDA stream; calls on one solver must not run
 *    concurrently.  Different solvers are independent.
 *  - The library allocates and owns all device work memory and the Gamma^p
 *    table; the caller owns every buffer it passes in.
 */
#ifndef FFTHOMOG_H
#define FFTHOMOG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FH_OK = 0,
  FH_NOT_CONVERGED = 1,   /* max_iter reached; results are valid            */
  FH_DIVERGED = 2,        /* residual kept growing; results are valid        */
  FH_NONFINITE = 3,       /* NaN/Inf met in the residual; iteration stopped  */
  FH_ERR_ARG = -1,        /* invalid argument                                */
  FH_ERR_SINGULAR_M = -2, /* det M = 0                                       */
  FH_ERR_OVERFLOW = -3,   /* sizes or integer index maps exceed int64/int32  */
  FH_ERR_NO_ONB = -4,     /* alias sum of |c_k(f)|^2 vanishes: translates not
                             linearly independent (Lemma FI:Props (ii))      */
  FH_ERR_CUDA = -5,       /* a CUDA runtime call failed                      */
  FH_ERR_TIMEOUT = -6,    /* reserved: a bounded device wait gave up         */
  FH_ERR_INTERNAL = -7,   /* internal consistency check failed               */
  FH_ERR_UNSUPPORTED = -8,/* e.g. an FFT axis longer than 4096               */
  FH_ERR_STATE = -9       /* call order violated (e.g. solve before stiffness) */
} fh_status;

/* Generator f of the space of translates V^f_M (Sec. 2.2). */
typedef enum {
  FH_GEN_DIRICHLET = 0,  /* Dirichlet kernel D_M; on boundary frequencies
                            |(M^-T h)_i| = 1/2 the modified kernel's symbol
                            1/2 is used so that Gamma^p is even (real).      */
  FH_GEN_DLVP = 1,       /* de la Vallee Poussin mean, Def. dlVP: per-axis
                            trapezoid g, flat for |u_i| <= 1/2 - alpha_i, zero
                            for |u_i| >= 1/2 + alpha_i, linear in between.   */
  FH_GEN_BOXSPLINE = 2   /* periodised pattern box spline: g(u) =
                            prod_{xi in Xi} sinc(pi xi^T u); the alias sums
                            (Sec. 3.2, end) keep the aliases k = h + M^T z
                            with |(M^-T k)_i| <= r + 1/2, a cube symmetric in
                            k so that Gamma^p stays even.                    */
} fh_gen_kind;

#define FH_MAX_XI 16
#define FH_MAX_LOADS 16
#define FH_TUNE_CANDIDATES 8   /* launch configurations the autotuner times */

typedef struct {
  int kind;                 /* fh_gen_kind                                   */
  double alpha[3];          /* FH_GEN_DLVP: half ramp width per axis, [0,1/2];
                               1/2 is the Fejer kernel, 0 the modified
                               Dirichlet kernel                              */
  int n_xi;                 /* FH_GEN_BOXSPLINE: number s of directions      */
  double xi[3 * FH_MAX_XI]; /* FH_GEN_BOXSPLINE: direction k is
                               xi[3k .. 3k+d-1]                               */
  int alias_radius;         /* FH_GEN_BOXSPLINE: r in 0..16                  */
} fh_generator;

/* FH_PREC_FP64: every stage in FP64.  FH_PREC_FP32: FFT, stress and Green
 * stages in FP32 (table built in FP64 and rounded; residual sums carried with
 * about 48 bits; mean stress in FP64).  FH_PREC_MIXED: FP32 iterations until a
 * load meets the tolerance or its residual stops improving (no 1% progress in
 * 50 iterations: the FP32 rounding floor), then FP64 iterations from that
 * iterate until the FP64 Cauchy residual meets the tolerance (at least one),
 * which removes the FP32 rounding from E and C_eff.  Iteration counts and the
 * residual history cover both phases; status and residual are the FP64
 * phase's. */
typedef enum { FH_PREC_FP64 = 0, FH_PREC_FP32 = 1, FH_PREC_MIXED = 2 } fh_precision;

typedef struct {
  double tol;      /* Cauchy tolerance: a load stops after the first iteration n
                      with r_n = ||E_n - E_{n-1}|| / ||E_n + eps0|| <= tol
                      (Sec. 4; Frobenius l2 over P(M)).  0 = run max_iter.   */
  int max_iter;    /* >= 1                                                    */
  int precision;   /* fh_precision of the FFT, stress and Green stages; the
                      table build, residual norms and mean stresses are FP64
                      in every mode                                          */
  int init;        /* 0: start from E = 0; 1: start from the strain left by
                      the previous solve or set by fh_set_strain (resume)    */
  int chunk;       /* iterations per captured CUDA-graph replay; 0 = 32      */
  int path;        /* 0 = automatic; 1 = whole-GPU passes (one kernel per axis
                      per iteration, CUDA-graph replays); 3 = the same, but
                      FP32 3-D grids with axis-1 and axis-2 lengths in {32, 64,
                      128} fuse both inner axes and the constitutive stage into
                      one plane pass per 2-CTA cluster (an iteration is two
                      kernels; measured slower than path 1 at 128^3, kept for
                      comparison); 2 = cluster-resident
                      (2-axis grids only: one thread-block cluster per load
                      case holds the fields in distributed shared memory and
                      runs every iteration in one launch).  Automatic picks 2
                      when the fields fit, else 1.                            */
  int cluster;     /* cluster size for path 2: 0 = automatic (fh_solve: 16
                      where the fields fit, else 8; fh_solve_batch: 8 where
                      they fit, else 16), 8 or 16                            */
  int form;        /* 0: the Lippmann-Schwinger discretisation, Eq.
                      (pde_coefficients) of Thm. pde_discretization:
                      E <- -Gamma^p (C - C0)(E + eps0).
                      1: the variational discretisation, Eq.
                      (pde_coefficients_variational) of Thm.
                      ls_discretization, whose fixed point solves
                      C0 Gamma^p C (E + eps0) = 0: E <- E - Gamma^p C (E + eps0).
                      The two coincide for the Dirichlet kernel only (Remark
                      constants).  For dlVP and box splines Gamma^p(h) is
                      invertible at most frequencies, so form 1's limit has
                      zero stress there and its iterates contract slowly
                      (thousands of iterations at contrast 8); E is kept in
                      range(Gamma^p), not restricted to the compatible fields
                      of V^f_M that the theorem assumes.                     */
  int tune;        /* 1 with path = cluster = 0 and init = 0: on the first such
                      solve of each bulk precision, time every eligible launch
                      configuration for 24 iterations of these loads and use
                      the fastest from then on (see fh_get_tuning): the
                      whole-GPU passes with the default shapes and radix
                      schedules, clusters of 8 and 16 CTAs, the fused plane
                      pass, and the passes with twice the rows per block of
                      the block row pass, twice the line tile width, every
                      axis's radix schedule reversed, or radix-4 stages in
                      place of radix-8 / radix-2.  The trials overwrite the
                      strain before the actual solve starts from E = 0.
                      2 + c (c < FH_TUNE_CANDIDATES): run candidate c of the
                      list of fh_get_tuning without timing (FH_ERR_UNSUPPORTED
                      where it does not apply); its shapes stay with the
                      solver.                                                 */
  int method;      /* 0: the fixed point of Sec. 4 (Basic Scheme).
                      1: BiCGStab (van der Vorst 1992) on the same discrete
                      equation, (I + Gamma^p (C - C0)) E = -Gamma^p (C - C0)
                      eps0 (the Krylov solvers the paper's introduction cites),
                      two operator applications per iteration, on the
                      whole-GPU passes (path 0 or 1; path 2 gives
                      FH_ERR_UNSUPPORTED), form 0, tune 0.  It stops by the
                      same rule: the fixed point's step from E is b - A E, so
                      a load stops after the first iteration with
                      |b - A E| <= tol |E + eps0|; iterations count BiCGStab
                      iterations and the residual history holds that ratio.
                      With FH_PREC_MIXED the FP32 BiCGStab phase aims at
                      tol / 2 (its recursively updated residual drifts from
                      the true one) and the FP64 phase is the fixed point, as
                      for method 0.                                           */
} fh_solve_opts;

typedef struct {
  int iterations[FH_MAX_LOADS];        /* iterations run, per load            */
  double residual[FH_MAX_LOADS];       /* last r_n, per load                  */
  int status[FH_MAX_LOADS];            /* fh_status per load (0, 1, 2 or 3)   */
  double mean_stress[FH_MAX_LOADS * 6];/* <C:(E+eps0)> per load, Mandel, FP64 */
  double elapsed_ms;                   /* device time from first launch to
                                          the mean-stress reduction          */
  long long kernel_launches;           /* CUDA kernels launched by the solve */
  int path;                            /* path taken (1 or 2)                 */
  int cluster;                         /* cluster size used by path 2         */
} fh_result;

typedef struct fh_pattern fh_pattern;
typedef struct fh_solver fh_solver;

/* Pattern P(M) and generating set G(M^T) of a regular integer matrix M
 * (Sec. 2.1).  d in {2,3}; M is d x d row-major.  Builds the Smith normal form
 * U M V = diag(d_1..d_d) in exact int64 arithmetic and the index maps
 *   point n -> y = M^-1 U^-1 n reduced to [-1/2,1/2)^d,
 *   frequency l -> h = V^-T l reduced to G(M^T),
 * so that exp(-2 pi i h^T y) = exp(-2 pi i sum_i l_i n_i / d_i) and the pattern
 * DFT of Eq. (Fouriermatrix) is a plain FFT on the grid.  Errors:
 * FH_ERR_SINGULAR_M, FH_ERR_OVERFLOW (entries so large that the exact maps
 * could overflow int64, or m >= 2^31), FH_ERR_ARG. */
fh_status fh_pattern_create(int d, const int64_t* M, fh_pattern** out);
void fh_pattern_destroy(fh_pattern* p);

/* m = |det M|, the number of non-trivial SNF axes and their lengths in storage
 * order (dims[ndims-1] is the contiguous one).  dims must hold 3 ints. */
fh_status fh_pattern_info(const fh_pattern* p, int64_t* m, int* ndims, int* dims);

/* Host array y[m*d]: coordinates of the stored points, y = a / m exactly with
 * the integer numerators a of fh_pattern_numerators(). */
fh_status fh_pattern_points(const fh_pattern* p, double* y);
/* Host array a[m*d] of int64 numerators: y = a / m, -m <= 2a < m. */
fh_status fh_pattern_numerators(const fh_pattern* p, int64_t* a);
/* Host array h[nh*d] of the frequencies of the stored half spectrum: row-major
 * over (l_0, .., l_{ndims-2}, l_last in [0, dims_last/2]).  nh is returned in
 * *nh when h is NULL. */
fh_status fh_pattern_half_freqs(const fh_pattern* p, int64_t* h, int64_t* nh);

/* Solver for one pattern and generator on one CUDA stream (cudaStream_t,
 * NULL = legacy default stream).  Allocates device work memory for up to
 * nload_max load cases (1..FH_MAX_LOADS).  The pattern may be destroyed
 * afterwards.  Every axis length up to 4096 is supported: radices 2, 3, 4,
 * 5, 8 are written out, 7, 11, 13 and any larger prime factor run as direct
 * DFT stages (slower for large primes).  Errors: FH_ERR_ARG,
 * FH_ERR_UNSUPPORTED (an SNF axis longer than 4096, or |det M| = 1: a single point has
 * no fluctuation, E = 0 and C_eff = C there), FH_ERR_CUDA. */
fh_status fh_solver_create(const fh_pattern* p, const fh_generator* gen,
                           int nload_max, void* cuda_stream, fh_solver** out);
void fh_solver_destroy(fh_solver* s);

/* Piecewise-constant stiffness (Sec. 3.1, C in SSym_d(L^inf)): phase[m]
 * (uint8, storage order, host or device) selects one of nphase (1..16)
 * Mandel matrices Cp[nphase*n_v*n_v] (host).  C is sampled at the pattern
 * points (collocation, Thm. pde_discretization).  Errors: FH_ERR_ARG when a
 * phase id >= nphase is found (checked on the device). */
fh_status fh_set_stiffness_phases(fh_solver* s, const uint8_t* phase, int nphase,
                                  const double* Cp);

/* Stiffness given point by point (Sec. 3.1, C in SSym_d(L^inf), sampled at
 * the pattern points): C[m*n_v*n_v] Mandel matrices in storage order (the
 * order of fh_pattern_points), host or device memory, read once.  A field of
 * at most 16 distinct matrices (exact, bitwise comparison) is reduced to phase
 * ids and a table and solved exactly as fh_set_stiffness_phases with those
 * matrices.  A field with more distinct matrices (a graded or continuously
 * varying material) is kept point by point: its upper triangles live on the
 * device (21 doubles per point in 3-D, plus FP32 copies and C - C0 after
 * fh_set_reference), the constitutive stage reads them per point, and such
 * solves run on the whole-GPU passes with the block row pass (path 2 gives
 * FH_ERR_UNSUPPORTED).  The reference-medium rule of fh_set_reference then
 * takes its ranges over all points.  Errors: FH_ERR_ARG (non-finite or
 * non-symmetric matrix). */
fh_status fh_set_stiffness_field(fh_solver* s, const double* C);

/* Reference medium C0 (n_v x n_v Mandel, host).  NULL selects the rule of
 * Moulinec & Suquet (1998): isotropic with lambda0, mu0 the midpoints of the
 * phases' ranges (phases read as isotropic: lambda = C[0][1], 2 mu = C[n_v-1]
 * [n_v-1]).  The paper leaves C0 open.  Builds the Gamma^p table of
 * Def. gamma_tilde_fourier on the device in FP64: for every stored frequency
 * h, sum_z w_z(h) Gamma^0(h + M^T z) with the orthonormalised alias weights
 * w_z = g(u+z)^2 / sum_z' g(u+z')^2, u = M^-T h (Lemma FI:Props (iii)), and
 * Gamma^0(k) : tau = sym(k (x) K(k)^-1 tau k), K_ik = C0_ijkl k_j k_l
 * (Def. projection).  Must follow fh_set_stiffness_phases.  Errors:
 * FH_ERR_STATE, FH_ERR_NO_ONB, FH_ERR_ARG (C0 not positive definite). */
fh_status fh_set_reference(fh_solver* s, const double* C0);

/* Run the fixed point for nload (1..nload_max) macroscopic strains
 * eps0[nload*n_v] (host, Mandel), all load cases together on the device:
 *   tau = (C - C0):(E + eps0);  E^_h = -Gamma^p_h tau^_h,  E^_0 = 0;
 *   E = inverse DFT;  r_n as in fh_solve_opts.tol.
 * Each load stops on its own.  Fills *res (host).  Returns FH_OK when every
 * load converged, else the worst per-load status (FH_NONFINITE >
 * FH_DIVERGED > FH_NOT_CONVERGED), or an error code. */
fh_status fh_solve(fh_solver* s, int nload, const double* eps0,
                   const fh_solve_opts* opts, fh_result* res);

/* Batched solve: runs fh_solve on n distinct solvers (patterns of any sizes)
 * with one shared set of options; nload[i] and eps0[i] are solver i's load
 * count and strains, res[i] (host, may be NULL) its result.  Every solver's
 * set-up is enqueued on its own stream before any is waited for; the cluster-
 * resident solves of all solvers then run as one persistent launch per
 * cluster-kernel variant, whose clusters take (solver, load) tasks from a list
 * ordered largest pattern first; solvers that need the whole-GPU pass path
 * run their host-driven loops in turn.  With path and
 * cluster left at 0 (and no earlier tuning of the solver), a batch takes the
 * 8-CTA cluster wherever the fields fit: two of those run per GPC, where a
 * 16-CTA cluster occupies a GPC alone, so the batch finishes sooner even
 * though each solve alone is slower.  Returns the worst per-load status over
 * the batch or an error code (nothing is run when an argument check fails). */
fh_status fh_solve_batch(fh_solver* const* solvers, int n, const int* nload, const double* const* eps0,
                         const fh_solve_opts* opts, fh_result* res);

/* Copy the strain fluctuation E of one load (component-major: E[c*m + i] is
 * component c at stored point i) into host or device memory, as doubles. */
fh_status fh_get_strain(const fh_solver* s, int load, double* E);
/* Set the start E of one load for the next solve with init = 1 (host or
 * device, layout of fh_get_strain). */
fh_status fh_set_strain(fh_solver* s, int load, const double* E);

/* FP32 variants of fh_get_strain / fh_set_strain (same layout), for starting
 * strains produced in FP32 (e.g. by the FNO below).  Setting an FP32 strain
 * makes the next init = 1 solve start from it in either precision. */
fh_status fh_get_strain_f32(const fh_solver* s, int load, float* E);
fh_status fh_set_strain_f32(fh_solver* s, int load, const float* E);

/* Effective stiffness C_eff (Sec. 3.1, read as <C:(E+eps0)> = C_eff eps0)
 * from the last solve, which must have had nload = n_v linearly independent
 * eps0.  Ceff[n_v*n_v] host, row-major; voigt != 0 converts Mandel to Voigt
 * (C_V = C_M / (s_a s_b), s = 1 normal, sqrt2 shear). */
fh_status fh_get_ceff(const fh_solver* s, double* Ceff, int voigt);

/* Host copy of the Gamma^p table: G[nh * n_v * n_v], the full symmetric
 * matrix for every stored half-spectrum frequency (order of
 * fh_pattern_half_freqs). */
fh_status fh_get_green(const fh_solver* s, double* G);

/* Autotuner result for a bulk precision (FH_PREC_FP64 or FH_PREC_FP32): the
 * chosen path (0 = not tuned yet; 1 passes, 2 cluster-resident, 3 passes with
 * the fused plane pass), cluster size and candidate index, and the measured
 * microseconds per iteration of every candidate (-1 where it does not apply):
 * [0] passes, [1] cluster 8, [2] cluster 16, [3] passes with the plane pass,
 * [4] twice the rows per block of the block row pass, [5] twice the line tile
 * width, [6] reversed radix schedules, [7] radix-4 schedules.  candidate and
 * us_per_iter[FH_TUNE_CANDIDATES] may be NULL. */
fh_status fh_get_tuning(const fh_solver* s, int precision, int* path, int* cluster, int* candidate,
                        float* us_per_iter);

/* Residual history r_1..r_n of one load from the last solve: hist[n] host;
 * *n receives the count (hist may be NULL to query it). */
fh_status fh_get_residuals(const fh_solver* s, int load, double* hist, int* n);

/* Profiling aid: time each kind of iteration pass of the current solver in
 * isolation with CUDA events on the solver's stream, `reps` back-to-back
 * launches each after one warm-up launch, for `nload` loads in the given
 * precision.  ms[4] (host) receives the mean duration per launch of
 *   [0] the row pass (contiguous axis, fused constitutive stage + residual),
 *   [1] the axis-0 line pass with the Green step (or the Green step alone on
 *       1-axis grids),
 *   [2] a forward middle-axis line pass (3-axis grids, else 0),
 *   [3] an inverse middle-axis line pass (3-axis grids, else 0).
 * The passes run on the solver's own buffers and advance its iterate: call it
 * after the results of the last solve have been read.  Requires a prior
 * fh_solve with the same nload (it reuses that solve's eps0). */
fh_status fh_profile_passes(fh_solver* s, int nload, int precision, int reps, double* ms);

/* Mean stress <C:(E+eps0)> per load case, computed without allocating any
 * device memory.  The paper has no counterpart: this is an interface for
 * callers that cannot call cudaMalloc when they need the result -- real-time
 * loops where an allocation could block or fail, and applications (a larger
 * simulation embedding this solver, say) whose device memory is owned entirely
 * by their own allocator with a fixed budget.  All scratch (per-block partial
 * sums, a block counter, an error word, the result) lives in one fixed array
 * of 6272 doubles (49 KB) inside the library, held by every GPU that loads the
 * library until the process exits.
 *
 *   E[nload * n_v * m]   device, FP64, layout of fh_get_strain per load
 *   phase[m]             device, uint8 phase ids < nphase
 *   Cp[nphase*n_v*n_v]   host, Mandel phase stiffnesses (nphase 1..16)
 *   eps0[nload*n_v]      host, Mandel macroscopic strains
 *   mean_stress[nload*n_v] host or device output
 *   cuda_stream          stream to run on (NULL = legacy default); the call
 *                        synchronises it before returning.
 * n_v = 3 (d = 2) or 6 (d = 3).  nload above 16 is rejected with FH_ERR_ARG
 * before anything runs.  A phase id >= nphase is detected on the device (the
 * point is skipped, never used as an index) and the call returns FH_ERR_ARG;
 * mean_stress is then not valid.  The first call on a device looks up and
 * caches the array's device address: make that first call before any stream
 * capture, and do not call again after cudaDeviceReset on that device.  Calls
 * that overlap on the GPU share the array and race: serialise them. */
fh_status fh_mean_stress_noalloc(int d, long long m, int nload, const double* E, const uint8_t* phase,
                                 int nphase, const double* Cp, const double* eps0, double* mean_stress,
                                 void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned start: a Fourier neural operator (FNO) that predicts the starting
 * strain fluctuation E of fh_solve from the microstructure and eps0.  The
 * paper has no counterpart; the Basic Scheme started from the prediction
 * still iterates to the same tolerance, so the network only saves iterations.
 * Network on an n^3 grid (z fastest, the storage order of a diagonal M):
 *   v0 = P x + p;  u_l = W_l v_l + w_l + K_l v_l,  v_{l+1} = gelu(u_l);  y = Q v_L + q,
 *   K_l v = n^-3 Re sum_k w(kz) R_l(k) v^(k) e^{+2 pi i k.x/n},  v^ = truncated DFT,
 *   kx, ky in {-modes..modes-1}, kz in {0..modes-1}, w(0) = 1, w(kz>0) = 2.
 * R_l and W_l are applied in BF16 (from FP32 master weights), all sums FP32.
 * Arrays x [batch][cin][n^3], y and targets [batch][cout][n^3] are device FP32.
 * The parameter vector (host FP32) is, in order: P[width][cin], p[width],
 * W[layers][width][width], w[layers][width], Re R[layers][2m][2m][m][width][width],
 * Im R[...], Q[cout][width], q[cout]. */
typedef struct fh_fno fh_fno;
fh_status fh_fno_create(int n, int cin, int cout, int width, int modes, int layers, int max_batch,
                        void* cuda_stream, fh_fno** out);
void fh_fno_destroy(fh_fno* f);
fh_status fh_fno_param_count(const fh_fno* f, long long* count);
fh_status fh_fno_set_params(fh_fno* f, const float* params);
fh_status fh_fno_get_params(const fh_fno* f, float* params);
fh_status fh_fno_get_grads(const fh_fno* f, float* grads);
fh_status fh_fno_zero_grad(fh_fno* f);
/* y = network(x) for `batch` samples (x, y device).  FH_ERR_TIMEOUT when a
 * tensor-core layer's bounded wait for its MMAs gave up (y not valid). */
fh_status fh_fno_forward(fh_fno* f, int batch, const float* x, float* y);
/* The hidden 1 x 1 layers W_l v + w_l run on the tensor cores (tcgen05, BF16
 * weights as above, each FP32 activation split into three BF16 terms, FP32
 * accumulation in tensor memory) when width is 16, 32 or 64 and n^3 is a
 * multiple of 128; enable = 0 selects the SIMT layers (default 1).  Not in
 * the paper: the network is this library's own. */
fh_status fh_fno_set_tensor_cores(fh_fno* f, int enable);
/* Forward and backward of the mean squared error against `target`
 * (mean over samples, channels and voxels); the loss goes to *loss (host,
 * may be NULL) and the gradient is ADDED to the accumulated gradient. */
fh_status fh_fno_loss_grad(fh_fno* f, int batch, const float* x, const float* target, double* loss);
/* One Adam update of the master weights with the accumulated gradient
 * (step counts from 1 for the bias corrections). */
fh_status fh_fno_adam_step(fh_fno* f, float lr, float beta1, float beta2, float eps, int step);
/* Input channels of one sample: log10(E(x))/2 from a phase map (device
 * uint8[n^3]) and per-phase log10 Young moduli (host); for cin = 7 followed
 * by the six Mandel components of eps0 (host) as constant channels (for
 * cin = 1 eps0 is not used).  x device [cin][n^3]. */
fh_status fh_fno_make_input(const fh_fno* f, const uint8_t* phase, int nphase, const double* phase_logE,
                            const double* eps0, float* x);

const char* fh_status_string(fh_status st);
const char* fh_last_error(void);

/* ---- checked build --------------------------------------------------------
 * The library compiled with -DFH_CHECKED (build(checked=True) of the Python
 * package, libffthomog_checked.so) tests the global-memory and tile indices
 * of its solver kernels against the extents of the arrays they address.  A
 * violating access is skipped and recorded; fh_solve, fh_solve_batch,
 * fh_set_reference and fh_profile_passes then return FH_ERR_INTERNAL and
 * fh_last_error() names the kernel and array, the index and the extent.  The
 * checks stand in for a memory checker; they cost time and are off in the
 * normal build. */
/* 1 in the checked build, else 0. */
int fh_checked_build(void);
/* Checked build: launches a one-thread kernel that tests one index inside and
 * one outside a declared extent (inside its buffer either way) and returns
 * FH_ERR_INTERNAL naming the self test when the check caught the second.
 * Normal build: FH_ERR_UNSUPPORTED, nothing launched. */
fh_status fh_check_selftest(void);

#ifdef __cplusplus
}
#endif
#endif /* FFTHOMOG_H */
