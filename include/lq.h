/*
 * lq.h -- C ABI of the GB300 library for two-sided-Lanczos approximations of the
 * matrix sign function sgn(H(mu)) x and of its derivative d_t sgn(H(mu)) x, where
 * H(mu) = gamma5 Dw(mu) is the finite-density Wilson kernel of the overlap operator
 * (Puhr & Buividovich, Lattice 2016: Sec. 1, Eq. (1.1); the derivative through
 * Mathias' block identity, Sec. 2, Eqs. (2.5)-(2.6)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Lattice  dims (nt, nx, ny, nz); V = nt*nx*ny*nz; site s = x + nx*(y + ny*(z + nz*t)).
 *  Spinor   colour-spinor field of n = 12 V complex numbers, index 12*s + 3*spin + colour,
 *           stored as interleaved complex128 (re, im) doubles: double[V][4][3][2].
 *           A batch of nsrc fields is double[nsrc][V][4][3][2].  The boundary always
 *           carries FP64 values; the internal precision is set by lq_lattice_desc.precision.
 *  Gauge    U_nu(s) in SU(3) (nu = 0..3 = x, y, z, t; link s -> s + nu-hat), row-major,
 *           interleaved complex128: double[4][V][3][3][2].
 *  Operator (Dw psi)(s) = (4r + m_w) psi(s) - 1/2 sum_nu [ f+ (r - g_nu) U_nu(s) psi(s+nu)
 *           + f- (r + g_nu) U_nu(s-nu)^dag psi(s-nu) ],  f+- = exp(+-mu) on time hops, 1
 *           otherwise; a hop across the time boundary carries -1 when t_antiperiodic;
 *           chiral gamma basis, gamma5 = diag(1, 1, -1, -1); H = gamma5 Dw; H^dag = H(-mu).
 *  Memory   every pointer argument may point to host memory (pageable or pinned) or to
 *           device memory of the context's GPU; the library detects which and stages host
 *           data through buffers reserved by lq_reserve.  The caller owns every buffer it
 *           passes; the library owns the context, its device copy of the gauge field, the
 *           direction field, the Krylov workspace and the deflation space.
 *  Streams  `stream` is a cudaStream_t (0 = legacy default stream).  Entry points that
 *           return a report (lq_report) synchronise the stream before returning; the others
 *           are asynchronous on the stream.
 *  Errors   every int-returning function returns LQ_OK (0) or a negative LQ_ERR_* code;
 *           lq_last_error() gives a one-line description.  Soft, per-source failures
 *           (Lanczos breakdown, Newton not converged) are reported in lq_report.status and do
 *           not fail the call.
 *  Threads  a context is not thread safe; use one context per host thread.
 */
#ifndef LQ_H
#define LQ_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return / status codes ---------------------------------------------------------- */
#define LQ_OK               0
#define LQ_ERR_ARG         -1   /* invalid argument (null pointer, bad size, r != 1, ...)   */
#define LQ_ERR_LAYOUT      -2   /* pointer in an unsupported memory space / misaligned       */
#define LQ_ERR_OOM         -3   /* device allocation failed in lq_reserve / uploads          */
#define LQ_ERR_CUDA        -4   /* a CUDA runtime call failed                                */
#define LQ_ERR_BREAKDOWN   -5   /* (status) serious Lanczos breakdown: k_eff < k             */
#define LQ_ERR_NEWTON      -6   /* (status) Newton sign iteration did not converge           */
#define LQ_ERR_TIMEOUT     -7   /* a bounded device-side wait gave up                        */
#define LQ_ERR_NOT_READY   -8   /* gauge / workspace / direction / deflation not set         */
#define LQ_ERR_NONFINITE   -9   /* (status) NaN or Inf met in a reduction                    */
#define LQ_ERR_NOT_CONVERGED -10 /* (status) an iterative solve stopped at its iteration cap  */

/* ---- internal precision ------------------------------------------------------------- */
#define LQ_FP64   0   /* stencil, vectors, dots, scalars and Newton all in FP64                */
#define LQ_MIXED  1   /* FP32 links, spinors and stencil (FP32 accumulation); FP64 compensated
                         dots, FP64 Lanczos coefficients, FP64 Newton, FP64 recombination      */
#define LQ_MIXED_BF16 2 /* as LQ_MIXED with the links stored in BF16 (real and imaginary parts,
                         4 bytes per complex entry).  The uploaded links are rounded once, FP64
                         -> FP32 (nearest) -> BF16 (nearest even), and every operator of the
                         context (stencil, derivative directions, adjoint force, eigensolver)
                         uses the rounded links: H(mu) of the rounded gauge field.  Stencil
                         schedules 6-8 are not available (schedule 3 runs instead)          */
#define LQ_FLOAT_FLOAT 3 /* links, spinors, stencil and update in float-float: pairs of FP32
                         numbers (hi + lo, about 48 significant bits) with compensated sums and
                         FMA-exact products, on the FP32 units (FP64 runs at 1/64 of their
                         rate on this GPU); dots in float-float, coefficients, Newton and
                         recombination in FP64.  Per-step rounding near 2^-47 instead of 2^-24:
                         the accuracy class of LQ_FP64 at a fraction of its time.  Stencil
                         schedules 0 (one thread per site and side), 1 and 2 (one thread per
                         site and output field, at least 3 / 4 blocks per SM); no split
                         loop.  The adjoint's pair vectors are recombined in FP64 and stored
                         in float-float; the force contraction runs in FP64              */

/* ---- derivative directions (d_t of Eq. (2.5)) --------------------------------------- */
#define LQ_DIR_MU   0   /* d/dmu: field unused                                               */
#define LQ_DIR_SU3  1   /* U_nu(x) -> exp(i t Omega_nu(x)) U_nu(x), Omega = sum_a w^a lambda_a/2;
                           field = double[4][V][8] coefficients w^a_nu(x)                      */
#define LQ_DIR_U1   2   /* U_nu(x) -> exp(i t theta_nu(x)) U_nu(x) (the external U(1) field of
                           Sec. 4); field = double[4][V]                                       */

typedef struct lq_ctx lq_ctx;

typedef struct {
    int nt, nx, ny, nz;    /* lattice extents, each >= 1                                     */
    double m_w;            /* Wilson mass (the paper's workloads: -2.0)                       */
    double r;              /* Wilson parameter; only r = 1 is supported (spin projectors)     */
    double mu;             /* chemical potential                                              */
    int t_antiperiodic;    /* 1: antiperiodic in time (default), 0: periodic                  */
    int precision;         /* LQ_FP64, LQ_MIXED, LQ_MIXED_BF16 or LQ_FLOAT_FLOAT             */
} lq_lattice_desc;

typedef struct {
    int kmax;              /* Krylov depth k = number of applications of the operator, and the
                              dimension of the projected tridiagonal T_k; 1 <= k <= reserved  */
    double breakdown_tol;  /* serious breakdown if |<w^,v^>| < tol |w^| |v^| (default 1e-14)   */
    int newton_max_iter;   /* cap on Newton iterations for sgn(T_k) (default 50)              */
    double newton_tol;     /* stop when ||X_{i+1}-X_i||_F <= tol ||X_{i+1}||_F (default 1e-13) */
    int deflate;           /* 1: deflate with the uploaded eigenpairs (Sec. 3): Eq. (3.1) for
                              the sign, Eqs. (3.2)-(3.4) for the derivative; 0: no deflation  */
    int projected;         /* solver for the projected sign sgn(T_k) e_1 (default LQ_PROJ_AUTO)  */
    int quad_nodes;        /* quadrature nodes N (default 64, at most 128)                      */
    double proj_tol;       /* accept the quadrature when ||Q(T)Q(T)e_1 - e_1|| <= proj_tol
                              (default 1e-11)                                                   */
    int hop_variant;       /* stencil schedule: -1 = autotuned on first use (default; the
                              autotuner leaves out 7 and 8, measured slower), 0 = one
                              thread per (site, side), 1 = one thread per (site, output field),
                              2 / 3 = as 0 with at least 5 / 4 resident blocks per SM, 4 = as
                              1 with 64 sites per block, 5 = as 1 with at least 5 resident
                              blocks per SM, 6 = shared-memory tiles of whole x rows x 2x2x2
                              (needs even y, z, t extents; else 3), 7 = as 3 in packed FP32
                              pair arithmetic (identical results), 8 = as 7 with the next
                              hop's neighbour spinors prefetched into shared memory, 9 = as 3
                              with both sides of 64 sites in one block (the second load of a
                              link hits L1).  2-9 are FP32 only (FP64 runs 0, 1; float-float
                              0, 1 and 2, where 1 / 2 are the one-thread-per-output-field
                              kernel at 3 / 4 blocks per SM, any other value runs 0);
                              lq_report.hop_variant gives the schedule that ran               */
    int defl_kmax;         /* depth of the shifted solves for the eigenvector derivatives of the
                              generalised deflation (0 = the reserved kmax)                    */
    int defl_nderiv;       /* Jordan blocks of the derivative deflation: the first defl_nderiv
                              uploaded pairs (0 = all); the shifted solves still project out all
                              uploaded pairs (the paper deflates the derivative with fewer pairs
                              than the sign, Sec. 4)                                           */
    int two_pass;          /* 1: two passes over the Krylov process with O(n) memory instead of
                              O(k n): the first keeps a ring of basis vectors and yields T_k,
                              the second reruns the (deterministic) process and recombines
                              windows of 16 vectors as they appear; twice the operator work.
                              Required for kmax beyond the ring of a LQ_RESERVE_TWO_PASS
                              workspace.  lq_sign_bilinear_grad (without deflation) keeps rings
                              of the right and the left basis and accumulates the pair vectors
                              of the force window by window in its second pass (default 0)  */
    int graph;             /* -1 / 1: the Krylov loop (2k - 1 launches) is captured once per
                              configuration into a CUDA graph and replayed (default -1); 0:
                              plain launches.  Off while lq_profile_enable times kernels.  The
                              first call of a configuration captures: make it outside any stream
                              capture of the caller's own                                    */
    int split;             /* -1 / 1: a derivative solve in FP32 with an even nsrc >= 8 runs the
                              Krylov loops of its two source halves as concurrent branches, so
                              that the bandwidth-bound update of one half overlaps the
                              issue-bound stencil of the other (default -1); 0: one batch.  Off
                              while lq_profile_enable times kernels, for two-pass runs and for
                              the adjoint.  Results differ from the unsplit run by FP32
                              rounding only (each half has its own reduction grids)           */
    int nested_m;          /* inner Krylov size of LQ_PROJ_NESTED and of that rung of LQ_PROJ_AUTO
                              (default 100, the paper's; capped by k and the reserved kmax)   */
    int update_variant;    /* FP32 Lanczos update kernel: 1 = inputs staged in shared memory by
                              bulk asynchronous copies, 0 = register-streaming kernel, -1
                              (default) = 1 for a loop run as one batch, 0 for the split loop
                              (the bulk kernel's shared memory would take the L1 of the stencil
                              running beside it).  The vectors are bitwise the same; the inner
                              products differ by the order of their partial sums              */
    int rebiorth;          /* 0 (default): plain three-term recurrences.  p > 0: the new pair
                              (vh, wh) of step j (v_{j+1}, counting from v_0) is made
                              biorthogonal to all earlier pairs when j + 1 or j (j > 0) is a
                              multiple of p, vh -= sum_i v_i <w_i, vh>, wh -= sum_i w_i <v_i,
                              wh>, before omega and the next beta, delta are formed (two
                              consecutive pairs per period: the recurrence builds each pair
                              from the last two); T keeps its three-term entries.  Costs
                              O(j n) bytes per corrected step (p = 1: every step, O(k^2 n) per
                              solve).  The projection's own rounding is amplified by the
                              condition |v_i| |w_i| of the pairs (FP32 data: float-float sums,
                              one rounding per stored element), so on strongly non-normal
                              kernels it can add more error than it removes: on the Wilson
                              kernel at 14^4, mu = 0.3, k = 400 it moves even float-float
                              results by 0.1.  It restores exactness where the bases stay
                              well conditioned.  Sign and derivative solves only (not the
                              adjoint, two-pass runs or lq_batch_apply); needs a workspace
                              reserved with LQ_RESERVE_REBIORTH (LQ_ERR_NOT_READY otherwise).
                              Runs with it do not split into source halves                    */
} lq_opts;

/* Projected step sgn(T_k) e_1 (Sec. 2):
 *  LQ_PROJ_NEWTON  scaled Newton iteration on the dense k x k matrix (FP64, O(k^3));
 *  LQ_PROJ_QUAD    midpoint quadrature of sgn(T) = (2/pi) T int_0^inf (t^2 + T^2)^{-1} dt
 *                  with t = c tan(theta): 2N complex tridiagonal solves (FP64, O(N k));
 *  LQ_PROJ_NESTED  the nested two-sided Lanczos process of Sec. 4 (one level of nesting): an
 *                  inner process of opts.nested_m steps from e_1 on M = T/c + c T^{-1} (a
 *                  function of T with the same sign), c = sqrt(|lambda|_min |lambda|_max)
 *                  estimated as for the quadrature, then the scaled Newton iteration on the
 *                  inner nested_m x nested_m tridiagonal; accepted per source only if the
 *                  involution residual of a second pass from the result is <= proj_tol
 *                  (O(m k) sequential work per source plus an m x m Newton);
 *  LQ_PROJ_AUTO    the quadrature, accepted per source only if its involution residual
 *                  ||Q(T) Q(T) e_1 - e_1|| <= proj_tol; a failing source is retried once
 *                  with 2048 nodes, then by the nested process, and only what still fails
 *                  goes to Newton on the k x k matrix.                                   */
#define LQ_PROJ_AUTO    0
#define LQ_PROJ_NEWTON  1
#define LQ_PROJ_QUAD    2
#define LQ_PROJ_NESTED  3

typedef struct {
    int k_eff;             /* dimension of T actually built (< kmax after a breakdown)        */
    int newton_iters;      /* Newton iterations taken on sgn(T_k) (0 if not used)             */
    int status;            /* LQ_OK, LQ_ERR_BREAKDOWN, LQ_ERR_NEWTON or LQ_ERR_NONFINITE      */
    int projected;         /* solver that produced sgn(T_k) e_1: LQ_PROJ_NEWTON, LQ_PROJ_QUAD or
                              LQ_PROJ_NESTED                                                  */
    double newton_change;  /* last relative Frobenius change of the Newton iterate            */
    double x_norm;         /* |x| of the source                                               */
    double proj_check;     /* involution residual of the quadrature or of the nested process
                              that produced the result (0 if neither was attempted)            */
    int hop_variant;       /* stencil schedule used (see lq_opts.hop_variant)                  */
    int reserved;
} lq_report;

typedef struct {
    int kind;              /* LQ_DIR_MU, LQ_DIR_SU3 or LQ_DIR_U1                              */
    const double* field;   /* see the LQ_DIR_* descriptions; host or device memory           */
} lq_direction;

/* Fill *opts with the defaults named above (kmax = 0 must still be set by the caller). */
void lq_default_opts(lq_opts* opts);

/* Create a context on the current CUDA device for the lattice and Wilson parameters of
 * Sec. 1 (Eq. (1.1)).  Allocates nothing on the device.  Returns LQ_ERR_ARG for extents
 * < 1, r != 1 or an unknown precision. */
int  lq_create(const lq_lattice_desc* desc, lq_ctx** out);
void lq_destroy(lq_ctx* ctx);
const char* lq_last_error(const lq_ctx* ctx);

/* Upload the SU(3) gauge field (layout above, host or device).  Allocates the device copy
 * in the internal layout and precision on first use.  Asynchronous on `stream`. */
int  lq_upload_gauge(lq_ctx* ctx, const double* U, void* stream);

/* Change mu (Eq. (1.1)) without re-uploading the gauge field. */
int  lq_set_mu(lq_ctx* ctx, double mu);

/* Reserve all workspace for Krylov depth <= kmax and <= nsrc sources per call.  flags:
 * LQ_RESERVE_BLOCK for the derivative path (2n-dimensional block vectors of Eq. (2.6)),
 * LQ_RESERVE_ADJOINT for lq_sign_bilinear_grad (stored left basis, nsrc >= 2); 0 for the sign
 * path only.  LQ_RESERVE_TWO_PASS keeps a ring of 32 basis vectors per source instead of kmax
 * (runs deeper than 32 then need lq_opts.two_pass = 1; with LQ_RESERVE_ADJOINT the stored left
 * basis becomes a ring of 32 as well).  No later
 * solve call allocates device memory.  LQ_ERR_OOM on failure. */
#define LQ_RESERVE_BLOCK    1
#define LQ_RESERVE_ADJOINT  2
#define LQ_RESERVE_TWO_PASS 4
#define LQ_RESERVE_SOLVE    8   /* nine more FP64 fields per source for lq_overlap_solve and
                                   lq_axial_current */
#define LQ_RESERVE_REBIORTH 16  /* the whole left basis (kmax vectors per source, NF fields each)
                                   and the dot scratch for lq_opts.rebiorth; LQ_ERR_ARG together
                                   with a two-pass ring (LQ_RESERVE_TWO_PASS and kmax > 32) */
int  lq_reserve(lq_ctx* ctx, int kmax, int nsrc, int flags);

/* y = H(mu) x (dagger = 0) or y = H(mu)^dag x = H(-mu) x (dagger = 1) for nsrc fields
 * (Eq. (1.1)); the single stencil application.  Needs the gauge field and lq_reserve(nsrc). */
int  lq_apply_H(lq_ctx* ctx, const double* x, double* y, int nsrc, int dagger, void* stream);

/* Set the derivative direction d_t (Eq. (2.5)): for LQ_DIR_SU3 / LQ_DIR_U1 the library
 * builds dU/dt = i Omega U on the device.  Must follow lq_upload_gauge. */
int  lq_set_direction(lq_ctx* ctx, const lq_direction* dir, void* stream);

/* Apply the block operator B = [[A, dA], [0, A]] of Eq. (2.5) with A = H(mu) and dA the
 * derivative of H along the current direction (dagger = 0), or B^dag (dagger = 1), to
 * nsrc stacked vectors (top, bottom), each half in the spinor layout. */
int  lq_apply_block(lq_ctx* ctx, const double* x_top, const double* x_bot,
                    double* y_top, double* y_bot, int nsrc, int dagger, void* stream);

/* y ~ sgn(H(mu)) x by the two-sided Lanczos method of Sec. 2: k steps from
 * v_1 = w_1 = x/|x|, then y = |x| V_k sgn(T_k) e_1 with sgn(T_k) from a scaled FP64 Newton
 * iteration on the device.  x, y: nsrc fields.  report: host array of nsrc entries (may be
 * NULL).  Synchronises `stream`. */
int  lq_sign_apply(lq_ctx* ctx, const double* x, double* y, int nsrc,
                   const lq_opts* opts, lq_report* report, void* stream);

/* Eq. (2.6): sgn(B)(0, x) = (d_t sgn(H) x, sgn(H) x) by the two-sided Lanczos method on the
 * 2n x 2n block operator B of Eq. (2.5), with v_1 = (0, x)/|x| and w_1 = (x, x)/|x|, along
 * `dir` (which replaces the current direction).  y_sign, y_deriv: nsrc fields each.
 * Needs lq_reserve(..., block = 1).  Synchronises `stream`. */
int  lq_sign_derivative_apply(lq_ctx* ctx, const lq_direction* dir, const double* x,
                              double* y_sign, double* y_deriv, int nsrc,
                              const lq_opts* opts, lq_report* report, void* stream);

/* Upload the l eigenpairs of A = H(mu) closest to zero for the deflation of Sec. 3:
 * lambda: host double[l][2]; R: right eigenvectors (A R_i = lambda_i R_i), spinor layout
 * double[l][V][4][3][2]; L: the left eigenvectors as kets, Lk_i = L_i^dag (so L_i A = lambda_i L_i
 * and <Lk_i|R_j> = delta_ij), same layout.  Host or device memory; copied (FP64).  l = 0 removes
 * the space.  Used by lq_sign_apply and lq_sign_derivative_apply when opts->deflate = 1.  Must
 * follow lq_reserve; lq_compute_deflation below computes such a space itself. */
int  lq_upload_deflation(lq_ctx* ctx, int l, const double* lambda, const double* R, const double* L,
                         void* stream);

/* Eigensolver of lq_compute_deflation. */
#define LQ_EIG_SHIFT_INVERT 0   /* implicitly restarted Arnoldi on H^{-1} (default)               */
#define LQ_EIG_CHEBYSHEV    1   /* Chebyshev-filtered subspace iteration on H^2                    */

/* Options of lq_compute_deflation. */
typedef struct {
    int nev;          /* eigenpairs wanted: the nev eigenvalues of H(mu) closest to zero          */
    int nsub;         /* shift-and-invert: Arnoldi basis size m (nev + 4 <= m <= 63; default
                         min(2 nev + 10, 63)).  Chebyshev: subspace size (nev + 2 <= nsub <= 64;
                         default min(nev + 12, 64))                                              */
    int degree;       /* Chebyshev filter degree in H^2 (default 40; unused by shift-and-invert)  */
    int max_iter;     /* restarts (shift-and-invert, default 300) or filtered subspace iterations
                         (Chebyshev, default 60)                                                   */
    double tol;       /* stop when ||H r - lambda r|| <= tol * ||H||_est for the nev pairs
                         (default 1e-10; the eigensolver's FP64 stencil runs in both precisions)  */
    int method;       /* LQ_EIG_SHIFT_INVERT (default, 0) or LQ_EIG_CHEBYSHEV                      */
    int inner_max;    /* shift-and-invert: iteration cap of each FP32 inner solve (0: 20000)      */
} lq_eig_opts;

/* Statistics of the last lq_compute_deflation of a context (lq_eig_stats_read). */
typedef struct {
    int method;              /* the eigensolver that ran                                          */
    int restarts;            /* Arnoldi restarts (shift-and-invert)                                */
    long long solves;        /* operator inverse applications, both processes together            */
    long long inner_iterations; /* FP32 CGNR iterations over all solves                           */
    long long refinements;   /* FP64 defect-correction steps over all solves                       */
    double norm_estimate;    /* ||H||_est, the scale of the reported residuals                     */
    double max_residual;     /* largest returned residual                                           */
    double pair_mismatch;    /* largest |lambda_i - conj(lambda'_j)| / |lambda_i| of the pairing of
                                right and left eigenvalues                                          */
    double seconds;          /* device time of the call                                             */
} lq_eig_stats;

/* Compute and install the deflation space of Sec. 3 with the library's own eigensolver (the
 * paper uses ARPACK's Arnoldi): the nev right eigenpairs of H(mu) closest to zero and the
 * matching left eigenvectors (from H(mu)^dag = H(-mu)), biorthonormalised so that
 * <Lk_i|R_j> = delta_ij.  Methods (eo->method):
 *   LQ_EIG_SHIFT_INVERT: ARPACK's method, the implicitly restarted Arnoldi process with exact
 *     shifts, on OP = H^{-1} (the wanted eigenvalues are the largest of OP, which polynomial
 *     methods cannot isolate when the spectrum surrounds zero) and on (H^dag)^{-1} for the left
 *     vectors, both in lockstep.  Each OP application is an FP64 solve: defect correction whose
 *     corrections are FP32 CGNR solves (conjugate gradients on H^dag H).  X0: two start fields
 *     (right, left).
 *   LQ_EIG_CHEBYSHEV: Chebyshev-filtered subspace iteration on H^2 with Rayleigh-Ritz
 *     (lq_dense_eig); converges only when the wanted eigenvalues are not surrounded by the rest
 *     of the spectrum.  X0: nsub start fields.
 * X0: host or device, spinor layout double[.][V][4][3][2] (random numbers are the caller's).
 * lambda, resid: host outputs double[nev][2] and double[nev] (may be NULL); resid is the larger of
 * the right and left residuals ||H r - lambda r|| / ||H||_est.  The FP64 operator applications run
 * in FP64 whatever the context's precision (a mixed-precision context converts its FP64 copy of
 * the links for the call): the generalised deflation of the derivative needs eigenpairs accurate
 * to FP64 rounding.  Allocates its own temporary workspace (a set-up call).  Synchronises. */
int  lq_compute_deflation(lq_ctx* ctx, const lq_eig_opts* eo, const double* X0, double* lambda,
                          double* resid, void* stream);

/* Statistics of the context's last lq_compute_deflation (no device work). */
int  lq_eig_stats_read(const lq_ctx* ctx, lq_eig_stats* out);

/* The massless overlap operator at finite density, Eq. (1.1) with lattice spacing 1:
 *   y = D_ov x = x + gamma5 sgn(H(mu)) x,   dy = d D_ov x = gamma5 d_t sgn(H(mu)) x,
 * the sign (and its derivative along `dir`, Eqs. (2.5)-(2.6)) by the two-sided Lanczos process
 * with the options and reports of lq_sign_apply / lq_sign_derivative_apply (deflation included).
 * dy may be NULL (then dir may be NULL and only y is computed; the workspace needs no
 * LQ_RESERVE_BLOCK).  x, y, dy: double[nsrc][V][4][3][2], host or device.  Synchronises. */
int  lq_overlap_apply(lq_ctx* ctx, const lq_direction* dir, const double* x, double* y, double* dy, int nsrc,
                      const lq_opts* opts, lq_report* rep, void* stream);

/* Per-source outcome of an overlap solve. */
typedef struct {
    int iterations;        /* BiCGStab iterations (two operator applications each)            */
    int status;            /* LQ_OK, LQ_ERR_NOT_CONVERGED, LQ_ERR_BREAKDOWN or a status of the
                              inner sign solves                                                */
    double residual;       /* ||b - D(m) z|| / ||b|| recomputed with one more application      */
} lq_solve_report;

/* z = D(m)^{-1} b for nsrc sources: the overlap operator with a bare mass,
 *   D(m) = (1 - m/2) D_ov + m,   D_ov = 1 + gamma5 sgn(H(mu))   (Eq. (1.1), lattice spacing 1),
 * mass = 0 giving the paper's massless operator.  BiCGStab with per-source scalars; every
 * application of D(m) is one batched two-sided Lanczos solve for sgn(H) x with opts (deflated with
 * the installed eigenpairs when opts->deflate = 1).  The Lanczos approximation at a fixed depth
 * is not linear in x, so the solve converges only down to the accuracy of that approximation:
 * choose opts->kmax (or deflation) so that sgn(H) is as accurate as tol asks.  Stops for a source
 * when ||r|| <= tol ||b|| or after max_iter iterations.  b, z: double[nsrc][V][4][3][2], host or
 * device.  Needs lq_reserve(..., LQ_RESERVE_SOLVE).  rep: nsrc entries (may be NULL).
 * Synchronises `stream`. */
int  lq_overlap_solve(lq_ctx* ctx, const double* b, double* z, int nsrc, double mass, double tol, int max_iter,
                      const lq_opts* opts, lq_solve_report* rep, void* stream);

/* Stochastic estimates of the conserved axial current of the paper's conclusion,
 *   J = Tr(D(m)^{-1} dD(m)/dt gamma5),   dD(m)/dt = (1 - m/2) gamma5 d_t sgn(H(mu)),
 * along the direction `dir` (for the current through the links that a U(1) field theta moves,
 * LQ_DIR_U1): out[s] = eta_s^dag D(m)^{-1} dD(m) gamma5 eta_s for each noise vector eta_s (Z2 noise
 * gives an unbiased estimate of J; the random numbers are the caller's).  Per source: one
 * derivative solve (Eq. (2.6)) for d sgn(H) gamma5 eta, then lq_overlap_solve's BiCGStab.  eta:
 * double[nsrc][V][4][3][2], host or device; out: host double[nsrc][2] (complex).  Needs
 * lq_reserve(..., LQ_RESERVE_BLOCK | LQ_RESERVE_SOLVE).  Synchronises `stream`. */
int  lq_axial_current(lq_ctx* ctx, const lq_direction* dir, const double* eta, int nsrc, double mass, double tol,
                      int max_iter, const lq_opts* opts, double* out, lq_solve_report* rep, void* stream);

/* One member of a ragged batch (lq_batch_apply). */
typedef struct {
    lq_ctx* ctx;               /* the member's own context: lattice, links, mu, precision and
                                  workspace; each context at most once per batch               */
    const lq_direction* dir;   /* direction of d_t (Eq. (2.6)), or NULL for sgn(H) x alone     */
    const double* x;           /* double[nsrc][V][4][3][2] sources, host or device            */
    double* y_sign;            /* sgn(H(mu)) x, same layout, host or device                   */
    double* y_deriv;           /* d_t sgn(H(mu)) x when dir != NULL (else unused)             */
    int nsrc;                  /* sources of this member, 1 <= nsrc <= its reserved nsrc      */
    const lq_opts* opts;       /* opts->kmax is this member's Krylov depth; deflate and two_pass
                                  must be 0                                                     */
    lq_report* report;         /* host array of nsrc reports, or NULL                         */
} lq_batch_item;

/* Up to LQ_BATCH_MAX independent two-sided Lanczos problems (Sec. 2) at once: lattices of
 * different extents and parameters, with their own sources and Krylov depths.  Member i gives
 * exactly (bit for bit) what lq_sign_derivative_apply (dir != NULL) or lq_sign_apply (dir ==
 * NULL) gives with the same context and options: the same kernels, stencil schedule and
 * reduction order.  The Krylov loops of all members (2k_i - 1 launches each) are one CUDA graph
 * with one branch per member, captured the first time the batch configuration is met (the
 * contexts, and per member k, nsrc, direction kind, stencil schedule and mu) and replayed with a
 * single launch on `stream`; the branches are independent, so the GPU runs the members' kernels
 * side by side and small lattices fill it together.  With opts->graph = 0 for some member, or
 * kernel timing on for some context (lq_profile_enable), the loops run as plain launches on
 * per-context streams forked from and joined into `stream`.  The projected signs and the
 * recombinations follow on the same per-context streams.  No device allocation beyond
 * lq_reserve's, except the first capture of a configuration (the CUDA graph; at most 8 batch
 * configurations are kept, dropped when a member context is reserved again or destroyed).
 * Errors: LQ_ERR_ARG for n outside [1, LQ_BATCH_MAX], a null member context or buffer, a
 * context named twice, members on different devices, or deflate / two_pass set; a member's
 * own errors as in the single-problem calls, stored on that context (lq_last_error).
 * Synchronises `stream`. */
#define LQ_BATCH_MAX 16
int  lq_batch_apply(const lq_batch_item* items, int n, void* stream);

/* The derivatives of the uploaded eigenpairs along `dir` (end of Sec. 3), as used by the
 * generalised deflation: dlambda_i = L_i E R_i; dR_j = sum_{i != j} R_i (L_i E R_j)/(lambda_j -
 * lambda_i) + Pbar (lambda_j - A)^{-1} Pbar E R_j and its left analogue, with the shifted solves on
 * the deflated complement done by two-sided Lanczos approximations of the resolvent at depth
 * opts->kmax (Sec. 2 with f(a) = 1/(lambda_j - a)).  Outputs (host or device, may be NULL):
 * dlambda double[l][2]; dR, dL (kets of dL_i) double[l][V][4][3][2].  Synchronises `stream`. */
int  lq_deflation_derivatives(lq_ctx* ctx, const lq_direction* dir, const lq_opts* opts,
                              double* dlambda, double* dR, double* dL, void* stream);

/* Opt-in timing of the library's own kernels with CUDA events recorded on the launch
 * stream (no effect on results).  Enabling resets the totals.  Times are accumulated when a
 * reporting call synchronises its stream.  launches counts every kernel the library has
 * launched since the last reset, whether or not timing is enabled. */
typedef struct {
    int enabled;
    int reserved;
    long long launches;        /* kernel launches since the last reset                      */
    double hop_ms;             /* stencil kernel (H, H^dag, block operator; Eq. (1.1)/(2.5)) */
    long long hop_launches;
    double update_ms;          /* Lanczos three-term update + omega dot                      */
    long long update_launches;
    double newton_ms;          /* projected sign sgn(T_k), all Newton kernels               */
    long long newton_iterations;
    double other_ms;           /* start vectors, recombination, layout conversion            */
    long long other_launches;
} lq_profile;

int  lq_profile_enable(lq_ctx* ctx, int enable);
int  lq_profile_read(lq_ctx* ctx, lq_profile* out);

/* The bilinear S = Re <y| sgn(H(mu)) |x> and its gradient: the fermionic force
 * force[nu][s][a] = dS/dw^a for U_nu(s) -> exp(i w^a lambda_a/2) U_nu(s) (the use named in
 * Secs. 1 and 5), and dS/dmu.  Uses dS/dt = Re tr(E L_sgn(H, x y^H)) with the Krylov
 * approximation L ~ |x||y| V_1 X W_2^H: V_1, T_1 from the Lanczos process started at x, W_2, T_2
 * from the process started at y, X the top-right block of sgn([[T_1, e_1 e_1^T], [0, T_2]]) by
 * Mathias' identity (Eq. (2.5)), evaluated by the quadrature of the projected sign (2 quad_nodes
 * rank-one terms).  With opts->deflate = 1 the installed eigenpairs (Sec. 3) split
 * L_sgn(H, x y^H) by the spectral projectors Pi = sum_j R_j L_j, Pbar = 1 - Pi: the deflated block
 * exactly (divided differences of sgn at the eigenvalues), the two mixed blocks through
 * (sgn z - sgn lambda_j) / (z - lambda_j) of the two Lanczos runs, and the rest by the Krylov route
 * on the deflated sources Pbar x, Pbar^H y; S is deflated by Eq. (3.1).  This needs
 * 2 quad_nodes + 3 l <= 256.  With opts->two_pass = 1 (no deflation; workspace reserved with
 * LQ_RESERVE_ADJOINT | LQ_RESERVE_TWO_PASS) both processes run twice with rings of 32 right and
 * left basis vectors: the first pass gives T_1, T_2 and the projected sign, the second reruns them
 * and accumulates the 2N pair vectors of the contraction window by window (O(n) memory, twice
 * the operator work).  x, y: one field each (host or device); S, dS_dmu: host double*; force:
 * double[4][V][8] (host or device, may be NULL).  Needs lq_reserve(kmax, nsrc >= 2,
 * LQ_RESERVE_ADJOINT).  Synchronises `stream`. */
int  lq_sign_bilinear_grad(lq_ctx* ctx, const double* x, const double* y, const lq_opts* opts,
                           double* S, double* force, double* dS_dmu, void* stream);

/* Copy the projected tridiagonal T_k of source `src` from the last lq_sign_apply /
 * lq_sign_derivative_apply (Sec. 2): alpha[j] = T[j][j], beta[j] = T[j][j+1],
 * delta[j] = T[j+1][j] (real, > 0).  alpha, beta: host double[k][2] (complex); delta:
 * host double[k].  Entries beyond the source's k_eff are zero.  Synchronous. */
int  lq_tsl_coefficients(lq_ctx* ctx, int src, int k, double* alpha, double* beta, double* delta);

/* The self-check of Sec. 4: eps_A = ||sgn(A)^2 psi - psi|| / (2 ||psi||), each sgn(A) one TSL
 * approximation of depth opts->kmax.  dir == NULL: the sign (two lq_sign_apply solves).
 * dir != NULL: the derivative version with B of Eq. (2.5) and the source (0, x): the second
 * application to the non-sparse (y_d, y_s) = sgn(B)(0, x) is taken by linearity,
 * sgn(B)(y_d, y_s) = (sgn(A) y_d + d_t sgn(A) y_s, sgn(A) y_s) (two derivative solves and one
 * sign solve).  x: nsrc fields (host or device); eps: host double[nsrc].  Needs
 * lq_reserve(..., block = 1) for the derivative version.  Synchronises `stream`. */
int  lq_error_estimate(lq_ctx* ctx, const lq_direction* dir, const double* x, int nsrc,
                       const lq_opts* opts, double* eps, void* stream);

/* Host-only utility (no GPU): eigenvalues w[n][2] and unit right eigenvectors V (columns,
 * row-major double[n][n][2], may be NULL) of a general complex matrix A double[n][n][2]
 * (row-major), by Householder reduction to Hessenberg form and the shifted QR algorithm.
 * Used for the Rayleigh-Ritz steps of lq_compute_deflation.  LQ_ERR_NEWTON if QR does not
 * converge. */
int  lq_dense_eig(int n, const double* A, double* w, double* V);

/* Batched dense FP64 sign of nb complex k x k matrices by the scaled Newton iteration
 * X <- (m X + (m X)^{-1})/2, m = sqrt(||X^{-1}||_F / ||X||_F) (Higham 2008, ch. 5; the
 * projected step of the Lanczos approximation, Sec. 2).  X, S: double[nb][k][k][2]
 * row-major, device memory only.  Uses workspace reserved by lq_reserve(ctx, kmax >= k,
 * nsrc >= nb, ...).  iters (host, nb entries, may be NULL) receives the iteration counts.
 * Synchronises `stream`. */
int  lq_newton_sign(lq_ctx* ctx, const double* X, double* S, int k, int nb,
                    int max_iter, double tol, int* iters, void* stream);

/* sgn(T) e_1 of nb complex tridiagonal k x k matrices by the nested two-sided Lanczos process of
 * LQ_PROJ_NESTED (Sec. 4): m inner steps on M = T/c + c T^{-1} from e_1, the inner projected sign
 * by the scaled Newton iteration, and the involution residual of a second pass.
 * alpha: diagonal double[nb][k][2]; beta: super-diagonal double[nb][k-1][2]; delta: real
 * sub-diagonal double[nb][k-1] (the layout of lq_tsl_coefficients); scale: double[nb], the c of
 * each matrix, or NULL for the library's estimate of sqrt(|lambda|_min |lambda|_max); host or
 * device.  out: double[nb][k][2] (host or device); check: host double[nb] (may be NULL).
 * Needs a workspace reserved with kmax >= k, nsrc >= nb and kmax >= m; overwrites the projected
 * coefficients of the context's last solve (lq_tsl_coefficients).  Returns LQ_ERR_NEWTON if an
 * inner Newton iteration did not converge.  Synchronises. */
int  lq_nested_sign(lq_ctx* ctx, const double* alpha, const double* beta, const double* delta,
                    const double* scale, int k, int nb, int m, double* out, double* check, void* stream);

/* Allocation-free variant of lq_newton_sign, for callers that cannot allocate device
 * memory: for example a process whose device memory is handed in full to a pool allocator
 * (a framework's caching allocator), where a cudaMalloc of the library's own would fail or
 * fragment the pool, or a service that forbids allocation after start-up.  The paper has no
 * counterpart: this entry point only changes where the workspace lives.
 *   - Needs no context and calls no cudaMalloc / cudaFree or other allocating routine.  Its
 *     workspace is one static device array of about 4.2 MB that every GPU loading the
 *     library holds until the process exits.
 *   - Limits: k <= 128 and nb <= 8; larger sizes return LQ_ERR_ARG and run nothing.
 *   - The first call on a device looks up the array's device address for that device
 *     (cudaGetSymbolAddress, with that device current); make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array and it keeps the last call's contents (the
 *     call clears what must start at zero).  Calls that overlap on the GPU -- from several
 *     host threads or on several streams at once -- race on it and give wrong results:
 *     serialise them.
 * X, S: device double[nb][k][k][2] row-major; iters: host int[nb] or NULL.  Returns LQ_OK,
 * LQ_ERR_ARG, LQ_ERR_LAYOUT if X or S is not device memory (checked before any launch),
 * LQ_ERR_CUDA, or LQ_ERR_NEWTON if a matrix did not converge.  Synchronises `stream`. */
int  lq_newton_sign_noalloc(const double* X, double* S, int k, int nb, int max_iter, double tol,
                            int* iters, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LQ_H */
