/*
 * fcrkpm.h -- C ABI of the GB300 fast-convolving RKPM library (FC-RKPM,
 * arXiv 2403.19854): the matrix-free Galerkin operator of the 3D Poisson problem
 * (Eq. 8-9) written as circular convolutions on a periodic node box (Sec. 4),
 * evaluated with FFTs on the GPU, and the conjugate-gradient solve around it
 * (Alg. 5).
 *
 * Conventions shared by every entry point
 *  - Grid: a periodic box of n[0] x n[1] x n[2] nodes with spacing h[k]
 *    (Eq. 70), x fastest: a field is an array of n0*n1*n2 values indexed
 *    i + n0*(j + n1*k).  n[0] must be even and n[1]*n[2] even; each n[k] must be
 *    one of the FFT line lengths the library was built for (rk_supported_length).
 *  - Domain: chi (Eq. 40) is 1 on the nodes of Omega and 0 on the gap; chi_gamma
 *    (Eq. 95) is 1 on the nodes where d = g is imposed (Eq. 29), a subset of chi.
 *    The gap must be at least l_e = (floor(a_tilde) + 1) h wide on every axis
 *    (Eq. 66): a node of Omega may not see another node of Omega across the
 *    periodic boundary within the support; rk_setup checks this.
 *  - Basis: degree 1 (s = 4, H = [1, x, y, z]) or 2 (s = 10, H = [1, x, y, z,
 *    x^2, xy, xz, y^2, yz, z^2]), Eq. 4-5, evaluated on the scaled offset
 *    (x - x_I)/a (each monomial divided by a^|alpha|; Psi is unchanged).  Kernel:
 *    tensor cubic B-spline of Eq. 6-7 with a_k = a_tilde * h[k] (Eq. 64).
 *  - Pointers: every array argument may be a host pointer or a device pointer of
 *    the current device (the library asks the CUDA driver which).  Device
 *    arrays are used in place and must be aligned to 16 bytes; host arrays are
 *    staged through library-owned device buffers and the call returns only after
 *    the host output is written.  The caller owns all arrays it passes; the
 *    handle owns everything it allocates.
 *  - Streams: stream is a cudaStream_t (NULL = legacy default stream).  Work on
 *    device arrays is stream-ordered; calls that report a convergence status
 *    (rk_solve, rk_solve_adjoint) synchronise the stream before returning.
 *  - Errors: no call aborts or prints.  Every call returns an rk_status;
 *    rk_status_string() names it and rk_last_error_message() describes the last
 *    failure of the calling thread.
 *  - Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef FCRKPM_H
#define FCRKPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rk_status {
  RK_OK = 0,
  RK_ERR_INVALID_ARG = 1,      /* bad pointer, size, alignment or option */
  RK_ERR_CUDA = 2,             /* a CUDA runtime call failed */
  RK_ERR_OOM = 3,              /* device allocation failed */
  RK_ERR_SINGULAR_MOMENT = 4,  /* M(x) not positive definite at some node of Omega */
  RK_ERR_NOT_CONVERGED = 5,    /* iteration cap reached before the tolerance */
  RK_ERR_BREAKDOWN = 6,        /* CG breakdown: p^T A p <= 0 or not finite */
  RK_ERR_TIMEOUT = 7,          /* a bounded device-side wait ran out: a pass waited too
                                  long for an input tile (the TMA tiles of the y/z
                                  passes, the bulk row copies of the x passes inside
                                  CG); the kernel gave up and the result is invalid.
                                  Reported by the next call of the handle that
                                  synchronises (solves, calls with host arrays). */
  RK_ERR_UNSUPPORTED = 8       /* grid size not built, gap too narrow, odd n[0] ... */
} rk_status;

typedef enum rk_dtype { RK_F64 = 0, RK_F32 = 1 } rk_dtype;

typedef enum rk_precision {
  RK_PREC_FP64 = 0,  /* every convolution and CG vector in FP64 */
  RK_PREC_MIXED = 1  /* FP32 convolutions and CG vectors, FP64 dots, FP64 refinement */
} rk_precision;

typedef struct rk_grid {
  int32_t n[3]; /* box nodes per axis */
  double h[3];  /* node spacing per axis */
} rk_grid;

typedef struct rk_handle rk_handle;

/* Preconditioner of the CG solve.  The paper's Alg. 5 runs plain CG; the spectral
 * preconditioner is an addition of this library (see rk_apply_precond). */
typedef enum rk_precond {
  RK_PRECOND_NONE = 0,
  RK_PRECOND_SPECTRAL = 1
} rk_precond;

typedef struct rk_solve_opts {
  double tol;         /* stop when ||F - A d||_2 / ||F||_2 <= tol, FP64 residual (default 1e-10) */
  int32_t max_iter;   /* cap on CG iterations, all refinement steps together (default 200000) */
  int32_t precision;  /* rk_precision (default RK_PREC_MIXED) */
  double inner_tol;   /* mixed: the FP32 CG residual is replaced by the true FP64 residual each time
                         it has dropped by this factor (default 0.1) */
  int32_t max_outer;  /* mixed: cap on refinement steps (default 60) */
  int32_t check_every;/* iterations between host-side convergence checks (default 25) */
  int32_t x0_given;   /* 1: on entry d holds an initial guess on the free nodes */
  int32_t fp64_finish;/* mixed: 1 (default) finishes with FP64 CG from the current iterate
                         when the FP32 iterations stop reducing the FP64 residual (three
                         replacements in a row without halving it, or max_outer reached);
                         0 returns RK_ERR_NOT_CONVERGED there instead */
  int32_t precond;    /* rk_precond: RK_PRECOND_NONE (default, the plain CG of Alg. 5) or
                         RK_PRECOND_SPECTRAL (see rk_apply_precond) */
  int32_t reserved;   /* 0 */
} rk_solve_opts;

typedef struct rk_solve_info {
  int32_t iterations;   /* CG iterations (inner iterations in mixed mode) */
  int32_t outer;        /* refinement steps (mixed) */
  int32_t matvec_f32;   /* FP32 K.u applications */
  int32_t matvec_f64;   /* FP64 K.u applications */
  double rel_residual;  /* final ||F - A d|| / ||F|| in FP64 */
  double f_norm;        /* ||F||, F = chi_Omega (f^r - K d_Gamma) */
  double setup_ms;      /* unused by rk_solve (0) */
  double solve_ms;      /* wall time of the call on the stream */
  int32_t status;       /* rk_status of the solve */
  int32_t fp64_iterations; /* FP64 CG iterations (included in iterations): all of
                              them for RK_PREC_FP64; for mixed, those run after the
                              FP32 iterations stopped reducing the FP64 residual
                              (0 when the mixed scheme alone reached tol) */
} rk_solve_info;

/* Default options (tol 1e-10, mixed precision). */
void rk_default_solve_opts(rk_solve_opts* opts);

/* 1 if the library holds FFT kernels for a box side of n nodes, else 0. */
int rk_supported_length(int n);

/*
 * rk_setup -- Alg. 1 and the "Initialize" block of Alg. 5.
 * Builds the per-axis kernel tables (the separable factors of H_p, H^a_p and
 * their spectra, Eq. 72-79), the moment fields M_pq = (1 - chi) delta_pq +
 * chi o F^-1[F(chi) o F(H_p o H^a_q)] (Eq. 80) in FP64, solves the s x s system
 * at every node (FP64 Cholesky) and stores b^0, b^x, b^y, b^z (Eq. 83-85) in FP64
 * and FP32, plus chi*V (Eq. 87).
 *   grid       box size and spacing; n[2] == 1 makes the problem two-dimensional
 *              (Sec. 6.1.2: no z axis, kernel phi(x)phi(y), basis [1, x, y] or
 *              [1, x, y, x^2, xy, y^2], b^z = 0, V the 2D cell measure); n[1] ==
 *              n[2] == 1 makes it one-dimensional (Sec. 6.1.1: kernel phi(x), basis
 *              [1, x] or [1, x, x^2], b^y = b^z = 0, V the 1D cell length; n[0] a
 *              multiple of 4); n[0] == 1, or n[1] == 1 < n[2], is invalid
 *   chi        uint8[nbox], Eq. 40
 *   chi_gamma  uint8[nbox], Eq. 95 (NULL: no Dirichlet nodes)
 *   V          double[nbox], nodal volumes of direct nodal integration (Eq. 54, 87)
 *   degree     1 or 2 (Eq. 4-5)
 *   a_tilde    support in units of h (Eq. 64), 0.5 < a_tilde < 16
 *   stream     cudaStream_t for the set-up work (synchronised before return)
 *   out        receives the handle
 * Errors: RK_ERR_INVALID_ARG, RK_ERR_UNSUPPORTED (size not built, odd sizes, gap
 * narrower than Eq. 66, a 1D side not a multiple of 4), RK_ERR_OOM, RK_ERR_CUDA, RK_ERR_SINGULAR_MOMENT (the
 * handle is still returned; rk_singular_nodes gives the count and first node).
 */
rk_status rk_setup(const rk_grid* grid, const uint8_t* chi, const uint8_t* chi_gamma, const double* V,
                   int32_t degree, double a_tilde, void* stream, rk_handle** out);

/* Number of nodes of Omega whose moment matrix was singular, and the flat index
 * of the first one (-1 if none). */
rk_status rk_singular_nodes(const rk_handle* h, int64_t* count, int64_t* first);

/*
 * rk_apply_K -- Alg. 2: f^int = K d (Eq. 57, 91) with direct nodal integration.
 *   d  [nbox] coefficients (values off chi are ignored: Eq. 91 uses chi o d)
 *   f  [nbox] output, 0 off chi
 *   dtype  RK_F64: double arrays, FP64 path;  RK_F32: float arrays, FP32 path
 */
rk_status rk_apply_K(rk_handle* h, const void* d, void* f, int32_t dtype, void* stream);

/*
 * rk_apply_precond -- z = M^{-1} r, the spectral preconditioner of
 * RK_PRECOND_SPECTRAL (no counterpart in the paper, whose Alg. 5 runs plain CG):
 *   z = chi_Omega o F^{-1}[ F(r) / (lam + shift) ]
 * with F the 3D DFT of the periodic box (Eq. 30), lam(theta) = V sum_k |D^_k(theta)|^2
 * the eigenvalues of K on a box of regular nodes (whole support in chi, interior V;
 * D^_k = sum_p b^k_p prod_axis T^_{alpha(p)}, the DFTs of the separable kernel
 * tables of Eq. 77-79 and the interior correction coefficients of Eq. 83-85), and
 * shift = 1e-3 lam(2 pi / n_x, 0, 0), which keeps the constant mode invertible.  M^{-1}
 * is symmetric positive definite on chi_Omega, as PCG requires.
 * r, z: box arrays (x fastest) of dtype RK_F64 or RK_F32, host or device.
 * Errors: RK_ERR_UNSUPPORTED when the domain has no regular node, a box side
 * exceeds 256, or the box is two-dimensional.
 */
rk_status rk_apply_precond(rk_handle* h, const void* r, void* z, int32_t dtype, void* stream);

/* rk_rhs -- Alg. 4 with the reflected kernel of Eq. 60/92:
 * f^r = chi o F^-1[ sum_p F(chi o V o b^0_p o r) o F(Hbar^a_p) ].  r, fr: double[nbox]. */
rk_status rk_rhs(rk_handle* h, const double* r, double* fr, void* stream);

/* rk_eval_u -- Alg. 3: u^h = chi o sum_p b^0_p o F^-1[F(chi o d) o F(H^a_p)] (Eq. 63, 94).
 * d, u: double[nbox]. */
rk_status rk_eval_u(rk_handle* h, const double* d, double* u, void* stream);

/* rk_eval_u_transpose -- transpose of Alg. 3 (the operator of Alg. 4 without V):
 * w = chi o F^-1[ sum_p F(chi o b^0_p o e) o F(Hbar^a_p) ].  e, w: double[nbox]. */
rk_status rk_eval_u_transpose(rk_handle* h, const double* e, double* w, void* stream);

/* rk_get_b -- the correction coefficients of Eq. 83-85 (FP64, scaled basis):
 * b[(i*s + p)*nbox + idx] for i = 0 (b^0), 1 (b^x), 2 (b^y), 3 (b^z). */
rk_status rk_get_b(rk_handle* h, double* b, void* stream);

/* Sizes of the handle: box nodes, s, and the number of nodes with chi = 1. */
rk_status rk_get_shape(const rk_handle* h, int32_t n[3], int32_t* s, int64_t* n_omega);

/*
 * rk_solve -- Alg. 5 with strong Dirichlet conditions (Eq. 29, Sec. 5.4.2):
 * d = g on chi_gamma; on the free nodes chi_Omega = chi - chi_gamma (Eq. 96)
 * conjugate gradients solve chi_Omega o K(chi_Omega o x) = F with
 * F = chi_Omega o (f^r - K d_Gamma) until ||F - A x|| <= tol ||F|| (FP64
 * residual); then u^h = Alg. 3 (d).  In RK_PREC_MIXED the CG runs in FP32
 * (FP32 convolutions and vectors, FP64 dot products) and its residual is
 * periodically replaced by the true FP64 residual (FP64 operator), the FP32
 * correction being accumulated into the FP64 iterate (iterative refinement
 * without restarting the Krylov recurrence).
 *   r  [nbox] source (read on chi);  g  [nbox] Dirichlet data (read on chi_gamma)
 *   d  [nbox] output coefficients (input guess if opts->x0_given);  u [nbox] output
 *      u^h (NULL: not computed)
 *   opts NULL: defaults;  info NULL: not reported
 * Errors: RK_ERR_NOT_CONVERGED, RK_ERR_BREAKDOWN (outputs hold the last iterate),
 * and the argument errors above.
 */
rk_status rk_solve(rk_handle* h, const double* r, const double* g, double* d, double* u,
                   const rk_solve_opts* opts, rk_solve_info* info, void* stream);

/*
 * rk_boundary_rhs -- f^q of Alg. A.1, the boundary integral of Eq. 28 in the
 * convolutional form of Eq. A.4-A.5 (DNI on the boundary nodes, Eq. A.2):
 *   f^q = chi o F^{-1}[ sum_p F(chi o A o b0_p o q) o F(Hbar^a_p) ]
 * q: Neumann data at the nodes of Gamma_q; A: quadrature weight (area) of each
 * boundary node, 0 elsewhere (Eq. A.6-A.7).  FP64 box arrays, host or device.
 * fq: FP64 box array, 0 off chi.
 */
rk_status rk_boundary_rhs(rk_handle* h, const double* q, const double* A, double* fq, void* stream);

/*
 * rk_solve_neumann -- Alg. 5 with Neumann data as well: the right-hand side of
 * Eq. 25 becomes f^r + f^q (rk_boundary_rhs) before the strong Dirichlet data
 * g on Gamma_g enter (Eq. 29).  Arguments as rk_solve, plus q and A as in
 * rk_boundary_rhs (both required).
 */
rk_status rk_solve_neumann(rk_handle* h, const double* r, const double* g, const double* q, const double* A, double* d,
                           double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream);

/*
 * Time-dependent problems (Appendix C; diffusion u_t = lap u + r, Eq. C.1-C.4:
 * M d' + K d = f^r + f^q).
 *
 * rk_apply_M -- f^m = M v, the consistent mass action of Alg. C.1 (Eq. C.7-C.12):
 *   A^0 = sum_q b0_q o F^{-1}[F(chi o v) F(H^a_q)],  f^m = chi o F^{-1}[sum_p F(chi V b0_p A^0) F(Hbar^a_p)].
 *   v, fm: box arrays of dtype RK_F64 or RK_F32, host or device.
 * rk_lumped_mass -- M^l, the row sums of M (Alg. C.2, Eq. C.9-C.13), FP64.
 * rk_transient_explicit -- Alg. C.3 with forward Euler and the lumped mass:
 *   n_steps times  d <- d + dt (M^l)^{-1} (f - K d) on the free nodes chi_Omega,
 *   with d = g on Gamma_g (g may be NULL: 0) and 0 off chi.  f = f^r + f^q (rk_rhs,
 *   rk_boundary_rhs), fixed over the steps; call with n_steps = 1 per step when it
 *   changes.  d: FP64 box array, in/out.  Stable for dt below 2 / lam_max((M^l)^{-1} K)
 *   (not checked).
 * rk_transient_implicit -- Alg. C.4 with backward Euler: n_steps times
 *   (M + dt K) d_{k+1} = M d_k + dt f on the free nodes, d = g on Gamma_g, each step
 *   by FP64 CG to opts->tol (relative residual of the step).  info: total CG
 *   iterations, steps (outer), FP64 operator applications, worst step residual.
 */
rk_status rk_apply_M(rk_handle* h, const void* v, void* fm, int32_t dtype, void* stream);
rk_status rk_lumped_mass(rk_handle* h, double* ml, void* stream);
rk_status rk_transient_explicit(rk_handle* h, const double* f, const double* g, double dt, int32_t n_steps, double* d,
                                void* stream);
rk_status rk_transient_implicit(rk_handle* h, const double* f, const double* g, double dt, int32_t n_steps, double* d,
                                const rk_solve_opts* opts, rk_solve_info* info, void* stream);

/*
 * Nonlinear reaction terms (Appendix B, the scalar form of Eq. B.1-B.4 and B.9):
 *   f^N = chi o F^{-1}[ sum_p F(chi V b0_p N(u^h)) F(Hbar^a_p) ],  u^h from Alg. 3,
 * with a built-in pointwise nonlinearity N (rk_nonlinearity; c >= 0 makes N
 * nondecreasing): RK_NL_CUBIC c u^3, RK_NL_SINH c sinh(u), RK_NL_EXP c exp(u).
 * rk_nonlinear_force -- f^N(d) (Alg. B.2 of the paper's listing for Eq. B.9).
 * rk_solve_nonlinear -- Alg. B.3: K d + f^N(d) = f^r on the free nodes, d = g on
 *   Gamma_g, by nonlinear CG (Polak-Ribiere+, exact line search by Newton's method
 *   on the convex energy), FP64, from d = d_Gamma, until |R| <= opts->tol |R_0|
 *   (opts->max_iter iterations at most; precision and the mixed options are not
 *   used).  u may be NULL.  info: iterations, relative residual, operator
 *   applications.  Errors: RK_ERR_NOT_CONVERGED, RK_ERR_BREAKDOWN (line search).
 */
/*
 * rk_solve_penalty -- essential boundary conditions imposed weakly by the penalty
 * method (Sec. 2.4) instead of Eq. 29: every chi node is free, and
 *   (K + beta U^T diag(A) U) d = f^r + beta U^T (A o g)
 * where U is the nodal interpolation of Alg. 3 (u^h at the nodes), A the boundary
 * quadrature weights (direct nodal quadrature on the boundary nodes, as Eq. A.2;
 * zero off the boundary) and beta > 0 the penalty parameter.  Solved by CG in FP64
 * to ||rhs - M d|| <= opts->tol ||rhs|| (opts->max_iter iterations at most; the
 * precision and mixed options are not used).
 *   r, g, A: [nbox] inputs (r the source of f^r, g the boundary data);
 *   d: [nbox] output; u: [nbox] output u^h (NULL: not computed).
 *   info: iterations, rel_residual, matvec_f64 (applications of the operator).
 * The solution tends to the one with u^h = g on the boundary nodes as beta grows,
 * at rate 1/beta; the CG iteration count grows with beta.
 * Errors: RK_ERR_INVALID_ARG (beta <= 0, NULL arrays, non-finite right-hand
 * side), RK_ERR_NOT_CONVERGED, RK_ERR_BREAKDOWN, RK_ERR_CUDA.
 */
rk_status rk_solve_penalty(rk_handle* h, const double* r, const double* g, const double* A, double beta, double* d,
                           double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream);

typedef enum rk_nonlinearity { RK_NL_CUBIC = 0, RK_NL_SINH = 1, RK_NL_EXP = 2 } rk_nonlinearity;
rk_status rk_nonlinear_force(rk_handle* h, const double* d, int32_t kind, double c, double* fN, void* stream);
/*
 * rk_nonlinear_grad_force -- the gradient-type nonlinear force of Eq. B.5-B.8 in
 * the form of Eq. B.10: f^N = B^T N with N^k(x) = a_k N(u^h(x)), i.e.
 * f^N_I = chi_I sum_S chi_S V_S sum_k b^k_p(x_S) a_k N(u^h(x_S)) Hbar^a_p(x_I - x_S)
 * (sum over p), evaluated as u^h (Alg. 3), the fields g_p = chi V sum_k a_k b^k_p N,
 * and the reflected passes of Alg. 2.  N is the pointwise nonlinearity kind with
 * coefficient c (as rk_nonlinear_force); a[3] (host) is the fixed direction of the
 * vector nonlinearity (a[2] is ignored on a 2D box, a[1] and a[2] on a 1D box).
 * d, fN: [nbox], FP64.  Errors: RK_ERR_INVALID_ARG, RK_ERR_CUDA.
 */
rk_status rk_nonlinear_grad_force(rk_handle* h, const double* d, int32_t kind, double c, const double* a, double* fN,
                                  void* stream);
rk_status rk_solve_nonlinear(rk_handle* h, const double* r, const double* g, int32_t kind, double c, double* d,
                             double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream);

/*
 * rk_solve_adjoint -- gradient of J = 1/2 sum_{chi} (u^h - u_target)^2 with respect
 * to the source r and the Dirichlet data g, for the solve of rk_solve.  The forward
 * solve is recomputed from (r, g) (nothing is kept between calls); one adjoint
 * solve chi_Omega K chi_Omega lambda = chi_Omega U^T e with e = chi o (u^h - u_target)
 * (K is symmetric) gives dJ/dr = chi V o U lambda and dJ/dg = chi_gamma o
 * (U^T e - K lambda), U being Alg. 3 (derivation from Eq. 25, 29, 59, 62).
 *   J (double, host) may be NULL;  dJ_dr, dJ_dg: [nbox] outputs.
 */
rk_status rk_solve_adjoint(rk_handle* h, const double* r, const double* g, const double* u_target,
                           double* dJ_dr, double* dJ_dg, double* J, const rk_solve_opts* opts,
                           rk_solve_info* info, void* stream);

/*
 * rk_solve_vjp -- vector-Jacobian product of the solve map (r, g) -> u^h of
 * rk_solve: given the cotangent u_bar of u^h, returns r_bar = (du/dr)^T u_bar and
 * g_bar = (du/dg)^T u_bar.  The map is linear (Eq. 25, 29, 59, 62), so one adjoint
 * solve chi_Omega K chi_Omega lambda = chi_Omega U^T (chi o u_bar) suffices:
 * r_bar = chi V o U lambda, g_bar = chi_gamma o (U^T (chi o u_bar) - K lambda).
 * Nothing of the forward solve is kept or needed.
 *   u_bar, r_bar, g_bar: double[nbox].
 */
rk_status rk_solve_vjp(rk_handle* h, const double* u_bar, double* r_bar, double* g_bar, const rk_solve_opts* opts,
                       rk_solve_info* info, void* stream);

/* ---- instrumentation ---------------------------------------------------- */

/* Kernel classes timed by rk_profile_read. */
enum {
  RK_PROF_X_SPLIT = 0,       /* x pass, forward chain (and set-up moments) */
  RK_PROF_Y_SPLIT = 1,       /* y pass, forward chain */
  RK_PROF_Z_SPLIT = 2,       /* z pass, forward chain (set-up moments; in Alg. 2 it also applies
                                the pointwise stage to the regular nodes when n_x % 4 == 0) */
  RK_PROF_Z_STIFF = 3,       /* pointwise stage of Alg. 2 (Eq. 90-91): the boundary nodes left by
                                the z pass, or every node when n_x % 4 != 0 */
  RK_PROF_Z_EVAL_U = 4,      /* fused z pass of Alg. 3 */
  RK_PROF_Z_TRANSPOSE_U = 5, /* fused z pass of Alg. 4 / transpose of Alg. 3 */
  RK_PROF_Y_MERGE = 6,       /* y pass, reflected chain */
  RK_PROF_X_MERGE = 7,       /* x pass, reflected chain */
  RK_PROF_MOMENT_SOLVE = 8,  /* per-node M^{-1} of Alg. 1 */
  RK_PROF_CG_VECTOR = 9,     /* CG dot products and vector updates (per iteration) */
  RK_PROF_Z_MERGE = 10,      /* z pass, reflected chain */
  RK_PROF_PRECOND = 11,      /* spectral preconditioner (five passes) */
  RK_PROF_CLASSES = 12
};

/* Total number of kernels this library has launched in the process. */
int64_t rk_kernel_launches(void);

/* Start (enable = 1) or stop (0) timing every kernel class of this handle with
 * CUDA events recorded on the launching stream; counters are cleared. */
rk_status rk_profile_enable(rk_handle* h, int32_t enable);

/* Accumulated milliseconds and launch counts per class since rk_profile_enable,
 * entry c for the FP32 kernels of class c and entry RK_PROF_CLASSES + c for the
 * FP64 ones (arrays of n_classes <= 2*RK_PROF_CLASSES entries, either may be
 * NULL).  Waits for the recorded events. */
rk_status rk_profile_read(rk_handle* h, double* ms, int64_t* launches, int32_t n_classes);

/* Name of a kernel class ("" if out of range). */
const char* rk_profile_class_name(int32_t cls);

/*
 * rk_debug_short_waits -- a diagnostic switch for tests of the time-out path (the
 * paper has no counterpart).  While enable = 1, the first bounded wait of every
 * block of this handle's TMA- or bulk-copy-fed passes for an input tile gives up at
 * once: the block records the time-out in the handle's error word, still waits
 * (with the normal limit) for its copy in flight to land, and returns without
 * writing its outputs (the x merge of a CG step instead completes, its outputs
 * invalid, so that its p . Ap reduction ends).  The next call of the handle that synchronises (a solve, or a call on
 * host arrays) then returns RK_ERR_TIMEOUT and clears the word; results computed
 * meanwhile are invalid.  enable = 0 restores the normal waits of 2^26 polls.
 * Passes fed by cp.async copies (boxes whose rows are not a multiple of 16 bytes)
 * have no bounded wait and are unaffected.  Drops the handle's captured CUDA
 * graph of CG iterations (it holds the pass arguments it was captured with).
 * Errors: RK_ERR_INVALID_ARG for a NULL handle or enable not 0 or 1.
 */
rk_status rk_debug_short_waits(rk_handle* h, int32_t enable);

/*
 * rk_apply_K_noalloc -- f = K d (the FP64 result of rk_apply_K) without allocating
 * any memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory -- code running inside a host application
 * that owns all device memory through its own pool, or latency-critical loops in
 * which a cudaMalloc/cudaFree (which may synchronise the device) is not allowed.
 * The caller passes every input and the output; the intermediate fields and the
 * per-axis tables live in one fixed device array of RK_NOALLOC_MAX_DOUBLES doubles
 * (about 16.8 MB), plus a few KB of flags and axis projections, that every GPU
 * loading this library holds until the process exits.
 *   grid, degree, a_tilde  as for rk_setup (the same built box sides)
 *   chi   uint8[nbox]  device, Eq. 40 (input and output mask)
 *   chiV  double[nbox] device, chi o V
 *   b     double[4*s*nbox] device, the coefficients in the layout of rk_get_b
 *   d, f  double[nbox] device, input and output
 * Every array must be device memory of the current device, aligned to 16 bytes
 * (host arrays, which the other entry points stage, would need buffers): else
 * RK_ERR_INVALID_ARG before any device work.
 * Limit: (n+1 + 2*n_Y) * nbox + 8192 <= RK_NOALLOC_MAX_DOUBLES with n_Y = 3 (degree
 * 1) or 6 (degree 2): up to a 64^3 box for degree 1 and a 48^3 box for degree 2
 * (any built sides whose product fits); larger boxes return RK_ERR_UNSUPPORTED
 * before any device work.
 * Gap: like rk_setup, the call checks the Eq. 66 gap of chi (a circular run of
 * empty node indices at least as long as the support's reach on every axis), on
 * the device; it waits for that check (a synchronisation of `stream`) and returns
 * RK_ERR_UNSUPPORTED, with f untouched, when chi is too close to its periodic
 * image.  The rest of the work is queued on `stream` without waiting.
 * Every call looks up the device addresses of the fixed arrays for the current
 * device (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device also loads the library's kernels there, so make it before any stream
 * capture.  Should a bounded wait for an input tile give up inside the passes, f
 * is filled with NaN.  All calls share the one array and overwrite it (every value
 * is written before it is read within a call; the flags are cleared at the start
 * of each call), so calls whose GPU work overlaps -- on different streams or host
 * threads -- race and must be ordered by the caller.
 */
#define RK_NOALLOC_MAX_DOUBLES 2105344LL
rk_status rk_apply_K_noalloc(const rk_grid* grid, int32_t degree, double a_tilde, const uint8_t* chi,
                             const double* chiV, const double* b, const double* d, double* f, void* stream);

/*
 * rk_clone -- a handle for another right-hand side of the same domain: it shares
 * the parent's set-up (tables, coefficients, masks -- the parent must outlive it)
 * and owns its own workspaces and solver state, so several solves of one domain
 * can run at the same time on different streams (rk_solve_batched).
 */
rk_status rk_clone(const rk_handle* parent, rk_handle** out);

/* One problem of rk_solve_batched: the handle of its domain (distinct per item;
 * use rk_clone for several right-hand sides of one domain) and the arrays of
 * rk_solve (u may be NULL). */
typedef struct rk_batch_item {
  rk_handle* h;
  const double* r;
  const double* g;
  double* d;
  double* u;
} rk_batch_item;

/*
 * rk_solve_batched -- Alg. 5 for many (domain, right-hand side) problems at once,
 * in mixed precision.  Every item runs on its own stream (forked from `stream`);
 * the CG iterations of all items advance together, each chunk of check_every
 * iterations of an item being one replay of a CUDA graph captured at its first
 * use.  Returns after every item finished; infos (NULL or n_items entries)
 * receives each item's report.  Errors: the first failing item's status.
 */
rk_status rk_solve_batched(const rk_batch_item* items, int32_t n_items, const rk_solve_opts* opts,
                           rk_solve_info* infos, void* stream);

/* Release the handle and everything it owns (NULL is accepted). */
rk_status rk_destroy(rk_handle* h);

/* Static string naming a status code. */
const char* rk_status_string(rk_status s);

/* Description of the last error raised on the calling host thread ("" if none). */
const char* rk_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* FCRKPM_H */
