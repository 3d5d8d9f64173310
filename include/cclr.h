/*
 * cclr.h -- C ABI of libcclr, the GB300 (sm_103a) Cholesky-decomposed relativistic
 * LR-CCSD response library.
 *
 * The operation: the CC Jacobian-vector product sigma = A X (Sec. 2.2, the Jacobian
 * A_mu,nu = <mu|[H-bar_0, tau_nu]|Phi_0>), its transpose Y A (the left / Lambda
 * equations, Sec. 2.2), and the linear solve (A - omega) X = -xi whose solution gives
 * the polarisability alpha_AB(omega) = -<<A;B>>_omega through the CC linear response
 * function with the P(A,B) symmetrisation (Sec. 2.2).  Two-electron integrals enter
 * only as Cholesky vectors (Sec. 3): <pq|rs> = (pr|qs) = sum_P L^P_pr L^P_qs, with each
 * L^P Hermitian; integrals with more than two virtual indices are formed on the fly on
 * the GPU and never stored.
 *
 * Conventions common to every entry point:
 *  - Complex numbers are interleaved (re, im) pairs of doubles (the layout of C99
 *    double _Complex and numpy complex128).  A "complex array of N entries" is 2N doubles.
 *  - All arrays are row-major.  n = o + v spinors, occupied first.
 *      eps [n]            real orbital (spinor) energies; the Fock matrix is diag(eps)
 *      L   [naux][n][n]   complex, each L[P] Hermitian
 *      mu  [3][n][n]      complex Hermitian dipole integrals (x, y, z)
 *      t1  [o][v]         t_i^a             (NULL: zero)
 *      t2  [o][o][v][v]   t_ij^ab, antisymmetric in (i,j) and in (a,b)
 *                         (NULL: first-order amplitudes <ab||ij>/(e_i+e_j-e_a-e_b))
 *      x1/s1 [nrhs][o][v], x2/s2 [nrhs][o][o][v][v]  amplitude-shaped vectors; doubles
 *                         blocks are full antisymmetric tensors (not packed).
 *  - Ownership: inputs are copied (to the device) during the call; the caller keeps
 *    ownership and may free them after return.  Outputs are caller-allocated.
 *  - device_ptrs = 0: every array argument is host memory; 1: device memory of the
 *    current CUDA device (e.g. torch tensors), used on the context's stream.
 *  - Errors: every call returns a cclr_status and never aborts or exits.  On error the
 *    outputs are unspecified; cc_lr_last_error() describes the failure.
 *  - Threading: a context is used by one host thread at a time.
 */
#ifndef CCLR_H
#define CCLR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cclr_ctx cclr_ctx;

typedef enum {
  CCLR_OK = 0,
  CCLR_EINVAL = 1,      /* bad argument (size, pointer, mode)                         */
  CCLR_ENOMEM = 2,      /* device allocation failed or the HBM budget is exceeded       */
  CCLR_ENOCONV = 3,     /* solver stopped without meeting the tolerance (alpha filled)  */
  CCLR_EDEVICE = 4,     /* CUDA runtime / driver error                                  */
  CCLR_ETIMEOUT = 5,    /* a bounded device-side wait gave up                           */
  CCLR_EUNSUPPORTED = 6 /* mode not available on this device or build                   */
} cclr_status;

/* Arithmetic of sigma and sigma^T.  FP64: complex128 everywhere.  The others run the
 * contractions in complex64 (tensor cores for the dominant ones) and keep the solver
 * state, residuals, subspace algebra and alpha in FP64. */
typedef enum {
  CCLR_FP64 = 0,
  CCLR_C64_TF32 = 1,     /* one TF32 tensor-core pass (kind::tf32)                      */
  CCLR_C64_3XTF32 = 2,   /* split hi/lo TF32, three products (about FP32 accuracy)      */
  CCLR_C64_FP32 = 3,     /* complex64 on FP32 CUDA cores (no tensor cores)              */
  CCLR_BF16X3 = 4        /* split hi/lo BF16, three products on kind::f16 (about 2^-16
                            relative per product, at twice the TF32 rate per pass)     */
} cclr_prec;

typedef struct {
  int iterations;        /* total solver iterations over all right-hand sides          */
  int sigma_calls;       /* number of sigma (or sigma^T) vectors formed                */
  int refinements;       /* FP64-accurate residual evaluations (mixed modes)           */
  int converged;         /* 1 if every right-hand side met the tolerance               */
  double max_rel_residual; /* max over RHS of ||r|| / ||b|| at exit                     */
  double time_solve_ms;  /* X solves                                                   */
  double time_lambda_ms; /* ground-state Lambda solve (cached after the first call)    */
  double time_alpha_ms;  /* eta.X, F.X.X and the alpha contraction                     */
} cclr_stats;

/* Create a context: copy the inputs to the device, T1-dress the Cholesky vectors,
 * build the stored intermediates (integrals with at most two virtual indices, the
 * one-body and o^2v^2 / o^3v / o^4 elements of H-bar) and the diagonal preconditioner.
 * lam1/lam2 ([o][v], [o][o][v][v]) give the ground-state Lambda; NULL means it is
 * solved on first use (lambda A = -dE/dT).
 * hbm_budget_bytes: the most device memory the context may hold (0 = no limit).  Every
 * device allocation the context makes -- at init and later, in any call on it (workspace,
 * solver vectors, ladder blocks, graph staging) -- is charged to it and checked before it is
 * made; a call that would exceed the budget returns CCLR_ENOMEM and allocates nothing more
 * (cc_lr_memory reports the bytes held).
 * cuda_stream: a cudaStream_t (NULL: the legacy default stream). */
cclr_status cc_lr_init(cclr_ctx **ctx, int o, int v, int naux,
                       const double *eps, const double *L, const double *mu,
                       const double *t1, const double *t2,
                       const double *lam1, const double *lam2,
                       int prec, size_t hbm_budget_bytes, int device_ptrs,
                       void *cuda_stream);

/* sigma = A X for nrhs vectors (Sec. 2.2 Jacobian).  s1/s2 are overwritten. */
cclr_status cc_lr_sigma(cclr_ctx *ctx, int nrhs, const double *x1, const double *x2,
                        double *s1, double *s2);

/* sigma^T = Y A (bilinear, no conjugation) over unique amplitudes: with
 * <Y, Z> = sum_ia Y_ia Z_ia + 1/4 sum_ijab Y_ijab Z_ijab it satisfies
 * <Y, A X> = <sigma^T(Y), X>.  Used by the Lambda and left response equations. */
cclr_status cc_lr_sigma_T(cclr_ctx *ctx, int nrhs, const double *y1, const double *y2,
                          double *s1, double *s2);

/* sigma (transpose = 0) or sigma^T (transpose = 1) of nrhs vectors in the packed
 * unique-amplitude layout the solvers use: each vector is n1 + n2p complex numbers,
 * singles [o][v] then doubles [(i<j)][(a<b)] (pairs numbered row by row), so a doubles
 * block is a quarter of the full tensor; the bilinear product of two vectors is the plain
 * sum over entries.  x and s are device arrays of nrhs vectors each (the batch forms every
 * <ab||ef>~ block once for all of them); host arrays return CCLR_EINVAL. */
cclr_status cc_lr_sigma_packed(cclr_ctx *ctx, int nrhs, int transpose, const double *x, double *s);

/* Right-hand side xi^B = <nu|e^{-T} mu^B e^{T}|Phi_0> (Sec. 2.2) for component
 * comp (0 = x, 1 = y, 2 = z). */
cclr_status cc_lr_xi(cclr_ctx *ctx, int comp, double *xi1, double *xi2);

/* Solve (A - omega) X = -xi^comp (Sec. 2.2, alpha -> 0+) and return X. */
cclr_status cc_lr_solve_x(cclr_ctx *ctx, double omega, int comp, double tol, int diis_depth,
                          double *x1, double *x2, cclr_stats *stats);

/* alpha_AB(omega) = -<<A;B>>_omega for every omega in omegas and A, B in comps:
 * alpha[w][a][b], complex (2 doubles per entry), host memory.  Solves X^B(+-omega) for
 * each component (batched), the ground-state Lambda if not given, and evaluates
 * g(A,B;w) = eta^A.X^B(w) + eta^B.X^A(-w) + (F X^A(-w)).X^B(w),
 * <<A;B>>_w = 1/2 [g(A,B;w) + conj g(A,B;-w)].  tol is the relative residual target
 * ||r||/||b||.  On CCLR_ENOCONV alpha and stats still hold the last estimate. */
cclr_status cc_lr_solve(cclr_ctx *ctx, int nomega, const double *omegas, int ncomp,
                        const int *comps, double tol, int diis_depth, double *alpha,
                        cclr_stats *stats);

/* The same alpha by the left-hand route of Sec. 2.2 (the response function written with the
 * perturbed left amplitudes Y): X^B(w) from (A - w) X = -xi^B, Y^B(w) from
 * Y (A + w) = -(eta^B + F X^B(w)) (transpose products, shift -w), and
 * g(A,B;w) = Y^B(w) . xi^A + eta^A . X^B(w), <<A;B>>_w = 1/2 [g(A,B;w) + conj g(A,B;-w)].
 * Equal to cc_lr_solve's alpha within the solver tolerance ("alpha from both sides").  Same
 * arguments, outputs and error behaviour as cc_lr_solve (real omega only). */
cclr_status cc_lr_solve_left(cclr_ctx *ctx, int nomega, const double *omegas, int ncomp,
                             const int *comps, double tol, int diis_depth, double *alpha,
                             cclr_stats *stats);

/* alpha to an absolute tolerance tol_alpha (a.u.) instead of a residual target: the left-hand
 * route and the X-only route are evaluated from the same X and F X (dot products only), their
 * largest difference over the entries is the a-posteriori error estimate written to
 * *alpha_err, and the solves are tightened, warm-started from the previous solutions, until it
 * is below tol_alpha.  alpha holds the left-hand route's values.  The ground-state Lambda, which
 * both routes share, is solved near the arithmetic's residual floor (5e-7 relative with 3xTF32
 * refinement).  Returns CCLR_ENOCONV (alpha and *alpha_err filled) when the floor is reached
 * with the estimate still above tol_alpha. */
cclr_status cc_lr_solve_alpha_tol(cclr_ctx *ctx, int nomega, const double *omegas, int ncomp,
                                  const int *comps, double tol_alpha, int diis_depth, double *alpha,
                                  double *alpha_err, cclr_stats *stats);

/* eta^A = <(1 + Lambda)|[A-bar, tau_nu]|Phi_0> (Sec. 2.2) for component comp as a vector:
 * eta1 [o][v], eta2 [o][o][v][v] (full antisymmetric).  Formed as dE_A/dT + lambda A[mu^A], with
 * A[mu^A] the Jacobian of the dipole operator alone; solves the ground-state Lambda first
 * (relative residual tol) if it is not known. */
cclr_status cc_lr_eta(cclr_ctx *ctx, int comp, double tol, double *eta1, double *eta2);

/* Damped response (complex frequency z = omega + i gamma, gamma >= 0; the pole widths and
 * absorption of Sec. 2.2's response function continued off the real axis): the same as
 * cc_lr_solve with X^C solved at the complex shifts z, -z, z*, -z* ((A - s) X = -xi^C, complex
 * shift in the solver and the diagonal preconditioner) and
 * <<A;B>>_z = 1/2 [g(A,B;z) + conj g(A,B;-z*)], alpha = -<<A;B>>_z.  gamma = 0 gives
 * cc_lr_solve. */
cclr_status cc_lr_solve_damped(cclr_ctx *ctx, int nomega, const double *omegas, double gamma, int ncomp,
                               const int *comps, double tol, int diis_depth, double *alpha,
                               cclr_stats *stats);

/* Ground-state Lambda (solved if needed) copied out: lam1 [o][v], lam2 [o][o][v][v]. */
cclr_status cc_lr_lambda(cclr_ctx *ctx, double tol, double *lam1, double *lam2);

/* Ground-state CCSD on the device (Sec. 2.2): the amplitude equations
 * Omega_mu(T) = <mu|e^{-T} H e^{T}|Phi_0> = 0 and the correlation energy
 * E(T) = <Phi_0|e^{-T} H e^{T}|Phi_0> - E_ref = sum_ia f_ia t_ia + 1/4 sum <ij||ab> t_ijab
 * + 1/2 sum <ij||ab> t_ia t_jb (f = diag(eps), so f_ia = 0).
 * The residual is formed from the Jacobian products the context already runs: Omega(sT) is a
 * polynomial of degree four in s with d/ds Omega(sT) = A(sT) T, so
 * Omega(T) = Omega(0) + 1/2 [A(s1 T) T + A(s2 T) T], s1,2 = 1/2 -+ 1/(2 sqrt 3), exactly
 * (two-point Gauss-Legendre quadrature of a cubic), with Omega(0) = <mu|H|Phi_0> (zero singles,
 * <ab||ij> doubles).  Each residual costs two builds of the intermediates and two sigma
 * products.
 * prec: the arithmetic of those products (a cclr_prec; -1 = the context's precision).  FP64
 * gives the exact residual; the tensor-core modes give it to their product accuracy.
 *
 * cc_lr_ccsd_residual: Omega(T) and E(T) at the given amplitudes (t1 [o][v], t2 [o][o][v][v]
 * antisymmetric in (i,j) and (a,b); r1, r2 the same shapes; energy NULL or 2 doubles, complex).
 * The context's own amplitudes and intermediates are unchanged.
 *
 * cc_lr_ccsd: solves Omega(T) = 0 starting from the context's amplitudes by quasi-Newton steps
 * T <- T - Omega(T) / D (D the orbital-energy differences) with Pulay (DIIS) extrapolation over
 * the last diis_depth steps (2..16), until the norm of the residual over unique amplitudes
 * (singles, i<j a<b doubles) is below tol, or max_iterations residuals were formed.  The context
 * then holds the final T and rebuilds or resets everything that depends on it (intermediates,
 * preconditioner, Lambda, eta).  energy (NULL or 2 doubles): E at the final T; res_norm: the last
 * residual norm; iterations: residuals formed.  CCLR_ENOCONV if the tolerance was not met (the
 * context then holds the last iterate).  CCLR_EUNSUPPORTED for FP64 products in a budgeted
 * context that released its FP64 inputs. */
cclr_status cc_lr_ccsd_residual(cclr_ctx *ctx, int prec, const double *t1, const double *t2,
                                double *r1, double *r2, double *energy);
cclr_status cc_lr_ccsd(cclr_ctx *ctx, int prec, double tol, int max_iterations, int diis_depth,
                       double *energy, double *res_norm, int *iterations);

/* The amplitudes the context holds (useful when t2 was NULL at init). */
cclr_status cc_lr_get_t(cclr_ctx *ctx, double *t1, double *t2);

/* Switch the arithmetic of subsequent sigma / sigma^T / solves. */
cclr_status cc_lr_set_precision(cclr_ctx *ctx, int prec);

/* CUDA graphs for the sigma / sigma^T programs (off by default).  On: a product whose
 * arguments (direction, precision, constant set, buffer addresses) repeat those of the
 * previous product, with no device memory freed and no constants rebuilt in between, is
 * captured once into a CUDA graph (thread-local capture on the context's stream) and later
 * products with those arguments replay it with one cudaGraphLaunch; the solvers' products
 * qualify after their first iterations.  Freeing memory or rebuilding constants invalidates
 * the captured graphs.  While a graph is replayed, cc_lr_last_timings reports the total only
 * (the other entries are -1).  If a capture fails the context turns graphs off and stays
 * eager.  Off: every product is issued kernel by kernel (and cached graphs are destroyed).
 * Needs a context created with its own stream (not the default stream): CCLR_EUNSUPPORTED
 * otherwise. */
cclr_status cc_lr_set_graphs(cclr_ctx *ctx, int on);

/* Result of the pp-ladder autotuner for the tensor-core mode prec (CCLR_C64_TF32,
 * CCLR_C64_3XTF32 or CCLR_BF16X3): on its first use in that mode the ladder times one product per candidate
 * group size (how many a values each formed <ab|ef>~ block covers) and keeps the fastest.
 * Writes the group size in use, the number of candidates timed (*n; 0 before the first use)
 * and up to cap of them (candidate group size, milliseconds). */
cclr_status cc_lr_ladder_tuning(cclr_ctx *ctx, int prec, int *group_size, int cap, int *cand, double *ms,
                                int *n);

/* Ablation of the on-the-fly ladder (off by default): with store = 1 the tensor-core modes keep
 * the whole antisymmetrised, packed <ab||ef>~ (P_v x P_v, P_v = v(v-1)/2; 8 bytes per entry in
 * TF32 mode, 24 in 3xTF32: 6.6 GB and 19.7 GB at v = 240) once the first sigma product has
 * formed it, and later sigma products contract it in one GEMM instead of forming it again.
 * The transpose product and the FP64 mode still form the blocks on the fly.  A rebuilt
 * constant set (new amplitudes) re-forms it on the next product. */
cclr_status cc_lr_set_ladder_storage(cclr_ctx *ctx, int store);

/* Number of graph captures and graph launches made by the context so far. */
cclr_status cc_lr_graph_stats(cclr_ctx *ctx, int *captures, int *launches);

/* Arithmetic of the mixed modes' accurate sigma products: the residual of every refinement
 * step, the polish that finishes a refinement which stalls, and the sigma^T products of the
 * F X stencil.  CCLR_FP64 (default): FP64 on CUDA cores; CCLR_C64_3XTF32: complex64 with
 * 3xTF32 on the tensor cores (about FP32 accuracy; the residual norms, vector updates, Krylov
 * subspace and alpha contractions stay FP64 either way).  The FP64 sigma is slow on GPUs with
 * a reduced FP64 rate, so large systems use CCLR_C64_3XTF32 with CCLR_C64_TF32 corrections. */
cclr_status cc_lr_set_refinement(cclr_ctx *ctx, int prec);

/* Linear solver of cc_lr_solve / cc_lr_solve_x / cc_lr_lambda: method 1 = restarted
 * GMRES with the diagonal preconditioner (default; subspace = restart length),
 * method 0 = DIIS extrapolation of preconditioned Jacobi steps (subspace ignored; the
 * calls' diis_depth applies), method 2 = block GMRES: cc_lr_solve advances the X systems of
 * all its components and frequency signs in lockstep, so every iteration applies the operator
 * to all unconverged systems in one batched product (the ladder's integral blocks formed once
 * for all); each system keeps its own GMRES, the restart length shrinks when the bases would not
 * fit in half of the free device memory, and single-system solves use method 1.  In the mixed
 * modes every method solves the corrections of the iterative refinement.  max_iterations bounds the sigma products of
 * each linear solve (default 300; 0 keeps the current value); a solve that reaches it
 * returns CCLR_ENOCONV with its best iterate. */
cclr_status cc_lr_set_solver(cclr_ctx *ctx, int method, int subspace, int max_iterations);

/* Tensor-core GEMM tile autotuner (on by default): the first eager use of each GEMM shape
 * (operand type, M, N, K, output layout) on a device times a handful of launch configurations
 * -- tile width, K splits, raster band -- around the rules' choice on the real operands (an
 * accumulated output is tuned into a scratch block) and keeps the fastest for that shape and
 * device; later products, and other contexts on the device, launch it.  on = 0: untuned shapes
 * keep the rules. */
cclr_status cc_lr_set_autotune(cclr_ctx *ctx, int on);

/* The tuned GEMM shapes of the current device: writes *n (the number of shapes) and the first
 * min(*n, cap) rows of 10 doubles (operand type 0 TF32 / 1 BF16, M, N, K (real elements), tile
 * width, K splits, raster band, best milliseconds, the rules' milliseconds, candidates timed). */
cclr_status cc_lr_gemm_tuning(cclr_ctx *ctx, int cap, int *n, double *rec);

/* Device memory held by the context now (*in_use), the most it has held (*peak), and its
 * budget (*budget, 0 = none), in bytes.  Host-side bookkeeping only (no device call). */
cclr_status cc_lr_memory(cclr_ctx *ctx, size_t *in_use, size_t *peak, size_t *budget);

/* Device-side timing (CUDA events on the context's stream) of the last sigma or
 * sigma^T product, in milliseconds; writes the first min(n, 5) of: [0] particle-particle
 * ladder (formation of <ab|ef>~ from L~_vv and its contraction with X), [1] every other
 * kernel, [2] total, [3] the ladder's formation GEMMs alone (tensor-core modes; 0 otherwise),
 * [4] the number of batched products the last multi-vector call was split into to fit the
 * device memory (1: all its vectors in one product). */
cclr_status cc_lr_last_timings(cclr_ctx *ctx, double *ms, int n);

void cc_lr_free(cclr_ctx *ctx);
const char *cc_lr_strerror(cclr_status status);
/* Thread-local text of the most recent failure (never NULL). */
const char *cc_lr_last_error(void);

/* Diagnostic: number of GPU kernels this library has launched in this process. */
unsigned long long cc_lr_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* CCLR_H */
