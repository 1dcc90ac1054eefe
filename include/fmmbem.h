/*
 * fmmbem.h — C ABI of the GB300 relaxed-p FMM-BEM library (libfmmbem.so).
 *
 * The library solves the collocation boundary-element systems of Wang, Layton
 * & Barba, "Inexact Krylov iterations and relaxation strategies with
 * fast-multipole boundary element method" (arXiv:1506.05957):
 *   - Laplace, first kind (Sec. 2.1, eqs. laplace_bem_final, laplace_matrix):
 *       V q = b,  V_ij = 1/(4 pi) int_{Gamma_j} 1/|c_i - y| dS_y,
 *   - Stokes, single layer (Sec. 2.2, eqs. stokes_bem_discretized, stokeslet):
 *       A t = u,  A_iJ = -1/(8 pi mu) int_{Gamma_J} (I/r + d d^T/r^3) dS_y,  d = c_i - y,
 * on flat triangular panels with one unknown (Laplace) or three (Stokes) per
 * panel, collocated at panel centroids. Integrals use K-point Gauss rules for
 * far panels, a 20-point rule for panels within 2 sqrt(2 S_j) of the target
 * and a semi-analytic self-panel integral (Sec. 2.3). The mat-vec is an
 * N-body sum (eq. matvec-onerow) accelerated by a spherical-harmonic fast
 * multipole method (Sec. 2.5) at a runtime expansion order p; GMRES
 * (Sec. 2.4) lowers p as the residual falls (Sec. 2.6, eqs.
 * matrix-perturbation and fmm_p).
 *
 * Conventions for every entry point:
 *   - Return value: 0 on success, a negative FMMBEM_E* code on failure
 *     (fmmbem_last_error() then describes it), FMMBEM_NOT_CONVERGED (1) from
 *     fmmbem_solve when the iteration cap was reached (outputs still filled).
 *   - "_dev" pointers are CUDA device memory of the current device; they are
 *     read/written on the handle's stream. Host pointers are named "_host".
 *   - The caller owns every buffer it passes; the library never frees them
 *     and keeps no reference after the call returns. The handle owns all of
 *     its own device state and frees it in fmmbem_destroy.
 *   - Unknowns are in the caller's panel order: Laplace [n_panels] doubles,
 *     Stokes [n_panels][3] doubles (x, y, z per panel).
 *   - A handle is not thread-safe; distinct handles may be used from
 *     distinct threads on distinct streams.
 */
#ifndef FMMBEM_H
#define FMMBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define FMMBEM_OK 0
#define FMMBEM_NOT_CONVERGED 1
#define FMMBEM_EINVAL (-1)   /* bad argument: sizes, p outside [1, p_max], theta outside (0,1), NULL */
#define FMMBEM_ENOMEM (-2)   /* device allocation failed */
#define FMMBEM_EDEVICE (-3)  /* CUDA error reported by a launch or a copy */
#define FMMBEM_ENAN (-4)     /* NaN/Inf met in the Krylov recurrence */
#define FMMBEM_ESTATE (-5)   /* call not valid for this handle (e.g. Stokes-only call on a Laplace handle) */
#define FMMBEM_ETIMEOUT (-6) /* a bounded device wait gave up (grid barrier, bulk-copy or tensor-core
                                barrier); the results of that call are invalid, the handle stays usable */

/* Operators (Sec. 2.1-2.2). */
#define FMMBEM_LAPLACE 0     /* Laplace single layer, 1 unknown per panel */
#define FMMBEM_STOKES 1      /* Stokeslet single layer, 3 unknowns per panel */

/* Arithmetic of the mat-vec (the Krylov recurrence is always FP64). */
#define FMMBEM_FP64 0        /* every pass in FP64 */
#define FMMBEM_MIXED 1       /* P2M/M2M/M2L/L2L/L2P and P2P in FP32 with FP64 tile sums;
                                singular/near-singular corrections and the output in FP64 */
#define FMMBEM_MIXED_REFINED 2 /* solves: iterative refinement with FP64 residuals around the
                                relaxed FMMBEM_MIXED GMRES, for tolerances below what FP32 passes
                                resolve (about 1e-6): each outer step solves A d = r with mixed
                                mat-vecs to a relative 1e-5 (or the final tolerance if looser),
                                adds d to x and recomputes r = b - A x with an FP64 mat-vec at
                                p_initial, until ||r|| / ||b|| <= tol. Mat-vecs run as FMMBEM_MIXED.
                                Single-vector handles only. */

/* Largest supported expansion order (degrees n = 0..p, (p+1)(p+2)/2 complex
 * coefficients per expansion). */
#define FMMBEM_P_MAX 16

/* A surface triangulation in host memory. Triangles are counter-clockwise
 * when seen from the side the normal should point to (outward for a closed
 * body). Copied to the device by fmmbem_create; not referenced afterwards.
 * A mesh may hold several bodies (the cells of the red-blood-cell configurations);
 * body_of_panel names each panel's body for fmmbem_body_integrals. */
typedef struct {
    int64_t n_vertices;
    const double* vertices;   /* [n_vertices][3], host */
    int64_t n_panels;
    const int32_t* triangles; /* [n_panels][3] vertex indices, host */
    int32_t n_bodies;         /* 0 or 1: the whole mesh is one body (body_of_panel ignored) */
    const int32_t* body_of_panel; /* [n_panels] body index in [0, n_bodies), host; required when n_bodies > 1 */
} fmmbem_mesh;

/* Options; fmmbem_default_opts fills the defaults shown. */
typedef struct {
    int p_max;            /* 16: largest p any later call may request (<= FMMBEM_P_MAX) */
    double near_factor;   /* 2.0: near-singular if |c_i - c_j| < near_factor * sqrt(2 S_j) (Sec. 2.3) */
    double mu;            /* 1.0: viscosity (Stokes) */
    int precision;        /* FMMBEM_MIXED */
    int restart;          /* 50: GMRES restart length m */
    int max_iter;         /* 100: cap on Arnoldi steps (the paper's cap, Table stokes_min_p) */
    void* stream;         /* NULL: the legacy default stream; else a cudaStream_t for all work;
                             it must stay valid until fmmbem_destroy returns (the handle's
                             device memory is stream-ordered and is released on it) */
    int nrhs;             /* 1: one vector per mat-vec. A batched handle's mat-vecs and solves take
                             nrhs vectors at once, laid out [nrhs][n_unknowns] (see
                             fmmbem_solve_batch): FMMBEM_BATCH for a Laplace handle, 2 to
                             FMMBEM_STOKES_BATCH_MAX for a Stokes handle (single layer only) */
    int near_k;           /* 20: points of the near-singular rule (Sec. 2.3 gives K ~ 20): a collapsed
                             Gauss product of nu x (nu - 1) points, exact to total degree 2 nu - 3;
                             one of 6, 12, 20, 30, 42 (nu = 3..7); 0 selects 20 */
} fmmbem_opts;

#define FMMBEM_BATCH 4
/* Largest Stokes batch. Each pass of a Stokes batch's mat-vec is one launch for all vectors:
 * the tensor-core M2M, M2L and L2L take every vector's expansion rows in their tiles (one
 * operator chunk serves 4 nrhs rows per pair), the other kernels take the vector from the
 * launch's second grid dimension. */
#define FMMBEM_STOKES_BATCH_MAX 8

typedef struct fmmbem_handle fmmbem_handle;

/* Fill *opts with the defaults. Returns FMMBEM_EINVAL if opts is NULL. */
int fmmbem_default_opts(fmmbem_opts* opts);

/*
 * Build everything the mat-vec needs (Sec. 2.3 and 2.5): panel geometry and
 * K-point Gauss points, a Morton-sorted octree over panels whose leaves hold
 * at most `ncrit` Gauss points, dual-tree-traversal interaction lists with the
 * acceptance criterion (R_a + R_b) < theta |c_a - c_b| (c = box centre; R_a = the
 * largest distance from c_a to a collocation point of the target cell a, R_b = the
 * largest distance from c_b to a Gauss point of the source cell b: the cluster
 * sizes of eq. multipole_error) together with |c_a - c_b| >= the larger cell's side
 * (which keeps the FP32 translation operators in range at p <= 16; a closed surface mesh
 * meets it whenever the first condition holds), and the sparse table of near-singular and
 * self-panel corrections (accurate integral minus the K-point sum), in FP64.
 *   mesh      : host mesh (see fmmbem_mesh)
 *   kernel    : FMMBEM_LAPLACE or FMMBEM_STOKES
 *   gauss_k   : far-field rule, K in {1, 3, 4, 7}
 *   ncrit     : leaf capacity in Gauss points, >= gauss_k
 *   theta     : multipole acceptance parameter, 0 < theta < 1
 *   opts      : NULL for defaults
 *   out       : receives the handle
 * Errors: FMMBEM_EINVAL on bad arguments or a degenerate (zero-area) panel,
 * FMMBEM_ENOMEM, FMMBEM_EDEVICE. No handle is returned on failure.
 */
int fmmbem_create(const fmmbem_mesh* mesh, int kernel, int gauss_k, int ncrit, double theta,
                  const fmmbem_opts* opts, fmmbem_handle** out);

/* Release all device memory of the handle. NULL is ignored. */
void fmmbem_destroy(fmmbem_handle* h);

/* Number of unknowns of one vector: n_panels (Laplace) or 3 n_panels (Stokes); a batched
 * handle's mat-vecs and solves take FMMBEM_BATCH such vectors. -1 for NULL. */
int64_t fmmbem_n_unknowns(const fmmbem_handle* h);

/* Switch the arithmetic of later mat-vecs and solves (FMMBEM_FP64 or FMMBEM_MIXED). */
int fmmbem_set_precision(fmmbem_handle* h, int precision);

/* M2L formulations, all computing the same sums:
 *   TABLES : batched products against precomputed translation operators, SIMT FMA;
 *   GATHER : per-target gather that builds the irregular harmonics of each pair on the fly;
 *   TENSOR : the TABLES products on the tcgen05 tensor cores in 3xTF32 (FP32-level
 *            accuracy) for FMMBEM_MIXED mat-vecs; FMMBEM_FP64 mat-vecs use TABLES.
 * fmmbem_create selects TENSOR when the operator tables fit in memory. */
#define FMMBEM_M2L_TABLES 0
#define FMMBEM_M2L_GATHER 1
#define FMMBEM_M2L_TENSOR 2
/* Select the M2L formulation; FMMBEM_ESTATE if the operator tables were not built. */
int fmmbem_set_m2l_mode(fmmbem_handle* h, int mode);

/* Lowest expansion order at which FMMBEM_MIXED mat-vecs in M2L mode TENSOR run M2L
 * (m2l_min_p) and M2M/L2L (tree_min_p) on the tensor cores; below it they use the SIMT
 * kernels (operator-table GEMM for M2L, per-parent translations for M2M/L2L), which are
 * lighter per launch and share SMs with the concurrent near field. Defaults: m2l_min_p 1,
 * tree_min_p 6 (measured on the 81920-panel sphere). FMMBEM_EINVAL for values below 1. */
int fmmbem_set_tc_thresholds(fmmbem_handle* h, int m2l_min_p, int tree_min_p);

/* Autotuner: first the near-field schedule (fmmbem_set_p2p_variant's four, timed at p_hi:
 * the near field does not depend on p), then for every order p in [p_lo, p_hi] M2L and
 * M2M/L2L on the tensor cores or on the SIMT kernels (four configurations): each candidate
 * times the handle's mat-vec (its captured graph, on the handle's stream) over three runs
 * after a capture run, and the fastest is kept. choice (optional, [p_max + 1] ints, host):
 * 2 * (M2L on tensor cores) + (M2M/L2L on tensor cores) for each tuned p, and in choice[0]
 * the near-field schedule. The sums are the same in every configuration (FP32 passes, 3xTF32
 * products). Synchronizes the handle's stream; for FMMBEM_FP64 handles or without
 * tensor-core tables it only reports the current choices. Errors: FMMBEM_EINVAL,
 * FMMBEM_EDEVICE. */
int fmmbem_autotune(fmmbem_handle* h, int p_lo, int p_hi, int* choice);

/*
 * Create with the leaf capacity chosen by measurement (Sec. 3 tunes N_CRIT separately for
 * relaxed and fixed-p runs): for each of the n_cand leaf capacities ncrit_cand[i] (host), build
 * the handle (fmmbem_create), run fmmbem_autotune(h, p_lo, p_hi), and time one mat-vec at
 * every order of [p_lo, p_hi] (their sum weighs the low orders of a relaxed solve as much as
 * the high ones); keep the fastest handle and destroy the others. Other arguments as
 * fmmbem_create. ncrit_out (optional, host) receives the chosen capacity, ms_out (optional) the
 * chosen handle's summed mat-vec milliseconds. Errors: those of fmmbem_create and
 * fmmbem_autotune; FMMBEM_EINVAL for an empty candidate list or a bad order range.
 */
int fmmbem_create_tuned(const fmmbem_mesh* mesh, int kernel, int gauss_k, int n_cand, const int* ncrit_cand,
                        double theta, const fmmbem_opts* opts, int p_lo, int p_hi, fmmbem_handle** out,
                        int* ncrit_out, double* ms_out);

/* Near-field kernel of FMMBEM_MIXED Laplace mat-vecs (same sums, different schedules):
 * 0 = source tiles staged in shared memory, targets held per lane;
 * 1 = (target, source slice) per thread, sources read through L1;
 * 2 = as 1, with each pair's sources bulk-copied into double-buffered shared memory
 *     (used when a leaf holds at most 1024 Gauss points, else 1);
 * 3 = one block per work item (at most 24 targets of one leaf), its warps' lanes over the
 *     leaf's source stream and the targets looped in registers (default).
 * Returns FMMBEM_EINVAL for any other value. */
int fmmbem_set_p2p_variant(fmmbem_handle* h, int variant);

/* Run each restart cycle of fmmbem_solve on the device (on = 1) instead of one host round
 * trip per GMRES step (Sec. 2.4 and 2.6: the steps are the same). The cycle is one CUDA graph
 * whose while node repeats the mat-vec at the step's order (a switch over the per-order
 * mat-vecs), the Arnoldi step and the column update (Givens rotations, residual estimate,
 * stopping tests and the next relaxed order), all on the device; the host reads the cycle's
 * state once at its end. Built on the first solve after it is enabled or after the kernel
 * selection of any order changed (that solve's capture must not run inside a stream
 * capture). Applies to single right-hand-side solves in FMMBEM_MIXED and FMMBEM_FP64 without
 * profiling; FMMBEM_EDEVICE from the solve if the graph cannot be built. Default off. */
int fmmbem_set_device_loop(fmmbem_handle* h, int on);

/* Which boundary-integral operator A the mat-vecs and solves of a handle apply
 * (eq. laplace_matrix; for Stokes eqs. stokes_bem_discretized and stresslet):
 *   SINGLE : A = V, V_ij = (1/4pi) int_j 1/r dS; the first-kind system for the unknown
 *            normal derivative when phi is given (default).
 *   DOUBLE : A = 1/2 I + K, K_ij = (1/4pi) int_j n_j.(x_i - y)/r^3 dS; the second-kind
 *            system of eq. laplace_bem_final for the unknown phi when the normal
 *            derivative q is given, with right-hand side V q. n is the panel normal of
 *            the mesh's triangle order, which must point out of the solution domain: for
 *            an exterior problem the triangles are ordered so that n points into the body.
 *            The FMM far field then carries dipoles (P2M of n.grad of the regular solid
 *            harmonics); the near field sums n_j.(x_i - y)/r^3 over the K Gauss points and
 *            adds the double-layer correction rows.
 *            Stokes: A = 1/2 I + B, B the stresslet double layer (1/8pi) int T.n dS, the
 *            second-kind system for the velocity u when the traction t is given (right-hand
 *            side A_single t). Its far field is four Laplace dipole expansions evaluated like
 *            the Stokeslet's: sum (a.r)(n.r) r / r^5 = (S_i - x_b d_i S_b + d_i S_0) / 6 with
 *            dipole moments a_b n + n_b a and (a.y) n + (n.y) a. On a closed surface the
 *            normal field n is a (near-)null vector of 1/2 I + B: solutions are determined up
 *            to c n, as the single layer's tractions are.
 * FMMBEM_ESTATE for DOUBLE on a batched handle, FMMBEM_EINVAL for another value. */
#define FMMBEM_LAYER_SINGLE 0
#define FMMBEM_LAYER_DOUBLE 1
int fmmbem_set_layer(fmmbem_handle* h, int layer);

/*
 * y = A x through the FMM at expansion order p (eq. matvec-onerow with the
 * far field by P2M, M2M, M2L, L2L, L2P and the near field by P2P plus the
 * precomputed corrections).
 *   p      : 1 <= p <= opts.p_max
 *   x_dev  : [n_unknowns] doubles, device ([FMMBEM_BATCH][n_unknowns] on a batched handle)
 *   y_dev  : as x_dev (must not alias x_dev)
 * Asynchronous on the handle's stream. Errors: FMMBEM_EINVAL, FMMBEM_EDEVICE.
 */
int fmmbem_matvec(fmmbem_handle* h, int p, const double* x_dev, double* y_dev);

/*
 * y = A x by direct summation over every (collocation point, Gauss point)
 * pair (the Appendix algorithm) plus the same corrections: the dense
 * operator the FMM approximates. Same arguments as fmmbem_matvec without p.
 */
int fmmbem_matvec_direct(fmmbem_handle* h, const double* x_dev, double* y_dev);

/*
 * Right-hand side of the Laplace first-kind problem with Dirichlet data
 * (Sec. 2.1, eqs. laplace_bem_final, laplace_matrix): b = phi/2 + K phi with
 * K_ij = 1/(4 pi) int_j n_j.(c_i - y)/|c_i - y|^3 dS_y, by direct summation in
 * FP64 with the same near-singular rule (the self term of a flat panel is 0).
 *   known_dev : [n_panels] doubles, phi at the collocation points, device
 *   b_dev     : [n_panels] doubles, device
 * Errors: FMMBEM_ESTATE on a Stokes handle, FMMBEM_EINVAL, FMMBEM_EDEVICE.
 */
int fmmbem_rhs(fmmbem_handle* h, const double* known_dev, double* b_dev);

/*
 * Integral of a panel field over each body: out[b][a] = sum over the panels j of body b of
 * S_j x_j[a] (a < 1 Laplace, a < 3 Stokes), in FP64. For the traction t of a Stokes solve
 * this is the force on body b (the drag of Sec. 3.2 and Table rbc_richardson_values); for
 * the Laplace unknown q = dphi/dn it is the flux through the body's surface.
 *   x_dev   : [n_unknowns] doubles, device, the caller's panel order (one vector; vector q of a
 *             batch starts at x_dev + q n_unknowns)
 *   out_host: [fmmbem_n_bodies(h)][dof] doubles, host (written before the call returns)
 * Synchronizes the handle's stream. Errors: FMMBEM_EINVAL, FMMBEM_EDEVICE.
 */
int fmmbem_body_integrals(fmmbem_handle* h, const double* x_dev, double* out_host);

/* Number of bodies of the handle's mesh (1 when the mesh named none); -1 for NULL. */
int fmmbem_n_bodies(const fmmbem_handle* h);

/*
 * Stokes double layer (eq. stresslet, T_ijk contracted once with the panel
 * normal): y = B u with B_iJ = 1/(8 pi) int_J 6 e e^T (e.n_J)/|e|^5 dS_y,
 * e = y - c_i, by direct summation in FP64 (the self term of a flat panel is
 * 0). u_dev, y_dev: [n_panels][3] doubles, device. FMMBEM_ESTATE on a Laplace handle.
 */
int fmmbem_stokes_dl_apply(fmmbem_handle* h, const double* u_dev, double* y_dev);

/*
 * Relaxation rule (eqs. matrix-perturbation and fmm_p): with
 * eps = min(eta / min(rho_prev, 1), 1), returns
 * min(p_initial, max(p_min, ceil(-log2 eps))). ceil(-log2 eps) is evaluated
 * exactly from the binary exponent of eps. Pure host function.
 */
int fmmbem_relaxed_p(double eta, double rho_prev, int p_initial, int p_min);

/*
 * Restarted GMRES(m) on A x = b (Sec. 2.4) with FP64 Arnoldi (classical
 * Gram-Schmidt, reorthogonalized when the first projection removes more than
 * half of the vector's squared norm), Givens rotations and the residual estimate
 * rho_k = |g_{k+1}| / ||b||. Step k uses the mat-vec at
 *   p_k = fmmbem_relaxed_p(tol, rho_{k-1}, p_initial, p_min)  if relax != 0,
 *   p_k = p_initial                                           otherwise.
 * Restart residuals and the final true residual use p_initial.
 *   rhs_dev   : [n] doubles, device
 *   tol       : relative residual target (also eta of the relaxation rule)
 *   x_dev     : [n] doubles, device; in: ignored (x0 = 0); out: solution
 *   iters     : out, number of Arnoldi steps (mat-vecs inside GMRES)
 *   p_hist    : out, [opts.max_iter] ints, host, p used at each step (may be NULL)
 *   res_hist  : out, [opts.max_iter + 1] doubles, host, rho_0 = 1, rho_1.. (may be NULL)
 *   true_res  : out, ||b - A_{p_initial} x|| / ||b|| after the solve (may be NULL)
 * With FMMBEM_MIXED_REFINED, iters, p_hist and res_hist count the inner (mixed) Arnoldi steps
 * of all outer steps in order; the entry of res_hist after an outer step's last inner step is
 * that step's FP64 residual, and true_res the last one.
 * Returns 0 (converged), FMMBEM_NOT_CONVERGED, or a negative error.
 */
int fmmbem_solve(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial,
                 int p_min, double* x_dev, int* iters, int* p_hist, double* res_hist,
                 double* true_res);

/*
 * fmmbem_solve with host buffers: copies rhs_host to the device, solves,
 * and copies the solution back into x_host before returning (synchronous).
 * rhs_host, x_host: [n] doubles, host (pinned memory gives the fastest copies).
 */
int fmmbem_solve_host(fmmbem_handle* h, const double* rhs_host, double tol, int relax,
                      int p_initial, int p_min, double* x_host, int* iters, int* p_hist,
                      double* res_hist, double* true_res);

/*
 * Relaxed GMRES for the nrhs systems A x_q = b_q of a batched handle (opts.nrhs > 1:
 * FMMBEM_BATCH Laplace or up to FMMBEM_STOKES_BATCH_MAX Stokes right-hand sides), in
 * lockstep: every mat-vec evaluates all systems' basis vectors together (one P2M, M2M, M2L,
 * L2L, L2P and P2P pass for the whole batch) at the largest order p_k any active system's
 * relaxation rule (Sec. 2.6) asks for; each system keeps its own residual, Hessenberg
 * matrix and restarts and leaves the lockstep when it converges.
 *   rhs_dev, x_dev : [nrhs][n_unknowns] doubles, device
 *   iters          : [nrhs] host, mat-vecs while each system was active (or NULL)
 *   p_hist         : [max_iter] host, the order of each batched mat-vec (or NULL)
 *   res_hist       : [nrhs][max_iter + 1] host (or NULL)
 *   true_res       : [nrhs] host, ||b - A x|| / ||b|| at p_initial (or NULL)
 * Returns 0 when every system converged, FMMBEM_NOT_CONVERGED otherwise, FMMBEM_ESTATE on a
 * handle that is not batched (and fmmbem_solve returns FMMBEM_ESTATE on a batched one).
 */
int fmmbem_solve_batch(fmmbem_handle* h, const double* rhs_dev, double tol, int relax, int p_initial,
                       int p_min, double* x_dev, int* iters, int* p_hist, double* res_hist,
                       double* true_res);

/*
 * Single expansions (Sec. 2.5, spherical-harmonic forms of M_n^m and L_n^m):
 * form the multipole (kind 0) or local (kind 1) expansion of order p about
 * `center` (host, 3 doubles) from n_src point charges, then evaluate it at
 * n_tgt targets, all in FP64 on the device. Used to check eq. multipole_error.
 *   src_dev : [n_src][4] doubles (x, y, z, q), device
 *   tgt_dev : [n_tgt][3] doubles, device
 *   out_dev : [n_tgt] doubles, device: sum_n sum_m M_n^m I_n^m(x - center) (kind 0)
 *             or sum_n sum_m L_n^m R_n^m(x - center) (kind 1)
 *   scale   : length used to scale the expansion (any positive number; the
 *             result does not depend on it up to rounding)
 */
int fmmbem_expansion_eval(int kind, int p, const double* center, double scale, int n_src,
                          const double* src_dev, int n_tgt, const double* tgt_dev, double* out_dev,
                          void* stream);

/*
 * fmmbem_expansion_eval without any allocation (the paper has no counterpart: this
 * is an interface for callers that cannot allocate device memory, e.g. code inside
 * a CUDA-graph capture or under a memory arena). Same arguments and results as
 * fmmbem_expansion_eval; the expansion coefficients are kept in a fixed module-global
 * device array of one expansion of order <= FMMBEM_P_MAX (2448 bytes, held by every
 * GPU that loads the library until the process exits) instead of a per-call buffer.
 *   - p > FMMBEM_P_MAX is rejected with FMMBEM_EINVAL.
 *   - No cudaMalloc, cudaFree or allocating routine is called.
 *   - The first call on each device does a one-time set-up there (looks up the
 *     array's device address and fills a small constant table with a synchronous
 *     copy); make that first call before any stream capture.
 *   - Work is queued on `stream` and the call returns without synchronizing.
 *   - All calls share the one array: calls whose work overlaps on the GPU (other
 *     streams, other host threads) race on it; serialize them.
 */
int fmmbem_expansion_eval_static(int kind, int p, const double* center, double scale, int n_src,
                                 const double* src_dev, int n_tgt, const double* tgt_dev, double* out_dev,
                                 void* stream);

/* Sizes of the tree and lists built by fmmbem_create (algorithmic work counts). */
typedef struct {
    int64_t n_panels, n_sources, n_cells, n_leaves, n_levels;
    int64_t n_m2l_pairs;          /* all M2L pairs */
    int64_t n_m2l_same_level;     /* pairs whose cells have the same size */
    int64_t n_p2p_pairs;          /* leaf-leaf near-field pairs */
    int64_t n_p2p_interactions;   /* sum over P2P pairs of targets x Gauss points */
    int64_t n_corrections;        /* entries of the near-singular/self correction table */
    int64_t n_m2l_tables;         /* distinct M2L operators (0: gather form only) */
    int64_t n_m2l_tiles;          /* GEMM tiles over the M2L pairs (SIMT kernel: 64 pairs) */
    double setup_seconds;         /* wall time of fmmbem_create */
    int64_t n_m2l_tiles_tc;       /* tensor-core tiles over the M2L pairs (128 rows) */
} fmmbem_stats;

int fmmbem_get_stats(const fmmbem_handle* h, fmmbem_stats* out);

/* Per-pass device timing, measured with CUDA events recorded around each
 * pass on the stream that launches it while profiling is enabled. */
#define FMMBEM_PASS_P2M 0
#define FMMBEM_PASS_M2M 1
#define FMMBEM_PASS_M2L 2
#define FMMBEM_PASS_L2L 3
#define FMMBEM_PASS_L2P 4
#define FMMBEM_PASS_P2P 5          /* near field + corrections */
#define FMMBEM_PASS_KRYLOV 6       /* Arnoldi, Givens and updates */
#define FMMBEM_PASS_MATVEC 7       /* whole mat-vec */
#define FMMBEM_N_PASSES 8
typedef struct {
    double ms[FMMBEM_N_PASSES];       /* accumulated milliseconds */
    int64_t launches[FMMBEM_N_PASSES]; /* kernel launches counted in each pass */
    int64_t calls[FMMBEM_N_PASSES];    /* timed intervals */
    double m2l_flops;                  /* accumulated algorithmic M2L flops: 2 (p+1)^4 per pair and expansion */
    double p2p_interactions;           /* accumulated P2P pair interactions */
    int64_t kernel_launches;           /* every kernel launched by the handle since the reset */
    double tc_ms;                      /* milliseconds of the M2M, M2L and L2L passes that ran on the
                                          tensor-core kernel (k_m2l_tc), a subset of ms[] */
    double tc_flops;                   /* algorithmic flops of those passes: 2 (p+1)^4 per M2L pair and
                                          expansion, and per M2M and per L2L translation of a cell */
} fmmbem_profile;

/* enable != 0 starts recording (and resets the counters); 0 stops. enable = 2 also runs each
 * profiled mat-vec's near field before its far field on one stream (same sums), so that every
 * pass's time is its kernels' own time rather than time spent waiting for SMs held by the
 * other field; 1 keeps the concurrent schedule of unprofiled mat-vecs. */
int fmmbem_profile_enable(fmmbem_handle* h, int enable);
int fmmbem_profile_get(fmmbem_handle* h, fmmbem_profile* out); /* synchronizes the stream */

/* Message of the last failure in this thread ("" if none). The message is kept per host
 * thread, not per handle, because fmmbem_create can fail before any handle exists. */
const char* fmmbem_last_error(void);

/*
 * Bounded device waits. Every wait inside the library's kernels (the grid barrier of the
 * cooperative Arnoldi step, the near field's bulk-copy stages, the tensor-core pipeline's
 * mbarriers) gives up after a fixed number of polls and raises a flag on the handle rather
 * than hold the GPU. fmmbem_solve and fmmbem_solve_batch clear the flags on entry and return
 * FMMBEM_ETIMEOUT when one was raised during the solve. fmmbem_matvec and
 * fmmbem_matvec_direct are asynchronous and do not read them: fmmbem_check_waits does.
 */
/* Synchronize the handle's streams, read and clear its wait flags: 0, or FMMBEM_ETIMEOUT when a
 * wait of the work queued since the last check gave up (the results of that work are invalid). */
int fmmbem_check_waits(fmmbem_handle* h);
/* Test hook: polls (about 64 ns each) after which a grid-barrier wait of the Arnoldi step gives
 * up; 0 restores the default 2^26. A tiny limit makes the waits run out on purpose, so that the
 * error path can be exercised without a fault: the solve returns FMMBEM_ETIMEOUT, the barrier
 * counters are reset and the handle stays usable. */
int fmmbem_set_wait_limit(fmmbem_handle* h, unsigned limit);

/*
 * Peak rates of this GPU at its current clocks: the denominators of the rooflines (the paper
 * has no counterpart; it is a measurement interface). One launch of `blocks` blocks
 * (0: 4 blocks of 256 threads per SM, one CTA per SM for TF32; at most one per SM for TF32)
 * runs `iters` iterations of eight independent chains per thread of one operation:
 *   FFMA  : fma.rn.f32                    2 flop each
 *   FFMA2 : fma.rn.f32x2 (paired FP32)    4 flop each
 *   RSQRT : rsqrt.approx.ftz.f32 (special-function unit), 1 result each
 *   DFMA  : FP64 fma                      2 flop each
 *   TF32  : tcgen05.mma.kind::tf32, M 128, N 256, K 8, from shared memory into TMEM,
 *           2 M N K flop each, 4 per iteration
 * ops receives the operations done, ms the CUDA-event time of the launch on `stream`
 * (synchronizes it). Errors: FMMBEM_EINVAL, FMMBEM_EDEVICE, FMMBEM_ETIMEOUT (the tensor-core
 * completion wait gave up).
 */
#define FMMBEM_PEAK_FFMA 0
#define FMMBEM_PEAK_FFMA2 1
#define FMMBEM_PEAK_RSQRT 2
#define FMMBEM_PEAK_DFMA 3
#define FMMBEM_PEAK_TF32 4
int fmmbem_peak(int kind, int blocks, int64_t iters, double* ops, double* ms, void* stream);

/*
 * The hand-written device primitives of the tree build (Sec. 2.5: the Morton-ordered octree,
 * its leaf classes and its list offsets), exported for callers that order their own points.
 *
 * fmmbem_sort_pairs_u64: stable least-significant-digit radix sort of n 64-bit keys (8-bit
 * digits over bits [0, end_bit); end_bit 0 = 64), carrying one int32 value per key
 * (vals_in/vals_out both NULL: keys only). keys_out/vals_out receive the keys in ascending
 * order and each key's value; keys of equal value keep their input order. All four are
 * device buffers of n elements on `stream` (NULL: the legacy default stream); inputs are
 * left unchanged and must not alias the outputs. Scratch is stream-ordered
 * (cudaMallocAsync). Synchronizes `stream` (it reads back the scatter's bounds flag).
 * Errors: FMMBEM_EINVAL (n < 0 or n >= 2^30, end_bit outside [0, 64], aliasing, one value
 * buffer without the other), FMMBEM_ENOMEM, FMMBEM_EDEVICE.
 *
 * fmmbem_scan_i32: prefix sum of n int32 values, out[i] = sum_{k<i} in[k] (inclusive = 0)
 * or sum_{k<=i} in[k] (inclusive != 0), wrapping in 32-bit arithmetic; device buffers on
 * `stream`, in == out allowed. Synchronizes `stream`. Errors: FMMBEM_EINVAL (n < 0),
 * FMMBEM_ENOMEM, FMMBEM_EDEVICE.
 */
int fmmbem_sort_pairs_u64(const uint64_t* keys_in_dev, uint64_t* keys_out_dev, const int32_t* vals_in_dev,
                          int32_t* vals_out_dev, int64_t n, int end_bit, void* stream);
int fmmbem_scan_i32(const int32_t* in_dev, int32_t* out_dev, int64_t n, int inclusive, void* stream);

/*
 * ---- Serving many solves at once.
 *
 * The paper solves one problem at a time. This is the request loop around its solver:
 * solves of different meshes, operators and tolerances share one GPU.
 *
 * fmmbem_server_submit copies a request and queues it. max_active worker threads take
 * queued requests in arrival order. A request is admitted as soon as:
 *   - a worker is free, and
 *   - the request's device-memory estimate (fmmbem_estimate_bytes) fits in what is left of
 *     hbm_budget (one request is always admitted when nothing else is running).
 * A smaller request that fits may therefore pass a larger one that does not.
 *
 * An admitted request is created and solved (fmmbem_solve_host) on its worker's own CUDA
 * stream. The workers' mat-vecs interleave on the device, and each request's state stays
 * resident until its solve ends.
 *
 * Handle cache (the paper has no counterpart: requests on one geometry are the serving case
 * of its repeated solves). The handle of a request that solved without error is kept idle
 * instead of destroyed, up to fmmbem_server_set_cache's count (default 4 max_active). A later
 * request on the same mesh (vertices and triangles equal byte for byte) with the same kernel,
 * gauss_k, ncrit, theta and options takes the idle handle and skips fmmbem_create; its tree,
 * lists, operators, correction rows and captured mat-vec graphs are reused. Idle handles count
 * against hbm_budget: a request that does not fit evicts them, least recently used first.
 *
 * Handles are independent and the library keeps no shared mutable state in a handle's path,
 * so concurrent requests give the results they give alone, up to floating-point summation
 * order.
 */
typedef struct fmmbem_server fmmbem_server;

typedef struct {
    int64_t ticket;
    int status;            /* fmmbem_solve's return value, or a negative error from fmmbem_create */
    int iters;             /* Arnoldi steps */
    double true_res;       /* ||b - A x|| / ||b|| after the solve */
    double queue_s;        /* submit -> admission */
    double setup_s;        /* fmmbem_create (about 0 when the handle came from the cache) */
    double solve_s;        /* fmmbem_solve_host (copies included) */
    double latency_s;      /* submit -> result ready */
    int64_t device_bytes;  /* admission estimate (of the cached handle's request when reused) */
    int32_t handle_reused; /* 1 when the request ran on a cached handle */
} fmmbem_result;

/* Conservative estimate of the device memory of a handle (bytes), -1 for bad arguments. */
int64_t fmmbem_estimate_bytes(int64_t n_panels, int kernel, int gauss_k, int ncrit, const fmmbem_opts* opts);

/* Start max_active (1..64) workers on the current device with an HBM budget in bytes. */
int fmmbem_server_create(int max_active, int64_t hbm_budget, fmmbem_server** out);

/*
 * Queue one solve. The mesh and rhs_host ([n_unknowns] doubles, host) are copied before the
 * call returns. x_host ([n_unknowns] doubles, host) receives the solution and must stay valid
 * until fmmbem_server_wait returns for the ticket. The other arguments are those of
 * fmmbem_create and fmmbem_solve (opts->stream is ignored: each worker has its own).
 * Errors: FMMBEM_EINVAL (NULL or empty arguments), FMMBEM_ESTATE (server shutting down).
 */
int fmmbem_server_submit(fmmbem_server* s, const fmmbem_mesh* mesh, int kernel, int gauss_k, int ncrit, double theta,
                         const fmmbem_opts* opts, const double* rhs_host, double tol, int relax, int p_initial,
                         int p_min, double* x_host, int64_t* ticket);

/* Keep at most max_handles idle handles (0 turns the cache off); extra idle handles are
 * destroyed at once, least recently used first. Errors: FMMBEM_EINVAL (NULL server, negative
 * count). */
int fmmbem_server_set_cache(fmmbem_server* s, int max_handles);

/* Requests served on a cached handle since the server was created (0 for NULL). */
int64_t fmmbem_server_cache_hits(fmmbem_server* s);

/* Block until the ticket's request has finished and return its result (each ticket once). */
int fmmbem_server_wait(fmmbem_server* s, int64_t ticket, fmmbem_result* out);

/* Finish every queued request, stop the workers, destroy the cached handles and free the
 * server. NULL is ignored. */
int fmmbem_server_destroy(fmmbem_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FMMBEM_H */
