/*
 * st.h - C ABI of the GB300 (sm_103a) space-time (p,delta)-Navier-Stokes
 * slab solver: matrix-free residual and Jacobian action of one DG-in-time
 * slab, the space-time Vanka smoother, the multigrid V-cycle and the
 * modified Newton step.
 *
 * Discretisation (arXiv 2603.28706):
 *   - Omega = [0,Lx]x[0,Ly](x[0,Lz]), uniform mesh of nx x ny (x nz) cells;
 *   - Q2 continuous velocity, Q1 continuous pressure (Taylor-Hood), Sec. 3.1;
 *   - DG(k) in time, Lagrange basis on the right (k+1)-point Gauss-Radau
 *     nodes of the slab I_n = (t0, t0+dt], Sec. 3.1, Rem. 3.2;
 *   - Nitsche boundary terms B_gamma of eq. def-b-gam on Gamma_D, the
 *     convective boundary term of eq. Defc on all of Gamma;
 *   - optional convection-aligned CIP on the interior faces, eq. scip-def
 *     (gamma_cip > 0), h_F = the face diameter (diagonal).
 *
 * Vector layout (all vector arguments): a slab vector is
 *     U = [V_1 ... V_{k+1} | P_1 ... P_{k+1}]            (eq. slab-system)
 * V_mu is component-major (component c = 0..dim-1), each component
 * lexicographic on the Q2 node grid (2nx+1)(2ny+1)(2nz+1), x fastest;
 * P_mu is lexicographic on the Q1 grid (nx+1)(ny+1)(nz+1) (pressure_space = 1:
 * (dim+1) coefficients per cell, cells lexicographic).  A velocity field
 * (v_prev, one time node) is dim*(2nx+1)(2ny+1)(2nz+1) values.  On level l
 * of the multigrid hierarchy the mesh is n/2^(L-l) cells per direction.
 *
 * Ownership: every vector argument is a caller-owned, contiguous DEVICE
 * pointer, 16-byte aligned, of dtype double (ST_FP64) or float (ST_FP32).
 * The handle owns all other device memory (coefficient caches, patch
 * factorisations, coarse operators, Krylov workspace).  Calls are enqueued
 * on the stream given to st_setup_mesh and return before the GPU finishes,
 * except st_newton_step and st_mnorm which synchronise that stream (their
 * results steer host control flow).  Calls on one handle must not overlap.
 *
 * Errors: every call returns an st_status.  Invalid arguments give ST_EINVAL
 * before anything is launched; CUDA failures give ST_ECUDA; st_last_error()
 * returns a message for the last failure on the handle.  After a status other
 * than ST_ECUDA the handle stays usable.  No call allocates or frees caller
 * memory; no call falls back to the CPU.
 */
#ifndef ST_H_
#define ST_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ST_OK = 0,
  ST_EINVAL = 1,            /* bad argument, size or state                     */
  ST_ECUDA = 2,             /* a CUDA call or kernel failed                    */
  ST_ENOMEM = 3,            /* device allocation failed                        */
  ST_NOT_CONVERGED = 4,     /* Newton or FGMRES missed its tolerance (Sec. 6.2) */
  ST_LINESEARCH_FAILED = 5, /* Armijo backtracking hit lambda_min (Sec. 6.2)  */
  ST_SINGULAR_PATCH = 6,    /* a Vanka patch matrix has a zero pivot          */
  ST_DEVICE_TIMEOUT = 7     /* a bounded device wait ran out                   */
} st_status;

/* Linearisation of the constitutive term (Sec. 4): Picard eq.
 * local-tangent-picard, exact Newton eq. local-tangent-exact, modified
 * Newton (stress-clipped rank one) eq. local-tangent-clip. */
typedef enum { ST_PIC = 0, ST_EXN = 1, ST_MODN = 2 } st_tangent;

typedef enum { ST_FP64 = 0, ST_FP32 = 1 } st_prec;

/* Problem and solver parameters, copied at setup (plain old data). */
typedef struct {
  int dim, nx, ny, nz;        /* dimension 2 or 3; cells per direction (nz ignored in 2D) */
  double Lx, Ly, Lz;          /* box lengths                                         */
  int k;                      /* DG degree in time, 0 <= k <= 3 (k+1 Radau nodes)    */
  double t0, dt;              /* slab I_n = (t0, t0 + dt]                            */
  double p, delta, nu, nu_inf;/* stress law eq. constitutive-law: 1 < p <= 2, delta > 0 */
  double sigma_max;           /* modN stress clip (Sec. 4.4); may be +inf             */
  double gamma1, gamma2;      /* Nitsche penalties, eq. def-b-gam-3                   */
  unsigned dirichlet_mask;    /* bit s = 2*axis + (upper side): side is Gamma_D      */
  int inflow_profile;         /* 0: g_D = 0; 1: u_x = vbar*6y(1-y)[*6z(1-z)] scaled,
                                 lifting constant in x                                */
  double vbar;                /* inflow mean velocity                                */
  double q_sign;              /* coefficient of (u.n, q)_{Gamma_D} in B^s; -1 = as
                                 printed in eq. def-b-gam-2.5                          */
  int levels;                 /* multigrid levels (1 = no coarsening)                */
  int pre_smooth, post_smooth;/* Vanka sweeps per level (Sec. 6.3, Sec. 7: 2 + 2)    */
  double omega;               /* Vanka damping, eq. stmg-vanka-update                */
  double rho_refresh;         /* patch refresh threshold rho (Sec. 6.3)              */
  int fgmres_restart, fgmres_maxit, newton_maxit;
  double tol_abs, tol_rel;    /* Newton stop, eq. nk-stop                            */
  double lin_rtol;            /* fixed relative FGMRES tolerance (Picard)            */
  double ew_gamma, ew_alpha, ew_max; /* Eisenstat-Walker forcing, eq. nk-inexact-newton */
  double armijo_c, lambda_min;/* Armijo backtracking on phi = 1/2 |R|_M^2 (Sec. 6.2) */
  int coarse_sweeps;          /* Vanka sweeps (exact patches) on the coarsest level  */
  double gamma_cip;           /* CIP weight gamma_CIP of eq. scip-def; 0 = no CIP,
                                 must be finite and >= 0                             */
  int finest_patches;         /* 0: surrogate patches on the finest level (eq.
                                 surrogate-diag, Sec. 6.3); 1: exact patches
                                 R_K J_n R_K^T of the linearisation, under the same
                                 refresh rule (not with gamma_cip > 0)               */
  int coarse_solve;           /* coarsest level of the V-cycle: 0 = coarse_sweeps
                                 Vanka steps; 1 = FP64-accurate direct solve of the
                                 Galerkin operator A_0 (dense FP64 assembly, FP32
                                 Gauss-Jordan inverse, FP64 iterative refinement to
                                 |b - A_0 x|_2 <= 1e-12 |b|_2, at most 10 steps);
                                 needs a nonsingular A_0 (a Gamma_N side fixes the
                                 pressure constant) of at most 20000 dofs          */
  int pressure_space;         /* 0: Q1 continuous pressure (Taylor-Hood); 1: P1disc,
                                 the pair of the paper's experiments (Sec. 7): per
                                 cell the basis 1, 2 r_a - 1 (r_a the cell's
                                 reference coordinates), P_mu = [cell][1 + dim]
                                 with cells lexicographic, x fastest                */
  int smoother;               /* 0: additive Vanka step of eq. stmg-vanka-update (one
                                 defect per step); 1: the same update taken class by
                                 class over the 2^dim colour classes of cells (cell
                                 parities px + 2 py + 4 pz, in that order), a fresh
                                 defect before each class: multiplicative between
                                 classes, additive inside one (its cells share no
                                 dof); 2^dim defects per step; 2: the class-by-class
                                 step on the finest level, the additive step with
                                 omega_coarse on the coarser levels                  */
  int patch_type;             /* Vanka patches (Sec. 6.3): 0 = cell patches (every dof
                                 of a cell); 1 = vertex-star patches: the velocity
                                 nodes of the 2^dim cells around a vertex that are not
                                 on the star's outer boundary, and the vertex's
                                 pressure, all k+1 time nodes, classes by vertex
                                 parity; exact patches only (finest_patches = 1,
                                 gamma_cip = 0, pressure_space = 0)                  */
  double omega_coarse;        /* Vanka damping below the finest level with smoother = 2
                                 (0 = omega)                                          */
} st_params;

typedef struct {
  int newton_iters;           /* nonlinear iterations taken                          */
  int fgmres_iters_total;     /* FGMRES iterations over all Newton steps             */
  int fgmres_iters_last;
  int patch_rebuilds;         /* surrogate patch inverses built                      */
  double lambda_last;         /* last accepted damping                               */
  double res_norm_initial;    /* |R_n(U^0)|_M                                        */
  double res_norm_final;      /* |R_n(U^m)|_M at exit                                */
  int status;                 /* st_status of the solve                              */
} st_newton_info;

typedef struct st_problem st_problem;

/* Create a problem on the current CUDA device; all work is enqueued on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream).  Validates the
 * parameters (ST_EINVAL), precomputes the colour classes of cells and the
 * boundary-face lists of every level, and allocates the handle's caches. */
st_status st_setup_mesh(const st_params* params, void* cuda_stream, st_problem** out);

/* Free everything the handle owns.  NULL is accepted. */
st_status st_destroy(st_problem* h);

/* (k+1)(M_v + M_p) on level `level` (0 = coarsest, levels-1 = finest), the
 * length of a slab vector (eq. slab-system); 0 for a bad level. */
size_t st_num_dofs(const st_problem* h, int level);

/* R = R_n(U) = -[(K_t (x) M_x) V - (m_t (x) M_x) v_prev ; 0] + (M_t (x) I) F(U)
 * (eq. slab-underint), residual convention "right-hand side minus left-hand
 * side" (eq. disc-residual).  F_mu at node t_n^mu is the spatial residual of
 * eq. disc with the form A_gamma of eq. def-a-gam (plus s_CIP(u; u, .) of eq.
 * scip-def when gamma_cip > 0) and data
 * B_gamma(g_D) of eq. def-b-gam.  v_prev: left trace u^-(t_{n-1}) (velocity
 * field); f: body force as Q2 nodal coefficients per time node ((k+1) velocity
 * fields, layout of V) or NULL.  Finest level.  prec selects the dtype of all
 * four vectors and the arithmetic. */
st_status st_residual(st_problem* h, st_prec prec, const void* U, const void* v_prev, const void* f, void* R);

/* Evaluate and keep the state-dependent coefficients of the linearisation at
 * the iterate U (FP64: A^m = D u^m, Delta^{m,2}, mu^m, eta^m and the rank-one
 * factor of the tangent at every quadrature point and Radau node, Sec. 4.1;
 * plus an FP32 copy).  Later st_jacobian_apply calls with U_state == NULL use
 * them.  Invalidates the preconditioner. */
st_status st_linearize(st_problem* h, st_tangent tangent, const void* U);

/* out = J_n(U) dU, eq. slab-underint-jac:
 *   J_n = [[K_t (x) M_x, 0], [0, 0]] + (M_t (x) I) diag(J_1 .. J_{k+1}),
 * J_mu the spatial linearisation with the selected tangent (Sec. 4.2-4.4,
 * eq. Jmu-block, eq. Amu-decomp; A_CIP with the advecting field lagged at the
 * linearisation state, Sec. 4.2-4.4, when gamma_cip > 0).  U_state != NULL: linearise
 * at U_state first (as st_linearize); NULL: use the last st_linearize, whose
 * tangent must equal `tangent` (else ST_EINVAL).  dU and out: slab vectors of
 * dtype prec; U_state is always double. */
st_status st_jacobian_apply(st_problem* h, st_tangent tangent, st_prec prec, const void* U_state, const void* dU,
                            void* out);

/* *out = |r|_M = sqrt(r_v^T M_v r_v + r_p^T M_p r_p) with M_v = M_t (x) M_x and
 * M_p = M_t (x) M_{x,p} (Sec. 6.1).  r: FP64 slab vector, finest level.
 * Synchronises the stream. */
st_status st_mnorm(st_problem* h, const void* r, double* out);

/* Build the Vanka smoother and coarse operators for the current
 * linearisation: finest-level surrogate patch matrices with the coefficients
 * frozen at t_rep = midpoint of I_n (eq. surrogate-diag), Galerkin coarse
 * operators A_l = P^T A_{l+1} P (Sec. 6.3) and their exact cell patches,
 * inverted explicitly (batched Gauss-Jordan with partial pivoting), on every
 * level including the coarsest (finest_patches = 1: exact finest patches
 * instead of the surrogate ones).  With CIP the finest-level defects and
 * the finest surrogate patches include it (R_K S R_K^T of the CIP matrix at
 * the representative state), while the Galerkin coarse operators and their
 * patches are built from the cell-local part of the Jacobian (all but the
 * interior-face CIP coupling).  prec: FP32 (mixed) or FP64
 * storage/arithmetic of the smoother.  Called implicitly by
 * st_vanka_smooth / st_vcycle when missing. */
st_status st_precond_setup(st_problem* h, st_prec prec);

/* `sweeps` Vanka steps on level `level` (eq. stmg-vanka-update):
 *   d <- d + omega sum_K R_K^T A_K^{-1} R_K (r - A_l d)
 * (smoother = 1: over one colour class at a time, a fresh defect each),
 * cell patches K with all k+1 time nodes; A_K exact on coarse levels and the
 * surrogate of eq. surrogate-diag on the finest level (exact there too with
 * finest_patches = 1).  r, d: slab vectors of
 * that level, dtype prec; d is updated in place. */
st_status st_vanka_smooth(st_problem* h, int level, int sweeps, st_prec prec, const void* r, void* d);

/* d = B^{-1} r: one space-time multigrid V-cycle on the finest level
 * (Sec. 6.3): pre_smooth Vanka sweeps, restriction P^T, recursion, coarsest
 * solve (coarse_solve: Vanka steps, or the FP64-accurate direct solve; with
 * levels = 1 the finest level is the coarsest), prolongation P, post_smooth
 * sweeps.  r, d: finest slab vectors of
 * dtype prec (d is overwritten). */
st_status st_vcycle(st_problem* h, st_prec prec, const void* r, void* d);

typedef struct {
  int iters;                  /* FGMRES iterations                                   */
  double res_norm;            /* |b - J x|_M at exit                                 */
  double rhs_norm;            /* |b|_M                                               */
} st_linsolve_info;

/* x = J^{-1} b for the current linearisation (st_linearize): right-
 * preconditioned FGMRES(fgmres_restart) in FP64 in the block mass inner
 * product of Sec. 6.1 (classical Gram-Schmidt twice), one V-cycle of
 * precision vcycle_prec per iteration (Sec. 6.3), from x = 0 until
 * |b - J x|_M <= rtol |b|_M or maxit iterations.  Builds the preconditioner
 * when it is missing or of the other precision.  b, x: FP64 finest slab
 * vectors.  Synchronous.  info may be NULL.  ST_NOT_CONVERGED when maxit is
 * reached first (x then holds the last iterate). */
st_status st_fgmres_solve(st_problem* h, st_prec vcycle_prec, const void* b, void* x, double rtol, int maxit,
                          st_linsolve_info* info);

/* Globalised (modified) Newton on the slab (Sec. 4.1, 6.1-6.3):
 *   repeat: R = R_n(U); stop if |R|_M <= tol_abs or <= tol_rel |R^0|_M
 *   (eq. nk-stop); linearise with `tangent`; refresh the preconditioner by the
 *   rule of Sec. 6.3; solve J dU = R by right-preconditioned FGMRES (FP64) with
 *   one V-cycle of precision vcycle_prec per iteration to the Eisenstat-Walker
 *   forcing (eq. nk-inexact-newton; Picard: lin_rtol); Armijo backtracking on
 *   phi = 1/2 |R|_M^2 (exN, modN; Picard takes lambda = 1); U += lambda dU.
 * U (FP64 slab vector) is updated in place.  Synchronous.  info may be NULL.
 * Returns ST_NOT_CONVERGED / ST_LINESEARCH_FAILED when the step fails
 * (Sec. 6.2: the time-step solve is declared unsuccessful). */
st_status st_newton_step(st_problem* h, st_tangent tangent, st_prec vcycle_prec, void* U, const void* v_prev,
                         const void* f, st_newton_info* info);

/* Message describing the last failure on h (never NULL). */
const char* st_last_error(const st_problem* h);

/* Launch shapes chosen by the library's autotuner in this process, one line
 * per tuned kernel and launch size: the choice and every candidate's time.
 * The first launch of the Jacobian action's volume kernel (cells per CTA),
 * of the Vanka patch solves and of the coarse-level operator (threads per
 * CTA, CTAs per SM) with a new size times the candidates on the real
 * arguments with CUDA events (not while the stream is being captured; not at
 * all when the environment sets ST_AUTOTUNE=0) and keeps the fastest; every
 * candidate computes the same values.  Writes at most len bytes (NUL-
 * terminated) into buf (may be NULL) and returns the length the whole report
 * needs, NUL included. */
size_t st_autotune_report(char* buf, size_t len);

/* Allocation-free variant of st_mnorm.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a memory
 * pool owned by another framework with a hard cap, a plugin host that forbids
 * device allocations, a latency-critical path that must not touch the
 * allocator).  It needs no handle: params gives the mesh, k and dt; r is an
 * FP64 finest-level slab vector (device pointer, caller-owned) and *out (host)
 * receives |r|_M, the block mass norm computed by st_mnorm.  The work vectors and
 * partial sums live in a static device array of 16 MiB that every GPU loading
 * the library holds until exit, so the slab may have at most
 * (2^21 - 2048) / 2 = 1 047 552 dofs; larger slabs give ST_EINVAL with a
 * message on stderr.  The first call on a device resolves the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The call calls no cudaMalloc or cudaFree
 * and synchronises `cuda_stream`.  All calls share the array: calls that
 * overlap on the GPU race and must be serialised by the caller. */
st_status st_mnorm_noalloc(const st_params* params, void* cuda_stream, const double* r, double* out);

/* ---------------------------------------------------------------- batches
 * Many independent slab problems solved side by side: each instance has its
 * own mesh, parameters and state (Sec. 3 and 6 per instance); all instances
 * share dim and k (one kernel instantiation).  The operator calls run the
 * volume terms of every instance in one persistent launch whose work queue
 * holds (instance, cell batch) items, so instances of uneven size keep all SMs
 * busy; the face terms and the node sums follow per instance.  Vector
 * arguments are host arrays of n caller-owned device pointers (instance i:
 * the layout and dtype of the single-problem calls).  Calls are enqueued on
 * `cuda_stream`; the batch owns its instances. */
typedef struct st_batch st_batch;

/* n instances from params[0..n-1] (n >= 1).  ST_EINVAL if a parameter block
 * is invalid or dim / k differ between instances. */
st_status st_batch_setup(const st_params* params, int n, void* cuda_stream, st_batch** out);
st_status st_batch_destroy(st_batch* b);
/* Space-time dofs of instance i (0 for a bad index). */
size_t st_batch_num_dofs(const st_batch* b, int i);

/* st_linearize for every instance at its state U[i] (FP64). */
st_status st_batch_linearize(st_batch* b, st_tangent tangent, const void* const* U);
/* out[i] = J_i dU[i] for every instance (the linearisation of st_batch_linearize
 * with the same tangent; ST_EINVAL otherwise). */
st_status st_batch_jacobian_apply(st_batch* b, st_tangent tangent, st_prec prec, const void* const* dU,
                                  void* const* out);
/* R[i] = R_n(U[i]) with data v_prev[i] and f[i] (f may be NULL: all forcings
 * zero; an entry may be NULL: that instance's forcing is zero). */
st_status st_batch_residual(st_batch* b, st_prec prec, const void* const* U, const void* const* v_prev,
                            const void* const* f, void* const* R);
/* st_newton_step for every instance, the instances driven concurrently (one
 * host thread and one internal CUDA stream each); U[i] updated in place,
 * info[i] filled (info may be NULL).  Synchronous.  Returns ST_OK when every
 * instance converged, else the status of the first instance that did not
 * (the others still complete). */
st_status st_batch_newton_step(st_batch* b, st_tangent tangent, st_prec vcycle_prec, void* const* U,
                               const void* const* v_prev, const void* const* f, st_newton_info* info);
/* st_fgmres_solve for every instance (after st_batch_linearize), the
 * instances driven concurrently (one host thread and one internal CUDA stream
 * each): x[i] = J_i^{-1} rhs[i] to |rhs[i] - J_i x[i]|_M <= rtol |rhs[i]|_M
 * with one V-cycle of precision vcycle_prec per iteration.  info[i] filled
 * (info may be NULL).  Synchronous.  Returns ST_OK when every instance met
 * rtol, else the status of the first instance that did not (the others still
 * complete). */
st_status st_batch_fgmres_solve(st_batch* b, st_prec vcycle_prec, const void* const* rhs, void* const* x,
                                double rtol, int maxit, st_linsolve_info* info);

/* Message describing the last failure on b (never NULL). */
const char* st_batch_last_error(const st_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* ST_H_ */
