/*
 * hfe.h — C ABI of the B300 hex8 finite-strain Hill-48 plasticity library.
 *
 * The library computes, on one GPU, the per-Newton-iteration sweep over all hex8 Gauss
 * points of a displacement-based finite element model in the additive logarithmic-strain
 * formulation (paper Sec. 2.2.2: geometric pre-processor Eq. c_decomp, log-space elasticity
 * Eq. T, Hill-48 effective stress Eq. Phi_hill with App. A.1, hardening Eq. Hard,
 * associative flow Eq. ep_evol and the Kuhn-Tucker conditions Eq. KT, return mapping
 * Eq. Tr_stress/Eq. local_cpp, geometric post-processor Eq. proj_lagrange/Eq. pk_stress),
 * the element residual and consistent tangent (Sec. 2.2.4, Eq. Stiffness_mat), their
 * assembly into a block-CSR matrix, the linear solve, the global Newton loop over load
 * steps, and the discrete adjoint (Sec. 2.3, Eq. dR_u, Eq. main_grad, Algorithm
 * adjoint_ad).
 *
 * Units are whatever the caller uses consistently (the tests use mm, N, MPa).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - hex8 node order C3D8: bottom face 0-1-2-3 counter-clockwise seen from +z, top 4-7;
 *  - Gauss points: 2x2x2 at +-1/sqrt(3), unit weights, gp = i + 2j + 4k (xi fastest);
 *    the global Gauss-point index is 8*element + gp;
 *  - degrees of freedom are node-major: dof = 3*node + component;
 *  - symmetric tensors are 6 tensor components in the order (11, 22, 33, 12, 23, 13);
 *  - history is structure-of-arrays [7][n_gp]: eps_p (6 components), alpha;
 *  - theta (material parameters) is [n_mat][11]: E, nu, F, G, H, L, M, N, h1, h2, h3
 *    with (h1, h2, h3) = (K, eps0, n) for Swift sigma_y = K (eps0 + alpha)^n and
 *    (sigma0, Q, b) for Voce sigma_y = sigma0 + Q (1 - exp(-b alpha)); the yield function
 *    is f = sqrt(T:H:T) - sqrt(2/3) sigma_y(alpha) with alpha-rate sqrt(2/3) gamma-rate;
 *  - Dirichlet data (dof[i], value[i]) prescribe u[dof] = t * value at load factor t;
 *  - pointer arguments marked "host or device" may point to either; the library detects
 *    which with cudaPointerGetAttributes and copies on its stream.  All other pointers
 *    are host pointers.
 *
 * Ownership: the caller owns every buffer it passes.  hfe_create copies what it needs;
 * the handle owns its device workspaces and frees them in hfe_destroy.
 *
 * Errors: every function returns an hfe_status; none aborts, exits or traps.  Device
 * loops are bounded (local Newton, Krylov iterations) and report through a device status
 * word that the host reads after each sweep and solve.  A non-zero status leaves the
 * handle usable; hfe_last_error() gives a one-line description.
 */
#ifndef HFE_H
#define HFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HFE_OK = 0,
  HFE_EINVAL = -1,      /* invalid argument (sizes, indices, NULL where required) */
  HFE_ENOMEM = -2,      /* device allocation failed */
  HFE_ECUDA = -3,       /* CUDA runtime error (message in hfe_last_error) */
  HFE_EDETJ = -4,       /* an element has det(dX/dxi) <= 0 or det F <= 0, or one that is not a
                           number (non-finite coordinates or displacements) */
  HFE_ENEWTON = 1,      /* global Newton did not converge within newton_maxit */
  HFE_ELOCAL = 2,       /* a local return mapping did not converge (count in stats) */
  HFE_EPCG = 3,         /* Krylov solve did not reach pcg_rtol within pcg_maxit, broke down, or (hfe_solve)
                           the matrix has diagonal blocks that are not positive definite */
  HFE_ENONFINITE = 4,   /* a non-finite value appeared in a residual, stress or solve */
  HFE_EBARRIER = 5      /* a grid-barrier wait of a one-launch Krylov solve ran out (options.
                           barrier_spin_limit): the solve was abandoned and every CTA left; the
                           handle stays usable.  Not retried by adaptive stepping: hfe_forward
                           returns it with the state of the last converged step */
} hfe_status;

typedef struct hfe_handle hfe_handle;

/* Mesh: X[n_nodes*3] reference coordinates, conn[n_el*8] node ids in C3D8 order. */
typedef struct {
  int64_t n_nodes;
  int64_t n_el;
  const double* X;
  const int32_t* conn;
} hfe_mesh;

/* Boundary data (Eq. equilibrium): n_fixed Dirichlet entries (sorted or not, no duplicates),
 * and an optional nodal dead load f_ext[n_dof] at t = 1 (NULL for none), scaled by t. */
typedef struct {
  int64_t n_fixed;
  const int64_t* dof;
  const double* value;
  const double* f_ext;
} hfe_bc;

#define HFE_HARDENING_SWIFT 0
#define HFE_HARDENING_VOCE 1

/* Material: n_mat = 1 (uniform) or n_el (per element); theta[n_mat*11] as above;
 * Theta NULL (material axes = global axes) or [n_mat*9] row-major 3x3 whose columns are the
 * material axes in global coordinates (App. A.1: H_g = Theta Theta : H_l : Theta^T Theta^T). */
typedef struct {
  int hardening;
  int64_t n_mat;
  const double* theta;
  const double* Theta;
} hfe_material;

#define HFE_PRECISION_FP64 0
#define HFE_PRECISION_MIXED 1
#define HFE_PRECOND_JACOBI 0
#define HFE_PRECOND_BLOCK3 1

/* Options (hfe_default_options fills the defaults). */
typedef struct {
  int precision;          /* HFE_PRECISION_FP64 or HFE_PRECISION_MIXED */
  double newton_rtol;     /* ||R_free|| <= newton_rtol * max(||R_free^0||, newton_atol);
                             default 1e-10 (FP64), 1e-7 (mixed) */
  double newton_atol;
  int newton_maxit;
  double newton_stag_tol; /* mixed only: stagnation accepted below this relative norm */
  double pcg_rtol;        /* ||r|| <= pcg_rtol * ||b||; default 1e-12 (FP64), 1e-6 (mixed); the
                             adjoint's reverse solves on the mixed path go to 0.3 pcg_rtol */
  int pcg_maxit;
  int pcg_check_every;    /* iterations per convergence read-back (one CUDA graph) */
  int precond;            /* HFE_PRECOND_JACOBI or HFE_PRECOND_BLOCK3 */
  int local_maxit;        /* bound of the local return-mapping Newton */
  double local_tol;       /* relative tolerance of the local yield residual */
  int ckpt_every;         /* adjoint: store the history every k steps, recompute between */
  int predictor;          /* initial guess of each (sub)step's Newton iteration:
                             2 (default) / 3: linear / quadratic extrapolation in the load
                             factor through the last 2 / 3 converged (sub)step solutions
                             (Sec. 2.2, automatic time stepping); linear while only two are
                             stored, and the tangent predictor while only the stored state is
                             known (after hfe_create, hfe_set_state, hfe_set_load,
                             hfe_set_material, hfe_set_barlat and at the start of
                             hfe_adjoint's forward pass);
                             1: the tangent predictor u = u_{n-1} + du_D + K^-1 (-(R + K du_D))
                             built on the converged start-of-step state, at every step;
                             0: u_{n-1} with the new Dirichlet values.
                             The Dirichlet values are those of the new load factor.  Modes 1-3
                             take the norm of the tangent predictor's right-hand side as the
                             Newton reference (2 and 3 form it without the solve); mode 0 the
                             residual at u_{n-1} with the new Dirichlet values */
  int ew_forcing;         /* 1: inexact Newton, the CG tolerance of each Newton solve follows the
                             Eisenstat-Walker forcing term (never below pcg_rtol) and a step is
                             accepted only after a correction solved to pcg_rtol; about 2x fewer
                             CG iterations on well-behaved runs, but loose solves can send the
                             iterates of ill-conditioned meshes astray.  0 (default): every
                             Newton solve to pcg_rtol */
  int pcg_persistent;     /* 1 (default): each CG solve is one cooperative kernel launch that runs
                             every iteration on the device (grid barriers, convergence tested each
                             iteration), its SpMV streaming FP32 K through shared memory by bulk
                             asynchronous copies in row chunks (FP64 K is loaded directly);
                             2: the same launch with K always loaded directly by the SpMV's lanes; 0: chunks of pcg_check_every iterations
                             as CUDA-graph launches with a host convergence check between chunks */
  int adaptive;           /* 1 (default): adaptive load stepping - a load step whose Newton
                             fails is rejected, the state restored, and retried with the
                             increment times cutback (substeps between the requested load
                             factors, which are hit exactly); 0: a failed step is an error */
  double cutback;         /* increment factor after a rejected step (default 0.5); the increment
                             grows by 1/cutback after two accepted substeps in a row */
  int max_cutbacks;       /* the increment is never cut below (requested interval) x
                             cutback^max_cutbacks (default 8: 1/256 of the interval) */
  int fbar;               /* 1: F-bar element (Sec. 2.2.4, Eq. Fbar): the constitutive model gets
                             Fbar = (Jbar/J)^(1/3) F, Jbar the element average of J; K is then
                             non-symmetric and every Krylov solve is BiCGSTAB (hfe_adjoint solves
                             with the transposed blocks).  0 (default): the standard element */
  int64_t barrier_spin_limit; /* polls (each >= 32 ns, backing off to 256 ns) after which a CTA
                             waiting at a grid barrier of a one-launch Krylov solve gives up; the
                             solve then returns HFE_EBARRIER.  Default 2^25 (seconds: a wait that
                             long means the CTAs are not all resident).  0 makes every wait give
                             up at its first poll (a way to exercise the failure path) */
  int64_t assembly_l2_bytes; /* launch order of the sweeps (set at hfe_create): the elements are
                             grouped into slabs by the K rows they write, each slab's rows holding
                             about this many bytes of K, and one launch runs one colour of one
                             slab; the colours of a slab then add into rows that are still in L2.
                             -1 (default): 3/4 of the device's L2; 0: one launch per colour over
                             the whole mesh.  Results differ from one setting to another by the
                             order of the additions only */
} hfe_options;

/* Statistics of the last hfe_forward / hfe_adjoint / hfe_gp_sweep call. */
typedef struct {
  int64_t newton_iters;   /* total over steps */
  int64_t pcg_iters;      /* total over solves */
  int64_t sweeps;         /* Gauss-point sweeps launched */
  int64_t plastic_gps;    /* plastic Gauss points in the last sweep */
  int64_t local_fail;     /* local return mappings that hit local_maxit (last sweep) */
  int32_t max_local_iters;/* largest local Newton iteration count (last sweep) */
  int32_t steps_done;     /* load steps completed */
  double last_residual;   /* ||R_free|| at the last Newton check */
  double sweep_ms;        /* device time in the sweep kernels */
  double solve_ms;        /* device time in the Krylov solves */
  double total_ms;        /* wall time of the call */
  int64_t bicgstab_solves;/* Newton corrections whose CG met negative curvature and that were
                             solved again by BiCGSTAB */
  int64_t substeps;       /* accepted load (sub)steps */
  int64_t cutbacks;       /* rejected attempts (adaptive stepping) */
  int64_t warm_steps;     /* requested load steps whose Newton iteration started from the
                             warm-start record (hfe_set_warm_start) */
  int64_t warm_retries;   /* of those, attempts that failed and were retried cold */
  int64_t refine_pcg_iters;  /* hfe_adjoint on a mixed handle: CG iterations of the FP64
                                refinement that ends each forward step (part of pcg_iters) */
  int64_t reverse_pcg_iters; /* hfe_adjoint: Krylov iterations of the reverse pass (part of
                                pcg_iters) */
} hfe_stats;

/* Sizes of the internal data (for tests and benchmarks). */
typedef struct {
  int64_t n_nodes, n_el, n_dof, n_gp, n_blocks, n_fixed;
  int32_t n_colors;
  int32_t precision;
  int64_t device_bytes;
  int64_t n_slabs;        /* slabs of the launch order (options.assembly_l2_bytes) */
  int64_t n_launches;     /* launches of one sweep: the non-empty (slab, colour) groups */
} hfe_info;

/* Fill *opt with defaults for the given precision. */
void hfe_default_options(hfe_options* opt, int precision);

/* Build the handle: copies the mesh, boundary data and material to the device, builds the
 * block-CSR pattern of K (3x3 blocks, one block per node pair sharing an element), the
 * element-to-block slot map, a conflict-free element colouring and the launch order of the
 * sweeps (options.assembly_l2_bytes); Sec. 2.2.5 describes the assembly this replaces.
 * stream: a cudaStream_t the library orders its work after and before (NULL = legacy
 * default stream).  Returns HFE_EINVAL for out-of-range node ids, HFE_EDETJ for an
 * element with det(dX/dxi) <= 0 at a Gauss point. */
hfe_status hfe_create(const hfe_mesh* mesh, const hfe_bc* bc, const hfe_material* mat,
                      const hfe_options* opt, void* stream, hfe_handle** out);
void hfe_destroy(hfe_handle* h);
const char* hfe_last_error(const hfe_handle* h);
hfe_status hfe_get_info(const hfe_handle* h, hfe_info* info);

/* Replace the material parameters (same hardening law and n_mat); used by inverse loops. */
hfe_status hfe_set_material(hfe_handle* h, const hfe_material* mat);

/* State: displacement u[n_dof] and history [7][n_gp] at t_n (host or device).  hist may be
 * NULL in set_state to mean zero history.  hfe_set_state resets the load factor of the
 * stored state to 0; a state taken at t_n > 0 (hfe_get_state after a forward run) is
 * continued correctly after hfe_set_load(h, t_n), since the next step's tangent predictor
 * linearises the Dirichlet increment from t_n.  hfe_get_load returns it. */
hfe_status hfe_set_state(hfe_handle* h, const double* u, const double* hist);
hfe_status hfe_get_state(hfe_handle* h, double* u, double* hist);
hfe_status hfe_set_load(hfe_handle* h, double t);
hfe_status hfe_get_load(const hfe_handle* h, double* t);

#define HFE_SWEEP_RESIDUAL 0   /* R and trial history only */
#define HFE_SWEEP_TANGENT 1    /* R, trial history and K (into the internal BSR values) */

/* One Gauss-point sweep at displacement u (host or device, [n_dof]) against the stored
 * history h_n (the per-Newton-iteration element pass, paper Sec. 2.2.5 "Parallel element-
 * wise residual and stiffness calculation"): R_out[n_dof] (host or device, may be NULL)
 * receives the internal force minus t*f_ext with t = load (Dirichlet rows included, no
 * elimination); rnorm_out (host or device, may be NULL) the FP64 norm of R over the free
 * dofs; hist_trial_out [7][n_gp] (host or device, may be NULL) the updated history; in
 * tangent mode K is assembled into the handle (read it with hfe_get_bsr).  With stats ==
 * NULL and device outputs the call does not synchronise (device status is checked by the
 * next call that passes stats). */
hfe_status hfe_gp_sweep(hfe_handle* h, const double* u, double load, int mode, double* R_out,
                        double* rnorm_out, double* hist_trial_out, hfe_stats* stats);

/* Export the block-CSR pattern (rowptr[n_nodes+1], cols[n_blocks]) and the values of the
 * last assembled K as float64 [n_blocks*9] (row-major 3x3 blocks); any pointer may be NULL;
 * host pointers. */
hfe_status hfe_get_bsr(hfe_handle* h, int64_t* rowptr, int32_t* cols, double* vals);

/* y = Kt x for the last assembled K with symmetric Dirichlet elimination (rows and columns
 * of fixed dofs zeroed, unit diagonal); x, y [n_dof] host or device, float64. */
hfe_status hfe_spmv(hfe_handle* h, const double* x, double* y);

/* Solve Kt x = b (Dirichlet components of b ignored, x_fixed = 0) with Jacobi or 3x3
 * block-Jacobi preconditioned CG; b, x [n_dof] host or device, float64. */
hfe_status hfe_solve(hfe_handle* h, const double* b, double* x, hfe_stats* stats);

/* Load-step loop with global Newton (Eq. Stiffness_mat) from the stored state.  t[n_steps]
 * load factors.  u_out [n_steps*n_dof] (all steps), sigma_out [n_gp*6] Cauchy stress
 * sigma = P F^T / J at the final step, hist_out [7][n_gp] at the final step; each host or
 * device or NULL.  On success the stored state is the final one. */
hfe_status hfe_forward(hfe_handle* h, int n_steps, const double* t, double* u_out,
                       double* sigma_out, double* hist_out, hfe_stats* stats);

/* Warm start of the load steps for repeated forward passes (Sec. 3.6: inside the inverse
 * loop the displacement of every step of the previous pass is the initial guess of the same
 * step of the next, enabled while every parameter moved by less than 10 %).  The library
 * records, on the device, the displacement each pass (hfe_forward, and the forward pass of
 * hfe_adjoint) converges to at each requested load factor t[n].  In HFE_WARM_USE a later
 * pass starts the Newton iteration of requested step n from record slot n when that slot was
 * recorded at the same load factor (|t_rec - t[n]| <= 1e-12 max(1, |t[n]|)), with the
 * Dirichlet values of t[n]; the step then spans the whole interval at once (an increment
 * reduced by cutbacks in an earlier interval is not carried into it), and no predictor solve
 * is made.  Its convergence reference is the cold step's (the predictor right-hand side norm,
 * or the residual at u_{n-1} with the new Dirichlet values when options.predictor = 0), so a
 * warm step meets the same tolerance as a cold one.  A warm attempt that fails is retried
 * cold over the same increment before any cutback (hfe_stats.warm_retries).
 *   mode: HFE_WARM_OFF (default): nothing recorded, every step cold, the record is freed;
 *         HFE_WARM_RECORD: record each pass, start cold;
 *         HFE_WARM_USE: record each pass and start from the record.
 * Memory: n_steps x n_dof doubles on the device, owned by the handle, grown to the longest
 * pass (older slots kept) and freed by HFE_WARM_OFF or hfe_destroy.  hfe_set_material,
 * hfe_set_state and hfe_set_barlat keep the record: deciding whether it is close enough to
 * the current parameters (the paper's 10 % rule) is the caller's.
 * Errors: HFE_EINVAL for a NULL handle or an unknown mode; HFE_ENOMEM if the record cannot
 * be allocated at the start of a pass (the pass then fails before its first step). */
#define HFE_WARM_OFF 0
#define HFE_WARM_RECORD 1
#define HFE_WARM_USE 2
hfe_status hfe_set_warm_start(hfe_handle* h, int mode);

/* Replaces the handle's options.barrier_spin_limit (>= 0) for the calls that follow, e.g. to
 * restore the default after a test of the failure path.  Errors: HFE_EINVAL for a NULL
 * handle or a negative limit. */
hfe_status hfe_set_barrier_spin_limit(hfe_handle* h, int64_t limit);

/* Misfit J = w sum_n ||u^n - u_target^n||^2 of a forward run from zero state over t, and its
 * gradient by the discrete adjoint (Eq. dR_u, Eq. main_grad) with the per-Gauss-point
 * implicit-function derivative of the return mapping (App. D).  u_target [n_steps*n_dof]
 * host or device; grad_out [n_mat*11] host or device (same layout as theta); J_out host.
 * The forward runs in the handle's precision; the adjoint in FP64 (on the mixed path each
 * step's state is first refined in FP64, and the reverse solves K^T lambda = rhs run FP32 CG
 * inside FP64 iterative refinement until the FP64 residual is 0.3 pcg_rtol ||rhs||). */
hfe_status hfe_adjoint(hfe_handle* h, int n_steps, const double* t, const double* u_target,
                       double w, double* J_out, double* grad_out, hfe_stats* stats);

/* ||r_free||_2 = sqrt(sum of r[d]^2 over the dofs with free_mask[d] != 0): the FP64 norm the
 * Newton iteration tests for convergence (the same quantity hfe_gp_sweep returns), here
 * without a handle and without allocating any device memory: its reduction scratch is a
 * static device array of the library (8,448 bytes per device, held until the process exits).
 * The paper has no counterpart.  It serves callers that cannot allocate: device memory held
 * by a caching allocator or exhausted, e.g. an error path that must still report the
 * residual, or a loop that has fixed its memory budget.
 *   r[n_dof] float64, free_mask[n_dof] uint8 (0 = Dirichlet dof), norm_out[1] float64: all
 *   device memory of the calling thread's current device, owned by the caller; n_dof = 0
 *   writes +0.0.  cuda_stream: the cudaStream_t the work is queued on (NULL = legacy
 *   default stream); the call does not synchronise, norm_out is valid once the stream has
 *   reached it.  The summation order is fixed, so the result is reproducible bit for bit.
 * Errors: HFE_EINVAL if n_dof < 0, n_dof > HFE_FREE_NORM_STATIC_MAX_DOF, a required pointer
 * is NULL or not on the current device (nothing is launched); HFE_ECUDA if a CUDA error was
 * already pending when the call began (it is left pending, nothing is launched), or if the
 * address look-up, the counter reset or the launch fails.
 * Rules: calls that overlap on one device (two host threads, or two streams with no
 * ordering between them) share the scratch and race — serialise them.  Every call looks up
 * the scratch's address in the current context (cudaGetSymbolAddress); the first call on a
 * device may load the module, so make it before any stream capture begins. */
#define HFE_FREE_NORM_STATIC_MAX_DOF 4194304
hfe_status hfe_free_norm_static(const double* r, const uint8_t* free_mask, int64_t n_dof, double* norm_out,
                                void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Barlat Yld2004-18p material points (no handle, no mesh)
 *
 * phi(T) = [1/4 sum_ij |s'_i - s''_j|^m]^(1/m) with s'_i, s''_j the eigenvalues of
 * s' = C' : P : T_l and s'' = C'' : P : T_l, P the deviatoric projector, T_l = Theta^T T Theta
 * the stress in the material frame (Eq. Phi_barlat, App. A.2).  C' and C'' are the 6x6
 * matrices of App. A.2 on the components (11, 22, 33, 12, 23, 13): off-diagonal normal
 * entries -c12, -c13, -c21, -c23, -c31, -c32 and the shear diagonal c44, c55, c66 acting on
 * the 12, 23, 13 components.  Associative flow N = dphi/dT with W = 1 (alpha-rate =
 * gamma-rate), yield function f = phi(T) - sigma_y(alpha) (Eq. ep_evol, Eq. alpha_update,
 * Eq. yield_final), isotropic log-space elasticity E, nu (Eq. T).
 *
 *   c1[9], c2[9]: (c12, c13, c21, c23, c31, c32, c44, c55, c66) of C' and C'';
 *   m: the exponent, an even integer 2 <= m <= HFE_BARLAT_MAX_M;
 *   hardening, h[3]: HFE_HARDENING_SWIFT (K, eps0, n) or HFE_HARDENING_VOCE (sigma0, Q, b);
 *     perfect plasticity is Voce with Q = 0;
 *   Theta[9]: row-major 3x3 whose columns are the material axes (orthonormal to 1e-10;
 *     the identity for material axes = global axes);
 *   orthotropic, d[9]: 0 = isotropic elasticity from E, nu; 1 = the orthotropic E of nine
 *     stiffness coefficients in the material frame (Eq. T): d = (E1111, E2222, E3333, E1122,
 *     E1133, E2233, E1212, E2323, E1313) with the minor and major symmetries, rotated by
 *     Theta (E_g,ijkl = Theta_ia Theta_jb Theta_kc Theta_ld E_l,abcd); E and nu are then
 *     unused by the return map but must still be valid.  d1, d2, d3, d7, d8, d9 > 0.
 * Voce hardening for this model is Eq. Hard as printed: sigma_y = sigma0 + sqrt(2/3) Q
 * (1 - exp(-b alpha)) (the Hill-48 handle path places sqrt(2/3) in f instead). */
#define HFE_BARLAT_MAX_M 32
typedef struct {
  double c1[9];
  double c2[9];
  int m;
  double E, nu;
  int hardening;
  double h[3];
  double Theta[9];
  int orthotropic;
  double d[9];
} hfe_barlat_material;

/* Local closest-point projection controls (App. B, App. C): at most kmax Newton iterations,
 * line_search = 1 for App. B's line search (0 = standard Newton), at most jmax + 1 merit
 * evaluations after the full step, Goldstein constant beta, safeguard eta, and convergence
 * when sqrt(|G_T / s|^2 + G_alpha^2 + (G_f / s)^2) <= tol with s = max(sigma_y(alpha_n),
 * |T_tr|).  precision HFE_PRECISION_FP64: every iteration in double;
 * HFE_PRECISION_MIXED: the same iteration in float down to a scaled residual of 1e-5 (at
 * most kmax iterations), then at most 6 double Newton iterations to tol (the FP32 phase
 * hitting kmax reports HFE_CPP_MAXIT), the elastic test in float outside |f_tr| <= 1e-5 s and
 * in double inside.  Defaults (hfe_default_cpp_options): kmax 40, line_search 1, jmax 10,
 * beta 1e-4, eta 0.1, tol 1e-13, precision HFE_PRECISION_FP64. */
typedef struct {
  int kmax;
  int line_search;
  int jmax;
  double beta, eta, tol;
  int precision;
} hfe_cpp_options;
void hfe_default_cpp_options(hfe_cpp_options* opt);

/* phi_out[i] = phi(T[i]) and, if N_out is not NULL, N_out[i*6 .. i*6+5] = dphi/dT as tensor
 * components (dphi = N : dT), for n stresses T[n*6] (components as above).  All arrays are
 * device memory of the current device owned by the caller; queued on cuda_stream (NULL =
 * legacy default stream), no synchronisation.  A pure pressure gives phi = 0 up to the
 * rounding of the deviatoric projection; T = 0 gives phi = 0 and N = 0; a non-finite stress
 * gives NaN.  Errors: HFE_EINVAL for an invalid material (odd or out-of-range m,
 * E <= 0, nu outside (-1, 0.5), unknown hardening, non-finite values, Theta not orthonormal),
 * n < 0, NULL or non-device pointers (nothing is launched); HFE_ECUDA if the launch fails. */
hfe_status hfe_barlat_phi(const hfe_barlat_material* mat, const double* T, int64_t n, double* phi_out,
                          double* N_out, void* cuda_stream);

/* Per-point outcome of hfe_barlat_return_map. */
#define HFE_CPP_CONVERGED 0   /* plastic, the residual test passed */
#define HFE_CPP_ELASTIC 1     /* f_tr = phi(T_tr) - sigma_y(alpha_n) <= 0: T = T_tr */
#define HFE_CPP_MAXIT 2       /* kmax Newton iterations without convergence: the last iterate */
#define HFE_CPP_SINGULAR 3    /* the Newton matrix was singular: the last iterate */
#define HFE_CPP_NONFINITE 4   /* a non-finite input or residual (or phi = 0 inside the iteration) */

/* Elastic predictor / plastic corrector for n material points driven by trial stresses
 * (App. C): for each i, from T_trial[i*6..] and alpha_n[i], the elastic test and, if
 * plastic, Newton on G(y) = 0, y = [T, alpha, dgamma] (Eq. local_cpp) from
 * y0 = [T_trial, alpha_n, 0], with the App. B line search when opt->line_search.
 * Outputs: T_out[n*6], alpha_out[n], dgamma_out[n], iters_out[n] (Newton iterations taken),
 * status_out[n] (HFE_CPP_*), and, if tangent_out is not NULL, tangent_out[n*36] =
 * dT/dT_trial row-major per point ([a*6 + c] = dT_a / dT_trial_c, a shear component moving
 * both symmetric entries) by implicit differentiation of the converged local system (App. D);
 * the identity for elastic points.  opt NULL = the defaults.  Every array is device memory of
 * the current device, owned by the caller; queued on cuda_stream (NULL = legacy default
 * stream), no synchronisation, no allocation.  One thread per point.
 * Errors: as hfe_barlat_phi, plus HFE_EINVAL for options out of range (kmax outside
 * [0, 100000], jmax outside [0, 1000], beta outside (0, 0.5), eta outside (0, 1), tol <= 0,
 * unknown precision).
 * Per-point failures are reported in status_out, not as an error. */
hfe_status hfe_barlat_return_map(const hfe_barlat_material* mat, const hfe_cpp_options* opt, const double* T_trial,
                                 const double* alpha_n, int64_t n, double* T_out, double* alpha_out,
                                 double* dgamma_out, int32_t* iters_out, int8_t* status_out, double* tangent_out,
                                 void* cuda_stream);

/* Give a handle the Barlat Yld2004-18p material (uniform, standard element) in place of
 * its Hill-48 parameters: every later sweep, solve and forward step updates the Gauss points
 * with App. C's stress update of this model from the total log strain (elastic test, the
 * projection with opt's controls in FP64, recovery eps_p,n+1 = eps_p,n + dgamma N,
 * T = E : (eps - eps_p,n+1)) and assembles with its tangent dT/deps = (dT/dT_tr) E, the
 * geometric pre- and post-processor and the element being those of the Hill-48 path.  The
 * history layout is unchanged (eps_p tensor components, alpha).  opt NULL = the defaults
 * (kmax 40); opt->precision selects the projection's arithmetic (FP64, or the FP32 iteration
 * with the FP64 finish to the same tolerance); the element path keeps the handle's precision
 * (FP64, or the mixed path's FP32 kinematics, post-processor and assembly).  mat NULL
 * returns the handle to Hill-48.  A local
 * projection that stops at kmax counts in stats.local_fail and the call returns
 * HFE_ELOCAL like the Hill-48 path.  hfe_adjoint returns HFE_EINVAL while the model is set.
 * Errors: HFE_EINVAL for per-element Hill parameters, the F-bar element, or invalid
 * material / options; HFE_ENOMEM if the exchange buffers (64 doubles and
 * 6 bytes per Gauss point) cannot be allocated. */
hfe_status hfe_set_barlat(hfe_handle* h, const hfe_barlat_material* mat, const hfe_cpp_options* opt);

#ifdef __cplusplus
}
#endif
#endif /* HFE_H */
