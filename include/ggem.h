/*
 * ggem.h -- C ABI of libggem, a GB300 (sm_103a) implementation of the GGEM
 * evaluation of Stokes flow driven by point forces in a planar slit, and of
 * the boundary-integral operators and Fredholm solve built on it.
 *
 * Paper: Kumar & Graham, "Accelerated boundary integral method for multiphase
 * flow in non-periodic geometries", arXiv 1109.6587.
 *
 * Geometry: walls at y = y0 and y = y0 + W (no slip), periodic in x (period
 * Lx) and z (period Lz); grid of Nx x Nz equispaced Fourier nodes times Ny
 * Gauss-Lobatto Chebyshev nodes y_j = y0 + W/2 (1 + cos(pi j/(Ny-1))).
 *
 * Conventions for every entry point:
 *  - Arrays of doubles; vectors are stored point-major, [n][3] (x, y, z).
 *    Stresses are [n][6] in the order xx, xy, xz, yy, yz, zz.
 *  - Array arguments may be device pointers (cudaMalloc, torch CUDA tensors)
 *    or host pointers (pageable or pinned); the library detects which.  Host
 *    inputs are copied to plan-owned device buffers and host outputs are
 *    copied back before the call returns.  With device pointers the call is
 *    asynchronous on the plan's stream.
 *  - The caller owns every input and output array; the plan owns all
 *    workspaces.  No entry point below allocates device memory except
 *    ggem_plan, ggem_mesh_set (which sizes its mesh tables once),
 *    ggem_set_offgrid (the oversampled grid) and the first bie_solve on a
 *    plan (Krylov workspace; FP64 twin of a mixed plan).
 *  - Every entry point returns a ggem_status; no C++ exception crosses the
 *    ABI.  On error ggem_last_error(plan) gives a message.
 */
#ifndef GGEM_H
#define GGEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GGEM_OK = 0,
    GGEM_ERR_INVALID_ARG = 1,   /* bad size, pointer, or geometry parameter   */
    GGEM_ERR_CAPACITY = 2,      /* more points/triangles than the plan holds  */
    GGEM_ERR_CUDA = 3,          /* a CUDA runtime call failed                 */
    GGEM_ERR_NUMERICAL = 4,     /* NaN/Inf detected                            */
    GGEM_ERR_NOT_CONVERGED = 5, /* iterative solve hit its iteration limit     */
    GGEM_OK_BREAKDOWN = 6       /* GMRES happy breakdown: exact solution found */
} ggem_status;

enum { GGEM_FP64 = 0, GGEM_MIXED = 1, GGEM_FP64_EMULATED = 2 };  /* ggem_params.precision */
enum { GGEM_NODAL = 0, GGEM_ELEMENT = 1 };       /* ggem_params.quadrature */

typedef struct ggem_plan ggem_plan_t;

/*
 * Parameters of a plan (Sec. 3.2 and Sec. 5 of the paper).
 *   alpha        splitting parameter of Eq. (rho_l_g); 0 selects
 *                1/(2 max(Lx/Nx, W/(Ny-1), Lz/Nz)), i.e. alpha*dy_m <= 0.5.
 *   rcut_factor  r_cut = rcut_factor/alpha; 0 selects 4 (Sec. 3.2.1).
 *   precision    GGEM_FP64: every step in FP64.  GGEM_MIXED: local sum,
 *                spreading, FFT, Chebyshev transforms and interpolation in
 *                FP32; per-mode tau solves in FP64.  GGEM_FP64_EMULATED: as
 *                GGEM_FP64, except that the element-rule local sum runs in
 *                double-float arithmetic (pairs of floats, ~48-bit
 *                significand; GB300's FP32 rate is 64x its FP64 rate), at FP64
 *                parity; the FP64 twin of a mixed plan uses it.
 *   quadrature   GGEM_ELEMENT: local part by the 4x4 Gauss product rule per
 *                triangle with the polar rule on triangles touching the
 *                target (Sec. 3.4.1, 3.5.2).  GGEM_NODAL: nodal point forces
 *                A_b q_b with the self pair left out.
 *   max_points   capacity for nodes / point sources / targets.
 *   max_tris     capacity for triangles (element quadrature).
 * Requirements: Nx, Nz powers of two in [16, 1024]; 9 <= Ny <= 257;
 * alpha*Lx > 2*rcut_factor and alpha*Lz > 2*rcut_factor (Sec. 3.2.2: r_cut
 * below half the period); W > 0; mu > 0.
 */
typedef struct {
    double Lx, Lz, W, y0;
    int Nx, Ny, Nz;
    double alpha;
    double rcut_factor;
    double mu;
    int precision;
    int quadrature;
    int max_points;
    int max_tris;
} ggem_params;

/* Create a plan on a CUDA stream (cudaStream_t passed as void*; NULL = the
 * legacy default stream).  Builds the grid, the Chebyshev and FFT tables and,
 * for every Fourier mode, the homogeneous Kleiser-Schumann solutions and the
 * inverse 2x2 influence matrix (App. C: "solved just once ... and stored").
 * Allocates all workspaces.  *out receives the plan, or NULL on error. */
ggem_status ggem_plan(const ggem_params *params, void *stream, ggem_plan_t **out);

/* Free a plan and all its device memory.  NULL is accepted. */
ggem_status ggem_plan_destroy(ggem_plan_t *plan);

/* Message describing the last error on this plan (static text for NULL). */
const char *ggem_last_error(const ggem_plan_t *plan);

/* Effective alpha and r_cut of the plan (host values). */
ggem_status ggem_plan_info(const ggem_plan_t *plan, double *alpha, double *rcut);

enum { GGEM_OFFGRID_LAGRANGE = 0, GGEM_OFFGRID_SPECTRAL = 1 };   /* ggem_set_offgrid */

/*
 * How the global solution is evaluated at points off the grid (every entry
 * point that returns velocities, stresses or layer values at nodes or
 * targets).
 *   GGEM_OFFGRID_LAGRANGE (the default): 5-point Lagrange interpolation in
 *     each direction, error ~ h^5 (Sec. 3.2.2).
 *   GGEM_OFFGRID_SPECTRAL: the Fourier (x, z) x Chebyshev (y) expansion of the
 *     global solution itself, evaluated to a tolerance rather than
 *     interpolated, so that the error off the mesh decays as fast as on it
 *     (the non-uniform FFT route that Sec. 3.2.3 points to): Greengard &
 *     Lee's type-2 non-uniform FFT with a Gaussian window in x, z and
 *     theta = arccos of the normalised y (where the Chebyshev series is a
 *     cosine series) -- modes deconvolved by the window, transformed onto a
 *     grid oversampled 2x in each direction, and the window gathered over
 *     2 half_width points per direction at each target.  half_width: 0
 *     selects 12 for FP64-accurate plans (window error ~1e-13) and 6 for
 *     GGEM_MIXED (~2e-7); otherwise 2..16.  Cost per target (2 half_width)^3
 *     per output component, against 125 for Lagrange.
 * Allocates the oversampled grid ((2Ny - 1) x 9 x 2Nz x 2Nx values of the
 * plan's precision, plus (2Ny - 1) x 9 x Nz x Nx) on the first switch to
 * GGEM_OFFGRID_SPECTRAL; a mixed plan's FP64 twin follows the setting (with
 * its own default width).
 * Returns GGEM_ERR_INVALID_ARG for an unknown mode or width.
 */
ggem_status ggem_set_offgrid(ggem_plan_t *plan, int mode, int half_width);

/*
 * Set the surface mesh (Sec. 3.3): n_nodes nodes x [n][3] and n_tris
 * outward-oriented triangles tri [m][3] (node indices).  Each particle's
 * nodes must be unwrapped (one periodic image per triangle).  Computes
 * element areas A_k, nodal areas A_b = sum A_k / 3, area-averaged unit node
 * normals (Sec. 3.4.2, 3.5.2), the cell list of the nodes and, for element
 * quadrature, the quadrature points.  Every node must satisfy
 * y0 < y < y0 + W.  n_tris may be 0 for GGEM_NODAL.
 */
ggem_status ggem_mesh_set(ggem_plan_t *plan, int n_nodes, const double *x,
                          int n_tris, const int *tri);

/* Nodal areas A_b [n] and unit normals [n][3] of the current mesh (either
 * pointer may be NULL). */
ggem_status ggem_mesh_geometry(ggem_plan_t *plan, double *area, double *normal);

/*
 * Velocity and stress at n_tgt targets due to n_src point forces g [n][3] at
 * x_src (Sec. 3.2, Eqs. (u_g), (tot_l_g)):
 *   u_i(x)      = 1/(8 pi mu) sum_nu G_ij(x, x_nu) g_nu_j
 *   sigma_ik(x) = 1/(8 pi)    sum_nu T_ijk(x, x_nu) g_nu_j
 * with G, T the slit Green's function and its stress.  tgt_is_src != 0 means
 * the targets are the sources themselves (x_tgt ignored, n_tgt = n_src): the
 * self pair is left out of the local sum and the free-space global self
 * velocity (4 alpha/sqrt(pi)) g/(8 pi mu) is removed, so u is the regular
 * part of the slit solution at each source.  u [n_tgt][3] and sigma
 * [n_tgt][6] may each be NULL.  Sources and targets must lie strictly
 * inside the slit.
 */
ggem_status ggem_point_forces(ggem_plan_t *plan, int n_src, const double *x_src,
                              const double *g, int n_tgt, const double *x_tgt,
                              int tgt_is_src, double *u, double *sigma);

/*
 * Local part alone, Eq. (u_loc) of Sec. 3.2.1: the free-space response to the
 * local densities rho_l of the point forces, truncated at r_cut,
 *   u^l_i(x)      = 1/(8 pi mu) sum_{0 < |x - x_nu*| < r_cut} G^l_ij g_nu_j
 *   sigma^l_ik(x) = 1/(8 pi)    sum_{0 < |x - x_nu*| < r_cut} T^l_ijk g_nu_j
 * (x_nu* the minimum image in x and z).  Same arguments and layouts as
 * ggem_point_forces; no global part and no self term.
 */
ggem_status ggem_local_sum(ggem_plan_t *plan, int n_src, const double *x_src,
                           const double *g, int n_tgt, const double *x_tgt,
                           int tgt_is_src, double *u, double *sigma);

/*
 * Single-layer integral at the mesh nodes (Sec. 3.4, Eq. (sl_t)):
 *   w_j(z) = int_S q_i(x) G_ji(z, x) dS(x),   q, w: [n_nodes][3].
 * Local part by the plan's quadrature, global part from the trapezoidal
 * nodal strengths A_b q_b spread with rho_g (Eq. (rhog_sum)) and evaluated at
 * the nodes by the plan's off-grid mode (ggem_set_offgrid).
 */
ggem_status ggem_single_layer(ggem_plan_t *plan, const double *q, double *w);

/*
 * Double-layer integral at the mesh nodes (Sec. 3.5, Eq. (wdbl)):
 *   v_j(z) = n_k(z) int_S q_i(x) T_jik(z, x) dS(x),   q, v: [n_nodes][3].
 * Element quadrature uses the n-tilde form of Eqs. (dbl_l1), (ntilde) on
 * triangles that have z as a vertex.
 */
ggem_status ggem_double_layer(ggem_plan_t *plan, const double *q, double *v);

/*
 * Fredholm solve of Sec. 5 (the linear system below Eq. (qa)):
 *     (I + kappa/(4 pi) D) q = b   at the mesh nodes,
 * D the double layer of ggem_double_layer, kappa the diagonal of per-node
 * kappa_m = (lambda_m - 1)/(lambda_m + 1), Eq. (qa).
 *   kappa   [n_nodes]
 *   b       [n_nodes][3]
 *   q       [n_nodes][3]; in: initial guess (e.g. the previous time step's
 *           density, or b), out: the solution
 *   tol     stop when the TRUE relative residual ||b - A q|| / ||b|| <= tol,
 *           A applied in FP64 (the paper stops at 1e-4 on the residual)
 *   restart GMRES cycle length m, 1..64
 *   maxit   limit on Arnoldi steps (operator applications inside cycles)
 *   use_mlp 0: start from q.  1: also form the learned guess q + delta,
 *           delta the network's estimate of A^-1 r0 for r0 = b - A q, and
 *           start from whichever of q and q + delta has the lower relative
 *           residual under the plan's operator (needs ggem_mesh_particles and
 *           a model from ggem_mlp_load or ggem_mlp_train).
 *   iters, true_relres  (out, may be NULL) Arnoldi steps taken and the final
 *           true relative residual
 * Method: restarted GMRES with FP64 Arnoldi vectors (classical Gram-Schmidt
 * applied twice); every cycle starts from the true residual.  An FP64 plan
 * uses its own operator throughout.  A mixed plan refines: true residuals
 * come from an FP64 twin plan on the same mesh (built by the first solve and
 * kept in step with later ggem_mesh_set calls; it doubles the plan's device
 * memory), and each correction is one GMRES cycle with the mixed operator,
 * solved to max(tol ||b|| / (2 ||r||), 1e-5) relative to its residual r.  The
 * residual of the initial guess is formed with the mixed operator (the first
 * correction needs only ~1e-4) unless it is within 10 tol, when FP64 decides.
 * Arrays may be device or host memory.  The first solve allocates the
 * Krylov workspace ((restart + 1) x 3 max_points doubles); later solves with
 * the same or a shorter restart allocate nothing.  Returns GGEM_OK,
 * GGEM_OK_BREAKDOWN (converged after a cycle whose Krylov space became
 * invariant), GGEM_ERR_NOT_CONVERGED (q holds the last iterate, iters and
 * true_relres are filled), GGEM_ERR_NUMERICAL (non-finite residual) or an
 * argument error.  ||b|| = 0 returns q = 0 with no iteration.
 */
ggem_status bie_solve(ggem_plan_t *plan, const double *kappa, const double *b, double *q,
                      double tol, int restart, int maxit, int use_mlp, int *iters,
                      double *true_relres);

/*
 * Per-particle block preconditioner of the Fredholm solve (the paper solves
 * Sec. 5's system by GMRES without one).  ggem_precond_set builds
 *     B = (I + kappa/(4 pi) D_ref)^-1,
 * D_ref the discrete double layer (this plan's precision, quadrature and
 * off-grid evaluation) of one reference capsule alone -- nodes x_ref
 * [n_ref][3] (any origin: they are centred on their centroid), triangles
 * tri_ref [n_tri_ref][3] -- placed at the centre of a periodic cell of
 * ref_nx x ref_nz grid intervals of this plan's x-z spacing, with this
 * plan's wall gap, Chebyshev grid, alpha and r_cut (ref_nx, ref_nz powers
 * of two >= 4; the cell must satisfy alpha L > 8).  It costs 3 n_ref
 * double-layer evaluations on that cell and an FP64 Gauss-Jordan inversion
 * (partial pivoting) on the device, and enables the preconditioner.
 *
 * bie_solve (and the capsule steps, which call it) then runs GMRES on
 * A M y = r, x += M y (flexible form: the products M V_j are kept), with
 *     M = blockdiag over particles of (I x R_p) B (I x R_p^T),
 * R_p the rotation carrying the reference nodes onto particle p's (the
 * polar factor of their cross-covariance, each particle unwrapped about its
 * first node in x, z): every particle (ggem_mesh_particles) must have n_ref
 * nodes, its l-th node (increasing index) matching reference node l.  The
 * block is best for particles with this kappa and valid for any.  M is
 * applied as one GEMM over all particles, FP32 in GGEM_MIXED plans, FP64
 * otherwise.  The solution and its stopping test (the true residual) do not
 * depend on M; the iteration count does.
 *
 * Errors: GGEM_ERR_INVALID_ARG for bad sizes or pointers (host or device),
 * GGEM_ERR_NUMERICAL for a singular block, a reference-cell plan's error
 * otherwise; a failed set leaves no preconditioner.  x_ref and tri_ref may be
 * host or device arrays; the plan keeps B (FP64 and FP32 copies).
 */
ggem_status ggem_precond_set(ggem_plan_t *plan, int n_ref, const double *x_ref, int n_tri_ref,
                             const int *tri_ref, double kappa, int ref_nx, int ref_nz);
/* Use (on = 1) or stop using (0) the block preconditioner that was set. */
ggem_status ggem_precond_enable(ggem_plan_t *plan, int on);
/* The block B [3 n_ref][3 n_ref] (row-major, FP64) into out (host or device). */
ggem_status ggem_precond_block(ggem_plan_t *plan, double *out);

/* The last bie_solve's initial guess: used_mlp = 1 when it started from the
 * learned guess, and the relative residuals of the caller's and the learned
 * guess (0 when use_mlp was 0). */
ggem_status ggem_solve_guess(const ggem_plan_t *plan, int *used_mlp, double *relres_plain,
                             double *relres_mlp);

/* Work counts of the last bie_solve or ggem_rigid_solve on this plan: GMRES
 * cycles, operator applications in FP64 and with the mixed operator. */
ggem_status ggem_solve_stats(const ggem_plan_t *plan, int *cycles, int *matvec_fp64,
                             int *matvec_mixed);

/*
 * Rigid particles in the slit (Sec. 6.1, Eq. (sl_r)): the surface tractions f
 * and the translational and angular velocities U_p, Omega_p of rigid
 * particles that move freely in an undisturbed flow u_inf, or under an
 * external force and torque.  At every node b of particle p
 *   U_p + Omega_p x (x_b - c_p) + 1/(8 pi mu) int_S f_i G_ji(x_b, x) dS = u_inf(x_b),
 * the integral being ggem_single_layer of f, and for every particle
 *   sum_{b in p} A_b f_b = -F_p,   sum_{b in p} A_b (x_b - c_p) x f_b = -T_p,
 * A_b the nodal areas (f is the traction the fluid exerts on the particle).
 * The balance rows enter the system scaled by 1/(6 pi mu R_p) and
 * 1/(8 pi mu R_p^2), R_p = sqrt(S_p / (4 pi)), S_p = sum A_b over the particle,
 * so that every residual entry is a velocity.
 *   n_particles  must equal the count given to ggem_mesh_particles, whose ids
 *                (set for the current mesh) assign the nodes to particles
 *   centres      [n_particles][3] reference points c_p (e.g. the centres)
 *   u_inf        [n_nodes][3] undisturbed velocity at the nodes, or NULL (0)
 *   ext          [n_particles][6] external force F_p and torque T_p about c_p,
 *                or NULL (force- and torque-free)
 *   f            [n_nodes][3]; in: initial guess (zeros if unknown), out: f
 *   uo           [n_particles][6]; in: guess, out: U_p (3), Omega_p (3)
 *   tol, restart, maxit, iters, true_relres  as for bie_solve; the residual
 *                is that of the whole system [rows | balance rows]
 * The tractions of a closed surface are fixed only up to a multiple of the
 * normal (a uniform pressure exerts no force and moves no fluid), so the
 * velocities are the well-determined output.  Method, precision handling
 * and workspace as for bie_solve (the first call also builds the node lists
 * of the particles, once per ggem_mesh_particles).  Arrays may be device or
 * host memory.  Returns GGEM_OK, GGEM_OK_BREAKDOWN, GGEM_ERR_NOT_CONVERGED
 * (f and uo hold the last iterate), GGEM_ERR_NUMERICAL or an argument error.
 */
ggem_status ggem_rigid_solve(ggem_plan_t *plan, int n_particles, const double *centres,
                             const double *u_inf, const double *ext, double *f, double *uo,
                             double tol, int restart, int maxit, int *iters,
                             double *true_relres);

/* ------------------------------------------------------------------------
 * Capsule dynamics (Sec. 4, 5, App. B): elastic capsules (neo-Hookean
 * membranes around a fluid of viscosity lambda mu) carried by an undisturbed
 * flow.  Node velocities come from Eqs. (bi_ua) and (qa); positions advance by
 * the midpoint rule.  All of it runs on the plan's mesh, which a step moves.
 * ------------------------------------------------------------------------ */
enum { GGEM_FLOW_NONE = 0, GGEM_FLOW_SHEAR = 1, GGEM_FLOW_POISEUILLE = 2 };

/* Reference (stress-free) shape of the membranes: x_ref [n_nodes][3] with the
 * current mesh's triangles (e.g. the initial mesh).  Stores each triangle's
 * reference metric; required by the traction and the step, kept until a
 * ggem_mesh_set brings new triangles. */
ggem_status ggem_membrane_reference(ggem_plan_t *plan, const double *x_ref);

/* Traction jump at the nodes (Sec. 4, Eqs. (cntr2), (eq_WNH)): every flat
 * triangle stores A0 W, W = (G/2)(lambda_1^2 + lambda_2^2 + 1/(lambda_1
 * lambda_2)^2 - 3) of its uniform deformation from the reference; the force
 * on a node is the gradient of the stored energy (principle of virtual work)
 * and df_b = grad_b E / A_b, A_b the node's area (a third of its triangles'
 * current areas).  df [n_nodes][3]; G = shear_modulus. */
ggem_status ggem_membrane_traction(ggem_plan_t *plan, double shear_modulus, double *df);

/* Undisturbed flow at the nodes (App. B): flow GGEM_FLOW_SHEAR, u = s (y -
 * y_mid) e_x with y_mid the slit's mid-plane and s the shear rate;
 * GGEM_FLOW_POISEUILLE, u = 4 s eta (1 - eta) e_x, eta = (y - y0)/W, s the
 * centre-line velocity, pressure -8 mu s x / W^2; GGEM_FLOW_NONE, u = 0.
 * u_inf [n_nodes][3] and f_inf = sigma_inf . n [n_nodes][3] (either may be
 * NULL; f_inf needs triangles for the normals). */
ggem_status ggem_undisturbed(ggem_plan_t *plan, int flow, double strength, double *u_inf,
                             double *f_inf);

typedef struct {
    int flow;              /* GGEM_FLOW_* */
    double strength;       /* shear rate or centre-line velocity */
    double shear_modulus;  /* G of the membranes */
    double dt;             /* time step (ggem_capsule_step) */
    double tol;            /* Fredholm solve of each stage: as bie_solve */
    int restart;
    int maxit;
    int use_mlp;
} ggem_step_params;

/* Node velocities of the capsules at the current mesh: b = -(df/(lambda + 1)
 * + kappa f_inf)/(4 pi mu), kappa = (lambda - 1)/(lambda + 1) (Eq. (qa)),
 * (I + kappa/(4 pi) D) q = b by bie_solve, u = u_inf + int q G dS
 * (Eq. (bi_ua)).  lambda [n_nodes] viscosity ratio of each node's capsule;
 * q [n_nodes][3] in: initial guess, out: the density; u [n_nodes][3].
 * iters, true_relres as for bie_solve.  Needs ggem_membrane_reference. */
ggem_status ggem_capsule_velocity(ggem_plan_t *plan, const ggem_step_params *sp,
                                  const double *lambda, double *q, double *u, int *iters,
                                  double *true_relres);

/* One midpoint step of dx/dt = u (Sec. 5): x_half = x + dt/2 u(x), x_new =
 * x + dt u(x_half), u as ggem_capsule_velocity; the second stage's solve
 * starts from the first stage's density.  Moves the plan's mesh to x_new
 * (cell lists, geometry, quadrature points rebuilt as by ggem_mesh_set; a
 * node leaving the slit is an error).  q [n_nodes][3] in: guess, out: the
 * second stage's density (the next step's guess); x_out [n_nodes][3] or NULL;
 * iters: GMRES steps of both stages; true_relres: the larger of the two. */
ggem_status ggem_capsule_step(ggem_plan_t *plan, const ggem_step_params *sp,
                              const double *lambda, double *q, double *x_out, int *iters,
                              double *true_relres);

/* The plan's current node positions [n_nodes][3]. */
ggem_status ggem_mesh_positions(const ggem_plan_t *plan, double *x);

/* Smallest distance between two nodes (any particles; minimum image in x,
 * z), the h_min of the time step rule gamma_dot dt = 0.5 Ca h_min / a
 * (Sec. 5).  Pairs are searched in neighbouring cells of the plan's cell
 * grid; with none there the result is the smallest cell width. */
ggem_status ggem_min_separation(ggem_plan_t *plan, double *h_min);

/* Enclosed volume of every particle of ggem_mesh_particles (divergence
 * theorem over its outward-oriented triangles), volumes [n_particles]. */
ggem_status ggem_particle_volumes(ggem_plan_t *plan, double *volumes);

/* Volume correction (Sec. 5): every particle whose volume differs from v0
 * [n_particles] by more than threshold * |v0| moves its nodes along their
 * normals by (v0 - V)/S, S its area; repeated at most max_passes times until
 * all are within the threshold (one pass leaves a second-order residual).
 * Moves the plan's mesh; passes (out, may be NULL): passes made. */
ggem_status ggem_volume_correct(ggem_plan_t *plan, const double *v0, double threshold,
                                int max_passes, int *passes);

/* Minimum-gap (overlap) correction (Sec. 7.1): every pair of particles whose
 * closest nodes (minimum image in x, z) are nearer than h_min moves apart
 * rigidly along its line of centres (node centroids, minimum image) by half
 * the deficit each; all pairs of a sweep move at once from the positions at
 * its start (a particle in several pairs moves by the sum), and sweeps repeat
 * (at most max_sweeps) until no pair is nearer than h_min (1 - 1e-9).  Gaps
 * are node to node: they see near contacts, not deep overlaps.  h_min must be
 * at most a cell width of the plan (pairs are searched in neighbouring
 * cells).  Moves the plan's mesh; moves (out, may be NULL): pair moves made.
 * GGEM_ERR_CAPACITY when a node lies within h_min of more than 4 other
 * particles (their pairs could not all be recorded). */
ggem_status ggem_overlap_correct(ggem_plan_t *plan, double h_min, int max_sweeps, int *moves);

/*
 * Allocation-free local velocity sum (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc -- code recording a CUDA graph
 * under stream capture, where allocation calls are not allowed; applications
 * whose device memory belongs to another allocator or a fixed budget; loops
 * that must avoid the device-wide synchronisation of cudaFree -- and that
 * therefore cannot create a plan either.  Computes the same local velocity
 * as ggem_local_sum (velocity only, FP64) from the geometry and alpha /
 * r_cut rules of *params (its precision, quadrature and capacity fields are
 * ignored), on `stream`.
 *
 * It allocates nothing: its cell list lives in one file-scope device array
 * of the library, sized for at most GGEM_NOALLOC_MAX_POINTS sources and
 * GGEM_NOALLOC_MAX_CELLS cells (about 7.8 MB, held on every GPU that loads
 * the library until the process exits); targets are taken in chunks of
 * GGEM_NOALLOC_MAX_POINTS, so their number is not limited.  The first call on each device
 * (and the first after that device's context was reset) looks up that array's device
 * address, so make it before any stream capture.
 * Every call reuses the same array: calls that overlap on the GPU (different
 * streams or threads) race and must be serialised by the caller.  The array
 * keeps the last call's contents; each call clears the counters it needs.
 *
 * Arrays must be device pointers.  Returns GGEM_ERR_CAPACITY when n_src or
 * the cell count exceeds the limits, GGEM_ERR_INVALID_ARG for bad sizes,
 * geometry or host pointers (no message is recorded: there is no plan).
 */
#define GGEM_NOALLOC_MAX_POINTS 65536
#define GGEM_NOALLOC_MAX_CELLS 32768
ggem_status ggem_local_velocity_noalloc(const ggem_params *params, void *stream, int n_src,
                                        const double *x_src, const double *g, int n_tgt,
                                        const double *x_tgt, int tgt_is_src, double *u);

/* (I + kappa/(4 pi) D) q at the mesh nodes, D as in ggem_double_layer:
 * kappa [n_nodes], q and out [n_nodes][3]. */
ggem_status ggem_bie_operator(ggem_plan_t *plan, const double *kappa, const double *q,
                              double *out);

/*
 * Learned warm start (no counterpart in the paper, which starts GMRES from the
 * previous time step, Sec. 5).  A 12-128-128-128-3 ReLU network estimates
 * A^-1 r - r node by node, A = I + kappa/(4 pi) D, for a right-hand side r
 * (the residual of a guess), from 12 features:
 *   0-2 r/s; 3-5 (kappa/4 pi)(D r)/s; 6-8 the node normal; 9 kappa;
 *   10 min(y - y0, y0 + W - y); 11 nodes of other particles within r_cut
 *   divided by the node count of the node's particle;
 * s = rms(r) over all nodes and components, so the estimate scales with r.
 * Inputs are standardised, (f - mu)/sigma; weights and hidden activations are
 * bfloat16 (round to nearest even), products accumulate in FP32:
 *   A^-1 r ~ r + s s_y MLP((f - mu)/sigma).
 * A model is 25 + 35075 doubles: mu[12], sigma[12], s_y, then W1[12][128],
 * b1[128], W2[128][128], b2[128], W3[128][128], b3[128], W4[128][3], b4[3]
 * (W[fan_in][fan_out]).  The first call that needs the model's buffers
 * allocates them.
 */

/* Particle id of each node (caller order), ids in [0, n_particles); needed
 * by the features.  Call after ggem_mesh_set. */
ggem_status ggem_mesh_particles(ggem_plan_t *plan, int n_particles, const int *particle);

/* The 12 features [n_nodes][12] of the right-hand side r [n_nodes][3] on the
 * current mesh (one double-layer evaluation), and s = rms(r) (may be NULL). */
ggem_status ggem_mlp_features(ggem_plan_t *plan, const double *kappa, const double *r,
                              double *feat, double *scale);

/* delta [n_nodes][3] = the learned estimate of A^-1 r. */
ggem_status ggem_mlp_guess(ggem_plan_t *plan, const double *kappa, const double *r,
                           double *delta);

/* Arithmetic of the network (forward, guess and training): GGEM_MLP_BF16
 * (the default; the rounding points above) or GGEM_MLP_FP32 (no rounding
 * point: FP32 master weights, FP32 inputs and activations), e.g. to check
 * the kernels entry by entry against an FP64 reference. */
#define GGEM_MLP_BF16 0
#define GGEM_MLP_FP32 1
ggem_status ggem_mlp_precision(ggem_plan_t *plan, int mode);

/* Load / save a model (count = 25 + 35075 doubles, layout above). */
ggem_status ggem_mlp_load(ggem_plan_t *plan, const double *model, size_t count);
ggem_status ggem_mlp_save(ggem_plan_t *plan, double *model, size_t count);

/* Adam state of the model (first and second moments [35075], FP32 on the
 * device, and the step count that sets the bias corrections): set = 0 reads
 * it into m, v, *step; set = 1 replaces it (checkpoint / resume of training).
 * m, v host or device. */
ggem_status ggem_mlp_adam_state(ggem_plan_t *plan, int set, double *m, double *v,
                                long long *step);

/* Raw network output [n][3] (units of s_y) for n feature rows [n][12]. */
ggem_status ggem_mlp_forward(ggem_plan_t *plan, int n, const double *feat, double *out);

/*
 * Train on n samples: features [n][12] and targets (A^-1 r - r)/s [n][3].
 * init != 0 starts a fresh model: mu, sigma (1 for a constant feature) and
 * s_y = rms(target) from these samples, He-uniform weights from seed, zero
 * biases.  Then `epochs` passes over minibatches of `batch` rows in an order
 * shuffled from seed; loss = mean over rows and components of
 * (output - target/s_y)^2; Adam (0.9, 0.999, 1e-8) at rate lr on FP32 master
 * weights.  *loss (may be NULL) gets the mean minibatch loss of the last
 * epoch.  With epochs = 0, one full-batch pass in row order computes *loss
 * and, when grad_out is not NULL, the gradient [35075] without updating.
 * Allocates and frees its own staging buffers.  GGEM_ERR_NUMERICAL when init
 * finds a non-finite feature or target.
 */
ggem_status ggem_mlp_train(ggem_plan_t *plan, int n, const double *feat, const double *target,
                           int init, unsigned long long seed, int epochs, int batch, double lr,
                           double *loss, double *grad_out);

/* Device-side status of the plan's kernels: waits with an iteration limit
 * (the tensor-core kernels' mbarrier waits) record a failure instead of
 * hanging; GGEM_ERR_CUDA here means results since the plan was created are
 * invalid.  Synchronises the plan's stream. */
ggem_status ggem_check(ggem_plan_t *plan);

/* Failure injection for tests of the bounded waits (no counterpart in the
 * paper): the next tensor-core Chebyshev transform launched in this process
 * (by any plan) issues no MMA for the first tile of each CTA and polls its
 * mbarrier at most `polls` times (1 .. 2^24), so its wait expires with no
 * work in flight: the kernel records the failure (seen by ggem_check),
 * releases its tensor memory and returns; the CUDA context stays usable. */
ggem_status ggem_inject_tc_wait_expiry(long polls);

/*
 * Tracing (no counterpart in the paper).  With tracing enabled, each stage
 * of an evaluation is bracketed by CUDA events on the plan's stream and the
 * host waits for its end, so per-stage device times can be read back; this
 * serialises the host with the device and is meant for measurement only.
 * ggem_trace_enable also resets the counters and the launch count.
 */
ggem_status ggem_trace_enable(ggem_plan_t *plan, int on);
int ggem_trace_stage_count(void);
const char *ggem_trace_stage_name(int stage);
ggem_status ggem_trace_read(const ggem_plan_t *plan, int stage, double *total_ms,
                            long *calls);
/* Measurement probe (no counterpart in the paper): the throughput of float4
 * vector reductions (atomic adds) into an L2-resident buffer of nvec 16-byte
 * vectors (a multiple of 32, at most 2^28) -- the operation the spreading is
 * bound by: 8 blocks of 256 threads per SM, every warp adding into 32
 * consecutive vectors at a pseudo-random position, `iters` times each; one
 * untimed launch, then one timed by CUDA events on `stream`.  *ms: the
 * timed launch; *vec_per_s: vector reductions per second.  Allocates and
 * frees its buffer. */
ggem_status ggem_probe_l2_reduction(long nvec, int iters, void *stream, double *ms,
                                    double *vec_per_s);
/* Measurement probe (no counterpart in the paper): the throughput of FP32
 * atomic adds into shared memory -- what a spreading staged in shared memory
 * (sources accumulated into a tile of the grid, one write per node) would be
 * bound by: 4 blocks of 256 threads per SM, each holding 4096 nodes x 3
 * components (48 KB); every warp adds into 32 consecutive nodes of each
 * component at a pseudo-random place of its block's tile, `iters` times
 * (1 <= iters <= 2^20); one untimed launch, then one timed by CUDA events on
 * `stream`.  *ms: the timed launch; *adds_per_s: scalar adds per second.
 * Allocates and frees a 48 KB result buffer. */
ggem_status ggem_probe_smem_reduction(int iters, void *stream, double *ms, double *adds_per_s);

/* Number of library kernels launched by this plan since creation or the
 * last ggem_trace_enable. */
ggem_status ggem_launch_count(const ggem_plan_t *plan, long *launches);

#ifdef __cplusplus
}
#endif
#endif /* GGEM_H */
