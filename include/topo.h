/*
 * topo.h - C ABI of the GB300 SIMP state-solve library (libtopo.so).
 *
 * The library computes, on one GPU, the state solve, compliance and element
 * sensitivities of density-based (SIMP) compliance topology optimisation on a
 * structured grid of trilinear 8-node bricks (arXiv 2605.04735):
 *
 *   E_e = Emin + rho_e^p (E0 - Emin)                        Sec. 2.1, Eq. (1)
 *   K(rho) U = F,  J = F^T U = U^T K U = sum_e u_e^T k_e u_e Sec. 2.1.1, Eq. (2)
 *   dJ/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e     Sec. 2.1.2, Eq. (3)
 *
 * k0 is the 24x24 matrix of the unit cube brick for unit Young's modulus
 * (Sec. 2.1.2), exact (2x2x2-point) integration of the trilinear element,
 * isotropic material with Poisson ratio nu; an element of edge h uses h*k0.
 * The paper does not say how K U = F is solved: the library solves it with
 * matrix-free preconditioned conjugate gradients (Jacobi or a geometric
 * multigrid V-cycle), either all in FP64 or in FP32 inside FP64 iterative
 * refinement, always to a true FP64 relative residual.
 *
 * Numbering (both for inputs and outputs):
 *   node    n = i + (nx+1) * (j + (ny+1) * k),  0 <= i <= nx, ...
 *   DOF     3 n + c, c = 0 (x), 1 (y), 2 (z)     (displacements: n_dof = 3 * nodes)
 *   element e = i + nx * (j + ny * k),           0 <= i < nx, ...
 *   local nodes of an element: (0,0,0) (1,0,0) (1,1,0) (0,1,0)
 *                              (0,0,1) (1,0,1) (1,1,1) (0,1,1)
 *
 * Conventions for every entry point:
 *   - Every call returns a topo_status; nothing throws across the ABI.
 *   - The library owns the mesh and all device memory it allocates; caller
 *     arrays are only read or written during the call (inputs are copied).
 *   - on_device != 0: the pointer is a device pointer on the mesh's device;
 *     on_device == 0: it is a host pointer (pageable or pinned).
 *   - Streams: each mesh runs its kernels on its own non-blocking stream and
 *     fences it against the caller's stream (given to topo_create_mesh or
 *     topo_set_stream; NULL = the legacy default stream) with events: a
 *     call's work starts after everything already enqueued on the caller's
 *     stream, and work the caller enqueues after the call starts after it.
 *     Calls that return host values synchronise; the others only enqueue.
 *     One mesh must not be used from two host threads at once; different
 *     meshes are independent.
 *   - Sizes are checked: a count that differs from the mesh's size returns
 *     TOPO_ERR_INVALID and touches nothing.
 */
#ifndef TOPO_H
#define TOPO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct topo_mesh topo_mesh; /* opaque, library-owned */

typedef enum {
  TOPO_OK = 0,
  TOPO_ERR_INVALID = -1,       /* bad argument, size or option */
  TOPO_ERR_OOM = -2,           /* device or host allocation failed */
  TOPO_ERR_CUDA = -3,          /* a CUDA runtime/driver call failed */
  TOPO_ERR_NO_DENSITY = -4,    /* solve before set_density */
  TOPO_ERR_NOT_SOLVED = -5,    /* compliance/sensitivity before a solve */
  TOPO_ERR_NOT_CONVERGED = -6, /* iteration limits reached above rtol */
  TOPO_ERR_NAN = -7,           /* NaN/Inf or out-of-range density, or a NaN in the solve */
  TOPO_ERR_TIMEOUT = -8        /* a bounded device-side wait ran out */
} topo_status;

/* Boundary conditions (zero displacement on the listed DOFs). */
enum {
  TOPO_BC_CANTILEVER = 0, /* every component of every node with i = 0 */
  TOPO_BC_MBB = 1,        /* u_x on i = 0; u_z on (i = nx, k = 0); u_y at (nx, ny/2, 0); ny even */
  TOPO_BC_ROLLER_BOX = 2, /* u_x on i = 0, u_y on j = 0, u_z on k = 0 (test problem) */
  /* the paper's problems (Sec. 4.2, 4.3) on a 2:1:1 domain, sizes relative to
   * the unit cross-section of ny x nz elements: */
  TOPO_BC_CORNERS = 3,   /* i = 0 fixed on four corner squares j, k <= 0.3 n or >= 0.7 n */
  TOPO_BC_MBB_STRIP = 4, /* u_x on i = 0; u_z on the bottom strip i >= nx-1; u_y pin; ny even */
  TOPO_BC_NONE = 5       /* no support: a slab of a larger grid whose supports the caller
                            applies (K is singular: for topo_apply and topo_jacobi_inverse,
                            not for solves) */
};

/* Loads (consistent nodal forces; total magnitude params.load). */
enum {
  TOPO_LOAD_EDGE_XL_BOTTOM = 0,  /* -z along the line i = nx, k = 0 */
  TOPO_LOAD_EDGE_X0_TOP = 1,     /* -z along the line i = 0, k = nz */
  TOPO_LOAD_FACE_XL_TRACTION = 2, /* uniform +x traction (per unit area) on i = nx */
  TOPO_LOAD_DISC_XL = 3,          /* -z on the x = L face quads within 0.1 ny of its centre */
  TOPO_LOAD_HALFDISC_X0_TOP = 4   /* -z on the top face quads within 0.1 ny of (0, ny/2) */
};

/* Arithmetic of the inner (preconditioned CG) solve. */
enum {
  TOPO_PREC_FP64 = 0, /* plain FP64 PCG (the reference GPU path) */
  TOPO_PREC_FP32 = 1, /* FP32 PCG inside FP64 iterative refinement */
  TOPO_PREC_DWORD = 2 /* topo_apply / topo_apply_internal only: the operator in double-word
                         arithmetic (two FP32 words per value, ~48 significand bits) */
};

/* Operator kernels (both compute the same K x; results agree to rounding). */
enum {
  TOPO_OPERATOR_MODAL = 0,  /* element-centric, k0 in the Walsh-Hadamard modal basis (default;
                               the library picks the FP32 kernel form per grid) */
  TOPO_OPERATOR_GATHER = 1, /* node-centric 27-node gather with the dense 24x24 k0 */
  TOPO_OPERATOR_MODAL_SINGLE = 2, /* modal, one element column per thread */
  TOPO_OPERATOR_MODAL_PAIR = 3,   /* modal, two element columns per thread in packed two-wide
                                     FP32 arithmetic, on FP32 grids with nx >= 65 (others fall
                                     back to one column) */
  TOPO_OPERATOR_TENSOR = 4  /* the element products K0 U_e (Eq. (3)'s k_e = E_e k0) as TF32
                               GEMMs on the tensor cores (tcgen05, accumulator in TMEM): the
                               CG operator and FP32 residuals in three TF32 passes (FP32-level
                               accuracy), the multigrid smoother's operator in one TF32 pass;
                               FP64 kernels and grids too small for the tiles (ny < 6) keep
                               the modal SIMT kernels */
  ,
  TOPO_OPERATOR_MODAL_CLUSTER = 5 /* modal, one element column per thread, the x tiles of a
                                     grid row as one thread-block cluster passing the halo
                                     column's sums through distributed shared memory (no
                                     recomputed halo column); FP32 grids with nx <= 128 (others
                                     use the tiled one-column kernel) */
};

enum {
  TOPO_PRECOND_JACOBI = 0, /* D^-1, D = diag K */
  TOPO_PRECOND_GMG = 1     /* one geometric multigrid V-cycle (2:1 vertex-nested grids) */
};

typedef struct {
  double E0;    /* solid Young's modulus (default 1) */
  double Emin;  /* void modulus (default 1e-9) */
  double nu;    /* Poisson ratio (default 0.3), 0 <= nu < 0.5 */
  double penal; /* SIMP exponent p (default 3), p >= 1 */
  double h;     /* element edge length (default 1) */
  double load;  /* total edge load, or traction per unit area (default 1) */
} topo_params;

typedef struct {
  int precision;     /* TOPO_PREC_* (default FP32) */
  int precond;       /* TOPO_PRECOND_* (default GMG) */
  double rtol;       /* target ||f - K u||_2 / ||f||_2 over free DOFs, in FP64 (default 1e-8) */
  double inner_rtol; /* relative residual reduction of each inner solve (default 1e-5) */
  int max_iter;      /* cap on inner CG iterations summed over the solve (default 100000) */
  int max_outer;     /* cap on refinement steps (default 12) */
  int warm_start;    /* 1: start from the stored displacement, 0: from zero */
  int gmg_levels;    /* 0: as many 2:1 levels as the grid allows (coarsest <= ~3000 DOF) */
  int smooth_degree; /* Chebyshev smoother degree per pre/post smoothing (default 3) */
  int check_every;   /* inner iterations between host convergence checks (default 8) */
  int residual;      /* TOPO_RESIDUAL_*: arithmetic of the refinement residual f - K u of
                        TOPO_PREC_FP32 solves (default DWORD); FP64 solves use FP64 */
} topo_solve_opts;

enum {
  /* K u in double-word arithmetic (two FP32 words, ~48 significand bits: rounding
     error ~2^-48 per operation, against 2^-53 in FP64), f - K u and ||r||^2 in
     FP64.  GB300 issues FP32 64 times as fast as FP64. */
  TOPO_RESIDUAL_DWORD = 0,
  TOPO_RESIDUAL_FP64 = 1 /* every operation in FP64 */
};

/* Where a failed solve stopped (topo_solve_info.detail). */
enum {
  TOPO_FAIL_NONE = 0,
  TOPO_FAIL_SETUP = 1,       /* options, allocation or setup before the first residual */
  TOPO_FAIL_RESIDUAL = 2,    /* a true FP64 residual was not finite */
  TOPO_FAIL_BREAKDOWN = 3,   /* inner CG breakdown (p.Ap <= 0 or r.z <= 0 or non-finite) */
  TOPO_FAIL_LIMIT = 4,       /* iteration or refinement caps reached */
  TOPO_FAIL_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  TOPO_FAIL_DEVICE = 6       /* a CUDA call failed */
};

typedef struct {
  int iters;           /* inner CG iterations (all refinement steps) */
  int outer;           /* FP64 refinement steps (residual evaluations after the first) */
  int status;          /* the topo_status the call returned */
  int detail;          /* TOPO_FAIL_* */
  double rel_residual; /* final true FP64 relative residual */
  double seconds;      /* wall time of the call */
} topo_solve_info;

/* Defaults as documented above. */
void topo_default_params(topo_params* p);
void topo_default_opts(topo_solve_opts* o);

/* Create a mesh of nx*ny*nz elements (each in [1, 4096], fewer than 2^31
 * nodes in all; TOPO_ERR_INVALID otherwise) with the given boundary
 * condition and load, on the current CUDA device.  stream: the caller's
 * cudaStream_t to order against (NULL = legacy default stream).  Allocates all device state of the
 * FP32/FP64 Jacobi paths; the multigrid hierarchy is built on first use.
 * Cites Eq. (2): K is assembled implicitly (matrix-free) from E_e k0. */
topo_status topo_create_mesh(int nx, int ny, int nz, int bc, int load, const topo_params* prm,
                             void* stream, topo_mesh** out);

/* Create a group of n_designs (1..1024) meshes of one grid, BC, load and
 * material whose solve state (vectors, scalars and a multigrid hierarchy built
 * now with gmg_levels / smooth_degree as in topo_solve_opts) shares one device
 * arena, design b at a fixed stride from design 0.  Each out[b] is an ordinary
 * mesh (every call works on it, topo_free frees it; the arena goes with the
 * last one).  topo_solve_many on exactly the group's meshes (any order)
 * solves them as one batch (one kernel launch per step for all designs,
 * FP64 refinement in lockstep, a design that has converged sits out) with
 *   - FP32 precision and the multigrid preconditioner with the group's
 *     gmg_levels and smooth_degree, or
 *   - the Jacobi preconditioner in FP32 (inside FP64 refinement) or FP64
 *     (the plain FP64 Jacobi-PCG path; its FP64 CG vectors are allocated
 *     for the whole group on first use, at the group stride);
 * other options solve the meshes one by one on their own streams.
 * Results equal the one-at-a-time solves up to FP rounding order. */
topo_status topo_create_batch(int nx, int ny, int nz, int bc, int load, const topo_params* prm,
                              void* stream, int n_designs, int gmg_levels, int smooth_degree,
                              topo_mesh** out);

/* Set element densities rho (n_elem float32 values in [0, 1], element
 * order) and derive E_e by Eq. (1).  NaN/Inf or values outside [0, 1] give
 * TOPO_ERR_NAN (checked on the device; the call synchronises).  Invalidates
 * the stored solution's compliance/sensitivity until the next solve; the
 * displacement itself is kept for warm starts. */
topo_status topo_set_density(topo_mesh* m, const float* rho, size_t n_elem, int on_device);

/* Solve K(rho) u = f (Eq. (2)) to opts->rtol in the true FP64 residual.
 * opts NULL = defaults.  info may be NULL; when given it is always filled.
 * Returns TOPO_ERR_NOT_CONVERGED (u kept, info->rel_residual set) if the
 * iteration caps are reached first. */
topo_status topo_solve(topo_mesh* m, const topo_solve_opts* opts, topo_solve_info* info);

/* Solve n distinct meshes at once (same options; NULL = defaults): each
 * mesh runs on its own stream and one host thread advances all of them, so
 * their kernels overlap on the GPU (batched / continuous solving); the meshes
 * of one group (topo_create_batch) run as one batch instead.  infos:
 * NULL or n entries, each filled as by topo_solve.  Returns TOPO_OK if every
 * solve succeeded, else the first failing status (see infos for each);
 * TOPO_ERR_INVALID if a mesh appears twice.  Blocks until all are done. */
topo_status topo_solve_many(topo_mesh* const* meshes, int n, const topo_solve_opts* opts,
                            topo_solve_info* infos);

/* Compliance J = f^T u (Eq. (2)) of the last solve, computed in FP64. */
topo_status topo_compliance(topo_mesh* m, double* c);

/* Compliance J = sum_e E_e u_e^T k0 u_e (Eq. (2), element form) of the last
 * solve; equals topo_compliance at equilibrium. */
topo_status topo_compliance_energy(topo_mesh* m, double* c);

/* Element sensitivities dJ/drho_e (Eq. (3)) of the last solve, FP64,
 * n_elem values in element order. */
topo_status topo_sensitivity(topo_mesh* m, double* dc, size_t n_elem, int on_device);

/* Batched forms of topo_set_density, topo_compliance and topo_sensitivity
 * for n meshes of one grid (n_elem elements each): design b's densities
 * (floats) or sensitivities (doubles) at b * n_elem in one contiguous array
 * (host, or device with on_device != 0); c receives n compliances (host).
 * Results equal the per-mesh calls'.  When the meshes are a whole mesh group
 * in its own order (topo_create_batch), each is one kernel launch for all
 * designs and one host synchronisation (set_density: the validity flags;
 * compliance: the values); otherwise the per-mesh calls run in turn.
 * Errors: TOPO_ERR_INVALID (NULL or repeated mesh, n < 1, n_elem not the
 * grid's), TOPO_ERR_NAN (set_density: a density outside [0, 1] in some
 * design, which then has none), TOPO_ERR_NOT_SOLVED.  Eqs. (1), (2), (3). */
topo_status topo_set_density_many(topo_mesh* const* meshes, int n, const float* rho,
                                  size_t n_elem, int on_device);
topo_status topo_compliance_many(topo_mesh* const* meshes, int n, double* c);
topo_status topo_sensitivity_many(topo_mesh* const* meshes, int n, double* dc, size_t n_elem,
                                  int on_device);

/* Copy the stored FP64 displacement out (n_dof = 3 * nodes, DOF order). */
topo_status topo_get_displacement(topo_mesh* m, double* u, size_t n_dof, int on_device);

/* The inverse Jacobi diagonal of K (Eq. (2)) from the current densities, in
 * FP64, DOF order: 1 / K_ii on free DOFs, 1 on fixed DOFs and where K_ii
 * vanishes.  n_dof = 3 * nodes.  TOPO_ERR_NO_DENSITY before set_density.
 * (With TOPO_BC_NONE, the diagonal of a slab: the caller's x-slab
 * decomposition supplies its supports.) */
topo_status topo_jacobi_inverse(topo_mesh* m, double* dinv, size_t n_dof, int on_device);

/* Replace the stored displacement (warm start, checkpoint restore).
 * Entries on fixed DOFs are ignored (held at zero). */
topo_status topo_set_displacement(topo_mesh* m, const double* u, size_t n_dof, int on_device);

/* y = M K M x with M the diagonal mask of free DOFs: entries of x on fixed
 * DOFs are taken as 0 and y is 0 there (the operator the solver inverts on
 * the free DOFs, Eq. (2)).  K comes from the current densities.  precision
 * TOPO_PREC_FP64, TOPO_PREC_FP32 or TOPO_PREC_DWORD selects the kernel (FP32
 * rounds x to float and returns y widened to double; DWORD splits x into two
 * FP32 words and evaluates K x in double-word arithmetic, the residual's
 * kernel).  n_dof values in DOF order. */
topo_status topo_apply(topo_mesh* m, int precision, const double* x, double* y, size_t n_dof,
                       int on_device);

/* Launch the fine-grid FP32 (or FP64, or double-word) operator kernel
 * `reps` times on the mesh's stream over the mesh's internal vectors (no
 * copies, no sync), for timing.  Cites Eq. (2) (K u). */
topo_status topo_apply_internal(topo_mesh* m, int precision, int reps);

/* ---------------------------------------------------------------------
 * The rest of a SIMP iteration (Sec. 2.1.3 Eq. (4) filter, Optimality
 * Criteria update named in Sec. 2.1.2 / Sec. 4.1).
 * --------------------------------------------------------------------- */
typedef struct {
  double volfrac;       /* target mean density V_f (default 0.4, Sec. 4.1) */
  double filter_radius; /* R in element edges (default 2: R = 2h, Sec. 4.1); <= 2.9 */
  double move;          /* OC move limit per iteration (default 0.2; not in the paper) */
  double eta;           /* OC damping exponent (default 0.5; not in the paper) */
  double rho_min;       /* lower density bound (default 1e-3) */
} topo_simp_opts;

typedef struct {
  double compliance; /* f^T u of the solved state the update used */
  double volume;     /* mean of the new densities */
  double change;     /* max_e |rho_new - rho| (the Delta rho_max of Sec. 4.1) */
  double lambda;     /* the OC Lagrange multiplier found */
} topo_simp_info;

void topo_default_simp_opts(topo_simp_opts* o);

/* One SIMP density update after a solve: sensitivities (Eq. (3)), filtered
 * by Eq. (4) with H = max(0, R - |x_e - x_i|) and the denominator density
 * guarded below by 1e-3, then the OC update rho_new = clip(rho (b/lambda)^eta,
 * max(rho_min, rho - move), min(1, rho + move)), b = max(-filtered dc, 0),
 * lambda bisected on the device so that mean(rho_new) = volfrac.  The new
 * densities replace the mesh's (E by Eq. (1)); the displacement is kept as
 * the warm start of the next solve.  Requires a solved state. */
topo_status topo_simp_update(topo_mesh* m, const topo_simp_opts* opts, topo_simp_info* info);

/* Filter an element field dc (n_elem doubles) by Eq. (4) with the mesh's
 * current densities; result in dcf.  Invalidates the stored solution's
 * sensitivities (call after compliance/sensitivity reads). */
topo_status topo_filter(topo_mesh* m, double radius, const double* dc, double* dcf, size_t n_elem,
                        int on_device);

/* Copy the mesh's current densities out (n_elem floats). */
topo_status topo_get_density(topo_mesh* m, float* rho, size_t n_elem, int on_device);

/* ---- the level-set stage's state problem (ersatz material) ----------------- */

/* Set the element moduli from a nodal level set instead of densities
 * (Sec. 2.2.2, Eqs. (7)-(9)): phi_e = phi at the element centroid (the mean of
 * the element's 8 nodal values), H_eta(phi_e) the regularised Heaviside of
 * Eq. (8) (0 below -eta, 1 above eta), I = (1 - H) + eps0 H, and
 * k_e(phi) = I(phi_e) k_e^0, i.e. E_e = E0 I(phi_e).  phi < 0 is material.
 *   phi      n_nodes = (nx+1)(ny+1)(nz+1) doubles, node i + (nx+1)(j + (ny+1)k),
 *            host or device (on_device); copied, not retained.
 *   eta      band half-width (> 0, element units of h);  eps0 in [0, 1].
 *   volume   if not NULL: V(phi) = sum_e V_e (1 - H(phi_e)) (Eq. (10)).
 * Later solves, compliance and displacement use these moduli until the next
 * topo_set_density / topo_set_levelset.  TOPO_ERR_NAN if phi holds a NaN. */
topo_status topo_set_levelset(topo_mesh* m, const double* phi, size_t n_nodes, int on_device,
                              double eta, double eps0, double* volume);
/* (phi may be NULL: the mesh's current level set, e.g. after topo_hj_evolve
 * or topo_reinit, is used.  The mesh keeps its own copy of phi.) */

/* Copy the mesh's current level set out (n_nodes doubles). */
topo_status topo_get_levelset(topo_mesh* m, double* phi, size_t n_nodes, int on_device);

/* Nodal right-hand sides of the relaxed shape derivatives (Sec. 2.2.5,
 * Eqs. (14), (15)) for the last solve and the level set of the last
 * topo_set_levelset, by 2x2x2 Gauss quadrature per element with phi and
 * grad(phi) of the Q1 interpolant:
 *   bJ[n] = int sigma(u):eps(u) N_n H'_eta(phi) |grad phi| dx
 *           (sigma:eps = eps^T D(E0, nu) eps, the solid's strain energy density)
 *   bV[n] = int N_n H'_eta(phi) |grad phi| dx   (C' of Eq. (15) is -bV / V_D)
 * The augmented-Lagrangian right-hand side (Eqs. (16)-(18)) is
 * bJ + ((lambda - Lambda C) / V_D) bV.  Either output may be NULL.
 * TOPO_ERR_NOT_SOLVED before a solve; TOPO_ERR_INVALID if the level set has
 * changed since the moduli were set. */
topo_status topo_shape_rhs(topo_mesh* m, double* bJ, double* bV, size_t n_nodes, int on_device);

/* Hilbertian extension-regularisation (Sec. 2.2.6, Eqs. (19), (20)): solve
 * A_H v = b, A_H the Q1 discretisation of int (ell^2 grad v . grad w + v w),
 * with v = 0 on the loaded nodes (the traction boundary Gamma_N), by
 * Jacobi-PCG in FP64 on the device from v = 0 to the relative residual rtol
 * (b, v: n_nodes doubles, host or device).  *iters: CG iterations.
 * TOPO_ERR_NOT_CONVERGED when max_iter is reached (v holds the last iterate). */
topo_status topo_hilbertian_solve(topo_mesh* m, double ell, const double* b, double* v,
                                  size_t n_nodes, int on_device, double rtol, int max_iter,
                                  int* iters);

/* Hamilton-Jacobi evolution (Sec. 2.2.7, Eqs. (21), (22)) of the mesh's level
 * set under the nodal speed v (phi decreases where v > 0: material grows):
 * `steps` forward-Euler steps of the first-order Godunov upwind scheme with
 * dt = gamma h / max|v| (*dt, if not NULL, receives it; 0 when v = 0).
 * Differences that would reach outside the grid are 0.  The moduli are not
 * updated: call topo_set_levelset(m, NULL, ...) for the next state solve. */
topo_status topo_hj_evolve(topo_mesh* m, const double* v, size_t n_nodes, int on_device,
                           double gamma, int steps, double* dt);

/* ---- SIMP -> level-set geometry transfer (Sec. 3.2-3.4) ------------------- */

/* Nodal densities from the mesh's current element densities (Eqs. (25)-(27)):
 * per node, the linear polynomial fitted by least squares (normal equations
 * X^T X a = X^T rho over the m elements sharing the node, X rows [1 x_e^T],
 * x_e the centroids) evaluated at the node when m >= 4 and the centroids are
 * not coplanar; otherwise the average weighted by 1 / |x_n - x_e| (m > 1) or
 * the single element's density.  rho_n: n_nodes doubles. */
topo_status topo_nodal_density(topo_mesh* m, double* rho_n, size_t n_nodes, int on_device);

/* The whole transfer: nodal densities, the iso-surface at rho_t (0 < rho_t < 1)
 * as a triangle soup, and the signed distance to it at every node (Eqs.
 * (28)-(30): exact closest points; phi = -d where rho_n >= rho_t), stored as
 * the mesh's level set (moduli unchanged until topo_set_levelset(m, NULL, ...)).
 * The surface is made by marching tetrahedra: linear interpolation on the
 * edges of the 6 tetrahedra of the Kuhn split of each hexahedron (a closed
 * surface).  *n_triangles: its size (topo_get_surface copies it).
 * TOPO_ERR_INVALID if no boundary exists at rho_t (nothing to measure from). */
topo_status topo_levelset_from_density(topo_mesh* m, double rho_t, long long* n_triangles);

/* Triangulate the zero level set of the mesh's current level set (material
 * phi <= 0) the same way: the discretisation of the final design (Sec. 3.6). */
topo_status topo_extract_levelset_surface(topo_mesh* m, long long* n_triangles);

/* Copy the last extracted surface: 9 doubles per triangle (x, y, z of its three
 * vertices), triangles grouped by cell in element order.  max_triangles must be
 * at least *n_triangles (which is always set). */
topo_status topo_get_surface(topo_mesh* m, double* tri, size_t max_triangles, int on_device,
                             long long* n_triangles);

/* Reinitialisation (Sec. 2.2.8, Eqs. (23), (24)): pseudo-time steps of
 * phi_t + S(phi)(|grad phi| - 1) = 0, S(phi) = phi / sqrt(phi^2 + h^2 |grad phi|^2)
 * recomputed from the current phi each step (central differences, one-sided on
 * the boundary), the same upwind scheme, dt = gamma h (0 < gamma <= 1), until
 * a step changes no node by more than tol h or after max_steps steps (the test
 * runs every 8 steps); *steps receives the count. */
topo_status topo_reinit(topo_mesh* m, double gamma, double tol, int max_steps, int* steps);

/* Element strain energies for unit Young's modulus, w_e = u_e^T k^0 u_e
 * (k^0 of edge h), of the last solve: the element factor of Eq. (3) and of
 * the level-set derivative dJ/dphi_e = E0 (1 - eps0) H'(phi_e) w_e.
 * n_elem doubles, element i + nx(j + ny k).  TOPO_ERR_NOT_SOLVED before a
 * solve. */
topo_status topo_element_energy(topo_mesh* m, double* w, size_t n_elem, int on_device);

/* Select the operator kernel family for all later calls on this mesh
 * (TOPO_OPERATOR_*); synchronises the mesh's stream.  Cites Eq. (2). */
topo_status topo_set_operator(topo_mesh* m, int kind);

/* Throughput form of the multigrid hierarchy (no counterpart in the paper),
 * for meshes that share the GPU with many others (the solve server turns it
 * on for every design it admits): the coarse levels of at most 1024 nodes
 * and the coarsest solve run as one kernel per V-cycle, and the coarsest grid
 * is chosen within 222 DOF so that its FP64 inverse is formed by one kernel
 * instead of one kernel per pivot.  Fewer, longer launches per solve: more
 * solves per second when many meshes run at once, more latency for a mesh
 * alone.  Results differ from the default form by rounding and by the
 * hierarchy's depth (both stop on the same true FP64 residual).  enable: 1
 * or 0; the hierarchy is rebuilt at the next solve.  TOPO_ERR_INVALID for a
 * mesh of a mesh group (its batched solves run their coarse end that way
 * already).  Synchronises the mesh's stream. */
topo_status topo_set_throughput_mode(topo_mesh* m, int enable);

/* Change the caller stream the mesh orders its calls against. */
topo_status topo_set_stream(topo_mesh* m, void* stream);

/* Sizes and memory: nodes, free DOFs, bytes of device memory held. */
topo_status topo_mesh_info(const topo_mesh* m, long long* n_nodes, long long* n_free_dof,
                           long long* device_bytes);

/* Device bytes a mesh of this size would hold after a solve with opts
 * (NULL = defaults), for admission control.  No allocation. */
long long topo_footprint_bytes(int nx, int ny, int nz, const topo_solve_opts* opts);

/* Kernel timing: when enabled, the library records CUDA events around every
 * launch of the fine-grid FP32 operator kernel during topo_solve and sums
 * their durations.  topo_profile_read returns (and with reset != 0 zeroes)
 * that total, the number of such launches, and the number of all kernel
 * launches the mesh has made (counted whether or not timing is enabled).
 * Any output pointer may be NULL. */
topo_status topo_profile_enable(topo_mesh* m, int enable);
topo_status topo_profile_read(topo_mesh* m, double* total_ms, long long* launches,
                              long long* all_launches, int reset);
/* With timing enabled, the library also records CUDA events around every
 * finest-level Chebyshev smoothing step of the multigrid V-cycle (the
 * operator kernel with the smoothing epilogue; mesh groups: design 0 holds
 * the batch's timing).  Returns (and with reset != 0 zeroes) their summed
 * duration, the number of design-launches they covered (a batched launch
 * counts once per design it advanced) and the algorithmic bytes those
 * launches moved: per node 60 B when the step stores x, 72 B when it adds to
 * it (direction and residual read, residual and new direction written, x),
 * plus 4 B per element (the modulus).  Cites Eq. (2) (K u). */
topo_status topo_profile_read_smoother(topo_mesh* m, double* total_ms, long long* launches,
                                       double* bytes, int reset);

/* Element sensitivities (as topo_sensitivity) and the element-form
 * compliance (as topo_compliance_energy) of a given displacement, for
 * callers that cannot allocate GPU memory: processes that hand all device
 * memory to their own allocator or budget it once at start-up, real-time
 * loops in which an allocation's latency or failure is not acceptable, and
 * embedded hosts with a fixed memory map.  It needs no mesh and calls no
 * cudaMalloc, cudaFree or allocating library routine.  The paper has no
 * counterpart: this is an interface variant of the Eq. (3) kernel.
 *   u   : device, n_dof = 3 (nx+1)(ny+1)(nz+1) doubles, DOF order above
 *         (fixed DOFs must hold 0, as a solved displacement does);
 *   rho : device, nx*ny*nz floats in [0, 1], element order (not checked:
 *         a value outside [0, 1] gives NaN or a meaningless dc and c);
 *   dc  : device output, nx*ny*nz doubles;  c : device output, 1 double.
 * The pointers' lengths cannot be checked here: arrays shorter than the
 * grid needs are read or written past their end.
 * prm NULL = defaults.  Work is enqueued on `stream` (NULL = legacy default
 * stream); the call does not synchronise.
 * Scratch: a fixed 32 KiB device array inside the library (one per GPU that
 * loads it, held until the process exits).  This bounds the size: at most
 * 8,388,608 elements; larger grids return TOPO_ERR_INVALID before anything
 * is enqueued.  Every call shares the array and keeps its last contents (the
 * call clears the part that must start at zero), so calls that overlap on
 * the GPU (e.g. on two streams without ordering) race: serialise them.  The
 * first call on each device sets up the array's device address
 * (cudaGetSymbolAddress, again after the device's context has been
 * re-created); make that first call before any stream capture begins. */
topo_status topo_sensitivity_noalloc(int nx, int ny, int nz, const topo_params* prm,
                                     const double* u, const float* rho, double* dc, double* c,
                                     void* stream);

/* ---------------------------------------------------------------------
 * Continuous-batching solve server (no counterpart in the paper: the
 * serving pattern of the hot path).  A design is opened once (grid, BC,
 * load) and then receives solve jobs (densities).  Designs are admitted in
 * arrival order, with backfill, while their estimated device footprint
 * (topo_footprint_bytes) fits mem_budget_bytes and fewer than max_active are
 * resident; an admitted design keeps its mesh, displacement (each new job
 * warm-starts from the last solution) and multigrid hierarchy on the device
 * until it is closed.  All admitted designs solve concurrently, each on its
 * own stream; topo_server_poll advances them from the caller's thread.
 * Every solve uses `opts` (NULL = defaults) and computes the compliance.
 * --------------------------------------------------------------------- */
typedef struct topo_server topo_server;

typedef struct {
  int job, design;       /* ids returned by topo_server_submit / topo_server_open */
  int status;            /* topo_status of the solve */
  int detail;            /* TOPO_FAIL_* (and 1 also when the density was rejected) */
  int iters, outer;      /* as in topo_solve_info */
  double rel_residual;   /* final true FP64 relative residual */
  double compliance;     /* f^T u (valid when status == TOPO_OK) */
  double submit_s, start_s, finish_s; /* seconds since topo_server_create */
} topo_job_result;

topo_status topo_server_create(long long mem_budget_bytes, int max_active, const topo_params* prm,
                               const topo_solve_opts* opts, void* stream, topo_server** out);
/* TOPO_ERR_OOM if the design alone exceeds the budget. */
topo_status topo_server_open(topo_server* s, int nx, int ny, int nz, int bc, int load,
                             int* design);
/* Queue a solve of `design` with densities rho (host, n_elem floats, copied). */
topo_status topo_server_submit(topo_server* s, int design, const float* rho, size_t n_elem,
                               int* job);
/* Advance all designs; return up to max_out finished jobs (in completion
 * order).  wait != 0: block until at least one job finished or nothing is
 * left to do. */
topo_status topo_server_poll(topo_server* s, int wait, topo_job_result* out, int max_out,
                             int* n_out);
/* Results of the last finished job of a resident, idle design. */
topo_status topo_server_sensitivity(topo_server* s, int design, double* dc, size_t n_elem,
                                    int on_device);
topo_status topo_server_displacement(topo_server* s, int design, double* u, size_t n_dof,
                                     int on_device);
/* Retire a design: its memory is released once its queued jobs are done
 * (immediately, dropping its jobs, if it was never admitted). */
topo_status topo_server_close(topo_server* s, int design);
topo_status topo_server_stats(const topo_server* s, long long* bytes_in_use, long long* peak_bytes,
                              int* active, int* waiting);
void topo_server_free(topo_server* s);

/* Fault injection for tests of the failure path (no counterpart in the
 * paper).  count = 1 arms the mesh so that the next launch of its
 * TMA-staged FP32 operator kernel (the default operator on grids with
 * nx < 150) runs one bounded device-side wait on a barrier that nothing ever
 * completes, with a short poll limit: the wait runs out, the kernel records a
 * timeout, and the solve that launched it ends with TOPO_ERR_TIMEOUT,
 * detail TOPO_FAIL_TIMEOUT (in a mesh group: that design only).  The
 * operator's own data transfers are not touched, so the GPU context and the
 * mesh stay usable; the next solve starts with the flag cleared.  count = 0
 * disarms.  Synchronises the mesh's stream. */
topo_status topo_debug_inject_timeout(topo_mesh* m, int count);

/* Release everything the mesh holds (NULL-safe). */
void topo_free(topo_mesh* m);

/* Static string for a status code. */
const char* topo_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* TOPO_H */
