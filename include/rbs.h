/*
 * rbs.h -- C ABI of the GB300 rigid-body Stokes mobility library.
 *
 * The library solves the mobility problem of Corona, Greengard, Rachh and Veerapaneni, "An
 * integral equation formulation for rigid bodies in Stokes flow in three dimensions"
 * (arXiv:1606.07428): given the force F_i and torque T_i on every rigid particle, find its
 * translational velocity v_i and rotational velocity omega_i (Section 2, Eqs. 1-5), by the
 * second-kind single-layer formulation (Section 2.3, Eq. 25)
 *
 *     (1/2 I + K + L) mu = -(1/2 I + K) rho,     u = S[rho + mu],
 *
 * with rho the incident density of Eq. 19, K the traction operator (Eqs. 13, 22-23), S the
 * single-layer operator (Eqs. 10-11) and L the rigid force/torque projection (Eq. 26); v_i and
 * omega_i follow from u by Eqs. 41-42.  Particles are ellipsoids discretised on the spherical
 * grid of Eq. 33 with the quadrature of Eq. 35.
 *
 * Conventions for every call:
 *  - Return value: RBS_OK (0) or a negative status below; rbs_last_error() then holds a message.
 *  - Pointers named *_dev are CUDA device pointers on the context's device; all other array
 *    pointers are host pointers.  Arrays are row-major float64 unless stated otherwise.
 *  - Inputs are copied in; the caller keeps ownership of every buffer it passes.  Outputs are
 *    written into caller-allocated buffers of the stated size.
 *  - Surface fields (densities, velocities on the surface) are (total_nodes, 3) arrays; nodes are
 *    ordered particle-major, then by the polar index j (Gauss-Legendre nodes t_j ascending, i.e.
 *    theta descending), then by the azimuthal index k, node = j * n_phi + k.
 *  - A context is not thread-safe; use one context per host thread.  All device work of a context
 *    runs on the stream given at creation (or the legacy default stream when it is NULL).
 */
#ifndef RBS_H
#define RBS_H

#ifdef __cplusplus
extern "C" {
#endif

#define RBS_OK 0
#define RBS_EINVAL -1    /* invalid argument (null pointer, bad size, non-finite input, p out of range) */
#define RBS_EOVERLAP -2  /* particles closer than the gap the quadrature is built for */
#define RBS_ENOTCONV -3  /* GMRES hit max_iters; outputs are still written, iterations reported */
#define RBS_ECUDA -4     /* a CUDA runtime error; the message names the call */
#define RBS_ENOMEM -5    /* device allocation failed */
#define RBS_ETIMEOUT -6  /* a bounded device wait expired */
#define RBS_ESTATE -7    /* call out of order (e.g. a solve before rbs_set_geometry) */

/* Arithmetic of a solve. */
#define RBS_PREC_FP64 0  /* every step in float64 */
#define RBS_PREC_MIXED 1 /* float32 inner GMRES; right-hand side, refinement residuals and velocity
                            in the arithmetic of rbs_options.refine_precision; float64 vectors,
                            Arnoldi, refinement updates, projection and velocity extraction */
#define RBS_PREC_MIXED_FP16 2 /* RBS_PREC_MIXED with the self blocks of the inner GMRES (the
                            block-diagonal preconditioner of Section 3.2 and the K self blocks of its
                            restarts) stored in float16 and applied with float32 accumulation: on the
                            tensor cores for particles sharing a shape (a batched GEMM), on CUDA cores
                            otherwise.  Refinement residuals and float32 corrections keep float32
                            blocks, so only the inner operator's accuracy changes (about 5e-4) */
#define RBS_PREC_DF 3    /* float64-class operator: pair sums in double-float arithmetic (unevaluated
                            sums of two float32 numbers, ~1e-12 relative), blocks and vectors in
                            float64 (rbs_apply_operator and rbs_options.refine_precision only) */
#define RBS_PREC_MIXED_BF16 4 /* as RBS_PREC_MIXED_FP16 with bfloat16 self blocks (about 4e-3) */

/* Operators for rbs_apply_operator (each acts on a surface field, Section 2). */
#define RBS_OP_A 0        /* (1/2 I + K + L), the system operator of Eq. 25 */
#define RBS_OP_HALF_K 1   /* (1/2 I + K), the right-hand-side operator of Eq. 25 */
#define RBS_OP_S 2        /* S, Eq. 11, as used for u = S[rho + mu] */
#define RBS_OP_K_OFF 3    /* K restricted to pairs of distinct particles (smooth and upsampled rules) */
#define RBS_OP_K_SELF 4   /* K restricted to each particle's own surface (singular rule) */
#define RBS_OP_S_OFF 5
#define RBS_OP_S_SELF 6
#define RBS_OP_L 7        /* L of Eq. 26 */

typedef struct rbs_ctx rbs_ctx;

typedef struct {
  int precision;       /* RBS_PREC_FP64 (default), RBS_PREC_MIXED, RBS_PREC_MIXED_FP16 or
                          RBS_PREC_MIXED_BF16 */
  int restart;         /* GMRES restart length (default 50) */
  int max_iters;       /* cap on GMRES iterations per solve (default 500) */
  int preconditioner;  /* 1 (default): right block-diagonal preconditioner, the inverse of each
                          particle's own 1/2 I + K_ii + L_i (Section 3.2); 0: none */
  double near_delta;   /* particles i, j are near when |c_i - c_j| < R_i + R_j + near_delta, R the
                          bounding radius: the largest semi-axis of an ellipsoid, see
                          rbs_set_geometry_sh for a coefficient surface (default 1.0); near
                          sources use an upsampled grid */
  int p_up_factor;     /* near sources are upsampled to order p_up_factor * p (default 2) */
  int p_self_factor;   /* singular self rule of order p_self_factor * p (default 2) */
  double viscosity;    /* fluid viscosity (default 1.0) */
  double inner_tol;    /* RBS_PREC_MIXED: relative tolerance of each float32 inner solve (default 1e-5) */
  int max_refinements; /* RBS_PREC_MIXED: cap on float64 refinement steps (default 20) */
  int device;          /* CUDA device ordinal (default 0) */
  void* stream;        /* cudaStream_t for all device work, NULL = legacy default stream */
  int timing;          /* 1: time the kernel classes below with CUDA events on the context stream
                          (default 0); results in rbs_stats.kernel_ms */
  int refine_precision; /* RBS_PREC_MIXED: arithmetic of the right-hand side, refinement residuals
                          and velocity evaluation, RBS_PREC_DF (default) or RBS_PREC_FP64 */
  int pair_variant;    /* pair-kernel variant: targets per thread 1, 2 or 4, or for the float32
                          kernels 9, 10 or 12 = 8 + targets per thread of the packed kernels that
                          evaluate two sources per instruction (the double-float kernels then use
                          the targets per thread alone); 0 (default) times the candidates once per
                          context and kernel and keeps the fastest */
  int warm_start;      /* initial GMRES guess: RBS_WARM_ZERO (default), RBS_WARM_PREVIOUS (the last
                          solved density of this context), RBS_WARM_LEARNED (the trained network's
                          density for the current configuration) or RBS_WARM_LEARNED_DELTA (the last
                          solved density plus the change the network predicts between the last
                          solve's configuration and the current one; the network's guess alone on
                          the first solve); the converged solution does not depend on it */
  int warm_record;     /* 1: rbs_advance records a training sample (rbs_warmstart_record) after every
                          stage solve (default 0) */
  double contact_gap;  /* 0 (default): no contact handling; > 0: the contact algorithm of Section
                          3.4 after every mobility solve (and so in every rbs_advance stage): two
                          particles of one suspension are in contact when the smallest distance
                          between the nodes of their upsampled grids is below contact_gap, at the
                          midpoint of that closest node pair; contact forces that make the two
                          rigid velocities agree there are found from 3 n_c extra solves, and the
                          velocities and density returned include them */
  double magnetic_field[3]; /* uniform applied field H0 for rbs_advance (default 0) */
  double mu_ratio;     /* permeability of the particles over that of the fluid, mu / mu0 (default 1);
                          with mu_ratio != 1 and a non-zero field, every rbs_advance stage adds the
                          magnetic forces and torques of rbs_magnetic_forces to F and T */
  int far_field;       /* RBS_FAR_DIRECT (default): every smooth pair sum runs over all node pairs.
                          RBS_FAR_TREECODE: the float32 applies of the mixed solve (inner GMRES and
                          float32 corrections) approximate the smooth sums over well-separated
                          clusters of particles with a barycentric Lagrange treecode, the
                          hierarchical far field in place of Section 3.1's fast multipole method;
                          the double-float and float64 passes, and so the converged result, stay
                          direct.  RBS_FAR_TREECODE_DF: the double-float passes use a treecode too,
                          at tree_df_theta and tree_df_degree (relative error about 5e-11 at the
                          defaults); float64 passes stay direct.  Only with precision
                          RBS_PREC_MIXED */
  double tree_theta;   /* treecode opening criterion: a cluster of radius r_C is approximated for a
                          target particle of radius r_B at centre distance d when r_B + r_C <
                          tree_theta d (default 0.5; 0 < tree_theta < 1) */
  int tree_degree;     /* treecode interpolation degree n per axis: (n + 1)^3 Chebyshev proxy points
                          per cluster (default 7; 2 <= n <= 10) */
  double tree_df_theta; /* opening criterion of the double-float passes' treecode (default 0.4) */
  int tree_df_degree;  /* its interpolation degree (default 12; 2 <= n <= 12); its cluster charges are
                          formed in float64 */
  int graphs;          /* 1 (default): the GMRES Arnoldi step of the mobility operator is captured once
                          per configuration into a CUDA graph whose conditional loop runs a whole
                          restart cycle on the device; 0: the same kernels are launched from the host,
                          with one host read of the stopping flags per iteration */
} rbs_options;

#define RBS_FAR_DIRECT 0
#define RBS_FAR_TREECODE 1
#define RBS_FAR_TREECODE_DF 2

#define RBS_WARM_ZERO 0
#define RBS_WARM_PREVIOUS 1
#define RBS_WARM_LEARNED 2
#define RBS_WARM_LEARNED_DELTA 3

/* Kernel classes timed when rbs_options.timing is set (indices into rbs_stats.kernel_*). */
#define RBS_KC_PAIR_K32 0 /* smooth traction pair sum, float32 */
#define RBS_KC_PAIR_S32 1 /* smooth Stokeslet pair sum, float32 */
#define RBS_KC_PAIR_K64 2 /* smooth traction pair sum, float64 */
#define RBS_KC_PAIR_S64 3 /* smooth Stokeslet pair sum, float64 */
#define RBS_KC_BLOCKS 4   /* particle-block kernel (self blocks, projection, preconditioner) with float32 or
                             16-bit entries (the inner solve's arithmetic) */
#define RBS_KC_NEAR 5     /* near correction (upsampling and upsampled pair sums) */
#define RBS_KC_PAIR_KDF 6 /* smooth traction pair sum, double-float */
#define RBS_KC_PAIR_SDF 7 /* smooth Stokeslet pair sum, double-float */
#define RBS_KC_PAIR_KSDF 8 /* smooth traction and Stokeslet sums of one density in one pass, double-float */
#define RBS_KC_TREE 9     /* treecode cluster charges (RBS_FAR_TREECODE); the treecode's pair sums count
                             under RBS_KC_PAIR_K32 / RBS_KC_PAIR_S32 with their evaluated pairs as units */
#define RBS_KC_GMRES_GRAPH 10 /* launches of the captured GMRES cycle graph (rbs_options.graphs); units =
                             Arnoldi steps it ran.  Kernels replayed inside it are not counted under
                             their own classes (their launches still count in rbs_stats.launches) */
#define RBS_KC_SELF_GEMM 11 /* tensor-core GEMM of the 16-bit self blocks of a shared shape (the GEMM kernel
                             alone; units = its flops, 2 n_g (3 N_p)^2 per launch) */
#define RBS_KC_BLOCKS_F64 12 /* particle-block kernel with float64 entries (the float64 and double-float
                             applies), and applies of the L term alone */
#define RBS_KC_COUNT 13

typedef struct {
  int iterations;        /* GMRES iterations of the last solve (inner iterations for mixed), the largest
                            over the suspensions (rbs_get_suspension_results gives each) */
  int refinements;       /* outer float64 refinement steps of the last solve (0 for FP64) */
  double residual;       /* final relative residual ||b_s - A mu_s|| / ||b_s|| in float64, the largest over
                            the suspensions s */
  double setup_ms;       /* wall time of the last rbs_set_geometry */
  double solve_ms;       /* wall time of the last rbs_mobility_solve */
  long long total_nodes;
  int n_particles;
  int n_shapes;          /* distinct body shapes: (semi-axes or input surface, p, n_phi) */
  long long near_pairs;  /* ordered (target, source) particle pairs treated as near */
  long long far_pairs;   /* (target node, source node) pairs of the smooth pair sum per apply */
  long long launches;    /* kernels launched by the context since creation or rbs_reset_stats */
  double kernel_ms[RBS_KC_COUNT];        /* summed device time per class (rbs_options.timing) */
  long long kernel_count[RBS_KC_COUNT];  /* launches per class */
  double kernel_units[RBS_KC_COUNT];     /* work per class: node pairs (pair sums, near), bytes of
                                            block entries read (particle blocks) */
  int n_contacts;        /* contacts found by the last mobility solve (rbs_options.contact_gap > 0) */
  int pair_variant[5];   /* variant in use (as rbs_options.pair_variant): float32 traction, float32
                            Stokeslet (the treecode kernel's with RBS_FAR_TREECODE), double-float
                            traction, double-float Stokeslet, fused double-float traction and
                            Stokeslet (the double-float treecode kernel's targets per thread with
                            RBS_FAR_TREECODE_DF; 0 = not yet chosen) */
  long long tree_pairs;  /* RBS_FAR_TREECODE: (target node, source) pairs one treecode apply evaluates,
                            direct node pairs (the target's own particle included, masked) plus
                            proxy pairs; 0 without a treecode */
  long long tree_proxy_pairs; /* of these, the (target node, cluster proxy point) pairs */
  int tree_cells;        /* clusters that carry proxy points */
  long long tree_df_pairs;       /* the same for the double-float passes' treecode (RBS_FAR_TREECODE_DF) */
  long long tree_df_proxy_pairs;
  int tree_df_cells;
} rbs_stats;

/* Fill *opt with the defaults listed above. */
void rbs_default_options(rbs_options* opt);

/* Create a context on opt->device (opt may be NULL for the defaults).  *out receives the handle. */
int rbs_create(const rbs_options* opt, rbs_ctx** out);

/* Release every device and host resource of the context.  NULL is ignored. */
void rbs_destroy(rbs_ctx* ctx);

/*
 * Define the suspension (Section 3: surfaces and grids; Section 3.1: self blocks computed once per
 * body shape and rotated, Eq. 38; Section 3.2: block-diagonal preconditioner).
 *  n            number of particles, n >= 1
 *  semi_axes    n x 3, ellipsoid semi-axes (a, b, c) along the body x, y, z axes, all > 0
 *  p            n, spherical-harmonic order per particle, 2 <= p <= 32
 *  nphi         n, azimuthal points per particle (even, >= 2p; NULL means 2p for every particle)
 *  centres      n x 3
 *  quats        n x 4, orientations as quaternions (w, x, y, z); normalised here
 *  suspension_id  n (NULL: all particles in one suspension); particles with different ids do not
 *               interact.  Particles of one suspension must be contiguous.
 * Returns RBS_EOVERLAP when two interacting particles certainly overlap (their inscribed spheres,
 * of radius the smallest semi-axis, intersect).
 */
int rbs_set_geometry(rbs_ctx* ctx, int n, const double* semi_axes, const int* p, const int* nphi,
                     const double* centres, const double* quats, const int* suspension_id);

/* Largest degree of a coefficient surface accepted by rbs_set_geometry_sh. */
#define RBS_MAX_SHAPE_DEGREE 24

/*
 * Define a suspension of general genus-0 particles whose surfaces are given by spherical-harmonic
 * coefficients (Section 3, Eq. 31; tangents by spectral differentiation, Eq. 37; area element Eq. 36).
 *  nshape       number of distinct input surfaces, >= 1
 *  shape_pg     nshape, degree p_g of each surface, 1 <= p_g <= RBS_MAX_SHAPE_DEGREE
 *  shape_coef   the surfaces' coefficients, one after another: surface k holds 3 x (p_g + 1)^2
 *               doubles, the x row, then the y row, then the z row; each row in the library's basis
 *               order of real orthonormal harmonics without the Condon-Shortley sign: m = 0..p_g,
 *               n = m..p_g, the cos(m phi) term then, for m > 0, the sin(m phi) term
 *  shape_of     n, the input surface of each particle, 0 <= shape_of[i] < nshape
 *  p, nphi, centres, quats, suspension_id   as for rbs_set_geometry
 * Each surface's body frame is centred at its area centroid on the particle's grid (the centroid of
 * Eq. 18), so centres give that centroid's lab position.  The bounding radius R of the near criterion
 * is the largest centroid distance over the nodes of the upsampled grid, and the overlap test uses the
 * smallest such distance.  Returns RBS_EINVAL for a surface whose area element vanishes on a grid or
 * whose parametrisation is inward (negative enclosed volume).  The learned warm start's features
 * take (R, R, R) as the semi-axes of such a particle.  All arrays are host memory, read during the call
 * and not retained.
 */
int rbs_set_geometry_sh(rbs_ctx* ctx, int n, int nshape, const int* shape_pg, const double* shape_coef,
                        const int* shape_of, const int* p, const int* nphi, const double* centres,
                        const double* quats, const int* suspension_id);

/*
 * The contacts of the last mobility solve (Section 3.4; rbs_options.contact_gap > 0), in ascending
 * (first, second) particle order: pairs (max x 2 ints: first < second particle), points (max x 3:
 * the contact point x*) and forces (max x 3: the contact force on the first particle; the second
 * receives its negative).  Any output may be NULL.  Returns the number of contacts (which may exceed
 * max; only the first max are written) or a negative status.
 */
int rbs_get_contacts(rbs_ctx* ctx, int max, int* pairs, double* points, double* forces);

/*
 * Magnetostatic coupling (Section 4.1.3): the net magnetic force and torque on every particle of the
 * current geometry in the uniform field H0 (3 doubles) for particles of permeability mu_ratio times
 * the fluid's.  The potential is phi = -H0 . x + S^L[q] with (1/2 I + eta K^L) q = eta H0 . n,
 * eta = (mu_ratio - 1) / (mu_ratio + 1), solved by float64 GMRES to relative tolerance tol with the
 * library's smooth, near and singular rules (scalar kernels); the fluid-side field
 * H = -grad_s phi + (H0 . n + q/2 - K^L[q]) n gives the Maxwell traction (H . n) H - |H|^2 n / 2 (the
 * fluid's permeability mu0 taken as 1), integrated over each surface.  F and T: n x 3 host outputs;
 * q: total_nodes host output or NULL; iterations may be NULL.  The scalar self blocks (every row, per
 * distinct shape) are built on the first call for a geometry.
 */
int rbs_magnetic_forces(rbs_ctx* ctx, const double* H0, double mu_ratio, double tol, double* F, double* T,
                        double* q, int* iterations);

/* The Laplace operators of the magnetostatic coupling on scalar node fields (host arrays of
 * total_nodes): kind 0 gives y = K^L x, kind 1 gives y = S^L x (Section 4.1.3). */
int rbs_apply_laplace(rbs_ctx* ctx, int kind, const double* x, double* y);

/* Number of surface nodes of the current geometry (3 * that many unknowns). */
long long rbs_total_nodes(const rbs_ctx* ctx);

/* Copy the lab-frame nodes, unit normals and quadrature weights (Eqs. 33-36) of the current
 * geometry: x and normal are total_nodes x 3, weight is total_nodes (any may be NULL). */
int rbs_get_surface(rbs_ctx* ctx, double* x, double* normal, double* weight);

/*
 * The mobility solve (the three steps at the start of Section 3; Algorithm 1 lines 3-5 without
 * contact).  Suspensions (rbs_set_geometry's suspension_id) do not interact, so each is its own
 * system and converges on its own: GMRES keeps one Krylov recursion per suspension, and a suspension
 * stops iterating once its own residual is within tolerance.
 *  F, T        n x 3 forces and torques
 *  tol         relative residual ||b_s - A mu_s||_2 / ||b_s||_2 at which GMRES stops, for every
 *              suspension s (b the right-hand side of Eq. 25); for RBS_PREC_MIXED the float64
 *              refinement stops when every suspension is at this tolerance
 *  v, omega    n x 3 outputs
 *  density     NULL, or total_nodes x 3 output receiving mu (lab frame)
 *  iterations  NULL, or rbs_suspension_count() ints receiving each suspension's GMRES iterations (in
 *              the order the suspensions appear; one int for a single suspension)
 * Returns RBS_ENOTCONV (outputs written) when max_iters is reached first.
 */
int rbs_mobility_solve(rbs_ctx* ctx, const double* F, const double* T, double tol, double* v,
                       double* omega, double* density, int* iterations);

/* The same solve on device buffers (F_dev, T_dev, v_dev, omega_dev: n x 3; density_dev: NULL or
 * total_nodes x 3).  Work is ordered on the context's stream; the call returns after it completes. */
int rbs_mobility_solve_device(rbs_ctx* ctx, const double* F_dev, const double* T_dev, double tol,
                              double* v_dev, double* omega_dev, double* density_dev, int* iterations);

/* Number of suspensions of the current geometry (runs of equal suspension_id; 1 without ids). */
int rbs_suspension_count(const rbs_ctx* ctx);

/* Per-suspension outcome of the last mobility solve: iterations (NULL or rbs_suspension_count() ints,
 * GMRES iterations, summed over refinements and contact solves) and residual (NULL or that many
 * doubles, the final relative residual ||b_s - A mu_s|| / ||b_s|| of suspension s; 0 when b_s = 0). */
int rbs_get_suspension_results(rbs_ctx* ctx, int* iterations, double* residual);

/* Explicit Runge-Kutta schemes for rbs_advance. */
#define RBS_RK_EULER 1
#define RBS_RK_TRAPEZOID 2
#define RBS_RK4 4

/*
 * Rigid-body time stepping (Section 3.3, Eqs. 40 and 43; Algorithm 1): `steps` explicit
 * Runge-Kutta steps of size dt (scheme RBS_RK_EULER, RBS_RK_TRAPEZOID or RBS_RK4) of dc_i/dt = v_i,
 * dq_i/dt = 1/2 (0, omega_i) q_i, with the forces F and torques T (n x 3 each, host) held fixed.
 * Every stage is one mobility solve to relative tolerance tol at the stage configuration (the
 * body-frame self blocks and preconditioner are reused, Eq. 38), with the contact correction of
 * Section 3.4 when rbs_options.contact_gap > 0; quaternions are renormalised after each step.  The
 * context's configuration is updated in place; iterations (may be NULL) receives the GMRES iterations
 * summed over the stage solves (each stage counting its largest suspension).  Returns RBS_EOVERLAP if the inscribed spheres of two particles intersect.
 */
int rbs_advance(rbs_ctx* ctx, const double* F, const double* T, double dt, int steps, int scheme, double tol,
                int* iterations);

/* Current centres (n x 3) and unit quaternions (n x 4) of the context's particles (host arrays). */
int rbs_get_state(rbs_ctx* ctx, double* centres, double* quats);

/* Incident density rho of Eq. 19 for forces F and torques T (n x 3 each); rho is total_nodes x 3. */
int rbs_incident_density(rbs_ctx* ctx, const double* F, const double* T, double* rho);

/* Rigid velocities of Eqs. 41-42 from a surface velocity u (total_nodes x 3): v, omega n x 3. */
int rbs_rigid_velocities(rbs_ctx* ctx, const double* u, double* v, double* omega);

/*
 * Allocation-free variant of rbs_rigid_velocities, on device buffers.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory at call time, such as
 * frameworks that reserve nearly all device memory for their own pool (a cudaMalloc from inside them
 * can fail), real-time stepping loops that forbid allocator calls, or hosts that give the library a
 * fixed memory budget.
 *  u_dev      total_nodes x 3 surface velocity (device)
 *  v_dev, omega_dev   n x 3 outputs (device), Eqs. 41-42
 * The per-particle intermediate lives in a fixed device array of 6 x 65,536 float64 (3 MiB), which
 * every GPU that loads the library holds until the process exits; geometries with more than 65,536
 * particles are rejected with RBS_EINVAL.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the process; do not reset the device (cudaDeviceReset)
 * afterwards, since the array may then move and the kept address would be stale.  All calls, from every context of the process, share the one array per
 * device, and each call overwrites the entries it reads, so calls whose work overlaps on the GPU
 * (other contexts or streams at the same time) race and must be ordered by the caller.  Work runs on
 * the context's stream and the call waits for it to complete before returning; the caller's current
 * device is restored.
 */
int rbs_rigid_velocities_noalloc(rbs_ctx* ctx, const double* u_dev, double* v_dev, double* omega_dev);

/*
 * Apply one discrete operator (RBS_OP_*) to a surface field: y = op(x), x and y total_nodes x 3 host
 * arrays.  precision RBS_PREC_FP64 applies it in float64; RBS_PREC_MIXED in the float32 arithmetic of
 * the inner solve (pair sums with compensated accumulation, float32 self blocks); RBS_PREC_MIXED_FP16
 * and RBS_PREC_MIXED_BF16 the same with the K self blocks in float16 or bfloat16 (float32 accumulation;
 * the context must have been created with that precision; the S self blocks stay float64);
 * RBS_PREC_DF with double-float pair sums and float64 blocks.
 */
int rbs_apply_operator(rbs_ctx* ctx, int op, int precision, const double* x, double* y);

/* The same with device buffers (x_dev, y_dev: total_nodes x 3 float64). */
int rbs_apply_operator_device(rbs_ctx* ctx, int op, int precision, const double* x_dev, double* y_dev);

/*
 * Learned warm start.  The paper's GMRES (Section 3.2) starts from zero; this network only changes
 * the initial guess, so the solve still converges to the same tolerance and the same solution.
 * Definitions (one (p, n_phi) grid for all particles):
 *  - features, 128 floats per particle: R_i^T F_i, R_i^T T_i, semi-axes, then for its 16 nearest
 *    neighbours in the same suspension (centre distance ascending, ties to the lower index) the
 *    body-frame offset R_i^T (c_j - c_i) and the relative rotation conj(q_i) q_j (scalar part >= 0);
 *    absent neighbours and entries 121-127 are zero;
 *  - targets, 3 n_basis floats per particle: the real orthonormal spherical-harmonic coefficients
 *    (Eq. 32, no Condon-Shortley sign) of the body-frame density R_i^T mu, component-major, each in
 *    the order m = 0..m_max, n = m..p, cos then (m > 0) sin;
 *  - network: y = W3 g(W2 g(W1 x + b1) + b2) + b3, widths 128 -> 256 -> 256 -> 3 n_basis, g the tanh
 *    form of GELU; bfloat16 operands, float32 accumulation and float32 master weights (Adam).
 *    Parameters are flattened as W1 (128 x 256, row-major), b1, W2 (256 x 256), b2, W3 (256 x 3 n_basis),
 *    b3.  The network predicts targets divided by a scale (the RMS of the training targets).
 */
/* Record the features of the current configuration for F, T (n x 3, host) and the coefficients of the
 * context's last solved density as one training sample per particle. */
int rbs_warmstart_record(rbs_ctx* ctx, const double* F, const double* T);
/* Train on the recorded samples: `epochs` passes of shuffled minibatches of `batch` rows, Adam with
 * learning rate lr; the first call draws initial weights from `seed`.  loss (may be NULL) receives
 * the mean loss of the last epoch. */
int rbs_warmstart_train(rbs_ctx* ctx, int epochs, int batch, double lr, unsigned seed, double* loss);
/* Read (out != NULL) or load (in != NULL) the flattened float32 parameters; count receives their
 * number, scale the output scale (read, or loaded with `in`). */
int rbs_warmstart_weights(rbs_ctx* ctx, float* out, const float* in, long long* count, float* scale);
/* Feature rows of the current configuration (X: n x 128, host). */
int rbs_warmstart_features(rbs_ctx* ctx, const double* F, const double* T, float* X);
/* Target coefficients of a density mu (total_nodes x 3, host) into coef (n x 3 n_basis, host). */
int rbs_warmstart_targets(rbs_ctx* ctx, const double* mu, float* coef);
/* Network on host rows X (rows x 128): outputs Y (rows x 3 n_basis, may be NULL); with targets Yt,
 * the gradients of mean((Y - Yt)^2) into grads (flattened like the parameters) and the loss. */
int rbs_warmstart_mlp(rbs_ctx* ctx, int rows, const float* X, const float* Yt, float* Y, float* grads, double* loss);

/* Statistics of the last rbs_set_geometry / rbs_mobility_solve, and the launch and kernel-time
 * counters accumulated since creation or the last rbs_reset_stats (waits for pending timing events). */
int rbs_get_stats(rbs_ctx* ctx, rbs_stats* out);

/* Zero the launch and kernel-time counters. */
int rbs_reset_stats(rbs_ctx* ctx);

/* Message describing the last error of the context (empty when none); valid until the next call. */
const char* rbs_last_error(const rbs_ctx* ctx);

/*
 * Host-only plan of the treecode far field (rbs_options.far_field): the tree, interaction lists and
 * work split that a context builds for a geometry, computed on the host without any device work (so
 * also without a GPU), from
 *  n              number of particles, >= 1 (particles of a suspension contiguous)
 *  nodes          n, node count per particle, >= 1
 *  centres        n x 3
 *  radius         n, bounding radius: every node lies within it of the centre
 *  node_box       n x 6, the bounding box of each particle's nodes: lo x, y, z, then hi x, y, z
 *  suspension_id  n, or NULL for one suspension
 *  theta, degree, near_delta   as rbs_options.tree_theta, tree_degree (2..12) and near_delta
 *  sm_count       SMs the work split is sized for (>= 1)
 *  out            6 values: direct node pairs, proxy pairs, clusters with proxy points, work items,
 *                 source segments, largest target count of a work item
 * Returns RBS_EINVAL for a NULL pointer or an argument out of range.  The paper has no counterpart:
 * its far field is a fast multipole method (Section 3.1).
 */
int rbs_treecode_plan(int n, const int* nodes, const double* centres, const double* radius, const double* node_box,
                      const int* suspension_id, double theta, int degree, double near_delta, int sm_count,
                      long long* out);

/*
 * Host-only near-pair list (Section 3: close particles take their sources from an upsampled grid):
 * the ordered pairs (i, j), i != j of one suspension with |c_i - c_j| < R_i + R_j + near_delta, as a
 * context builds them, without device work.
 *  n              number of particles, >= 1
 *  centres        n x 3
 *  radius         n, bounding radius R
 *  rmin           n, inscribed radius: two particles whose inscribed spheres intersect overlap
 *  suspension_id  n, or NULL for one suspension
 *  pairs          2 x max_pairs ints, or NULL: the pairs (i, j), by i, then j, ascending
 * Returns the number of near pairs (only the first max_pairs are written), RBS_EOVERLAP for
 * overlapping particles or RBS_EINVAL for a bad argument.
 */
int rbs_near_plan(int n, const double* centres, const double* radius, const double* rmin, const int* suspension_id,
                  double near_delta, int max_pairs, int* pairs);

/*
 * Host-only reflection-symmetry tables of the (p, n_phi) grid (Eq. 33), by which ellipsoid self blocks
 * are stored as the rows of representative nodes and the preconditioner is inverted per irreducible
 * representation.  The reflections h = 0..7 (bit 0: x -> -x, i.e. phi -> pi - phi; bit 1: y -> -y,
 * phi -> -phi; bit 2: z -> -z, theta -> pi - theta) map grid nodes to grid nodes (n_phi even).
 *  p, nphi   the grid: 2 <= p <= 32, n_phi even and >= 2p
 *  rep_of    (p + 1) n_phi ints, or NULL: the representative (j, k), j <= p/2, k <= n_phi/4, of each
 *            node's orbit, as j (n_phi/4 + 1) + k
 *  g_of      (p + 1) n_phi ints, or NULL: a reflection taking the representative to the node
 *  irrep_dim 8 ints, or NULL: the dimension of each irreducible representation's block of the
 *            3 (p + 1) n_phi surface-field components (they sum to 3 (p + 1) n_phi)
 * Returns the number of representatives, or RBS_EINVAL.  The paper has no counterpart (a storage
 * scheme of this library, exact up to rounding).
 */
int rbs_grid_symmetry(int p, int nphi, int* rep_of, int* g_of, int* irrep_dim);

#ifdef __cplusplus
}
#endif
#endif /* RBS_H */
