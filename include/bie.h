/*
 * bie.h -- C ABI of the GB300 library for the Stokes single- and double-layer operators on
 * drop surfaces represented by spherical-harmonic (SH) expansions, after Sorgentone & Tornberg,
 * "A highly accurate boundary integral equation method for surfactant-laden drops in 3D"
 * (arXiv 1707.02156).
 *
 * Conventions shared by every call
 * --------------------------------
 * Degrees.  Drop d has SH degree p[d] (1 <= p <= BIE_MAX_P).  Its Gauss grid (Sec. 2.1) has
 *   p+1 latitudes theta_j = arccos t_j (t_j the Gauss-Legendre nodes, ascending, so theta descends)
 *   and 2p+2 longitudes phi_k = pi k/(p+1); N_g(p) = (p+1)(2p+2) grid points.
 * Coefficients (Sec. 1.1, 1.2).  Real-packed per scalar: (p+1)^2 doubles, index n(n+1)+m holds
 *   Re f_n^m for m >= 0 and Im f_n^{|m|} for m < 0 (real functions: f_n^{-m} = (-1)^m conj f_n^m).
 *   Orthonormal Y_n^m with the Condon-Shortley phase.
 * Multi-drop arrays are drop-major: [drop][comp][(p[d]+1)^2] for coefficients and
 *   [drop][comp][j][k] for grids, each drop's block following the previous one.
 * Pointers.  Arrays named "coef", "grid" or "_dev" are DEVICE pointers (cudaMalloc'd memory of the
 *   context's device); the small per-drop arrays p, p_out, pq, lambda, euler are HOST pointers.
 *   The caller owns every buffer it passes; the library never frees them and keeps no pointer to
 *   them after the call returns (bie_geometry_setup copies what it needs).
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *   are asynchronous with respect to the host unless stated; results are ready when the stream is.
 * Errors.  Every call returns a status code; nothing throws or aborts.  On an error the output
 *   buffers are unspecified.  bie_strerror() names a code; bie_last_error() describes the last
 *   failure of the calling thread in words.
 * Normalisation (Eq. main_eq, mu = 1, xh = x0 - x, r = |xh|):
 *   G(xh) f = f/r + (xh.f) xh/r^3,   u.T(xh).n = -6 (u.xh)(xh.n) xh/r^5,
 *   single layer  S[f](x0) = -(1/4pi) sum_j int_{gamma_j} f.G dS,
 *   double layer  D[u](x0) = (1/4pi) sum_j (lambda_j - 1) PV int_{gamma_j} u.T.n dS,
 *   so Eq. main_eq reads (lambda_i + 1) u - D[u] = 2 u_inf + S[f].  With BIE_RAW the calls return
 *   the unscaled operators (1/8pi) int f.G and (1/4pi) PV int u.T.n instead.
 */
#ifndef BIE_H
#define BIE_H

#ifdef __cplusplus
extern "C" {
#endif

#define BIE_MAX_P 64

enum bie_status {
  BIE_OK = 0,
  BIE_EINVAL = 1,    /* bad argument (degree out of range, null pointer, bad flag) */
  BIE_ENOMEM = 2,    /* device or host allocation failed */
  BIE_ECUDA = 3,     /* a CUDA runtime call failed (see bie_last_error) */
  BIE_ENOCONV = 4,   /* iterative solve did not reach its tolerance: best iterate returned */
  BIE_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  BIE_EOVERLAP = 6,  /* drops intersect: a grid point lies inside, or on, another drop */
  BIE_ENOTSUP = 7    /* feature not supported for these arguments */
};

/* precision flags (the low byte), OR-able with BIE_RAW */
#define BIE_FP64 0   /* every step in double precision */
#define BIE_MIXED 1  /* rotation, synthesis and pair sums in FP32; geometry, analysis in FP64 */
#define BIE_DF 2     /* the rotation and contraction of the singular self term (projected form) and the
                        inter-drop pair sums (Omega_0, Omega_1) in double-float arithmetic (pairs of
                        FP32 numbers, about 44 significant bits) on the FP32 pipes; geometry, the
                        near-singular step and the analysis in FP64: FP64-grade results (relative
                        error ~1e-13) at a fraction of the FP64 pipe's cost */
#define BIE_RAW 0x100
#define BIE_GRID_OUT 0x200  /* applies: write the values at the grid targets, [drop][3][j][k], instead
                               of their Galerkin projection (for sampled checks against a reference) */

typedef struct bie_ctx bie_ctx;
typedef struct bie_geom bie_geom;

typedef struct bie_config {
  int device;        /* CUDA device ordinal */
  int upsample;      /* U: the intermediate region uses the grid of degree U(p+1)-1 (Sec. 2.3), >= 1 */
  double a_tilde;    /* A: Omega_0 / Omega_1 boundary at distance A*h (Sec. 2.3; the paper uses 5) */
  int n_interp;      /* L: check points of the near-singular interpolation (Sec. 2.3; 8) */
  int self_direct;   /* 0: singular self term in projected form (the kernel weights of each target's
                        rotated grid, phi-transformed and projected onto the associated Legendre
                        functions once per geometry; an apply rotates the density and contracts it
                        with them; the default); 1: direct form (synthesis on the rotated grid and
                        kernel evaluation at every quadrature point on every apply) */
  int use_graphs;    /* 1: an apply (kind, flags) is captured into a CUDA graph at its second call and
                        replayed afterwards (input and output pass through fixed internal buffers);
                        0: every apply launches its kernels one by one */
  int tensor_rotation; /* 1: in BIE_MIXED applies the Wigner rotation of the projected self form
                          (App. B) of degrees up to 58 runs on the tensor cores (TF32 with a 3-pass
                          split, FP32 accumulation, about FP32 accuracy); 0 (default): on the CUDA cores
                          in FP32, which measured 1.4-1.7 times faster on GB300.  FP64 and BIE_DF
                          applies always rotate on the CUDA cores */
} bie_config;

/* Fill a config with the paper's defaults: device 0, U = 4, A = 5, L = 8, projected self form, graphs
 * on, CUDA-core rotation. */
void bie_config_default(bie_config* cfg);

/* Create a context on cfg->device.  Plan tables are built lazily per degree and cached. */
int bie_create(bie_ctx** ctx, const bie_config* cfg);
void bie_destroy(bie_ctx* ctx);
const char* bie_strerror(int status);
const char* bie_last_error(void);

/* SH analysis, Eq. back_transf_discr (Sec. 2.1): grid values on the degree-p[d] grid ->
 * degree-p[d] coefficients, for ndrop drops with ncomp scalar components each.
 * grid: [drop][comp][p+1][2p+2] (device), coef: [drop][comp][(p+1)^2] (device). */
int bie_sh_analyze(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* grid, double* coef,
                   void* stream);

/* SH synthesis, Eq. spharm_ex, on the Gauss grid of degree p_out[d] (zero padding for
 * p_out > p: the upsampling of Sec. 1.3; p_out < p is rejected).
 * coef: [drop][comp][(p+1)^2], grid: [drop][comp][p_out+1][2p_out+2] (device). */
int bie_sh_synthesize(bie_ctx* ctx, int ndrop, const int* p, const int* p_out, int ncomp, const double* coef,
                      double* grid, void* stream);

/* Rotation of SH coefficients, App. B: coef_out holds the expansion of g(s) = f(R s) with
 * R = R_z(alpha) R_y(beta) R_z(gamma) (z-y-z Euler angles, active rotations), so the pole of g is
 * the point (theta, phi) = (beta, alpha) of f.  euler: host [ndrop][3] = (alpha, beta, gamma).
 * coef, coef_out: [drop][comp][(p+1)^2] (device, must not overlap). */
int bie_rotate(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* coef, const double* euler,
               double* coef_out, void* stream);

/* Allocation-free variant of bie_rotate.  The paper has no counterpart: this is an interface of
 * the library for callers that cannot allocate device memory -- frameworks that own all of the
 * device's memory through their own pool or arena and forbid any other allocation, and loops that
 * must not touch the allocator or wait on its implicit synchronisation.  bie_rotate allocates and
 * frees small per-call tables; bie_rotate_noalloc stages the same tables in one fixed array of
 * BIE_NOALLOC_SCRATCH_DOUBLES doubles (1.4 MiB) compiled into the library, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine, on the device or on the host: the tables are built on the host in a fixed
 * buffer of the same size and copied into the array with cudaMemcpyAsync on `stream`.
 *   Arguments, layout and result: as bie_rotate; degrees 1 <= p <= BIE_NOALLOC_MAX_P.  A request
 *   whose tables (the Wigner blocks of degree p, 2(p+1) phases and ncomp offsets) do not fit the
 *   array is rejected with BIE_EINVAL and a message in bie_last_error(), before any GPU work.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current.
 *   Device: the call makes the context's device current while it works and restores the caller's
 *   current device before it returns, on every path.
 *   Sharing: every call uses the same array and leaves the last drop's tables in it.  Each call
 *   writes every entry it reads before reading it, so nothing needs to start at zero.  Calls whose
 *   GPU work overlaps -- on different streams, or from several host threads -- race on the array:
 *   issue them on one stream or serialise them. */
#define BIE_NOALLOC_MAX_P 64
#define BIE_NOALLOC_SCRATCH_DOUBLES 184320
int bie_rotate_noalloc(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* coef, const double* euler,
                       double* coef_out, void* stream);

/* Geometry of ndrop drops (Table 2; Sec. 2.2 rotated-grid cache; Sec. 2.3 regions), built once per
 * shape and reused by every apply and solve on it.
 *   p[d]   SH degree of drop d (host), pq[d] degree of its self (singular) quadrature grid,
 *          p <= pq <= 2p+1 (pq = 2p+1 is the "upsampled 2x for quadrature" rule);
 *   xcoef  [drop][3][(p+1)^2] device coefficients of x(theta, phi);
 *   lambda host [ndrop] viscosity ratios.
 * Synchronous: returns when the geometry is ready.  With the projected self form (the default) this
 * includes the projected kernel factors of both layers, after which the rotated-grid cache is
 * released; with bie_config.self_direct the cache is kept for the per-apply evaluation.
 * BIE_EOVERLAP if a grid point of one drop lies inside another.  The geometry owns its device
 * memory until bie_geometry_destroy. */
int bie_geometry_setup(bie_ctx* ctx, int ndrop, const int* p, const int* pq, const double* xcoef,
                       const double* lambda, bie_geom** geom, void* stream);
void bie_geometry_destroy(bie_geom* geom);

typedef struct bie_geom_info {
  int ndrop;
  long long ncoef;        /* 3 * sum_d (p_d+1)^2: length of a vector-density coefficient array */
  long long ntarget;      /* sum_d N_g(p_d) */
  long long self_pairs;   /* sum_d N_g(p_d) * N_g(pq_d): pairs of the singular self rule */
  long long far_pairs;    /* (target, source) pairs of the regular rule on standard grids (Omega_0) */
  long long up_pairs;     /* pairs of the upsampled rule (Omega_1) */
  long long near_targets; /* (target, drop) pairs in Omega_2 */
  long long near_pairs;   /* pairs evaluated at Omega_2 check points */
  double cache_bytes;     /* device bytes held by the geometry */
  int interdrop_tpt;      /* targets per thread chosen by the pair-kernel autotuner (FP32) */
  long long pair_slots;   /* target slots x sources that the inter-drop pair kernels run: every work item
                             covers the 128 target slots of its tile, so (far_pairs + up_pairs) / pair_slots
                             is the share of that work that is useful */
} bie_geom_info;
int bie_geometry_info(const bie_geom* geom, bie_geom_info* info);

/* Interfacial force f = -2 sigma K n - grad_gamma sigma (Sec. 1, Table 2), computed on the grid of
 * degree 2p+1 and truncated to degree p (Sec. 1.3).  gammacoef: [drop][1][(p+1)^2] device surfactant
 * coefficients; sigma = 1 + E ln(1 - x_s Gamma) (Eq. langmuir) when x_s > 0, else 1 - E Gamma.
 * K is the mean curvature (E N - 2 F M + G L)/(2 W^2) of Table 2 (whose curvature labels are swapped)
 * with the outward normal, so K = -1/R on a sphere and f = 2 sigma/R n there.  Requires 0 <= x_s < 1.
 * fcoef: [drop][3][(p+1)^2] device output.  Synchronous. */
int bie_interfacial_force(bie_ctx* ctx, const bie_geom* geom, const double* gammacoef, double elasticity,
                          double x_s, double* fcoef, void* stream);

/* Single-layer apply (Eq. main_eq, Sec. 2.2-2.3, Galerkin projection of Sec. 1.2):
 * out = coefficients of S[f] at every drop's grid targets.  fcoef: [drop][3][(p+1)^2] (device);
 * precision: BIE_FP64, BIE_MIXED or BIE_DF, optionally | BIE_RAW. */
int bie_apply_single(bie_ctx* ctx, const bie_geom* geom, const double* fcoef, double* out_coef, int precision,
                     void* stream);

/* Double-layer apply, same layout: out = coefficients of D[u] (the GMRES matvec's operator part). */
int bie_apply_double(bie_ctx* ctx, const bie_geom* geom, const double* ucoef, double* out_coef, int precision,
                     void* stream);

/* Layer potentials at points off the surfaces (Sec. 1: the velocity can be evaluated anywhere in the
 * fluid from the interface densities).  out[c][t] = S[f](x_t) (bie_eval_single) or D[u](x_t)
 * (bie_eval_double), with the normalisations of bie_apply_single / bie_apply_double (or BIE_RAW's):
 * S[f] = -(1/4pi) sum_j int f.G ds, D[u] = (1/4pi) sum_j (lambda_j - 1) int u.T.n ds, ordinary
 * integrals here.  Each (point, drop j) pair takes the rule of its region, as the drops' own targets
 * do (Sec. 2.1-2.3): the regular rule on drop j's standard grid in Omega_0, on its upsampled grid in
 * Omega_1, and in Omega_2 the interpolation along the line through the closest point x* of drop j,
 * anchored at the exterior limit of drop j's on-surface value at x* (for the double layer the
 * principal value minus 4 pi (lambda_j - 1)/(4 pi) u(x*)); the check-point values are FP64 in every
 * precision.  precision: BIE_FP64, BIE_MIXED (FP32 pair sums and self term) or BIE_DF, optionally |
 * BIE_RAW.
 * points: [3][npoint] device FP64 (x of every point, then y, then z); fcoef / ucoef: the densities,
 * [drop][3][(p+1)^2] device; out: [3][npoint] device, overwritten.  0 <= npoint < 2^31.  Points must
 * lie in the fluid: a point inside (or on the inner side of the tangent plane at the nearest
 * upsampled grid point of) a drop gives BIE_EOVERLAP, the error text naming its 128-point tile and the
 * drop.  A single-drop geometry builds its upsampled grid and source data on the first call.  The
 * call uses the geometry's work buffers (not concurrently with other calls on the same geometry),
 * allocates its temporaries, and is synchronous. */
int bie_eval_single(bie_ctx* ctx, const bie_geom* geom, long long npoint, const double* points, const double* fcoef,
                    double* out, int precision, void* stream);
int bie_eval_double(bie_ctx* ctx, const bie_geom* geom, long long npoint, const double* points, const double* ucoef,
                    double* out, int precision, void* stream);

/* Velocity at fluid points: out = u_inf + (S[f] + D[u]) / 2, the representation whose limit onto an
 * interface is Eq. main_eq (the factor 1 of a fluid point against (lambda_i + 1)/2 there).  u: the
 * interface velocity (the solution of bie_solve), f: the interfacial force; uinf: [3][npoint] device
 * values of the far field at the points, or NULL for none.  Arguments otherwise as bie_eval_single;
 * BIE_RAW is refused (BIE_EINVAL). */
int bie_eval_velocity(bie_ctx* ctx, const bie_geom* geom, long long npoint, const double* points, const double* fcoef,
                      const double* ucoef, const double* uinf, double* out, int precision, void* stream);

/* Right-hand side of Eq. main_eq in coefficient space: rhs = 2 u_inf + S[f] with the single layer at
 * precision BIE_FP64 or BIE_DF (both FP64-grade).  uinf: [drop][3][(p+1)^2] device coefficients of the far field at the drop surfaces (a
 * linear flow is exactly band-limited: u_inf = (z, 0, 0) has the z coefficients of x in its first
 * component); fcoef: interfacial force coefficients; rhs: device output (must not alias the inputs). */
int bie_rhs(bie_ctx* ctx, const bie_geom* geom, const double* uinf, const double* fcoef, double* rhs,
            int precision, void* stream);

typedef struct bie_solve_opts {
  int precision;      /* BIE_FP64: FP64 GMRES; BIE_MIXED: mixed GMRES inside FP64 iterative refinement */
  double tol;         /* relative residual target ||b - A u|| / ||b|| (FP64-accurate residual) */
  int restart;        /* GMRES restart length (<= 64) */
  int max_iter;       /* total GMRES iterations allowed */
  double inner_tol;   /* mixed only: relative tolerance of each inner solve */
  int max_refine;     /* mixed only: outer refinement steps allowed */
  int residual_precision; /* mixed only: precision of the refinement residual b - A u, BIE_FP64 or
                             BIE_DF (the default: FP64-grade, inter-drop pairs on the FP32 pipes) */
} bie_solve_opts;

typedef struct bie_solve_info {
  int iterations;        /* GMRES iterations (all inner solves) */
  int refinements;       /* outer refinement steps (mixed) */
  int applies_fp64;      /* FP64-grade double-layer applies (BIE_FP64 or BIE_DF) */
  int applies_mixed;     /* mixed double-layer applies */
  double residual;       /* final FP64 relative residual */
  int converged;
} bie_solve_info;

void bie_solve_opts_default(bie_solve_opts* opts);

/* Solve Eq. main_eq in coefficient space: (lambda_i + 1) u_i - D[u]_i = b_i, Sec. 6 (GMRES).
 * rhs: [drop][3][(p+1)^2] device right-hand side b (form it as 2 u_inf + S[f] with
 * bie_apply_single); u: device initial guess in, solution out.  Synchronous (the Krylov loop reads
 * back one scalar block per iteration).  BIE_ENOCONV if tol was not reached (best iterate kept). */
int bie_solve(bie_ctx* ctx, const bie_geom* geom, const double* rhs, double* u, const bie_solve_opts* opts,
              bie_solve_info* info, void* stream);

/* Per-phase timing.  bie_profile(ctx, 1) starts recording CUDA events around each phase of the
 * library's work (on the stream each phase is launched on); bie_profile(ctx, 0) stops and discards.
 * bie_profile_read synchronises on the recorded events, returns per-phase totals (milliseconds and
 * number of timed calls, at most cap entries, *count = number of phases) and clears the record.
 * While profiling is on, applies launch their kernels one by one (no graph replay), so every phase
 * is timed.  Phases: "self_proj_f64/f32" (rotation + contraction with the projected kernel factors) and
 * "self_direct_f64/f32" (rotation + synthesis + the singular pair sum of Thm 1), "kernel_proj"
 * (projected kernel factors, once per geometry and kind), "analyze" (Galerkin
 * projection), "interdrop" (regular and upsampled pair sums), "near" (near-singular step),
 * "source_synth" (source densities on the standard/upsampled grids), "gmres_vec",
 * "surfactant_rates" and "surfactant_implicit" (bie_surfactant_rates, bie_surfactant_implicit). */
typedef struct bie_phase_stat {
  char name[24];
  double ms;
  long long calls;
} bie_phase_stat;
int bie_profile(bie_ctx* ctx, int enable);
int bie_profile_read(bie_ctx* ctx, bie_phase_stat* stats, int cap, int* count);

/* One midpoint time step of the drop shapes (Sec. 3, the drop update of Alg. 1, with the surfactant
 * held fixed over the step):
 *     x^{1/2} = x + (dt/2) u(x),    x^{new} = x + dt u(x^{1/2}),
 * where u(x) solves Eq. main_eq (bie_solve) for the shapes x, in the linear shear u_inf =
 * (shear z, 0, 0), with the interfacial force of the surfactant coefficients (bie_interfacial_force).
 *   p, pq, lambda   host [ndrop], as bie_geometry_setup;
 *   xcoef           [drop][3][(p+1)^2] device shapes: in at t, out at t + dt;
 *   gammacoef       [drop][1][(p+1)^2] device surfactant coefficients (not changed);
 *   elasticity, x_s as bie_interfacial_force;
 *   opts            options of both solves (zero initial guesses; the right-hand sides are formed at
 *                   BIE_FP64 for an FP64 solve, else at opts->residual_precision);
 *   info            NULL or an array of two: the solves at x and at x^{1/2}.
 * Builds and destroys the two geometries it needs.  Synchronous.  The status of the first failing
 * call is returned (xcoef unchanged unless both solves succeeded). */
int bie_step_midpoint(bie_ctx* ctx, int ndrop, const int* p, const int* pq, double* xcoef, const double* gammacoef,
                      double elasticity, double x_s, const double* lambda, double shear, double dt,
                      const bie_solve_opts* opts, bie_solve_info* info, void* stream);

/* ---- Insoluble surfactant (Eq. surfactant0, Sec. 1.2, Sec. 3, Alg. 1) ----
 * The surface points move with the full velocity (dx/dt = u), so Gamma is followed at fixed
 * parameters, with the rates
 *     f_E = -div(Gamma u_tan) + u_tan . grad Gamma + 2 K Gamma (u.n)   (= -Gamma div u),
 *     f_I = (1/Pe) lap Gamma,
 * K the mean curvature with the outward normal (-1/R on a sphere).  The surface gradient,
 * divergence and Laplacian are the coordinate forms in (theta, phi).  Every term is formed on the
 * grid of degree 2p+1 and projected on the degree-p SH basis (Galerkin, Eq. galerkin_surfactant).
 * Layouts: shapes and velocities [drop][3][(p+1)^2], surfactant [drop][(p+1)^2], device pointers,
 * per-drop degrees p on the host.  All in FP64. */

/* fe = projection of f_E at (x, u, Gamma); fi (NULL to skip) = projection of inv_pe * lap Gamma.
 * inv_pe = 1/Pe >= 0 (0: no surface diffusion). */
int bie_surfactant_rates(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* ucoef,
                         const double* gammacoef, double inv_pe, double* fe, double* fi, void* stream);

/* The implicit stage of Sec. 3 (Preconditioning): y with y - a P_p[lap_x y] = b per drop, by GMRES
 * (restart 60, at most 600 iterations, from y = 0) left-preconditioned with the diagonal the operator
 * has on the sphere of the drop's mean radius R, 1 + a n(n+1)/R^2; stops at relative residual tol.
 * a >= 0 (a = 0 copies b).  *iterations (may be NULL) = GMRES iterations.  Synchronous.
 * BIE_ENOCONV if tol was not reached. */
int bie_surfactant_implicit(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* b, double a,
                            double* y, double tol, int* iterations, void* stream);

/* Surfactant mass int_gamma Gamma dS per drop by the regular rule (Sec. 2.1) on the grid of degree
 * 2p+1: host mass[ndrop].  Synchronous. */
int bie_surfactant_mass(bie_ctx* ctx, int ndrop, const int* p, const double* xcoef, const double* gammacoef,
                        double* mass, void* stream);

typedef struct bie_coupled_info {
  double err_drop;          /* max over drops of ||dt (u^{t+dt/2} - u^t)||_inf / ||x^{t+dt}||_inf on the
                               degree-p grid: the embedded Euler estimate of the midpoint rule */
  double err_conservation;  /* max over drops of |M(t+dt) - M(t)| / |M(t)|, M the surfactant mass
                               (Eq. err_conservation) */
  double err_imex1;         /* max over drops of ||Gamma^{t+dt} - Gamma_IMEX1||_inf / ||Gamma^{t+dt}||_inf
                               (Eq. err_IMEX1), or -1 when not requested */
  int velocity_solves;      /* 1, or 2 when u^t was computed here */
  int implicit_iterations;  /* GMRES iterations of the implicit stage */
  bie_solve_info solve[2];  /* the velocity solves at t (when run) and at t + dt/2 */
} bie_coupled_info;

/* One step of Alg. 1 (Sec. 3): the midpoint rule for the shapes and the second-order IMEX scheme
 * (Eqs. systemforgammatpdt2, gammatpiudt) for the surfactant, coupled through the interfacial force:
 *   u^t = u(x^t, Gamma^t);  x_h = x^t + (dt/2) u^t;
 *   Gamma_h from (I - (dt/2)(1/Pe) lap_{x_h}) Gamma_h = Gamma^t + (dt/2) f_E(x^t, u^t, Gamma^t);
 *   u_h = u(x_h, Gamma_h);  x^{t+dt} = x^t + dt u_h;
 *   Gamma^{t+dt} = Gamma^t + dt (f_E(x_h, u_h, Gamma_h) + f_I(x_h, Gamma_h)),
 * u(x, Gamma) the solution of Eq. main_eq in the shear u_inf = (shear z, 0, 0) with the interfacial
 * force of Gamma (as bie_step_midpoint).
 *   u0         device [drop][3][(p+1)^2]: u^t in when u0_valid (a rejected attempt's), else written;
 *   x_out, gamma_out  device outputs at t + dt; they must not alias xcoef / gammacoef;
 *   inv_pe     1/Pe >= 0;  imex1_estimate  nonzero to compute info->err_imex1 (one more implicit solve);
 *   opts, p, pq, lambda, elasticity, x_s  as bie_step_midpoint.
 * Synchronous; builds and destroys the geometries it needs. */
int bie_step_coupled(bie_ctx* ctx, int ndrop, const int* p, const int* pq, const double* xcoef,
                     const double* gammacoef, double* u0, int u0_valid, double elasticity, double x_s,
                     const double* lambda, double shear, double inv_pe, double dt, int imex1_estimate,
                     const bie_solve_opts* opts, double* x_out, double* gamma_out, bie_coupled_info* info,
                     void* stream);

/* Step-size rule of Alg. 1: min(dt_max, dt (0.9 tol/err)^(1/2)); dt_max when err <= 0. */
double bie_next_dt(double dt, double err, double tol, double dt_max);

#define BIE_ERR_CONSERVATION 0  /* surfactant error of Alg. 1: the conservation error */
#define BIE_ERR_IMEX1 1         /* ... or the IMEX-1 estimate */

typedef struct bie_run_info {
  double t;                 /* time reached */
  double dt_next;           /* the step size the rule proposes next */
  double err_max_accepted;  /* largest err = max(err_drop, err_surfactant) of a kept step */
  int steps_accepted, steps_rejected, velocity_solves;
  int reparam_iterations;   /* angle steps of Alg. 2 over the run (summed over the kept steps) */
} bie_run_info;

/* ---- Angle reparametrisation (Sec. 4, Alg. 2) ----
 * The parameter points of each drop's working grid of degree P = u_rep (p+1) - 1 (zero-padded
 * coefficients) move in pseudo-time so that the spectral energy E = sum_n a_n sum_{m=-n..n} |x_n^m|^2
 * of the surface's parametrisation (Eq. energy_rep, |x_n^m| the Euclidean norm of the three complex
 * coefficients) decreases while the surface stays the same: the pseudo-velocity is the tangential
 * part g = (I - n n) grad E of the L2 gradient grad E = 2 sum a_n x_n^m Y_n^m (Eq. pseudo_rep, n the
 * normal of the original surface at the point), the angles follow the chain rule of Eq. system_rep
 * by forward Euler steps of size dtau, and after each step the original expansion, evaluated at the
 * new angles, is analysed on the grid (Eq. rep_trasf1).  a_n comes from the adaptive cutoff of
 * Eq. ncutoff_adaptive: n_cutoff = the smallest l with 1 < l <= P and
 * sum_{n >= l} sum_m |x_n^m| / sum_{n >= 1} sum_m |x_n^m| < p_cutoff (P if none), recomputed every
 * iteration; a_n = 1 (perfect filter) or n/P (smooth) for n >= n_cutoff, 0 below.  A drop stops when
 * max |g| over its points is below eps (the stopping test of Alg. 2) or after max_iter steps.  The
 * surfactant is evaluated at the final angles (Eq. rep_trasf2); shape and surfactant are analysed
 * back to degree p.  Readings: the working grid, the gradient and the pole crossing (an angle step
 * across a pole maps back to theta in [0, pi] with phi + pi) are those of the FP64 oracle. */
typedef struct bie_reparam_opts {
  int u_rep;        /* working-grid factor, >= 1 (P = u_rep (p+1) - 1 <= 4 BIE_MAX_P) */
  double p_cutoff;  /* fraction of Eq. ncutoff_adaptive, 0 < p_cutoff < 1 */
  int smooth;       /* 0: perfect low-pass filter, 1: smooth filter a_n = n/P */
  double dtau;      /* pseudo-time step (forward Euler is stable for dtau < 1/max a_n) */
  double eps;       /* stopping threshold on max |g| */
  int max_iter;     /* angle steps allowed per drop */
} bie_reparam_opts;

typedef struct bie_reparam_info {
  int iterations;           /* the largest number of angle steps a drop took */
  int converged;            /* drops that met the stopping test */
  double g_max;             /* the largest last max |g| over the drops */
  double energy_first_max;  /* the largest energy E at the first iteration */
  double energy_last_max;   /* the largest energy at the last evaluated iteration */
} bie_reparam_info;

/* Fill the options with u_rep 2, p_cutoff 0.05, perfect filter, dtau 0.5, eps 1e-10, max_iter 200. */
void bie_reparam_opts_default(bie_reparam_opts* opts);

/* Reparametrise ndrop drops in place: xcoef [drop][3][(p+1)^2] and, when non-NULL, gammacoef
 * [drop][(p+1)^2] (device), per-drop degrees p on the host; drops of one degree share every launch.
 * All in FP64.  Synchronous.  BIE_EINVAL for bad options or degrees (at most 65535 drops). */
int bie_reparametrize(bie_ctx* ctx, int ndrop, const int* p, double* xcoef, double* gammacoef,
                      const bie_reparam_opts* opts, bie_reparam_info* info, void* stream);

/* Alg. 1 from t = 0 to T with adaptive dt: each attempt is bie_step_coupled; it is kept when
 * err = max(err_drop, err_surfactant) < tol (estimator BIE_ERR_CONSERVATION or BIE_ERR_IMEX1);
 * after every attempt dt <- bie_next_dt(dt, err, tol, dt_max), the last step cut to end at T;
 * a rejected attempt reuses u^t.  xcoef, gammacoef: device, in at 0, out at the time reached.
 * reparam: NULL, or the options of an angle reparametrisation (bie_reparametrize, Sec. 4) applied to
 * the shapes and the surfactant after every kept step.  BIE_ENOCONV when max_steps attempts end
 * before T.  Synchronous. */
int bie_run_coupled(bie_ctx* ctx, int ndrop, const int* p, const int* pq, double* xcoef, double* gammacoef,
                    double elasticity, double x_s, const double* lambda, double shear, double inv_pe, double T,
                    double dt0, double tol, double dt_max, int estimator, int max_steps, const bie_solve_opts* opts,
                    const bie_reparam_opts* reparam, bie_run_info* info, void* stream);

/* Measured arithmetic rate of the context's GPU, the denominator of the pair kernels' ALU
 * rooflines (the paper has no counterpart; a measurement utility).  which: BIE_PEAK_FP32 (fma.rn.f32),
 * BIE_PEAK_FP32X2 (fma.rn.f32x2, two FP32 FMAs per instruction) or BIE_PEAK_FP64 (fma.rn.f64).
 * Runs a kernel of eight independent FMA chains per thread at full occupancy (eight 256-thread
 * blocks per SM), once to warm up and five times timed with CUDA events on the legacy default
 * stream; *tflops = 2 x FMAs / best time (FMA = 2 flops).  Synchronous; allocates one word of
 * device memory for the call; changes no setting of the GPU (the rate is whatever its clocks
 * give meanwhile).  BIE_EINVAL for a null pointer or an unknown `which`. */
#define BIE_PEAK_FP32 0
#define BIE_PEAK_FP32X2 1
#define BIE_PEAK_FP64 2
int bie_alu_peak(bie_ctx* ctx, int which, double* tflops);

/* Number of CUDA kernels the library has launched in this process (all contexts). */
long long bie_launch_count(void);

/* Host-side plan tables, exported so the host logic can be checked without a GPU.
 *   which 0: Gauss-Legendre nodes (n = P+1 doubles) then weights (n doubles), P = a
 *   which 1: Legendre table kind b (0 value, 1 d/dtheta, 2 d2/dtheta2) for degree a on the grid of
 *            degree c: layout [m][n][j], 0 <= m <= n <= a
 *   which 2: dense Wigner small-d matrix of degree a at angle x: [(2a+1)][(2a+1)], rows m', cols m
 *   which 3: singular weights of Thm 1 on the grid of degree a (a+1 doubles)
 * Writes at most `cap` doubles to out and returns the count needed (negative on bad arguments). */
long long bie_debug_table(int which, int a, int b, int c, double x, double* out, long long cap);

#ifdef __cplusplus
}
#endif
#endif /* BIE_H */
