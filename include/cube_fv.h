/*
 * cube_fv.h -- C-ABI of the GB300 (sm_103a) library for the Newton-Krylov and
 * Chebyshev-preconditioned Arnoldi stability analysis of air convection in a
 * laterally heated cube (Gelfgat, "Sequence of bifurcations of natural
 * convection of air in a laterally heated cube with perfectly insulated
 * horizontal and spanwise boundaries").
 *
 * Problem (Section 2, Eqs. 1-6), written with unit viscosity ("Form A"):
 *     dv/dt = -div(v v) + Lap v + Gr T e_z - grad p,   dT/dt = -div(v T) + Lap T / Pr,   div v = 0
 * in the cube [0,1]^3, no-slip walls, T = 1 at x = 0 and T = 0 at x = 1
 * (Eq. 4), dT/dy = 0 at y = 0, 1 (Eq. 5), dT/dz = 0 at z = 0, 1 (Eq. 6).
 * The paper's rescaled form (Section 2) has eigenvalues lambda_B with
 * lambda_A = Gr^(1/2) lambda_B.
 *
 * Discretisation: staggered (MAC) finite volumes on a tensor grid, conservative
 * central fluxes with linear interpolation, half-cell wall distances.
 *
 * ---------------------------------------------------------------- layout
 * A "state" or "vector" is ONE contiguous device buffer of 4 * nz*ny*nx
 * elements holding four blocks [u | v | w | T].  Each block is an (nz, ny, nx)
 * array, x fastest: element (k, j, i) is at (k*ny + j)*nx + i.
 *     u[k][j][i]: x-velocity on the x-face x_f[i] of cell row (j, k); slot i = 0
 *                 is the wall x = 0; the wall x = 1 is not stored;
 *     v[k][j][i]: y-velocity on the y-face y_f[j]; slot j = 0 is the wall y = 0;
 *     w[k][j][i]: z-velocity on the z-face z_f[k]; slot k = 0 is the wall z = 0;
 *     T[k][j][i]: temperature at the cell centre.
 * Wall slots are written as 0 by every entry point and ignored on input; a
 * caller that runs its own inner products must keep them 0.
 * Element type: double for FV_FP64, float for FV_FP32 (per call).
 *
 * ---------------------------------------------------------------- conventions
 * All vector arguments are DEVICE pointers owned by the caller, unless a
 * comment says "host".  The library never frees or reallocates caller memory;
 * its workspace belongs to the fv_grid handle.  Every call is ordered on the
 * handle's CUDA stream; entry points that return host scalars synchronise that
 * stream.  Every entry point returns a status (FV_OK = 0 or a negative
 * FV_E* code); nothing is thrown across the ABI.  fv_last_error() gives a
 * message for the last failure on the calling thread.
 */
#ifndef CUBE_FV_H
#define CUBE_FV_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FV_OK = 0,
    FV_EINVAL = -1,    /* bad argument (size, pointer, precision, option) */
    FV_ENOMEM = -2,    /* device or host allocation failed */
    FV_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    FV_ENOCONV = -4,   /* iteration limit reached; outputs hold the last iterate */
    FV_ENAN = -5,      /* NaN or Inf met in a reduction */
    FV_ETIMEOUT = -6   /* a bounded device-side wait gave up */
};

enum { FV_FP64 = 0, FV_FP32 = 1 };

typedef struct fv_grid_s* fv_grid;

/* Grid description.  Faces per axis: if xf/yf/zf are NULL the library builds
 * them: stretch == 0 gives the uniform grid i/n, otherwise the tanh law
 * x_f[i] = (1 + tanh(s (2i/n - 1)) / tanh(s)) / 2 mirrored about 1/2
 * (Section 4.1 only says "stretched near the borders"; the law is this
 * library's reading).  Given arrays are host, n+1 strictly increasing values
 * with x_f[0] = 0 and x_f[n] = 1.  2 <= n <= 1024 per axis. */
typedef struct {
    int nx, ny, nz;
    const double *xf, *yf, *zf;
    double stretch;
    double Pr;          /* Prandtl number (0.71 for air, Section 1) */
} fv_grid_desc;

/* Create a grid handle: metric arrays, the 1D generalised eigen-decompositions
 * used by the pressure solve (computed on the host in FP64), and workspace.
 * The FP32 pressure solve runs on the tensor cores when every axis has 32 to 256
 * cells, a multiple of 32, and faces mirror-symmetric about 1/2 (as the built-in
 * grids are); other grids take the CUDA-core passes, with the same results.
 * `stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: FV_EINVAL (sizes, faces), FV_ENOMEM, FV_ECUDA. */
int fv_grid_create(const fv_grid_desc* desc, void* stream, fv_grid* out);
int fv_grid_destroy(fv_grid g);
int fv_set_stream(fv_grid g, void* stream);
/* Number of elements of one state/vector buffer: 4*nx*ny*nz. */
long long fv_state_elems(fv_grid g);

/* Failure detection (no counterpart in the paper).  Every wait of the library's kernels on an mbarrier
 * (the TMA plane ring of the J.v stencils, the pipeline of the tensor-core pressure-solve passes) polls at
 * most `spins` times; a wait that runs out records a code in the handle's device error word, the kernel
 * stops issuing work, lets every bulk copy and tensor-core operation it has started complete, releases its
 * tensor memory and returns (its outputs are then undefined).  spins < 0 restores the default (2^22 polls,
 * seconds); 0 makes every such wait give up at once, which is how the give-up path is exercised.
 * Errors: FV_EINVAL (null handle). */
int fv_set_wait_limit(fv_grid g, long long spins);
/* Synchronise the handle's stream and report a device-side wait that gave up since the last check as
 * FV_ETIMEOUT (clearing it); the handle stays usable.  Calls that return host scalars make the same check.
 * Errors: FV_EINVAL, FV_ECUDA, FV_ETIMEOUT. */
int fv_sync(fv_grid g);

/* Residual F(q; Gr) of Eqs. 1-2 without the pressure gradient (Section 2),
 * FP64 always: F_u = -div(u u) + Lap u, F_w additionally + Gr T_face,
 * F_T = -div(u T) + Lap T / Pr with the Dirichlet data of Eq. 4.
 * q, F: device double[4*N].  F is not projected.  Errors: FV_EINVAL, FV_ECUDA. */
int fv_residual(fv_grid g, double Gr, const double* q, double* F);

/* Jacobian-vector product J(q) v, the exact derivative of F (F is quadratic):
 * J v = -div(q v) - div(v q) + Lap v + Gr T_v e_z, thermal Dirichlet data 0.
 * prec selects the element type of q, v and Jv.  The wall slot (slot 0 along
 * its own axis) of u, v and w must hold zero in q and in v, as every state
 * and vector this library writes does: the kernel reads it as the wall value.
 * Errors: FV_EINVAL, FV_ECUDA. */
int fv_jvp(fv_grid g, int prec, double Gr, const void* q, const void* v, void* Jv);

/* SIMPLE-like projection (Section 1 methods paragraph, Section 3): replaces the
 * velocity part of v by P v = v - G phi with DG phi = D v (cell-centred Neumann
 * problem, solved directly by fast diagonalisation), so that D P v = 0; T is
 * unchanged.  In place.  max_it >= 1 is the number of solves (each later one
 * corrects the divergence left by the previous); stops early when
 * ||D P v||_2 <= tol * ||D v||_2.  iters (host, may be NULL) gets the solves
 * done; div_rel (host, may be NULL) gets ||D P v||_2 / ||D v||_2 (computing it
 * costs one more pass).  Errors: FV_EINVAL, FV_ECUDA. */
int fv_project(fv_grid g, int prec, void* v, int max_it, double tol, int* iters, double* div_rel);

/* Fused hot path: out = P (J(q) v - sigma v) + sigma v.  With sigma = 0 this
 * is P J(q) v, one "J.v + projection".  For D v = 0 the result does not
 * depend on sigma; sigma < 0 moves the gradient complement, on which P J
 * vanishes, to the eigenvalue sigma (used by the Krylov drivers).
 * out must not alias q or v.  Errors: FV_EINVAL, FV_ECUDA. */
int fv_jvp_project(fv_grid g, int prec, double Gr, double sigma,
                   const void* q, const void* v, void* out);

/* Fused recurrence step (the Chebyshev filter's three-term recurrence, Section 1 ref. 21):
 *     out = alpha (P (J(q) v - sigma v) + sigma v) + beta v + gamma w
 * with the axpys folded into the projection's correction pass.  w may be NULL
 * (gamma ignored) and out may alias w, not q or v.  out_norm2 (host, may be
 * NULL) receives ||out||^2, summed in the same pass (deterministic, FP64-level
 * accumulation) and read back with a stream synchronisation.
 * Errors: FV_EINVAL, FV_ECUDA, FV_ENAN. */
int fv_jvp_project_lincomb(fv_grid g, int prec, double Gr, double sigma, const void* q, const void* v,
                           const void* w, double alpha, double beta, double gamma, void* out, double* out_norm2);

/* The same fused recurrence step, fully stream-ordered: ||out||^2 is summed in
 * the same pass and written to norm2_dev (device double, may be NULL) with no
 * host synchronisation, so that a caller running many steps reads it back only
 * when it needs it (the filter inside arnoldi_leading checks it every 16 steps).
 * Errors: FV_EINVAL, FV_ECUDA. */
int fv_jvp_project_lincomb_dev(fv_grid g, int prec, double Gr, double sigma, const void* q, const void* v,
                               const void* w, double alpha, double beta, double gamma, void* out,
                               double* norm2_dev);

/* Krylov inner product <a, b> over all 4N elements, accumulated in FP64 in a
 * fixed order (bit-reproducible).  result: host.  Errors: FV_EINVAL, FV_ECUDA, FV_ENAN. */
int fv_dot(fv_grid g, int prec, const void* a, const void* b, double* result);
/* Inner product <a, b> of two device vectors of n elements WITHOUT any allocation, for callers
 * that cannot allocate device memory (allocation-free real-time loops, fixed memory budgets,
 * memory owned by someone else's pool).  No counterpart in the paper: it is the fv_dot reduction
 * with its block partial sums kept in a library-owned static device array of 4096 doubles
 * (32 KiB, held by every GPU that loads the library until exit) instead of handle workspace.
 * No fv_grid handle is needed.  result: DEVICE double, written on `stream` (a cudaStream_t).
 * n <= 4096 * 2^18 elements; larger n, n < 1, null pointers or an unknown prec give FV_EINVAL.
 * The first call on each device looks up the array's address (make it before any stream capture).
 * All calls share the array: calls that overlap on the GPU race and must be serialised.
 * Errors: FV_EINVAL, FV_ECUDA. */
int fv_dot_noalloc(int prec, long long n, const void* a, const void* b, double* result, void* stream);

/* y <- alpha x + beta y over 4N elements (coefficients applied in FP64). */
int fv_axpby(fv_grid g, int prec, double alpha, const void* x, double beta, void* y);
/* Flags of the block calls below. */
enum { FV_BATCH_GRAPH = 1, FV_BATCH_AUTOTUNE = 2 };

/* Batched fused hot path: W_i = P (J(q) V_i - sigma V_i) + sigma V_i for the
 * nvec vectors stored one after another in V and W (device, nvec * 4N
 * elements each, precision `prec`).  Each stage runs as ONE launch over the
 * whole block where its kernel has a block form (FP32: the two-cell J.v
 * stencil for nx % 64 == 0, the divergence and correction for nx % 4 == 0;
 * both precisions: the six pressure-solve passes), else one launch per vector.
 * Block buffers (nvec * 6N elements) are owned by the handle and grown on
 * demand.  flags:
 *   FV_BATCH_AUTOTUNE: before the first block of a new size, time each z-chunk
 *     of the block stencil (4 ... 64 planes per CTA) with CUDA events on the
 *     handle's stream and keep the fastest for later blocks (fv_get_tuning);
 *   FV_BATCH_GRAPH: the block's launch sequence is captured once into a CUDA
 *     graph (on a private stream; the first call with a new argument set runs
 *     eagerly and captures) and replayed on the handle's stream by later calls
 *     with the same q, V, W, nvec, Gr and sigma.
 * The paper has no batched form (Krylov vectors are applied one at a time in
 * Section 1's methods); blocks of vectors and of continuation points (Section
 * 4.2's Gr sweeps) are how the same products fill one GPU.  W must not overlap
 * V or q.  Errors: FV_EINVAL, FV_ECUDA, FV_ENOMEM. */
int fv_jvp_project_batch(fv_grid g, int prec, double Gr, double sigma, const void* q, int nvec, const void* V,
                         void* W, int flags);

/* The block stencil's z-chunk picked by the autotuner (0 = not tuned: the
 * built-in 32 planes) and the block size it was timed on. */
int fv_get_tuning(fv_grid g, int* pair_zchunk, int* tuned_nvec);

/* Several problems (e.g. continuation points at different Gr on grids of
 * different sizes), each a block as in fv_jvp_project_batch, captured into ONE
 * CUDA graph whose branches run concurrently.  Problem i: handle grids[i]
 * (distinct handles: their workspaces run at the same time), Gr[i], sigma[i],
 * base state q[i], nvec[i] vectors V[i] -> W[i] (device, layouts as above, all
 * of precision `prec`).  Creation runs every block once eagerly (W is written)
 * and captures; fv_batch_plan_launch replays the graph on `stream` (a
 * cudaStream_t; NULL = legacy default).  The plan stores the pointers: the
 * buffers and the handles must outlive it, and a later fv_jvp_project_batch
 * call that grows a handle's block buffers invalidates it (launch then
 * returns FV_EINVAL).  flags: FV_BATCH_AUTOTUNE as above.  Errors: FV_EINVAL,
 * FV_ECUDA, FV_ENOMEM. */
typedef struct fv_batch_plan_s* fv_batch_plan;
int fv_batch_plan_create(int nprob, const fv_grid* grids, int prec, const double* Gr, const double* sigma,
                         const void* const* q, const int* nvec, const void* const* V, void* const* W, int flags,
                         fv_batch_plan* out);
int fv_batch_plan_launch(fv_batch_plan plan, void* stream);
int fv_batch_plan_destroy(fv_batch_plan plan);

/* out = L^-1 in, where L is the diffusion part of J (Eqs. 1-2 with homogeneous wall data): per
 * velocity component the Laplacian with no-slip walls, for T the Laplacian / Pr with T = 0 at the
 * x-walls (Eq. 4) and zero flux at the others (Eqs. 5-6).  Separable on the tensor-product grid, so
 * it is inverted directly by fast diagonalisation (six dense passes per field; nothing iterates).
 * The building block of newton_steady's optional preconditioner; the paper names no preconditioner
 * (Section 1 methods paragraph).  in, out: device, 4N elements of the precision `prec`, API layout;
 * the wall slots of the face fields must hold zero in `in` and hold zero in `out`; in and out may
 * alias.  Errors: FV_EINVAL, FV_ECUDA, FV_ENOMEM (workspace). */
int fv_diffusion_solve(fv_grid g, int prec, const void* in, void* out);

/* Transfer of an FP64 state between two grids of the cube (grid sequencing: a coarse steady state as the
 * Newton start on a finer grid; Section 4.1 refines its grids from 100^3 to 256^3 and continues solutions
 * between neighbouring states).  Every field is interpolated trilinearly in physical coordinates, with the
 * wall values of Eqs. 4-6 at the ends of each axis (no-slip velocity 0; T = 1 and 0 on the x-walls; zero
 * flux on the others: constant beyond the first and last centre); the velocity is then projected on the
 * target grid so that it is discretely divergence free.  q_from: device double[4 N_from], q_to: device
 * double[4 N_to] (must not alias); runs on the target handle's stream after synchronising the source's.
 * Both handles must belong to the current device.  Errors: FV_EINVAL, FV_ECUDA, FV_ENOMEM. */
int fv_transfer(fv_grid from, const double* q_from, fv_grid to, double* q_to);

/* Diagnostics of Section 4.2.3 for an FP64 state q (device double[4N]): ekin (host, may be NULL) gets
 * the total kinetic energy of Eq. 12, 1/2 sum of u_f^2 over the faces of every velocity component, each
 * weighted by its staggered control volume (centre spacing along its own axis times the cell widths
 * across); nu (host, may be NULL) the Nusselt number of Eq. 13 as printed, the sum over the hot wall's
 * cells of (T - 1) / (dx_0 / 2) dy dz (conduction gives -1).  Synchronises the handle's stream.
 * Errors: FV_EINVAL, FV_ECUDA. */
int fv_diagnostics(fv_grid g, const double* q, double* ekin, double* nu);

/* Time-dependent calculation (Section 4.2.3 runs the full equations in time at slightly sub- and
 * supercritical Gr and monitors E_kin and Nu): nsteps steps of size dt of the semi-implicit scheme
 *     q_{n+1} = q_n + P (I - dt L)^-1 dt F(q_n; Gr),
 * diffusion L backward in time (inverted directly, as fv_diffusion_solve does, with the shift 1/dt),
 * convection and buoyancy forward, the velocity increment made divergence free by the projection P (the
 * pressure correction).  First order in dt; stable for dt below the convective limit (cell size over
 * velocity).  q (device double[4N]) is advanced in place.  ekin, nu: host double[nsteps + 1] or NULL,
 * receive the diagnostics of fv_diagnostics before the first step and after every step.
 * Errors: FV_EINVAL, FV_ENAN (diagnostics not finite: an unstable step), FV_ECUDA, FV_ENOMEM. */
int fv_time_step(fv_grid g, double Gr, double dt, int nsteps, double* q, double* ekin, double* nu);

/* Element-type conversion of a state: FP64 -> FP32 (to_fp32 = 1) or back. */
int fv_convert(fv_grid g, int to_fp32, const void* src, void* dst);

/* ---------------------------------------------------------------- Newton */
typedef struct {
    int precision;        /* FV_FP64: everything FP64.  FV_FP32: Krylov vectors and
                             J.v+projection in FP32; residual, updates and inner
                             products FP64 (the outer loop refines to FP64); inner
                             tolerances are kept >= 1e-3 (preconditioned) or 1e-5 */
    double tol;           /* stop when ||P F||_inf <= tol * max(1, ||P F(q0)||_inf) (default 1e-10) */
    double krylov_tol;    /* relative residual of each inner solve (forcing = 0), or its floor
                             (default 1e-10) */
    int max_newton;       /* Newton steps per Gr (default 20) */
    int max_matvec;       /* J.v+projections per inner solve (default 8000) */
    int gmres_m;          /* restart length of the GMRES fallback (default 100; 30 stalled at
                             64^3, Gr = 4e7) */
    double gr_start;      /* > 0 and < Gr: continuation from gr_start up to Gr; 0 (default): none */
    double gr_ratio;      /* continuation factor per step (> 1) (default 2) */
    int precond;          /* 1 (default): right preconditioner M^-1 = P L^-1, L the diffusion
                             operator of J inverted by fast diagonalisation (see
                             fv_diffusion_solve): inner iteration counts stay nearly flat as the
                             grid is refined; 0: none */
    int forcing;          /* 1 (default): inner tolerance by Eisenstat-Walker, 0.9 (r_k/r_{k-1})^2
                             within [max(krylov_tol, target / (2 r_k)), 1e-2]; 0: krylov_tol */
    double ptc_dt0;       /* > 0: pseudo-transient continuation with this first pseudo-time step:
                             step k solves (P J - I/dt_k) delta = -P F (preconditioner
                             P (L - I/dt_k)^-1); dt grows by (r_{k-1}/r_k)^2 clipped to [1.5, 10]
                             after a step that lowered ||P F|| and halves (not below ptc_dt0) after
                             one that did not; plain Newton once dt_k > 1e4.  A globalisation for high Gr,
                             where the steady state is stable but far from the continuation's
                             previous point; it does not change the converged state.  0 (default): off */
} fv_newton_opts;

typedef struct {
    int status;           /* FV_OK or FV_ENOCONV */
    int newton_steps;     /* at the final Gr */
    int matvecs;          /* J.v+projections, all continuation steps */
    int gmres_fallbacks;  /* inner solves finished by GMRES */
    int continuation_steps;
    double residual0;     /* ||P F(q)||_inf at the start of the final Gr (or of the Gr that failed) */
    double residual;      /* ||P F(q)||_inf at the end (FP64) */
    double history[64];   /* ||P F||_inf per Newton step at the final (or failed) Gr */
} fv_newton_report;

void fv_newton_default_opts(fv_newton_opts* o);

/* Steady state by Newton's method (Section 1 methods paragraph): solve
 * P F(q) = 0 for divergence-free q; corrections from (P J(q)) delta = -P F(q)
 * by BiCGstab(2) (Sleijpen & Fokkema), with GMRES(m) taking over from the
 * current iterate on breakdown or stagnation.  Each correction is scaled
 * back (1, 1/2, .., 1/16) until ||P F||_inf decreases.  Converged when
 * ||P F||_inf <= tol max(1, r0), or when it is below its FP64 round-off
 * floor, estimated as 1e3 eps max|q| (Gr + sum_d 4 / h_min,d^2) (above
 * tol r0 on fine stretched grids; report->residual says where it stopped).  q_inout: device double[4N],
 * the initial state (its velocity must be divergence free, e.g. conduction
 * u = 0, T = 1 - x) and on return the last iterate.  Returns FV_OK,
 * FV_ENOCONV (report filled, q holds the last iterate), FV_ENAN, FV_EINVAL,
 * FV_ECUDA, FV_ENOMEM. */
int newton_steady(fv_grid g, double Gr, double* q_inout, const fv_newton_opts* opts,
                  fv_newton_report* report);

/* ---------------------------------------------------------------- Arnoldi */
typedef struct {
    int precision;        /* FV_FP64, or FV_FP32: a phase with FP32 Krylov vectors and
                             J.v + projection (FP64 Rayleigh-Ritz matrix, Gram-Schmidt
                             coefficients and inner products) down to residual low_tol, then
                             FP64 cycles started from its Ritz vectors refine to tol (each FP64
                             cycle picks its polynomial degree by the same rule as the FP32
                             ones, clamped to [min_degree, max_degree]) */
    int m;                /* Krylov subspace dimension per cycle (default 20) */
    double tol;           /* stop when every wanted Ritz pair has
                             ||A x - lam x|| <= tol |lam| ||x|| (true residual, FP64 reductions)
                             (default 1e-9) */
    int max_restarts;     /* cycle cap (default 30) */
    int max_degree;       /* Chebyshev polynomial degree cap per cycle (default 200) */
    int min_degree;       /* (default 10) */
    int guard;            /* extra Ritz values kept outside the filter's ellipse (default 2) */
    unsigned long long seed;   /* start vector: SplitMix64/Box-Muller N(0,1), projected (default 1) */
    double sigma;         /* shift of the gradient complement; 0 (default): automatic */
    double low_tol;       /* FV_FP32: residual tolerance of the FP32 phase (default 1e-3); the phase
                             also ends once its largest residual has not halved in 3 cycles */
    int low_max_restarts; /* FV_FP32: cycle cap of the FP32 phase (default 20) */
    double euler_dt;      /* > 0: spectral transform by one implicit-Euler step in place of the
                             Chebyshev polynomial: every cycle (the first included) runs its m
                             Arnoldi steps on B = (I - euler_dt P J)^-1, applied by a restarted
                             GMRES solve of (P J - I/euler_dt) y = x right-preconditioned with
                             P (L - I/euler_dt)^-1 (inner_m, inner_max, inner_tol below);
                             eigenvalues still come from V^T A V and are tested with A itself.  B
                             keeps the leading values of A near |mu| = 1/|1 - dt lam| and maps the
                             stiff, convection-dominated far spectrum towards 0.  0 (default): the
                             Chebyshev-preconditioned form of Section 1 */
    int inner_m;          /* euler_dt > 0: restart length of the GMRES shifted solves (default 50) */
    int inner_max;        /* euler_dt > 0: J.v + projections per shifted solve (default 3000) */
    double inner_tol;     /* euler_dt > 0: relative residual of each shifted solve (every solve runs to
                             it); 0 (default): max(1e-12, tol / 100) for FP64 solves, 1e-3 for FP32
                             ones (about their round-off floor).  In the FP64 cycles of the mixed form
                             every shifted solve is FP64-accurate by iterative refinement: FP64
                             residual x - (I - dt P J) y, FP32 GMRES correction to 1e-3, until the FP64
                             residual is below inner_tol or stops halving */
    int vecs_fp64;        /* 1: `vecs` holds FP64 vectors whatever the precision (the mixed form's FP64
                             cycles keep them in FP64; an FP32 copy would carry round-off of relative
                             size u32 ||A|| / |lam| into a residual check).  0 (default): the element
                             type of the precision */
} fv_arnoldi_opts;

typedef struct {
    int status;           /* FV_OK or FV_ENOCONV */
    int nconv;            /* number of values returned (k, or k+1 to complete a pair) */
    int restarts;
    long long matvecs;
    double residual[64];  /* ||A x - lam x|| / |lam| per returned value (FP64 recomputation) */
    double lam_scaled_re[64], lam_scaled_im[64];   /* lam / sqrt(Gr): the paper's scaling */
    int degrees[256];     /* Chebyshev degree per cycle */
    double seconds;
    int restarts_low;     /* FV_FP32: cycles of the FP32 phase (included in restarts) */
    long long matvecs_low;/* FV_FP32: J.v + projections of the FP32 phase (included in matvecs) */
    long long matvecs_fp64;  /* J.v + projections in FP64 (included in matvecs); the rest ran in FP32 */
    int solves;           /* euler_dt > 0: shifted solves */
    int solves_short;     /* euler_dt > 0: shifted solves that stopped above their tolerance */
    double solve_worst;   /* euler_dt > 0: largest final relative residual of a shifted solve */
} fv_arnoldi_report;

void fv_arnoldi_default_opts(fv_arnoldi_opts* o);

/* Leading eigenvalues (largest real part) of the linearised problem about
 * the steady state q: lam v = J(q) v - G p, D v = 0, i.e. of P J(q) on the
 * divergence-free subspace, by Chebyshev-preconditioned Arnoldi (Section 1
 * methods paragraph and its ref. 21; Section 4.1 uses four): cycle 0 runs m
 * Arnoldi steps on A = P(J - sigma) + sigma, every later cycle m steps on
 * p(A), the Chebyshev polynomial of an ellipse around the unwanted Ritz
 * values, with the eigenvalues of A from the Rayleigh-Ritz matrix V^T A V.
 * q: device
 * double[4N].  re, im: host double[k+1] (a conjugate pair straddling the cut
 * is completed, so up to k+1 values; report->nconv says how many), ordered by
 * real part descending, then +Im first.  vecs: NULL or a device buffer of
 * (k+1)*4N elements of the chosen precision; a complex pair occupies two
 * consecutive slots (Re, Im).  Form A units; report carries lam/sqrt(Gr).
 * Errors: FV_EINVAL (k < 1, k+guard+2 > m, m > 200), FV_ENOCONV, FV_ENAN,
 * FV_ECUDA, FV_ENOMEM. */
int arnoldi_leading(fv_grid g, int k, double Gr, const double* q, const fv_arnoldi_opts* opts,
                    double* re, double* im, void* vecs, fv_arnoldi_report* report);

/* ---------------------------------------------------------------- critical Gr (Section 4.1, Table 1) */
/* Which eigenvalue's real part the secant drives to zero. */
enum { FV_MODE_LEADING = 0, FV_MODE_REAL = 1, FV_MODE_OSCILLATORY = 2 };

typedef struct {
    double gr_a, gr_b;    /* the first two Gr of the iteration (ideally bracketing the crossing) */
    double tol;           /* stop when |Gr_{i+1} - Gr_i| <= tol Gr_i (default 1e-7) */
    int max_iter;         /* steady-state + eigenvalue evaluations after the first two (default 16) */
    int mode;             /* FV_MODE_LEADING: the largest real part among the k computed (the first of
                             several modes to cross); FV_MODE_REAL: the largest among the real ones (a
                             steady bifurcation); FV_MODE_OSCILLATORY: among the complex pairs (a Hopf
                             bifurcation, whose Im gives the critical frequency) */
} fv_critical_opts;

typedef struct {
    int status;           /* FV_OK, FV_ENOCONV (iteration cap, or an inner Newton / Arnoldi failure) */
    int evaluations;
    double gr_cr;         /* last iterate: Re lam(gr_cr) ~ 0 */
    double lam_re, lam_im;/* the tracked eigenvalue at gr_cr (Form A units) */
    double omega_scaled;  /* lam_im / sqrt(gr_cr): the angular frequency in the paper's time scale */
    double gr[40], re[40], im[40];   /* every evaluation */
} fv_critical_report;

void fv_critical_default_opts(fv_critical_opts* o);

/* Critical Grashof number of one grid (Section 4.1: the critical values on each grid are the input of
 * the Richardson extrapolation of Table 1): the Gr at which the real part of the tracked eigenvalue of
 * the linearised problem about the steady state crosses zero.  Each evaluation continues the steady
 * state by newton_steady (newton options `nopts`, its continuation ladder ignored: the start is the
 * state of the nearest Gr evaluated before) and computes k leading eigenvalues by arnoldi_leading
 * (`aopts`).  The iteration is the secant method on Re lam(Gr), switched to the Illinois variant of the
 * false-position method once a sign change brackets the crossing.  q_inout (device double[4N]): on entry
 * a divergence-free start for Newton at gr_a (e.g. a steady state nearby or conduction); on return the
 * steady state at gr_cr.  Errors: FV_EINVAL, FV_ENOCONV, FV_ENAN, FV_ECUDA, FV_ENOMEM. */
int fv_critical_gr(fv_grid g, int k, double* q_inout, const fv_newton_opts* nopts, const fv_arnoldi_opts* aopts,
                   const fv_critical_opts* copts, fv_critical_report* report);

/* A tracked eigenvalue as a function of Gr, supplied by the caller: returns FV_OK and the value's real
 * and imaginary parts at gr, or a nonzero status that ends the iteration. */
typedef int (*fv_tracked_fn)(double gr, void* ctx, double* re, double* im);

/* The root iteration of fv_critical_gr on a caller's function (Section 4.1), host only: evaluates f at
 * gr_a and gr_b, then takes secant steps (each at most twice the last spacing) until two values of
 * opposite sign bracket the crossing, then false-position steps with the Illinois halving of a retained
 * end.  Stops with FV_OK once a step moves Gr by at most tol Gr (or hits an exact zero), FV_ENOCONV after
 * max_iter steps or when two values coincide; a nonzero status of f ends it with that status.  `mode`
 * is not used (f returns the tracked value itself).  report (host, may be NULL): every successful
 * evaluation in order, gr_cr / lam_re / lam_im / omega_scaled at the last one.  Errors: FV_EINVAL (null
 * f, gr_a or gr_b not > 0 or equal, tol not > 0, max_iter outside 0..38). */
int fv_critical_root(const fv_critical_opts* copts, fv_tracked_fn f, void* ctx, fv_critical_report* report);

/* Richardson extrapolation to zero grid size (Section 4.1: the critical values depend linearly on the
 * squared average grid size): the least-squares line value = limit + slope h2 through n >= 2 points
 * (h2[i], value[i]) (host arrays), e.g. h2 = (nx ny nz)^(-2/3).  limit, slope: host, either may be NULL.
 * Errors: FV_EINVAL (n < 2, or all h2 equal). */
int fv_richardson(int n, const double* h2, const double* value, double* limit, double* slope);

/* ---------------------------------------------------------------- measurement */
/* Per-kernel-class timing with CUDA events recorded on the handle's stream around every launch.
 * fv_profile(g, 1) clears and starts recording, fv_profile(g, 0) stops.  fv_profile_read
 * synchronises the stream and returns, per class (host arrays of FV_PROF_CLASSES), the summed
 * milliseconds and the launch counts.  Classes: 0 stencil (F, J.v), 1 divergence, 2 pressure-solve
 * transforms (CUDA cores), 3 gradient correction, 4 reductions, 5 other vector kernels,
 * 6 pressure-solve transforms on the tensor cores (FP32 data, tcgen05).
 * Errors: FV_EINVAL, FV_ECUDA, FV_ENOMEM. */
enum { FV_PROF_CLASSES = 7 };
int fv_profile(fv_grid g, int enable);
int fv_profile_read(fv_grid g, double* ms, long long* launches);

const char* fv_strerror(int status);
const char* fv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CUBE_FV_H */
