/*
 * nop.h -- C ABI of the GB300 discrete-ordinates transport solver with
 * equation-recast neural-operator warm start (MD-PNOP, arXiv 2509.01416).
 *
 * The library solves the steady neutron transport equation by the S_N method
 * (diamond-difference sweeps inside source iteration, Sec. 5.1 Eq. 12 and the
 * iteration operator M of Sec. 3.1 Eq. 3a/4b), the k-eigenvalue problem by
 * power iteration with inner sweeps (Sec. 5.2 Eq. 26, App. A2 Eq. A2-A4),
 * multigroup problems (Sec. 5.3 Eq. 27-29), and warm-starts either solve with
 * a neural operator trained at one parameter point p* whose parameter mismatch
 * is recast as an extra source (Sec. 3.1 Eq. 7, Sec. 3.2 Eq. 8-10b, Sec. 5.1
 * Eq. 24, App. A2 Eq. A5-A6).
 *
 * Conventions for every entry point:
 *   - Return value: NOP_OK (0) on success, a negative NOP_E* code otherwise.
 *     nop_status_str() names a code; nop_last_error() returns a message for
 *     the last failing call on that context.
 *   - Pointers are host pointers unless an entry point or a flag says
 *     "device".  The caller owns every buffer it passes; the library copies
 *     inputs in and writes outputs into caller buffers before returning
 *     (device outputs: enqueued on the context stream, see NOP_OUT_DEVICE).
 *   - All floating-point host arrays are IEEE double; device-side arithmetic
 *     precision is chosen per call (nop_solve_opts.precision).
 *   - A context is used by one host thread at a time.  All GPU work of a
 *     context runs on its stream (nop_set_stream).
 *   - Array layouts are "group-major": for a field f with G groups over C
 *     cells the value of group g in cell c sits at f[g * C + c].  Slab cells
 *     are numbered instance by instance (all cells of instance 0, then of
 *     instance 1, ...); x-y cells are row-major, c = j * nx + i.
 */
#ifndef NOP_H
#define NOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define NOP_OK         0
#define NOP_EINVAL    -1   /* an argument is out of range or inconsistent      */
#define NOP_ECUDA     -2   /* a CUDA runtime call failed                        */
#define NOP_ENOMEM    -3   /* device or host allocation failed                  */
#define NOP_ENOCONV   -4   /* iteration cap reached; outputs hold the last iterate */
#define NOP_EDIVERGE  -5   /* recast iteration diverged; a plain guess was used */
#define NOP_ETIMEOUT  -6   /* a device-side wait hit its limit                  */
#define NOP_ENAN      -7   /* a non-finite value appeared in a norm             */
#define NOP_ESTATE    -8   /* call out of order (e.g. solve before set_problem) */
#define NOP_EIO       -9   /* a file could not be read or written, or is malformed */

/* ------------------------------------------------------------ enumerations */
#define NOP_GEOM_SLAB  1   /* batch of independent 1D slabs                  */
#define NOP_GEOM_XY    2   /* one 2D x-y rectangle                           */

#define NOP_BC_VACUUM      0
#define NOP_BC_REFLECTIVE  1

#define NOP_PREC_F32   0   /* FP32 sweeps; FP64 norms, k ratio and tests     */
#define NOP_PREC_F64   1   /* FP64 throughout                                */

#define NOP_WARM_NONE    0 /* plain guess: zero flux (fixed source), flat flux and k=1 (eigen) */
#define NOP_WARM_RECAST  1 /* neural-operator recast warm start (needs a network) */
#define NOP_WARM_RECAST_CP 2 /* eigen only: constrained preconditioning (App. A2
                                Eq. A7-A8) as the warm start; vacuum faces    */

/* flags of nop_solve_opts.flags */
#define NOP_PHI0_DEVICE  1 /* phi0 is a device pointer                        */
#define NOP_SP_CONSTRAINED 4 /* nop_sp_eigen: the constrained variant (Eq. A7-A8) */
#define NOP_OUT_DEVICE   2 /* phi_out / k_out are device pointers; the call does
                              not synchronise (results valid once the context
                              stream reaches this point)                      */
#define NOP_DSA          8 /* slabs: follow every group's sweep by a diffusion
                              synthetic correction (fixed source and the inner
                              iterations of eigen solves).  A classical
                              accelerator of the iteration itself, not the
                              paper's method (which keeps the iteration of
                              Sec. 3.1 Eq. 3a/4b and improves the first
                              iterate); the residual Sigma_s,gg (phi^{l+1/2} -
                              phi^l) drives the P1 equations written with the
                              sweep's diamond-difference closure, an edge-based
                              symmetric tridiagonal system per instance and
                              group, factored once per solve.  The converged
                              flux is unchanged.  NOP_EINVAL with sigma_s1 or
                              the x-y geometry.                               */

#define NOP_GAUSS_SEIDEL 64 /* x-y: Gauss-Seidel over groups with the newest
                              fluxes and quadrants in the order (-,-); (+,-)
                              and (-,+); (+,+) with the newest reflected flux
                              (the reference iteration).  Default: Jacobi in
                              energy with the reflected inflow of the previous
                              iteration, every group and quadrant swept in one
                              launch; same fixed point, other iterates.       */
#define NOP_SWEEP_CHUNKED 16 /* slabs: keep the chunked lane layout (angles x cell
                              chunks with a warp scan of the chunk maps) even
                              where the direct layout applies (vacuum faces,
                              isotropic scattering, no NOP_DSA: the two
                              direction halves swept at once, one lane per
                              angle over the whole slab).  Same iteration,
                              same answer up to rounding; a comparison and
                              tuning aid.                                     */

#define NOP_COLD_SCHEDULE 32 /* slabs: schedule without the iteration counts of
                              earlier solves of the same batch layout (as for a
                              batch seen for the first time); the answer is
                              unchanged                                       */

/* nop_solve_opts.schedule (slab batches).  NOP_SCHED_AUTO: each instance's
 * lane layout (direct or chunked lanes) and whether it runs on one warp or on
 * a 12-warp team come from costs measured on this device (the autotuner:
 * buckets of instances not yet measured are timed once per context, a few
 * milliseconds, on batches of NOP_SCHED_TUNE_MIN instances or more; smaller
 * batches use the analytic model); NOP_SCHED_MODEL: the analytic cost model
 * alone; NOP_SCHED_WARP / NOP_SCHED_BLOCK: every instance on one warp / on a
 * team where its layout allows. */
#define NOP_SCHED_AUTO   0
#define NOP_SCHED_WARP   1
#define NOP_SCHED_BLOCK  2
#define NOP_SCHED_MODEL  3
#define NOP_SCHED_TUNE_MIN 256

typedef struct nop_ctx nop_ctx;

/* Problem description, copied into device memory by nop_set_problem.
 *
 * geometry == NOP_GEOM_SLAB: n_inst independent slabs.  Instance b has
 *   n_cells[b] equal cells over [0, width[b]] and Gauss-Legendre order
 *   order[b] (even, 2..128).  C = sum_b n_cells[b].
 * geometry == NOP_GEOM_XY: one nx-by-ny rectangle of lx-by-ly with the
 *   level-symmetric S8 set (40 directions in the x-y plane); n_inst must be 1,
 *   order[0] must be 8.  C = nx * ny.
 *
 * Coefficients (Eq. 12, 26, 27-29), all group-major over C cells:
 *   sigma_t   [G*C]      total cross section (> 0)
 *   sigma_s   [G*G*C]    scattering from g' into g at [(g'*G + g)*C + c]
 *   source    [G*C]      isotropic external source S (NULL for eigenproblems)
 *   nu_sigma_f[G*C]      production nu*Sigma_f (NULL for fixed source)
 *   chi       [G]        fission spectrum (NULL for fixed source)
 * Boundary conditions: bc[0..1] = slab left/right (applied to every
 *   instance); bc[0..3] = x=0, x=lx, y=0, y=ly for x-y.
 * Linearly anisotropic scattering (Sec. 5.1 Eq. 25), slab fixed-source
 *   problems only (NULL otherwise):
 *   sigma_s1  [G*C]      first Legendre moment of the in-group scattering;
 *                        the emission of direction mu adds (3/2) sigma_s1 mu J
 *                        with the current J of the previous source iteration.
 *                        The recast warm start ignores it (Sec. 5.1: the
 *                        operator only knows isotropic scattering).
 */
typedef struct {
    int geometry;
    int n_inst;
    const int *n_cells;      /* slab: [n_inst] */
    const double *width;     /* slab: [n_inst] */
    const int *order;        /* [n_inst] quadrature order                   */
    int nx, ny;              /* x-y only */
    double lx, ly;           /* x-y only */
    int n_groups;
    const double *sigma_t;
    const double *sigma_s;
    const double *source;
    const double *nu_sigma_f;
    const double *chi;
    int bc[4];
    const double *sigma_s1;  /* slab fixed source only, may be NULL */
} nop_problem;

/* Solver options.  Convergence is the relative L2 change of the scalar flux
 * between successive iterates, ||phi_new - phi_old|| / ||phi_new|| over all
 * cells and groups of an instance, computed in FP64 on the device. */
typedef struct {
    double tol;            /* fixed source: flux tolerance; eigen: outer flux tolerance */
    double tol_k;          /* eigen: |k_new - k_old| / k_new                   */
    double tol_inner;      /* eigen: inner source-iteration tolerance          */
    int itmax;             /* fixed source: max iterations; eigen: max outers  */
    int itmax_inner;       /* eigen: max inner iterations per outer            */
    int precision;         /* NOP_PREC_F32 or NOP_PREC_F64                     */
    int warm_start;        /* NOP_WARM_NONE or NOP_WARM_RECAST                 */
    double recast_tol;     /* recast loop tolerance (Eq. 24)                   */
    int recast_itmax;      /* recast loop iteration cap                        */
    int flags;             /* NOP_PHI0_DEVICE | NOP_OUT_DEVICE | NOP_DSA       */
    int schedule;          /* slab batches: NOP_SCHED_AUTO, NOP_SCHED_MODEL,
                              NOP_SCHED_WARP (one warp per instance),
                              NOP_SCHED_BLOCK (a whole block per instance
                              where the layout allows it)                     */
} nop_solve_opts;

/* Per-call statistics (host struct).  Per-instance arrays are optional
 * caller buffers of n_inst entries (host memory), or NULL. */
typedef struct {
    int status;              /* worst status over instances (0 or NOP_E*)    */
    int max_iterations;      /* max over instances of source iterations (fixed
                                source) or total inner iterations (eigen)    */
    long long sum_iterations;/* sum over instances                           */
    int max_outer;           /* eigen: outer iterations                      */
    int recast_iterations;   /* NO recast iterations of the warm start (max)  */
    int recast_status;       /* worst recast status                          */
    double max_change;       /* final relative change, max over instances    */
    int *inst_iterations;    /* optional [n_inst] out                        */
    int *inst_status;        /* optional [n_inst] out                        */
} nop_stats;

/* ------------------------------------------------------------ lifecycle */

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Errors: NOP_EINVAL (out NULL), NOP_ECUDA (device unusable). */
int nop_create(nop_ctx **out, int device);

/* Free every device buffer of the context and the context itself.  NULL is
 * accepted and ignored. */
int nop_destroy(nop_ctx *ctx);

/* Use `stream` (a cudaStream_t, or NULL for the context's own stream) for all
 * later GPU work of the context.  The caller keeps the stream alive. */
int nop_set_stream(nop_ctx *ctx, void *stream);

/* Name of a status code (static string). */
const char *nop_status_str(int status);

/* Message describing the last failure on ctx (static per context). */
const char *nop_last_error(nop_ctx *ctx);

/* --------------------------------------------------------------- problem */

/* Copy a problem into device memory, replacing the previous one
 * (Sec. 5.1 Eq. 12, Sec. 5.2 Eq. 26, Sec. 5.3 Eq. 27-29 define its terms).
 * Also builds the angular quadratures on the device: Gauss-Legendre (1D) and
 * level-symmetric S8 (x-y).
 * Errors: NOP_EINVAL for bad sizes/orders/NULL arrays, NOP_ENOMEM, NOP_ECUDA. */
int nop_set_problem(nop_ctx *ctx, const nop_problem *p);

/* Read back the quadrature built for instance `inst` (slab: N nodes ascending
 * with weights summing to 2; x-y: 40 directions mu, eta with weights summing
 * to 1, order of quadrants (-,-), (+,-), (-,+), (+,+)).  `eta` may be NULL for
 * slabs.  n_out receives the node count; arrays must hold 128 (slab) / 40 (x-y)
 * entries. */
int nop_get_quadrature(nop_ctx *ctx, int inst, double *mu, double *eta,
                       double *w, int *n_out);

/* -------------------------------------------------------------- solvers */

/* Fixed-source solve by source iteration (Sec. 3.1 Eq. 3a/4b, Sec. 5.1
 * Eq. 20; multigroup: Gauss-Seidel over groups, Sec. 5.3).
 * phi0:    initial flux [G*C], or NULL for the zero guess (ignored when
 *          opts->warm_start == NOP_WARM_RECAST: the recast prediction, Eq. 9a,
 *          is used instead).
 * phi_out: converged scalar flux [G*C].
 * stats:   may be NULL.
 * Errors: NOP_ESTATE (no problem / source missing / warm start without a
 * network), NOP_ENOCONV (some instance hit itmax; phi_out holds the last
 * iterate), NOP_ENAN, NOP_ECUDA. */
int nop_solve_fixed_source(nop_ctx *ctx, const nop_solve_opts *opts,
                           const double *phi0, double *phi_out, nop_stats *stats);

/* k-eigenvalue solve by power iteration with inner source iteration
 * (Sec. 5.2 Eq. 26, App. A2 Eq. A2-A4).  The flux is normalised to unit
 * production, sum nu*Sigma_f * phi * cell volume = 1, and
 * k_{n+1} = k_n * production(phi_{n+1/2}).
 * phi0 / k0: initial guess (phi0 NULL: flat flux; k0 <= 0: 1.0); with
 *            NOP_WARM_RECAST the simple-preconditioning prediction (App. A2
 *            Eq. A5) replaces both (Eq. A6); with NOP_WARM_RECAST_CP the
 *            constrained-preconditioning result (Eq. A7-A8) does.
 * k_out:     [n_inst] eigenvalues.
 * Errors: as nop_solve_fixed_source. */
int nop_solve_eigen(nop_ctx *ctx, const nop_solve_opts *opts, const double *phi0,
                    double k0, double *phi_out, double *k_out, nop_stats *stats);

/* ------------------------------------------------------ neural operator */

#define NOP_NO_DEEPONET  1   /* Sec. 4.1, Eq. 11: <branch(sensors), trunk(x)>     */
#define NOP_NO_FNO1D     2   /* Sec. 4.2: lift, Fourier layers, projection (1D)   */
#define NOP_NO_FNO2D     3   /* the same on an x-y grid                           */

/* Shape of the solution operator N trained at p* = (sigma_t*, sigma_s*)
 * (Sec. 5.1 Eq. 19).  DeepONet: `sensors` uniform bins over [0, length]
 * feed the branch MLP (widths sensors -> width x (depth-1) -> basis); the trunk
 * MLP maps x/length (1 -> width x (depth-1) -> basis); ReLU after every hidden
 * layer, none after the last.  FNO: the operator acts on the problem's own
 * grid; `depth` Fourier layers of `width` channels keep `modes` modes (2D:
 * modes x modes in each of the two k_y half-planes), projection width `proj`.
 * Parameters are one FP32 array, concatenated in this order (W row-major
 * [out][in]):
 *   DeepONet: branch layer 0 W, b, ..., branch layer depth-1 W, b, then the
 *             trunk layers the same way.
 *   FNO1D:    lift W [width][2], b; per layer l: spectral re [modes][width][width],
 *             im [same], pointwise W [width][width], b; proj1 W [proj][width],
 *             b; proj2 W [1][proj], b.  Inputs per point: (S(x), x/length).
 *   FNO2D:    lift W [width][3], b; per layer: re1, im1, re2, im2 each
 *             [modes][modes][width][width] (blocks k_y < modes and k_y >= ny-modes),
 *             pointwise W, b; proj1 W, b; proj2 W, b.  Inputs (S, x/lx, y/ly). */
typedef struct {
    int kind;
    int sensors;
    int width;
    int basis;
    int depth;
    int modes;
    int proj;
    double sigma_t_star;
    double sigma_s_star;
    double length;
} nop_no_config;

/* Training options (App. A1, Table A1: MSE loss, Adam). */
typedef struct {
    int steps;               /* Adam steps                                       */
    int batch;               /* samples per step                                 */
    float lr, beta1, beta2, eps;
    const int *order;        /* [steps * batch] sample indices (host), or NULL for
                                sequential batches                              */
} nop_train_config;

/* Number of FP32 parameters of a configuration.  Errors: NOP_EINVAL. */
int nop_no_param_count(const nop_no_config *cfg, long long *n);

/* Install an operator and its parameters (host FP32 array in the order
 * above); resets the Adam state.  Errors: NOP_EINVAL, NOP_ENOMEM, NOP_ECUDA. */
int nop_no_set(nop_ctx *ctx, const nop_no_config *cfg, const float *params);

/* Copy the current parameters into a host array of nop_no_param_count entries. */
int nop_no_get(nop_ctx *ctx, float *params);

/* Operator files.  A trained operator (its configuration and FP32
 * parameters, Table A1's training result at p*) is kept in a binary file,
 * all numbers little-endian whatever the host:
 *   bytes  0..7   magic "NOPNET01"
 *          8..35  int32 kind, sensors, width, basis, depth, modes, proj
 *         36..59  float64 sigma_t_star, sigma_s_star, length
 *         60..67  int64 n = nop_no_param_count(config)
 *         68..    n float32 parameters in the order of nop_no_set.
 * nop_no_write_file / nop_no_read_file are host-only (no context, no GPU).
 * read: *n_inout holds the capacity of params (entries); on success it
 * receives n and params the values; params may be NULL to query n (cfg is
 * then still filled).  Errors: NOP_EINVAL (NULL path/cfg, invalid
 * configuration, params too small), NOP_EIO (cannot open, short read or
 * write, bad magic, n inconsistent with the configuration, trailing bytes).
 * nop_no_save writes the context's current operator (NOP_ESTATE without
 * one); nop_no_load reads a file and installs it as nop_no_set does. */
int nop_no_write_file(const char *path, const nop_no_config *cfg, const float *params);
int nop_no_read_file(const char *path, nop_no_config *cfg, float *params, long long *n_inout);
int nop_no_save(nop_ctx *ctx, const char *path);
int nop_no_load(nop_ctx *ctx, const char *path);

/* Raw network forward on n samples (no scaling): DeepONet inputs [n][sensors],
 * coords [n_coords] (x/length), out [n][n_coords]; FNO inputs [n][grid points]
 * with the grid given by coords (1D: n_coords = grid size; 2D: the current
 * x-y problem's nx * ny, coords ignored), out [n][grid points].  Host arrays. */
int nop_no_forward(nop_ctx *ctx, int n, const float *inputs, const float *coords,
                   int n_coords, float *out);

/* MSE loss and its gradient with respect to every parameter (same layout as
 * the parameters) for one batch, without updating anything.  Host arrays. */
int nop_no_loss_grad(nop_ctx *ctx, int n, const float *inputs, const float *coords,
                     int n_coords, const float *targets, double *loss, float *grad);

/* Train with Adam on n samples (inputs/targets as in nop_no_loss_grad);
 * loss_history (host, may be NULL) receives the loss of every step. */
int nop_no_train(nop_ctx *ctx, const nop_train_config *tc, int n, const float *inputs,
                 const float *coords, int n_coords, const float *targets,
                 double *loss_history);

/* Operator input map: average a cell field of the current slab problem (host
 * [C] doubles, one group) over each instance's `sensors` bins, out [n_inst][sensors]. */
int nop_no_sensors(nop_ctx *ctx, const double *field, float *out);

/* One application of the trained operator to an isotropic source per
 * instance of the current problem.  The network saw sources of unit integral
 * (Eq. 13) and the exact solution operator is linear, so a source s is applied
 * part by part as sigma+ N[s+/sigma+] - sigma- N[s-/sigma-], s+- its positive
 * and negative parts, sigma+- their integrals (a part with zero integral is
 * skipped).
 * src, phi_out: host [C] doubles (one group). */
int nop_no_predict(nop_ctx *ctx, const double *src, double *phi_out);

/* Equation-recast iteration of Sec. 5.1 Eq. 24 for the current fixed-source
 * problem (one group): phi <- N[S + ((Sigma_s - Sigma_s*) - (Sigma_t - Sigma_t*)) phi]
 * from phi = 0, per instance until the relative change <= tol or itmax.
 * phi_out: host [C] doubles (or device with NOP_OUT_DEVICE in flags); instances
 * whose iteration diverged get the zero flux and status NOP_EDIVERGE.
 * stats: recast_iterations / recast_status / inst_status are filled. */
int nop_recast_iterate(nop_ctx *ctx, double tol, int itmax, int flags, double *phi_out,
                       nop_stats *stats);

/* Simple-preconditioning warm start of an eigenproblem (App. A2 Eq. A5): a
 * power iteration whose inner solve is one application of the trained
 * operator per group and outer step, group g taking the recast source
 *   chi_g F / k + sum_{g' != g} Sigma_s^{g'->g} phi_g' + delta_g phi_g,
 *   delta_g = (Sigma_s^{g->g} - Sigma_s*) - (Sigma_t,g - Sigma_t*),
 * (newest fluxes of the groups already visited), then k <- k P, phi <- phi / P
 * with P the production integral.  Starts from the flat flux at unit
 * production and k = 1; an instance stops when |dk|/k <= tol and the relative
 * L2 change of its flux <= tol, or after itmax outer steps.  The operator is
 * the one installed (FNO-1D needs instances of equal cell counts).
 * phi_out: host [G*C] doubles (device with NOP_OUT_DEVICE in flags), unit
 * production per instance; k_out: host [n_inst].  Instances whose iteration
 * went non-finite get the plain guess (flat flux, k = 1) and NOP_EDIVERGE.
 * stats: recast_iterations (max outer steps), recast_status, inst_status,
 * inst_iterations.  Nothing of the problem is modified.  The result seeds
 * nop_solve_eigen with warm_start = NOP_WARM_RECAST (Eq. A6).
 *
 * With NOP_SP_CONSTRAINED in flags, the constrained preconditioning of App.
 * A2 Eq. A7-A8: every outer step refines the operator's prediction by one
 * model-based source iteration (a sweep per group, FP32) started from the
 * prediction, with the fission source chi F / k built from the prediction,
 * before the outer update.  Vacuum faces only (NOP_EINVAL otherwise). */
int nop_sp_eigen(nop_ctx *ctx, double tol, int itmax, int flags, double *phi_out,
                 double *k_out, nop_stats *stats);

/* --------------------------------------------------- allocation-free solve */

#define NOP_NOALLOC_MAX_CELLS  65536
#define NOP_NOALLOC_MAX_ORDER  128

/* Solve one single-group fixed-source slab (vacuum faces, zero initial flux,
 * FP32 sweeps with FP64 norms, Gauss-Legendre S_N) without allocating any
 * memory.  For callers that cannot call cudaMalloc: plug-ins whose host
 * application owns the device memory and forbids allocations outside the
 * budget it reserved, or real-time loops that must not touch the allocator
 * (a cudaMalloc can take milliseconds and synchronise the device).  The
 * paper has no counterpart; this is a library convenience.
 *
 * All pointers are device pointers: sigma_t, sigma_s (in-group scattering),
 * source (the isotropic S of Eq. 12) are [n_cells] doubles on equal cells
 * over [0, width]; phi_out receives the [n_cells] scalar flux; stats_out
 * receives {source iterations, status}: 0, NOP_ENOCONV (itmax reached; the
 * flux is the last iterate), NOP_ENAN, or NOP_EINVAL when a coefficient is
 * invalid (sigma_t not positive and finite, sigma_s or source not finite;
 * found on the device, the flux is then zero).  Work is enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and the call returns
 * without synchronising.
 *
 * Limits: n_cells <= NOP_NOALLOC_MAX_CELLS, even order <= NOP_NOALLOC_MAX_ORDER;
 * anything larger returns NOP_EINVAL at once.  The scratch is one fixed
 * device array of about 1.8 MB that every GPU loading the library holds
 * until exit; every call shares it, so calls that overlap on the GPU race on
 * it and must be serialised by the caller.  The first call on a device (with
 * that device current) looks up the array's address and sets the solve
 * kernel's shared-memory limit; make that first call before any stream
 * capture. */
int nop_slab_solve_noalloc(const double *sigma_t, const double *sigma_s,
                           const double *source, int n_cells, double width, int order,
                           double tol, int itmax, double *phi_out, int *stats_out,
                           void *stream);

/* --------------------------------------------------------------- tracing */

/* Device-side phase times accumulated since timing was enabled. */
typedef struct {
    double sweep_ms;         /* solver kernels (sweeps, norms, eigen updates)    */
    double operator_ms;      /* neural-operator kernels (inference, recast loop)  */
    double setup_ms;         /* data preparation / result conversion kernels      */
    long long launches;      /* kernels this library launched                    */
    long long sweep_launches;/* of which solver kernels                          */
    double cell_angle_updates; /* algorithmic sweep work: sum over solved
                                  instances of iterations x cells x angles x
                                  groups (one diamond-difference cell update per
                                  cell, direction and group)                     */
    double last_span_ms;     /* last slab solve: first instance start to last
                                instance end (device clock)                     */
    double last_inst_max_ms; /* last slab solve: longest single instance         */
    double last_inst_mean_ms;/* last slab solve: mean instance duration          */
    int last_block_instances;/* last slab solve: instances run on a whole block  */
    int last_direct_instances;/* last slab solve: instances on the direct lanes  */
    double last_tune_ms;     /* last slab solve: host time spent measuring layout
                                costs (0 when every bucket was known)          */
} nop_timings;

/* ----------------------------------------------------- diffusion batches */

/* A second PDE on the recast driver (Sec. 3.1, Table 1): a batch of n_inst
 * independent 1D slabs with -(D u')' + Sigma_a u = S on (0, width) and u = 0
 * at both faces.  Table 1's diffusion row is Sigma_a = 0 with parameter
 * p = D(x); its Helmholtz row -u'' - k^2 u = S is D = 1, Sigma_a = -k^2.
 * Discretisation: n_cells uniform cells per instance, cell-centred finite
 * volumes, face coefficients the harmonic mean of the two cells' D, a
 * boundary face half a cell from its centre.  diffusion (> 0), absorption
 * (finite; NULL = 0) and source are cell values of all instances
 * concatenated (host, FP64, copied).  After this call nop_recast_iterate and
 * nop_no_predict apply a DeepONet to the batch (its configuration's
 * sigma_t_star and sigma_s_star are read as D* and Sigma_a*; the mismatch
 * -dL = -(L(p) - L(p*)) of the discrete operators on the operator's grid is
 * the recast source term), nop_diffusion_solve gives the model-based
 * solution; the transport solves return NOP_ESTATE.  A later
 * nop_set_problem replaces the batch. */
int nop_set_diffusion(nop_ctx *ctx, int n_inst, const int *n_cells, const double *width,
                      const double *diffusion, const double *absorption, const double *source);

/* The model-based solution of the diffusion batch: every instance's
 * tridiagonal system solved by elimination in FP64; u_out: host, C doubles. */
int nop_diffusion_solve(nop_ctx *ctx, double *u_out);

/* Measured arithmetic ceilings of the sweep (a microbenchmark, not the
 * paper's method): the device's rate of the special-function reciprocal
 * rcp.approx.ftz.f32 (one per diamond-difference cell-angle update) and of
 * FP32 fused multiply-adds, in operations per second, from kernels of 8
 * independent chains per thread over 8 blocks of 256 threads per SM, timed
 * with CUDA events on the context stream (best of 3 after a warm-up).  Takes
 * a few milliseconds. */
int nop_measure_alu_peaks(nop_ctx *ctx, double *rcp_per_s, double *fma_per_s);

/* The slab batch scheduler's team selection, exported so that its logic can
 * be checked without a GPU (host arithmetic only).  lat_warp[b]: latency of
 * instance b on one warp; lat_team[b]: on a team of team_width warps (< 0:
 * no team).  mode 0: instances are taken in decreasing warp latency, and
 * each gets a team while margin x its warp latency exceeds the expected span
 * S = (warp latencies of the warp instances + team_width x team latencies of
 * the team instances) / warps, S updated after every pick; margin >= 1 covers
 * errors of the latency estimates (a team costs little extra SM time next to
 * the whole batch, an instance left on a warp that outlasts S costs the whole
 * difference); mode 1: every instance that can; mode 2: none.  team_out[b]
 * receives 0/1; *span_out (may be NULL) the final S.  NOP_EINVAL for
 * margin < 1, warps < 1 or team_width < 1. */
int nop_sched_select_teams(int n, const double *lat_warp, const double *lat_team, int warps,
                           int team_width, int mode, double margin, int *team_out,
                           double *span_out);

/* Failure detection.  Every wait of a tensor-core kernel on its own products
 * (an mbarrier poll) is bounded; when the bound runs out the kernel records
 * the failure, lets the products it committed finish, frees its tensor
 * memory and returns, and the call reports NOP_ETIMEOUT with the context
 * still usable.  polls < 0 restores the library default (2^26 polls, seconds
 * of waiting); polls >= 0 sets the bound, 0 giving up at the first wait (a
 * way to exercise the failure path).  Not in the paper: a library safeguard. */
int nop_set_wait_limit(nop_ctx *ctx, long long polls);

/* enable != 0: from now on record CUDA events around every kernel phase on
 * the context stream and count launches (totals reset); 0: stop recording.
 * Recording adds no synchronisation. */
int nop_set_timing(nop_ctx *ctx, int enable);

/* Synchronise the context stream and return the totals since the last
 * nop_set_timing(ctx, 1). */
int nop_get_timing(nop_ctx *ctx, nop_timings *out);

/* Per-instance trace of the last slab solve run with timing on (profiling
 * aid): start time relative to the first instance, duration (ms), and 1 where
 * the instance ran on a whole block rather than one warp.  n must be the
 * batch size; any output pointer may be NULL.  NOP_ESTATE if no such trace. */
int nop_get_trace(nop_ctx *ctx, int n, double *start_ms, double *duration_ms, int *block_path);

#ifdef __cplusplus
}
#endif
#endif /* NOP_H */
