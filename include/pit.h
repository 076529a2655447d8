/*
 * pit.h -- C ABI of libpit.so: the all-at-once BDF1 Newton iteration of
 * Yamaleev & Paudel, "A New Parallel-in-time Direct Inverse Method for
 * Nonlinear Differential Equations" (arXiv 2406.00878), on one GB300 GPU.
 *
 * The method (paper Sec. 2-4):
 *   eq. 1  u_t + f(u)_x + g(u)_y = (mu(u) u_x)_x + (mu(u) u_y)_y on a rectangle,
 *          Dirichlet data b on the boundary (eq. 2), initial data u0;
 *          nonlinear heat: f = g = 0, mu = mu_a + mu_b u^2;
 *          viscous Burgers: f = g = u^2/2, mu = mu_a (+ mu_b u^2).
 *   eq. 3  BDF1 in time, 2nd-order 3-point central differences in x and y,
 *          mid-point viscosity mu_{i+1/2} = mu((u_i + u_{i+1})/2).
 *   eq. 4  all time levels n = 1..M form one nonlinear system G(U) = 0.
 *   eq. 5  Newton: A_n du^n - du^{n-1} = r^n with A_n = I + tau dF/du(u^n)
 *          and r^n = -tau[(u^n - u^{n-1})/tau + F(u^n) - q^n].
 *   eq. 6  the Jacobian is block bidiagonal (A_n on the diagonal, -I below).
 *   eq. 7  its exact inverse, applied in nested form
 *          du^n = A_n^{-1}(r^n + du^{n-1}), one level solve per time level.
 *
 * Conventions for every entry point:
 *   - nx, ny count INTERIOR nodes; h_x = (xr - xl)/(nx + 1), node (j, i) sits at
 *     x = xl + (i + 1) h_x, y = yl + (j + 1) h_y; Ns = nx * ny.
 *   - All arrays are IEEE FP64 and C-contiguous with x fastest:
 *       level vector  [ny][nx]
 *       space-time    [M][ny][nx]       level n = 1..M at offset (n-1)*Ns
 *       boundary data [M][2*nx + 2*ny]  per level: south row (j = -1, nx values),
 *                                       north row (j = ny, nx), west column
 *                                       (i = -1, ny), east column (i = nx, ny)
 *       coefficients  [5][M][Ns]        C, W, E, S, N entries of each row of A_n
 *   - Pointers named *_dev are device pointers on the context's device; they are
 *     owned by the caller and must stay valid for the duration of the call.
 *     Pointers named *_host are host pointers (pinned memory is fastest).
 *   - Every call is ordered on the CUDA stream given to pit_create (NULL = the
 *     legacy default stream). Calls that return norms or statistics synchronise
 *     that stream before returning.
 *   - Errors are returned as pit_status; the library never aborts and never
 *     throws across the ABI. pit_last_error() gives a message for the last
 *     failing call on a context. Device-side waits are bounded: a wait that runs
 *     out of its budget ends the kernel with PIT_ETIMEOUT instead of hanging.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef PIT_H
#define PIT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pit_ctx pit_ctx;

typedef enum {
    PIT_OK = 0,
    PIT_EINVAL = 1,       /* invalid argument (sizes, NULL pointers, parameters) */
    PIT_ECUDA = 2,        /* a CUDA runtime call failed */
    PIT_ENOMEM = 3,       /* device allocation failed */
    PIT_ENOCONV = 4,      /* Newton or a level solve hit its iteration cap */
    PIT_EDIVERGED = 5,    /* NaN/Inf in the residual or the update */
    PIT_ETIMEOUT = 6,     /* a bounded device-side wait ran out of budget */
    PIT_EUNSUPPORTED = 7, /* the problem does not fit the kernels' limits */
    PIT_EBOUNDS = 8       /* bounds-checking build only: a kernel indexed an array out of range */
} pit_status;

typedef enum { PIT_HEAT = 0, PIT_BURGERS = 1 } pit_equation;

/* Level solver for the diagonal blocks A_n (eq. 7, one solve per level). */
typedef enum {
    PIT_LIN_AUTO = 0,     /* per level: SOR when the Jacobi-scaled Gershgorin bound of
                             A_n is below sor_rho_max, else BiCGStab */
    PIT_LIN_SOR = 1,      /* red-black SOR, omega from the Gershgorin bound */
    PIT_LIN_BICGSTAB = 2  /* Jacobi-preconditioned BiCGStab */
} pit_lin_solver;

typedef struct {
    int nx, ny;             /* interior nodes, >= 1 */
    double xl, xr, yl, yr;  /* domain, xr > xl, yr > yl */
} pit_grid;

typedef struct {
    int equation;           /* pit_equation */
    double mu_a, mu_b;      /* mu(u) = mu_a + mu_b u^2, both >= 0 (mu >= 0, Sec. 2) */
} pit_params;

typedef struct {
    int newton_max;         /* max Newton updates in pit_solve (default 30) */
    double tol_res;         /* pit_solve stops when ||R||_inf <= tol_res, R the tau-scaled
                               residual of eq. 5 (default 1e-12) */
    int lin_solver;         /* pit_lin_solver (default PIT_LIN_AUTO) */
    double eta_max;         /* inexact-Newton forcing: each level solve reduces its error
                               estimate to eta * ||rhs||, eta = min(eta_max, eta_gamma*||R||_inf)
                               (default 1e-2) */
    double eta_gamma;       /* (default 1.0) */
    double lin_atol;        /* absolute floor of SOR's error tolerance (default 1e-15); BiCGStab stops
                               relative to its Jacobi-scaled rhs */
    int lin_max_iter;       /* cap on sweeps / iterations per level solve (default 4000) */
    double sor_rho_max;     /* AUTO uses SOR below this Gershgorin bound (default 0.999; below 1 SOR
                               converges: symmetric levels are SPD, nonsymmetric ones get omega <= ~1) */
    int team_ctas;          /* CTAs that share one level in the chain kernel; > 0 also caps the
                               wavefront kernel's teams at this size, all equal (0 = auto) */
    long long wait_budget;  /* spin iterations before a device wait gives up (default 1<<26) */
    int wave_teams;         /* pit_solve: Newton iterations in flight in the wavefront kernel
                               (0 = auto: the most teams, up to 6, whose level strips fit in
                               shared memory; >= 1 that many; -1 = one launch per stage and
                               Newton iteration, as pit_newton_step). The SMs that K equal teams
                               leave over go to the teams nearest the middle (a row less per
                               strip), unless team_ctas > 0 fixes every team's size */
    int precision;          /* pit_solve level solves: PIT_FP64 (default) or PIT_FP32_INNER: the
                               Jacobian entries, right-hand sides and level-solve iterates are
                               held and updated in FP32, inside FP64 Newton (residual, update
                               and norms stay FP64; Newton then acts as iterative refinement) */
    int window;             /* pit_solve with the wavefront: 0 (default) = all M levels at once
                               from the caller's iterate; W > 0 = levels in consecutive windows of
                               W, each starting from the plain guess u^n = u^{s-1} at its first
                               level s. The all-at-once system is block lower-triangular in time,
                               so the solution is the same. In both modes a window whose Newton
                               diverges (a residual that is not finite, above 1e10, or in an
                               iteration k >= 1 above 1e3 times the first iteration's running
                               residual at that level) or does not converge is halved and
                               restarted from the plain guess, and grows back after a success */
    int batch_wave_nodes;   /* pit_batch_create: a problem with nx*ny >= batch_wave_nodes is a wavefront
                               job of the persistent launch (up to 6 teams, nearly every SM, several
                               Newton iterations of a window in flight), such jobs one after another;
                               <= 0 = one team per problem for all (default 65536, a 256 x 256 grid) */
    int window_start;       /* where a window's Newton iteration starts (pit_solve with window > 0, and
                               pit_batch_solve): PIT_START_PLAIN (default) = the plain guess
                               u^n = u^{s-1} for every level of the window; PIT_START_GIVEN = the
                               iterate the caller left in U_dev for those levels (a learned or
                               coarse-grid guess). A window that is retried after a failure starts
                               from the plain guess, as do later windows whose levels the failed
                               attempt overwrote */
} pit_options;

enum { PIT_FP64 = 0, PIT_FP32_INNER = 1 };
enum { PIT_START_PLAIN = 0, PIT_START_GIVEN = 1 };

#define PIT_MAX_NEWTON 64

typedef struct {
    double res_inf;         /* ||R||_inf of the iterate the step started from */
    double upd_rms;         /* sqrt(sum(dU^2) / (M Ns)), the update norm of Sec. 8 */
    double lin_iters_mean;  /* mean sweeps (SOR) or iterations (BiCGStab) per level */
    int lin_iters_max;
    int levels_sor;         /* levels solved by SOR in this step */
    int levels_capped;      /* levels that hit lin_max_iter */
    float ms_residual, ms_assemble, ms_solve;  /* device time of the three stages */
    float us_halo_wait;     /* time the first CTA of the level chain waited for neighbours */
    float us_reduce_wait;   /* time the first CTA of the level chain waited on team reductions */
    float us_chain;         /* the first CTA's total time in the level chain */
} pit_step_info;

typedef struct {
    int newton_iters;                      /* Newton updates applied */
    int converged;                         /* 1 when ||R||_inf <= tol_res was reached */
    double res_inf[PIT_MAX_NEWTON + 1];    /* ||R_k||_inf, k = 0..newton_iters */
    pit_step_info steps[PIT_MAX_NEWTON];
    double ms_total;                       /* device time of the whole solve */
    int wave_teams;                        /* Newton iterations in flight (0: per-stage launches) */
    int wave_team_ctas;                    /* CTAs per team (the smallest team's) */
    int wave_launches;                     /* wavefront launches (more than 1 after a restart) */
    float ms_wave;                         /* device time of the wavefront launches */
    float us_pred_wait;                    /* first CTA of team 0: waiting for the previous iteration */
    float us_halo_wait, us_reduce_wait;    /* first CTA of team 0: team synchronisation */
    int windows;                           /* windows of levels solved (1 without windowing) */
    int newton_iters_total;                /* Newton updates summed over the windows */
    float us_setup;                        /* first CTA of team 0: forming level systems (residual, Jacobian) */
    float us_level_solve;                  /* first CTA of team 0: level solves (includes halo/reduction waits) */
    float us_update;                       /* first CTA of team 0: iterate updates and progress publication */
    int windows_converged;                 /* windows whose Newton reached tol_res (windows minus restarts) */
    int wave_ctas;                         /* CTAs of the wavefront launch: SMs that K teams of
                                              wave_team_ctas leave over go to the middle teams */
} pit_solve_info;

/* Fill *opt with the defaults listed above. */
void pit_default_options(pit_options* opt);

/* Create a context for one problem: grid, M time levels of constant step dt
 * (tau_n = dt, t^n = n dt), closure parameters; opt may be NULL (defaults).
 * stream is a cudaStream_t (NULL = legacy default stream). Allocates every
 * device workspace here (residual, Jacobian planes, team workspace, the iterate of
 * pit_solve_host); only pit_set_data allocates later, once, for boundary data or
 * sources. Dirichlet data and sources are zero and u0 is zero until pit_set_data.
 * The chain kernel shares each level among a team of CTAs that must be co-resident
 * (cooperative launch); PIT_EUNSUPPORTED when a grid row does not fit. */
pit_status pit_create(const pit_grid* grid, int M, double dt, const pit_params* params, const pit_options* opt,
                      void* stream, pit_ctx** out);

/* Copy problem data into the context (device to device, stream ordered):
 * u0_dev [Ns] initial data u^0 (required); bc_dev [M][2nx+2ny] Dirichlet data at
 * t^n, or NULL for zero (eq. 2); q_dev [M][Ns] source q^n, or NULL for zero (eq. 4). */
pit_status pit_set_data(pit_ctx* ctx, const double* u0_dev, const double* bc_dev, const double* q_dev);

/* Write the plain initial iterate u^n = u^0, n = 1..M, into U_dev [M][Ns]. */
pit_status pit_fill_plain_guess(pit_ctx* ctx, double* U_dev);

/* The paper's initial iterate (Sec. 4): solve the context's problem on a grid
 * coarsened by cf >= 2 in both spatial directions and in time -- (nx+1)/cf - 1 by
 * (ny+1)/cf - 1 interior nodes on the same domain, M/cf levels over the same end time --
 * then interpolate the coarse solution to every fine node and level with natural cubic
 * splines along x, y and t, and write it to U_dev [M][Ns].
 * The coarse data are sampled from the context's data (pit_set_data): u^0 and sources
 * bilinearly in space, Dirichlet data linearly along each edge, both linearly in time
 * (exact injection where coarse and fine nodes coincide). The coarse problem is solved
 * all at once with the context's options (team sizes re-chosen); its converged result
 * is the sequential BDF1 solution on the coarse grid. coarse_info (may be NULL)
 * receives that solve's report.
 * Allocates and frees its temporaries (about (M/cf + 1) * Ns * 3 doubles) and
 * synchronizes the context's stream before returning.
 * PIT_EINVAL for cf < 2 or a grid too small to coarsen; a failed coarse solve returns
 * its status (PIT_ENOCONV, PIT_EDIVERGED, ...) and leaves U_dev unwritten -- fall back
 * to pit_fill_plain_guess. */
pit_status pit_coarse_guess(pit_ctx* ctx, int cf, double* U_dev, pit_solve_info* coarse_info);

/* Row (a1): the all-at-once residual of eq. 4-5 for all M levels at once,
 * R_dev[n] = -tau[(u^n - u^{n-1})/tau + F(u^n) - q^n] with F of eq. 3.
 * U_dev [M][Ns] in, R_dev [M][Ns] out (may not alias U_dev). If res_inf is not
 * NULL it receives ||R||_inf (synchronises the stream). */
pit_status pit_residual(pit_ctx* ctx, const double* U_dev, double* R_dev, double* res_inf);

/* Row (a2): the Jacobian blocks A_n = I + tau dF/du(u^n) of eq. 5-6 for all M
 * levels at once: coef_dev [5][M][Ns] receives the C, W, E, S, N entries of
 * every row (couplings to boundary nodes are 0). */
pit_status pit_assemble(pit_ctx* ctx, const double* U_dev, double* coef_dev);

/* Row (a3): solve the block-bidiagonal system of eq. 6 whose diagonal blocks are
 * the Jacobians A_n at U_dev, with right-hand side R_dev, by the exact block
 * inverse of eq. 7 in nested form: du^1 = A_1^{-1} r^1, du^n = A_n^{-1}(r^n + du^{n-1}),
 * one level solve per time level, chained. dU_dev [M][Ns] receives the solution;
 * U_dev is not modified. Each level solve stops when its error estimate (SOR) or
 * its preconditioned residual (BiCGStab) falls below max(eta * ||rhs||, lin_atol);
 * pass a small eta (e.g. 1e-14) for a nearly exact solve. info (may be NULL)
 * receives iteration statistics. PIT_ENOCONV: a level hit lin_max_iter (dU holds
 * the capped result). */
pit_status pit_block_solve(pit_ctx* ctx, const double* U_dev, const double* R_dev, double* dU_dev, double eta,
                           pit_step_info* info);

/* One Newton iteration in place on U_dev [M][Ns]: residual (a1), blocks (a2),
 * nested block inverse (a3) with the inexact-Newton forcing of pit_options, and
 * the update U += dU. info (may be NULL) receives norms and statistics. */
pit_status pit_newton_step(pit_ctx* ctx, double* U_dev, pit_step_info* info);

/* Phase timers of the last wavefront launch of pit_solve, for performance analysis:
 * for every team t of the launch (Newton iterations t, t + K, ...), 25 values from its
 * first CTA, out[25 t + j]: 0 halo waits (flag protocol), 1 team-reduction waits,
 * 2 waits for the previous Newton iteration, 3 total, 4 level setup, 5 level solves,
 * 6 updates, 7 setup: loading u^n_k, 8 setup: team reduction and boundary-row exchange
 * (nanoseconds), 9 cells solved, 10 sweeps or iterations (counts), 11 unused, 12..19 SM
 * cycles of its thread 0 in the steps of the SOR sweeps with deep rows: publishing the
 * boundary rows, interior rows of colour 0, fetching the neighbours' rows, boundary rows
 * and halo points, a barrier, colour 1, the lagged reduction and stop decision, a barrier;
 * 20..24 SM cycles of its thread 0 in the steps of the level setup: the node loop
 * (residual, couplings, rhs), the block reduction, publishing the level system's boundary
 * rows, the team reduction, fetching the neighbours' boundary rows.
 * Copies up to n values and returns how many there are (25 K), or -1 for a NULL argument. */
int pit_wave_timers(const pit_ctx* ctx, unsigned long long* out, int n);

/* The bounds-checking build. Compiled with PIT_CHECK_BOUNDS, every indexed access of the
 * residual, assembly, level-chain, wavefront and batched kernels to the problem's arrays
 * (U, u0, boundary data, source, right-hand sides, coefficient planes), to the per-iteration
 * records, and to the CTA's shared-memory arrays (couplings, rhs, iterate, solver vectors,
 * halo rows, u^n_k strip, neighbour rows) is checked against the array's extent, and every
 * bulk copy against its source and destination ranges and 16-byte alignment. An access out
 * of range is skipped (a load reads a scratch word, a store writes it; a bad bulk copy is
 * not issued), the array's id is recorded, and the kernel runs on: nothing traps. This call
 * synchronises the device, sets *enabled = 1 in that build (0 in the ordinary build, where
 * the checks are compiled out) and *first_id to the id of the first array found out of
 * range since the previous call (0 = none), then clears the record. Returns PIT_EBOUNDS
 * when an id was recorded, PIT_EINVAL for NULL arguments, PIT_ECUDA when the device
 * cannot be read. Ids: 1 U, 2 u0, 3 boundary data, 4 source, 5 R, 6 coefficient planes,
 * 7 dU; 16 + k the k-th shared array (cw ce cs cn bs x r rh p v t haloS haloN); 40 uprev,
 * 41 u^n_k strip, 42 neighbour rows; 50 running-residual record, 51 cell iterations, 52
 * update norms, 53 progress words, 58 per-level records; 60 a bulk copy. */
pit_status pit_bounds_status(int* enabled, int* first_id);

/* Row (a4): Newton from the iterate in U_dev until ||R||_inf <= tol_res or
 * newton_max updates (PIT_ENOCONV; U_dev holds the last iterate). By default all
 * Newton iterations run in one cooperative wavefront launch: iteration k works on
 * level n as soon as iteration k-1 has finished it, so up to wave_teams iterations
 * are in flight (same iterates as plain Newton; the level solves' forcing uses the
 * running max of ||r^j||_inf over the levels j <= n already visited). The final
 * ||R||_inf is always recomputed from U_dev by the residual kernel. */
pit_status pit_solve(pit_ctx* ctx, double* U_dev, pit_solve_info* info);

/* pit_solve with host buffers: copies u0_host [Ns] to the device (replacing u^0),
 * starts from the plain guess u^n = u^0, solves, and copies the solution to
 * U_host [M][Ns]. Uses the context-owned device iterate allocated by pit_create;
 * the boundary data and sources set by pit_set_data are kept. */
pit_status pit_solve_host(pit_ctx* ctx, const double* u0_host, double* U_host, pit_solve_info* info);

/* ----------------------------------------------------------- batched solves
 * Many independent problems (grids, level counts, closures and viscosities may
 * all differ) solved in ONE persistent cooperative launch. Each problem runs the
 * level chain of eq. 7 with Newton iterations until its residual is <= tol_res,
 * in windows of opt->window levels (default 32). A problem on a grid of at least
 * opt->batch_wave_nodes nodes is a wavefront job: K teams of G CTAs (K * G up to
 * the SM count, the SMs left over going to the middle teams) with K Newton
 * iterations of a window in flight, as in pit_solve; these jobs run first, one
 * after another. Every other problem gets one team of
 * CTAs, and teams of different sizes run side by side on the remaining SMs and
 * afterwards. pit_batch_create picks every such team's size with an autotuner
 * (short timed runs of each distinct grid size at candidate team sizes;
 * opt->team_ctas > 0 fixes it instead) and list-schedules the teams over the
 * SMs, longest first. pit_batch_solve replays the launch as a captured CUDA
 * graph after its first call; the batch works on a stream of its own, ordered
 * after the caller's `stream` at every solve, and returns when the solve is
 * complete. Level solves follow opt->precision (PIT_FP32_INNER is the intended
 * use). A window whose Newton diverges (a residual that is not finite or above
 * 1e10, or a level solve that breaks down) is restarted shorter, down to single
 * levels; a problem that still fails only ends unconverged (pit_batch_solve then
 * returns PIT_ENOCONV and its res_inf tells which); only a device wait that runs
 * out of budget ends the launch (PIT_ETIMEOUT). */
typedef struct pit_batch pit_batch;

typedef struct {
    pit_grid grid;
    int M;
    double dt;
    pit_params params;
    const double* u0_dev;   /* [Ns] initial data (required) */
    const double* bc_dev;   /* [M][2nx+2ny] Dirichlet data or NULL */
    const double* q_dev;    /* [M][Ns] source or NULL */
    double* U_dev;          /* [M][Ns] out: the solution; in: the starting iterate when
                               opt->window_start = PIT_START_GIVEN (ignored otherwise: every
                               window starts from the plain guess at its first level) */
} pit_instance;             /* all pointers caller-owned, valid until pit_batch_destroy */

typedef struct {
    int count;              /* problems */
    int ctas;               /* CTAs of the persistent launch */
    int teams;              /* teams (one per problem) */
    int min_team, max_team; /* team sizes chosen */
    int converged;          /* problems whose final ||R||_inf <= tol_res */
    int graph;              /* 1 when the launch was replayed from a CUDA graph */
    double ms;              /* device time of the launch */
    double est_makespan_ms; /* the schedule's estimate from the autotuner's timings */
    double ms_tuning;       /* host time spent in pit_batch_create's autotuner */
    int wave_jobs;          /* problems solved as wavefront jobs (several teams) */
} pit_batch_info;

pit_status pit_batch_create(const pit_instance* inst, int count, const pit_options* opt, void* stream,
                            pit_batch** out);
pit_status pit_batch_solve(pit_batch* batch, pit_batch_info* info);
/* Results of problem i after pit_batch_solve: final ||R||_inf of U (FP64), Newton
 * updates summed over windows, the number of windows that converged, and the CTAs
 * of each team that solved it (see pit_batch_placement). */
pit_status pit_batch_result(const pit_batch* batch, int i, double* res_inf, int* newton_iters, int* windows_converged,
                            int* team_ctas);
/* How problem i is solved: *teams teams (K > 1: a wavefront job with K Newton
 * iterations in flight; 1: one team) of *team_ctas CTAs each. Any pointer may be
 * NULL. */
pit_status pit_batch_placement(const pit_batch* batch, int i, int* teams, int* team_ctas);
const char* pit_batch_last_error(const pit_batch* batch);
void pit_batch_destroy(pit_batch* batch);

/* ------------------------------------------------- learned initial guess
 * A small residual conv net maps (u^0, log10 nu) on the grid to the corrections
 * u^n - u^0 of all M levels; u^0 + correction replaces the plain guess u^n = u^0
 * as Newton's starting iterate (the converged solution is the same; the net only
 * moves the start). Layers: 3x3 conv 2 -> C, ReLU; per block h = ReLU(conv(x)),
 * x = x + conv(h); head 3x3 conv C -> M. BF16 weights and activations, FP32
 * accumulation on the tensor cores, FP32 master weights, Adam, MSE loss. The head
 * starts at zero, so an untrained net returns the plain guess. Parameters travel
 * as one FP32 vector: per layer W [Cout][3][3][Cin] then bias [Cout], in the order
 * input, (block conv 1, block conv 2) x blocks, head. Targets are BF16 [B][H][W][M]
 * (pit_net_make_target). All calls are ordered on the stream of pit_net_create. */
typedef struct pit_net pit_net;

typedef struct {
    int height, width;      /* grid (interior nodes ny, nx) */
    int levels;             /* M, a multiple of 16 */
    int channels;           /* C, a multiple of 16 */
    int blocks;             /* residual blocks */
    int max_batch;          /* largest batch passed to the calls below */
} pit_net_shape;

long long pit_net_param_count(const pit_net_shape* shape);
pit_status pit_net_create(const pit_net_shape* shape, unsigned long long seed, void* stream, pit_net** out);
pit_status pit_net_get_params(pit_net* net, float* params_host);
pit_status pit_net_set_params(pit_net* net, const float* params_host);
/* U_dev [B][M][Ns] = u0 + net(u0, log10 nu): the starting iterate of B problems. */
pit_status pit_net_guess(pit_net* net, const double* u0_dev, const float* lognu_host, int B, double* U_dev);
/* target_dev (BF16 [H][W][M]) = U - u^0 for one solution U_dev [M][Ns]. */
pit_status pit_net_make_target(pit_net* net, const double* u0_dev, const double* U_dev, void* target_dev);
/* Mean squared error of a batch and its gradient (public layout, may be NULL). */
pit_status pit_net_gradients(pit_net* net, const double* u0_dev, const float* lognu_host, const void* target_dev,
                             int B, float* loss_out, float* grads_host);
/* One Adam step (beta 0.9 / 0.999) on a batch; loss_out (may be NULL) synchronises. */
pit_status pit_net_train_step(pit_net* net, const double* u0_dev, const float* lognu_host, const void* target_dev,
                              int B, float lr, float* loss_out);
const char* pit_net_last_error(const pit_net* net);
void pit_net_destroy(pit_net* net);

/* One layer of the network above, without a network: the same tensor-core kernels on
 * the caller's operands (for layer-by-layer checks, or nets of other shapes). NHWC BF16
 * activations X [B][H][W][Cin], weights W [Cout][3][3][Cin] BF16, bias FP32 [Cout];
 * Cin and Cout multiples of 16 (at most 4096).
 * Forward: Y [B][H][W][Cout] = act(conv3x3(X, W) + bias (+ res)), zero padding, FP32
 * accumulation, BF16 output; res (may be NULL) [B][H][W][Cout]; act = ReLU when relu != 0.
 * Backward, for the loss L = sum(dY * conv3x3(X, W)): dX [B][H][W][Cin] BF16 (may be NULL),
 * dW [Cout][3][3][Cin] FP32 and db [Cout] FP32 (device pointers).
 * Kernels (tcgen05 MMAs, FP32 accumulators in tensor memory): for Cin = 64 or 128 the
 * forward and data gradient run the row-stationary kernel, whose operands come from TMA
 * tensor loads of 128-byte-swizzled NHWC rows and 64-channel weight blocks (when X and W are
 * 16-byte aligned); for Cin = 64 and Cout a multiple of 64 the weight gradient reads the
 * TMA-staged NHWC rows as MN-major operands. Other shapes take the general TMA or cp.async
 * kernels; all give the same results up to FP32 summation order.
 * Both allocate their temporaries per call and synchronise `stream`. */
pit_status pit_conv3x3_forward(const void* X_dev, const void* W_dev, const float* bias_dev, const void* res_dev,
                               void* Y_dev, int B, int H, int W, int Cin, int Cout, int relu, void* stream);
pit_status pit_conv3x3_backward(const void* X_dev, const void* W_dev, const void* dY_dev, void* dX_dev,
                                float* dW_dev, float* db_dev, int B, int H, int W, int Cin, int Cout, void* stream);

/* ---------------------------------------------------------------- literal product form
 * The decoupled systems of Theorem 1 (eq. 8) exactly as the paper states them, built
 * by the recursion of Sec. 5: P^1 = A_1, P^n = P^{n-1} A_n, r~^1 = r^1,
 * r~^n = P^{n-1} r^n + r~^{n-1}; each P^n du^n = r~^n is scaled by diag(P^n) (the
 * preconditioner of Sec. 7) and solved by banded LU without pivoting (the direct solver
 * of Sec. 8), all levels in parallel. P^n has the 2n^2 + 2n + 1 diagonals of Remark 2
 * and is stored by diagonal offset; memory grows like (2/3) M^3 Ns doubles for the
 * products plus the dense bands (half width n nx) of the factorizations. The condition
 * number of P^n grows like K^n (Sec. 7, eq. 15): beyond eq. 15's bound on M the result
 * loses its digits, while pit_block_solve (nested form, same exact inverse) does not. */
typedef struct {
    int levels;           /* M */
    long long diagonals;  /* stored diagonals of P^M: 2M^2 + 2M + 1 */
    long long half_band;  /* half bandwidth of the factorization of P^M: M nx */
    double min_pivot;     /* smallest |pivot| met by the LU of the scaled systems */
    float ms_assemble, ms_products, ms_factor;  /* device time of the three stages */
} pit_product_info;

/* One product-form block solve: the Jacobians A_n at U_dev [M][Ns], right-hand sides
 * R_dev [M][Ns] (the tau-scaled residual, as for pit_block_solve), solution dU_dev
 * [M][Ns]. Allocates its workspace per call and synchronizes the stream.
 * PIT_EUNSUPPORTED for M > 180; PIT_ENOMEM when the products do not fit half the
 * free device memory; PIT_ECUDA when a band row of P^M does not fit shared memory. */
pit_status pit_product_form_solve(pit_ctx* ctx, const double* U_dev, const double* R_dev, double* dU_dev,
                                  pit_product_info* info);

/* Newton on the all-at-once system with the product-form block solve in every
 * iteration (the method as the paper states it), from the iterate in U_dev, until
 * ||R||_inf <= tol_res or newton_max iterations (context options). info as for pit_solve
 * (steps[k].ms_solve = products + factorization). */
pit_status pit_solve_product(pit_ctx* ctx, double* U_dev, pit_solve_info* info);

/* Limits of pit_block_solve_noalloc's built-in workspace. */
#define PIT_NOALLOC_MAX_NX 512       /* interior nodes per grid row */
#define PIT_NOALLOC_MAX_TEAM 160     /* CTAs sharing one level */
#define PIT_NOALLOC_MAX_LEVELS 4096  /* time levels M */

/* The paper has no counterpart to this entry point: it is pit_block_solve for
 * callers that cannot allocate device memory -- code that runs from a fixed
 * memory budget, a real-time loop that may not take an allocation's implicit
 * synchronisation, or an embedding that owns all GPU memory itself. It needs no
 * context and allocates nothing: the caller passes the raw Jacobian entries
 * coef_dev [5][M][Ns] (C, W, E, S, N of every A_n, e.g. from pit_assemble) and
 * R_dev [M][Ns]; dU_dev [M][Ns] receives the same block solve as pit_block_solve
 * (level tolerance eta, solver choice from opt, NULL = defaults).
 * The level chain's team workspace is a static device array of about 2.7 MB in
 * this library, held by every GPU that loads it until the process exits. The
 * first call on a device looks up that array's device address (with the device
 * current). Every call reads its status back and synchronises `stream`, so it must
 * never be made while `stream` is being captured into a CUDA graph: such a call
 * returns PIT_EUNSUPPORTED without doing anything. Sizes beyond the
 * workspace (nx > PIT_NOALLOC_MAX_NX, M > PIT_NOALLOC_MAX_LEVELS, a team larger
 * than PIT_NOALLOC_MAX_TEAM) return PIT_EUNSUPPORTED. All calls on a device share
 * the workspace: it is re-initialised at the start of each call, and calls that
 * overlap on the GPU race on it, so serialise them. Ordered on `stream`;
 * synchronises it before returning. err (may be NULL) receives a message of up to
 * err_len bytes. */
pit_status pit_block_solve_noalloc(int nx, int ny, int M, const double* coef_dev, const double* R_dev,
                                   double* dU_dev, double eta, const pit_options* opt, void* stream, char* err,
                                   int err_len);

/* Measurement helper, no counterpart in the paper: the fused multiply-add rate of
 * this GPU in TFLOP/s (FMA = 2 flops), precision 0 = FP64, 1 = FP32. A full-occupancy
 * grid runs eight independent FMA chains per thread; the best of five launches of
 * about 40 ms, timed with CUDA events on `stream`, is written to *tflops. It is the
 * peak that the FP64-bound level-chain kernels are compared against. Allocates a
 * small output buffer and synchronises `stream`. PIT_EINVAL for another precision. */
pit_status pit_probe_fma_peak(int precision, void* stream, double* tflops);

/* Message for the last failing call on ctx (never NULL). */
const char* pit_last_error(const pit_ctx* ctx);

/* Name of a status code (never NULL). */
const char* pit_status_string(pit_status s);

/* Release every device and host resource of ctx (NULL is ignored). */
void pit_destroy(pit_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PIT_H */
