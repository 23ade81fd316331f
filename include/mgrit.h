/*
 * mgrit.h -- C ABI of libmgrit.so: GB300 (sm_103a) MGRIT for 1D periodic
 * scalar conservation laws, after Danieli & MacLachlan, "Multigrid Reduction
 * in Time for non-linear hyperbolic equations" (arXiv:2104.09404).
 *
 * Problem (Sec. 2, Eq. consLaw): u_t + f(u)_x = 0 on [0, L) x [0, T],
 * periodic, f = u^2/2 (Burgers, Eq. burgers) or f = u (advection, speed 1).
 * Space: nx finite-volume cells of width dx = L/nx (Sec. 2.1, Eq. spaceDisc),
 * WENO5-JS reconstruction (Sec. 2.1.1, k = 2) or first-order (k = 0), global
 * Lax-Friedrichs flux (Sec. 2.1.2).  Time: nt steps of dt = T/nt with SSPRK3
 * (Eq. SSPRK3) or forward Euler (Eq. SSPRK1).
 * Solver: FAS MGRIT V-cycle (Sec. 3.2, Algorithm 1) with coarsening factor m
 * in time only, rediscretised coarse integrators Phi_l with step dt*m^l
 * (Sec. 3.3), F- or FCF-relaxation (Eq. relaxation), injection restriction
 * with the coarse initial guess of Eq. (restriction::u) or plain injection,
 * sequential coarsest solve (Eq. coarseCorr), ideal interpolation
 * (Eq. interpolation).
 *
 * Conventions for every entry point:
 *  - Arrays passed in and out are FP64, row-major [time][cell]; one row is nx
 *    contiguous cell values (cell i covers [i dx, (i+1) dx)).  Pointers named *_dev are
 *    device pointers on the current CUDA device; the caller allocates and
 *    owns them.  The context owns all level workspaces and CUDA graphs.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; functions that return a host value synchronise it.
 *  - Return value: MGRIT_OK or a negative MGRIT_E* code; nothing aborts.
 *    mgrit_last_error() gives a one-line description of the last failure.
 *  - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef MGRIT_H
#define MGRIT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgrit_ctx mgrit_ctx;

enum {
    MGRIT_OK = 0,
    MGRIT_EINVAL = -1,     /* bad argument or unsupported size */
    MGRIT_ECUDA = -2,      /* a CUDA runtime call failed */
    MGRIT_ENOMEM = -3,     /* device or pinned-host allocation failed */
    MGRIT_EDIVERGED = -4,  /* residual not finite or > 1e8 x first residual */
    MGRIT_ENOTCONV = -5,   /* max_iter cycles without reaching tol */
    MGRIT_ETIMEOUT = -6    /* a bounded device wait gave up (see mgrit_sync_status) */
};

/* spatial reconstruction + time integrator (Sec. 2.1.1, Sec. 2.2), or the
 * classical Lax-Friedrichs + forward Euler scheme of Sec. 3.3 Eq. (fineLF),
 * u_i <- (u_{i+1} + u_{i-1})/2 - dt (f(u_{i+1}) - f(u_{i-1}))/(2 dx)
 * (FP64, single-CTA sequential solves; numflux does not apply) */
enum { MGRIT_WENO5_SSPRK3 = 0, MGRIT_FO_FE = 1, MGRIT_LF_FE = 2 };
/* physical flux f (Sec. 2): Burgers u^2/2, or linear advection with speed 1 */
enum { MGRIT_BURGERS = 0, MGRIT_ADVECTION = 1 };
/* numerical flux (Sec. 2.1.2): global Lax-Friedrichs splitting
 * f^{+/-} = (f(u) +/- alpha u)/2 reconstructed left/right-biased, or the
 * state form of Eq. (LFflux) with the dissipative sign; alpha is the
 * global maximum of |f'| over the stage input (split) or over all
 * reconstructed states (state form), recomputed at every RK stage; or
 * Roe's flux on the reconstructed states with the Harten-Hyman entropy fix
 * (Eq. roeflux; Roe speed (u^+ + u^-)/2 for Burgers, 1 for advection):
 * F = (f(u^-) + f(u^+))/2 - q (u^+ - u^-)/2 with q = |lam|, or
 * (lam^2/delta + delta)/2 when |lam| < delta = max(0, lam - f'(u^-), f'(u^+) - lam) */
enum { MGRIT_LF_SPLIT = 0, MGRIT_LF_STATE = 1, MGRIT_ROE = 2 };
enum { MGRIT_RELAX_F = 0, MGRIT_RELAX_FCF = 1 };         /* Sec. 3.2 */
enum { MGRIT_GUESS_EQ17 = 0, MGRIT_GUESS_INJECT = 1 };   /* Eq. restriction::u */
enum { MGRIT_CYCLE_V = 0, MGRIT_CYCLE_F = 1 };           /* Algorithm 1; Sec. 3.2 */
/* coarse integrators (Sec. 3.3): rediscretisation with dt m^l, or, for
 * MGRIT_LF_FE, the integrators matched to M = m^l fine steps (dt the fine step):
 *   PSI0  E^M u - M dt D f(u)                          (Eq. coarseLFord0)
 *   PSI1  E^M u - dt sum_{i=1..M} E^{i-1} D f(E^{M-i} u)  (Eqs. coarseLFord1, fineLFxM)
 * with (E v)_i = (v_{i+1} + v_{i-1})/2 and (D v)_i = (v_{i+1} - v_{i-1})/(2 dx) */
enum { MGRIT_COARSE_REDISC = 0, MGRIT_COARSE_PSI0 = 1, MGRIT_COARSE_PSI1 = 2 };

typedef struct {
    double T;        /* final time (default 1) */
    double L;        /* domain length (default 1) */
    int relax;       /* MGRIT_RELAX_F / MGRIT_RELAX_FCF (default FCF) */
    int cycle;       /* MGRIT_CYCLE_V (Algorithm 1, default) or MGRIT_CYCLE_F (the
                        F-cycle of Sec. 3.2: below each level an F-cycle, then
                        one V-cycle) */
    int guess;       /* MGRIT_GUESS_EQ17 (default) / MGRIT_GUESS_INJECT */
    int numflux;     /* MGRIT_LF_SPLIT (default) / MGRIT_LF_STATE / MGRIT_ROE */
    double tol;      /* stop when the level-0 residual 2-norm < tol (default 1e-10) */
    int max_iter;    /* cycles before MGRIT_ENOTCONV (default 64, at most 254) */
    int precision;   /* 64: every sweep in FP64 (default when nx fits an FP64 slab).
                        32: relaxation and interpolation sweeps in FP32; the FAS
                        tau term (g rows), residual, norm, convergence test and
                        the coarsest sequential solve stay FP64.  The FP64
                        residual of an FP32 iteration levels off near FP32
                        rounding, so a solve also stops (MGRIT_OK, stats.stagnated
                        = 1) once two cycles reduce it by less than 10 %.
                        MGRIT_LF_FE accepts 64 only. */
    int coarse;      /* MGRIT_COARSE_REDISC (default), or PSI0 / PSI1 with the
                        MGRIT_LF_FE scheme (MGRIT_EINVAL otherwise) */
    int chunk_clusters; /* 1 (default): the relaxation / interpolation chunks of
                        a level whose chunks alone would leave SMs idle run
                        on thread-block clusters (mgrit_query 100 + l); and
                        with the WENO5 split form and nx > 8192, the chunks of
                        the other levels run on clusters of 2 or 4 CTAs of
                        the one-CTA slab's layout where that was timed faster
                        when the workspaces were allocated (mgrit_query
                        200 + l); 2 or 4: as 1, with those clusters taken
                        without timing, of 2 or 4 CTAs; 0: one CTA per chunk
                        wherever a slice fits one CTA.  FP64 slices beyond
                        one CTA use clusters either way. */
    int seq_stepper; /* kernel of the sequential chains (the coarsest solve and
                        mgrit_serial_step): 0 (default) the fastest of those
                        that fit, as timed when the workspaces are allocated;
                        1: one CTA; 2: a thread-block cluster; 3: the grid
                        stepper (split numerical flux).  A choice that does not
                        fit this nx falls back to the default.  All of them
                        perform the same floating-point operations per cell,
                        so their results are bit-identical. */
} mgrit_params;

typedef struct {
    int iters;            /* completed cycles when the solve stopped */
    int status;           /* same code as the return value */
    double res_hist[256]; /* res_hist[k] = residual 2-norm after the level-0
                             relaxation of cycle k, k = 0..iters */
    double t_total_ms;    /* device time of the solve (CUDA events) */
    double cell_updates;  /* cells x Phi applications executed on the GPU */
    int stagnated;        /* 1 if an FP32-sweep solve stopped on stagnation */
} mgrit_stats;

/* Fill *p with the defaults listed in mgrit_params. */
void mgrit_default_params(mgrit_params *p);

/*
 * Create a solver for nx cells, nt fine steps, coarsening factor m and
 * `levels` time levels (level l has nt/m^l steps).  Requires m >= 2,
 * levels >= 2, nt divisible by m^(levels-1), nx >= 5 (WENO5) or nx >= 3
 * (first order, classical Lax-Friedrichs), and nx <= 16384 (MGRIT_EINVAL
 * otherwise).  One CTA holds a slice of up to 8192 cells in FP64 and 16384 in
 * FP32; wider FP64 slices (WENO5 and first order) run every chunk on a
 * thread-block cluster, and the classical Lax-Friedrichs scheme stops at
 * 8192.  Device memory is allocated on the current device at the first solve.  Sec. 3.1 (C/F splitting, time chunks of m
 * steps); Eq. (monolithicSystem) for nt and the time grid.
 */
int mgrit_create(mgrit_ctx **out, int nx, int nt, int m, int levels, int scheme, int flux);

/* Replace the solver parameters (validated; MGRIT_EINVAL on bad values). */
int mgrit_set_params(mgrit_ctx *ctx, const mgrit_params *p);

/*
 * FAS MGRIT V-cycle solve (Algorithm 1) from u0_dev (nx values, cell
 * averages of the initial condition).  The level-0 initial iterate has every
 * C-point equal to u0.  Cycle k relaxes level 0, forms the residual
 *   r^i = Phi_0(u^{mi-1}) - u^{mi},  i = 1..nt/m,
 * and stops if ||r||_2 < tol; else it restricts (Eqs. restriction::rhs,
 * restriction::u), recurses and interpolates (Eq. interpolation).
 * Outputs (device, may be NULL): uC_out_dev = (nt/m + 1) x nx C-point
 * states after the last relaxation; uT_out_dev = the state at T (nx).
 * Returns MGRIT_OK, MGRIT_EDIVERGED or MGRIT_ENOTCONV (outputs written in
 * all three cases), or an error.  Synchronises `stream` once per cycle to
 * read the residual.  stats may be NULL.
 */
int mgrit_solve(mgrit_ctx *ctx, const double *u0_dev, double *uC_out_dev, double *uT_out_dev,
                void *stream, mgrit_stats *stats);

/*
 * Run exactly `ncycles` V-cycles from the initial iterate built from u0_dev,
 * with no stopping test and no host synchronisation (throughput
 * measurement).  The C-point states after the last level-0 relaxation are
 * left in the context (read them with mgrit_solve's outputs semantics via
 * mgrit_copy_cpoints).  Asynchronous on `stream`.
 */
int mgrit_run_cycles(mgrit_ctx *ctx, const double *u0_dev, int ncycles, void *stream);

/* Copy the C-point states after the last level-0 relaxation
 * ((nt/m + 1) x nx) to uC_out_dev.  Asynchronous on `stream`. */
int mgrit_copy_cpoints(mgrit_ctx *ctx, double *uC_out_dev, void *stream);

/*
 * Sequential fine time-stepping: uT_dev = Phi_0^nsteps(u0_dev), i.e. forward
 * substitution of Eq. (monolithicSystem).  Baseline for time-to-tolerance.
 * Steps in the context's sweep precision (FP32 rounds u0 once on entry).
 * u0_dev and uT_dev hold nx values and may alias.  Asynchronous.
 */
int mgrit_serial_step(mgrit_ctx *ctx, const double *u0_dev, double *uT_dev, int nsteps,
                      void *stream);

/*
 * Level-0 residual 2-norm of given C-point states uC_dev ((nt/m+1) x nx):
 *   ||r||_2,  r^i = Phi_0^m(u^{m(i-1)}) - u^{mi},  i = 1..nt/m
 * (the fine-level residual of the Schur system, Eq. schurComplement),
 * always with the FP64 operator (also for an FP32-sweep context, so it
 * measures FP32 results against the FP64 discrete system).  Requires nx to
 * fit an FP64 slab.  Writes the host double *norm_out; synchronises `stream`.
 */
int mgrit_residual(mgrit_ctx *ctx, const double *uC_dev, double *norm_out, void *stream);

/*
 * Profiling hook: launch one named kernel of the V-cycle `reps` times on
 * `stream` with the context's current level data, so that a caller can
 * time it with CUDA events.  which = 0: level-`level` relaxation;
 * 1: level-`level` residual/restriction; 2: coarsest solve;
 * 3: level-`level` interpolation (level >= 1).  Requires a prior
 * mgrit_solve or mgrit_run_cycles (ncycles = 0 is enough: it allocates the
 * workspaces and loads the initial iterate).  Asynchronous.
 */
int mgrit_launch_kernel(mgrit_ctx *ctx, int which, int level, int reps, void *stream);

/*
 * Measurement aid (the paper has no counterpart): the multiply-add throughput
 * of one SIMT pipe on the current device, the roofline denominator of the
 * arithmetic-bound sweeps.  kind = 0: FP64 fused multiply-add; 1: FP32;
 * 2: FP32 on packed pairs (one instruction, two multiply-adds).  Launches
 * blocks_per_sm x SMs CTAs of 256 threads, each thread running 8 independent
 * chains of 64 x iters multiply-adds, times the launch with CUDA events on
 * `stream` and writes the rate in flop/s (one multiply-add = 2 flops) to the
 * host double *flops_out.  Synchronises `stream`.  MGRIT_EINVAL for
 * kind outside 0..2, iters < 1 or blocks_per_sm outside 1..64.
 */
int mgrit_fma_probe(int kind, int iters, int blocks_per_sm, double *flops_out, void *stream);

/*
 * Allocation-free variant of mgrit_residual (the paper has no counterpart:
 * this is a deployment convenience).  Some callers cannot call cudaMalloc:
 * code that runs while the application owns all device memory through its
 * own pool or fixed budget (a plugin inside a host framework), code that must
 * not trigger the allocator's implicit device synchronisation inside a
 * latency-critical loop, and code that only has a stream and pointers handed
 * to it.  This entry point needs no context and allocates nothing: the Phi^m
 * rows and norm partials it needs live in one static device array of
 * MGRIT_STATIC_SCRATCH_DOUBLES + 2048 doubles (16 MiB + 16 KiB), which every
 * GPU that loads the library holds until the process exits.
 *
 *   uC_dev   (nt/m + 1) x nx C-point states (device, caller-owned, read only)
 *   norm_dev one device double that receives ||r||_2, with r as in
 *            mgrit_residual (caller-owned output)
 *   the other arguments as in mgrit_create / mgrit_params (dx = L/nx,
 *   dt = T/nt), with two restrictions: scheme MGRIT_WENO5_SSPRK3 or
 *   MGRIT_FO_FE (not MGRIT_LF_FE), and nx at most 8192 (the one-CTA FP64
 *   slab; wider slices, which mgrit_residual steps on clusters, are refused).
 *
 * Returns MGRIT_EINVAL for bad arguments, for the cases above, or when
 * (nt/m + 1) * nx exceeds MGRIT_STATIC_SCRATCH_DOUBLES (nothing is launched),
 * MGRIT_ECUDA if a launch fails.  Asynchronous on `stream`; the caller
 * reads norm_dev after synchronising.  Every call looks up the array's device
 * address (cudaGetSymbolAddress, with the caller's device current), so the
 * entry point keeps working after a device reset; the first call on each
 * device also raises the kernel's shared-memory limit.  Every call shares
 * the one array, so calls that overlap on the GPU (other streams, other host
 * threads) race; each call overwrites every scratch value it reads before
 * reading it, so no state carries over between calls.
 */
#define MGRIT_STATIC_SCRATCH_DOUBLES (1 << 21)
int mgrit_residual_static(int nx, int nt, int m, int scheme, int flux, int numflux, double T,
                          double L, const double *uC_dev, double *norm_dev, void *stream);

/*
 * Sequential stepping (the coarsest solve and mgrit_serial_step) runs, where
 * it measured faster at allocation, on a grid of up to one CTA per SM that
 * exchange boundary cells through global memory: once per Runge-Kutta stage
 * each CTA waits for the values it reads (its neighbours' boundary cells and,
 * with Burgers, every CTA's partial maximum of |f'|) (split numerical flux;
 * mgrit_query 3).  Every wait is bounded (0.5 s): a wait that gives up ends
 * the launch and sets a flag, which mgrit_solve reports as MGRIT_ETIMEOUT.
 * This call synchronises `stream` and returns MGRIT_ETIMEOUT (clearing the
 * flag) if a wait of an earlier asynchronous call on the context gave up,
 * else MGRIT_OK.
 */
int mgrit_sync_status(mgrit_ctx *ctx, void *stream);

/*
 * Test hook for the bounded waits above: launches the grid stepper for one
 * step with one CTA that never publishes its first stage, so the waits of the
 * CTAs that read it run out (and then those of their readers); returns what
 * mgrit_sync_status then returns (MGRIT_ETIMEOUT).  The context stays usable.  MGRIT_EINVAL if the context
 * does not use the grid stepper.
 */
int mgrit_test_grid_timeout(mgrit_ctx *ctx, void *stream);

/* Launch shape chosen for this context (for reports and tests):
 * what = 0: cells per thread of the slab kernel; 1: threads per CTA;
 * 2: CTAs per thread-block cluster used for sequential stepping (the
 * coarsest solve and mgrit_serial_step; 1 = a single CTA, 0 = the grid
 * stepper), known after the first call that allocates (0 before);
 * 3: CTAs of the grid stepper used for sequential stepping (0: not used); 100 + l (0 <= l <= levels-2): CTAs
 * per cluster of each relaxation / interpolation chunk of level l (1 = one
 * CTA per chunk; clusters are used where a level's chunks alone leave SMs
 * idle, and for FP64 slices beyond one CTA), 0 before the first allocating
 * call; 200 + l: 1 if those clusters hold run-major slabs (chunk_clusters),
 * else 0.  -1 for an unknown `what`. */
int mgrit_query(const mgrit_ctx *ctx, int what);

/* Cells x Phi applications of one cycle (V or F, for throughput figures). */
double mgrit_cycle_cell_updates(const mgrit_ctx *ctx);

/* ------------------------------------------------------------------------
 * Discrete adjoint (the paper has no adjoint: these entry points
 * differentiate the discrete scheme above, for gradients of an objective
 * J(u^nt) with respect to u^0).  The transpose of the derivative of one step
 * Phi (Eq. SSPRK3 or SSPRK1, through Eq. spaceDisc, the WENO weights of
 * Sec. 2.1.1 and the global Lax-Friedrichs splitting of Sec. 2.1.2, with
 * alpha = max|f'| differentiated at its first maximising cell) is applied
 * stage by stage with the forward stage states recomputed.  Split numerical
 * flux only (MGRIT_LF_SPLIT; MGRIT_EINVAL otherwise); FP64 in every
 * precision mode; nx <= 16384 (MGRIT_EINVAL otherwise).  One CTA holds a
 * transposed step of up to 4096 cells; wider slices, and the chunks of levels
 * whose chunks alone would leave SMs idle (unless chunk_clusters = 0), run on
 * thread-block clusters of up to 16 CTAs x 1024 cells.  Workspaces (the
 * regenerated fine trajectory, nt x nx, and the adjoint levels) are
 * allocated on the first call.
 * ------------------------------------------------------------------------ */

/* out_dev = Phi'(u_dev)^T lam_dev for one fine step (dt = T/nt).  Each
 * argument holds nx values; any of them may alias.  Asynchronous. */
int mgrit_step_vjp(mgrit_ctx *ctx, const double *u_dev, const double *lam_dev, double *out_dev,
                   void *stream);

/* Serial adjoint with C-point checkpointing: lam0_dev = dJ/du^0 given
 * lamT_dev = dJ/du^nt, through nt fine steps from u0_dev.  One CTA steps
 * forward keeping u^{mj}, j < nt/m, then for each chunk from the last it
 * recomputes the chunk's m states from its checkpoint and applies their m
 * transposed steps backward; for nx >= 512 on a thread-block cluster of up to
 * 16 CTAs, its size timed when the adjoint workspaces are allocated
 * (mgrit_adjoint_query(ctx, 2)).  Asynchronous.  Baseline for
 * mgrit_adjoint. */
int mgrit_adjoint_serial(mgrit_ctx *ctx, const double *u0_dev, const double *lamT_dev,
                         double *lam0_dev, void *stream);

/*
 * Adjoint MGRIT: lam^n = Phi'(u^n)^T lam^{n+1}, lam^nt = lamT_dev, solved
 * backward in time by the V-cycle of Algorithm 1 (same levels, m, relax,
 * guess, tol, max_iter as the context).  In reversed time k = nt - n the
 * system has the block-bidiagonal form of Eq. (monolithicSystem), so the
 * V-cycle applies unchanged with the propagator of level l = the transposed
 * linearisation of Phi_l (step dt m^l) at the forward state of the coarse
 * point: the fine states on level 0 and the injected forward C-states on
 * the coarse levels.
 *   uC_dev    forward C-point checkpoints ((nt/m + 1) x nx), e.g. the uC
 *             output of mgrit_solve; the fine states between them are
 *             regenerated by one parallel launch (u^{mj+r} = Phi^r(uC_j))
 *   lamT_dev  dJ/du^nt (nx)
 *   lam0_dev  output dJ/du^0 (nx), may be NULL
 *   lamC_dev  output (nt/m + 1) x nx, row i = lam at forward point m i,
 *             may be NULL
 * The residual is the level-0 adjoint residual after each relaxation, with
 * the stopping, divergence and iteration rules of mgrit_solve.  Returns
 * MGRIT_OK, MGRIT_EDIVERGED or MGRIT_ENOTCONV (outputs written in all
 * three cases) or an error.  Synchronises `stream` once per cycle.
 */
int mgrit_adjoint(mgrit_ctx *ctx, const double *uC_dev, const double *lamT_dev, double *lam0_dev,
                  double *lamC_dev, void *stream, mgrit_stats *stats);

/* Adjoint launch shape: what = 0 cells per thread, 1 threads per CTA of
 * the one-CTA adjoint slab (0 when the context's nx or numerical flux has
 * none); 2 CTAs per thread-block cluster of the sequential adjoint chains
 * (the coarsest adjoint solve and mgrit_adjoint_serial; 1 = a single CTA);
 * 100 + l (0 <= l <= levels-2): CTAs per cluster of each adjoint chunk of
 * level l (1 = one CTA per chunk); 2 and 100 + l are known after the first
 * adjoint call (0 before); -1 otherwise. */
int mgrit_adjoint_query(const mgrit_ctx *ctx, int what);

/* ------------------------------------------------------------------------
 * Batches: many independent problems advanced together (the paper treats
 * one problem at a time; batching is a throughput feature of this library).
 * Every instance has its own nx, nt, m, levels, flux and T (WENO5/SSPRK3
 * only); the other parameters are shared, the cycle (V or F) included.  Each
 * phase of a cycle is one launch per launch class (flux x CTA shape) over the
 * work items of all instances, and a cycle is two CUDA graphs, as for one
 * instance.  V-cycle phases align the instances by level; F-cycle phases
 * merge each instance's own launch order (one phase per operation kind that
 * most instances have next).
 * ------------------------------------------------------------------------ */
typedef struct mgrit_batch mgrit_batch;

typedef struct {
    int nx, nt, m, levels;   /* as in mgrit_create */
    int scheme;              /* MGRIT_WENO5_SSPRK3 */
    int flux;                /* MGRIT_BURGERS / MGRIT_ADVECTION */
    double T;                /* final time of this instance */
} mgrit_instance;

/* Create a batch of n instances (nx <= 8192 each; params may be NULL for
 * defaults; params->T is ignored, each instance has its own).  Allocates
 * every instance's workspaces on the current device and captures the
 * graphs.  MGRIT_EINVAL names the offending instance in mgrit_last_error(NULL). */
int mgrit_batch_create(mgrit_batch **out, const mgrit_instance *inst, int n,
                       const mgrit_params *params);

/* Exactly ncycles cycles (V or F) of every instance from u0_dev[i] (host array of n
 * device pointers).  Asynchronous. */
int mgrit_batch_run_cycles(mgrit_batch *b, const double *const *u0_dev, int ncycles, void *stream);

/* Solve every instance with the stopping rules of mgrit_solve, applied per
 * instance; an instance that has stopped is masked out on the device while
 * the others continue.  uT_dev[i] (may be NULL) receives u(T) of instance i;
 * status[i], iters[i], final_res[i] (each may be NULL) the per-instance
 * outcome.  Synchronises `stream` once per cycle. */
int mgrit_batch_solve(mgrit_batch *b, const double *const *u0_dev, double *const *uT_dev,
                      int *status, int *iters, double *final_res, void *stream);

/* Autotuner, each stage keeping the fastest candidate by CUDA-event timing
 * (reps >= 1 timed launches per candidate):
 *   1. CTA shape: for each group of instances with equal (flux, nx), the
 *      level-0 relaxation with 1x, 2x and 4x the minimal cells per thread;
 *   2. cluster shape of the coarsest solves, one policy for all instances
 *      timed on the whole coarsest phase: the single-instance occupancy rule
 *      K0 (nx >= 512), K0/2, 2 K0 (at most 16), or one CTA each;
 *   3. end to end: whole cycles with the policy of stage 2 and with the rule.
 * Slabs per CTA stay at one: a persistent variant (CTAs looping over work
 * items) was slower at every setting.  The graphs are then rebuilt.
 * Synchronises `stream`. */
int mgrit_batch_autotune(mgrit_batch *b, const double *const *u0_dev, int reps, void *stream);

/* Cells x Phi applications of one cycle (V or F) of all instances. */
double mgrit_batch_cycle_cell_updates(const mgrit_batch *b);

/* Profiling hook (as mgrit_launch_kernel): the batched level-0 relaxation of
 * every instance (Sec. 3.2: the FCF or F sweep of every chunk, in the
 * launches a cycle uses), `reps` times on `stream` from the instances'
 * current level-0 C-points, overwriting the level-0 relaxation outputs as a
 * cycle's first phase does.  Requires a prior mgrit_batch_run_cycles or
 * mgrit_batch_solve.  Synchronises `stream` (its launch tables are freed
 * afterwards).  MGRIT_EINVAL for reps < 1. */
int mgrit_batch_launch_relax(mgrit_batch *b, int reps, void *stream);

/* what = 0: cells per thread, 1: threads per CTA, 2: levels of instance i,
 * 3: slabs per CTA (always 1), 4: CTAs per cluster of its coarsest solve
 * (1 = one CTA); -1 for an unknown `what` or instance. */
int mgrit_batch_query(const mgrit_batch *b, int instance, int what);

/* C-points of instance i after its last level-0 relaxation (as
 * mgrit_copy_cpoints). */
int mgrit_batch_copy_cpoints(mgrit_batch *b, int instance, double *uC_out_dev, void *stream);

const char *mgrit_batch_last_error(const mgrit_batch *b);
void mgrit_batch_destroy(mgrit_batch *b);

/* One-line description of the last error on ctx (or of the last failed
 * mgrit_create when ctx is NULL). */
const char *mgrit_last_error(const mgrit_ctx *ctx);

/* Free every device/host resource of ctx (NULL is allowed). */
void mgrit_destroy(mgrit_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MGRIT_H */
