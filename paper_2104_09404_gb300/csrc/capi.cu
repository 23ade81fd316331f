// C ABI of libmgrit.so (declared in include/mgrit.h).
//
// Level data in HBM (nx cells per row, row-major [time][cell]):
//   level 0     : its C-points live in u[1] (level-1 point i = level-0 C-point i);
//                 newC[0], phirow[0] ((nt/m+1) rows), cstep[0] (nt/m rows)
//   0 < l < L-1 : u[l], g[l] ((nt_l+1) rows), newC/phirow/cstep[l]
//   l = L-1     : u[L-1], g[L-1]
// Precision: g rows and the coarsest level are always FP64.  The other rows
// (u, newC, phirow, cstep) hold the sweep precision: FP64, or FP32 in the
// FP32-sweep mode, where u32c mirrors the coarsest rows in FP32 for the
// level above it.  Level-0 F-points are never stored (Sec. 3.2: the level-0
// F-relaxation of the interpolation is redundant before the next relaxation).
//
// One cycle = graph A (level-0 relaxation, residual + restriction to level
// 1, norm) + graph B (levels 1..L-2 relaxation + restriction, coarsest
// solve, interpolation back to level 1).  Both are captured once per
// context and replayed; the solve reads the residual norm between them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/mgrit.h"
#include "kernel_table.cuh"
#include "restrict.cuh"

using namespace mgrit;

namespace {

constexpr int MAXLEV = 32;

struct Launch {
    const void *slab;   // k_slab instance for (precision, scheme, flux, cells per thread); null: unsupported
    int threads;
    int cpt;
    size_t smem;
};

// sequential stepping on a thread-block cluster (coarsest solve, serial stepper)
struct ClusterLaunch {
    const void *fn;     // k_seq_cluster instance; null: single-CTA k_slab
    int K;              // CTAs in the cluster
    int threads;
    size_t smem;
};

}  // namespace

struct mgrit_ctx {
    int nx, nt, m, L, scheme, flux;
    mgrit_params p;
    int nt_l[MAXLEV], nC_l[MAXLEV];
    double dt_l[MAXLEV];
    Launch ln64, ln32;
    ClusterLaunch lc64, lc32;
    int f32;             // precision the workspaces were allocated for (1: FP32 sweeps)
    bool alloc;
    bool prepared;       // workspaces, graphs and an initial iterate exist
    bool have_state;     // a level-0 relaxation has produced newC[0]
    int device;
    void *u[MAXLEV];
    double *g[MAXLEV];
    void *newC[MAXLEV], *phirow[MAXLEV], *cstep[MAXLEV];
    float *u32c;         // FP32 mirror of the coarsest rows (FP32-sweep mode)
    float *ser32;        // one FP32 row for the FP32 serial stepper
    double *resid_rows;  // mgrit_residual scratch ((nt/m+1) rows, FP64)
    double *partials;
    int nparts;
    double *d_norm;
    double *h_norm;
    cudaStream_t cap;
    cudaGraphExec_t gA, gB;
    cudaEvent_t ev0, ev1;
    char err[256];
};

static char g_create_err[256] = "";

static int fail(mgrit_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MGRIT_ENOMEM : MGRIT_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                      \
    } while (0)

static const KernelTable &table()
{
    static KernelTable t = [] {
        KernelTable k;
        memset(&k, 0, sizeof k);
        fill_all(k);
        return k;
    }();
    return t;
}

// smallest cells-per-thread giving at most MAX_THREADS threads per CTA
static bool choose_launch(int nx, int scheme, int flux, int f32, Launch *ln)
{
    memset(ln, 0, sizeof *ln);
    const size_t smem = f32 ? slab_smem_bytes<float>(nx) : slab_smem_bytes<double>(nx);
    if (smem > 227 * 1024) return false;
    const int ncpt = f32 ? NCPT : NCPT64;
    for (int ci = 0; ci < ncpt; ++ci) {
        const int cpt = CPT_VALUES[ci];
        const int need = (nx + cpt - 1) / cpt;
        if (need <= MAX_THREADS) {
            ln->cpt = cpt;
            ln->threads = ((need + 31) / 32) * 32;
            ln->smem = smem;
            ln->slab = f32 ? table().slab32[scheme][flux][ci] : table().slab64[scheme][flux][ci];
            return true;
        }
    }
    return false;
}

static cudaError_t launch1(const void *fn, int grid, const Launch &ln, cudaStream_t s, void *arg)
{
    void *args[] = {arg};
    return cudaLaunchKernel(fn, dim3(grid), dim3(ln.threads), args, ln.smem, s);
}

extern "C" void mgrit_default_params(mgrit_params *p)
{
    p->T = 1.0;
    p->L = 1.0;
    p->relax = MGRIT_RELAX_FCF;
    p->cycle = 0;
    p->guess = MGRIT_GUESS_EQ17;
    p->numflux = MGRIT_LF_SPLIT;
    p->tol = 1e-10;
    p->max_iter = 64;
    p->precision = 64;
}

static int check_params(mgrit_ctx *ctx, const mgrit_params *p)
{
    if (!(p->T > 0) || !(p->L > 0) || !std::isfinite(p->T) || !std::isfinite(p->L))
        return fail(ctx, MGRIT_EINVAL, "T and L must be positive and finite");
    if (p->relax != MGRIT_RELAX_F && p->relax != MGRIT_RELAX_FCF)
        return fail(ctx, MGRIT_EINVAL, "relax must be F (0) or FCF (1)");
    if (p->cycle != 0) return fail(ctx, MGRIT_EINVAL, "only the V-cycle (0) is built");
    if (p->guess != MGRIT_GUESS_EQ17 && p->guess != MGRIT_GUESS_INJECT)
        return fail(ctx, MGRIT_EINVAL, "guess must be 0 or 1");
    if (p->numflux != MGRIT_LF_SPLIT && p->numflux != MGRIT_LF_STATE)
        return fail(ctx, MGRIT_EINVAL, "numflux must be 0 or 1");
    if (!(p->tol >= 0)) return fail(ctx, MGRIT_EINVAL, "tol must be >= 0");
    if (p->max_iter < 0 || p->max_iter > 254)
        return fail(ctx, MGRIT_EINVAL, "max_iter must be in [0, 254]");
    if (p->precision != 64 && p->precision != 32)
        return fail(ctx, MGRIT_EINVAL, "precision must be 64 or 32");
    if (p->precision == 64 && !ctx->ln64.slab)
        return fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP64 single-CTA slab limit", ctx->nx);
    if (p->precision == 32 && !ctx->ln32.slab)
        return fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP32 single-CTA slab limit", ctx->nx);
    return MGRIT_OK;
}

static void set_level_steps(mgrit_ctx *ctx)
{
    double dt = ctx->p.T / ctx->nt;
    for (int l = 0; l < ctx->L; ++l) {
        ctx->dt_l[l] = dt;
        dt *= ctx->m;
    }
}

extern "C" int mgrit_create(mgrit_ctx **out, int nx, int nt, int m, int levels, int scheme,
                            int flux)
{
    mgrit_ctx *ctx = nullptr;
    if (!out) return fail(ctx, MGRIT_EINVAL, "out is NULL");
    *out = nullptr;
    if (scheme != MGRIT_WENO5_SSPRK3 && scheme != MGRIT_FO_FE)
        return fail(ctx, MGRIT_EINVAL, "unknown scheme %d", scheme);
    if (flux != MGRIT_BURGERS && flux != MGRIT_ADVECTION)
        return fail(ctx, MGRIT_EINVAL, "unknown flux %d", flux);
    if (m < 2) return fail(ctx, MGRIT_EINVAL, "m must be >= 2");
    if (levels < 2 || levels >= MAXLEV) return fail(ctx, MGRIT_EINVAL, "levels must be in [2, 31]");
    if (nt < 1) return fail(ctx, MGRIT_EINVAL, "nt must be >= 1");
    if (nx < (scheme == MGRIT_WENO5_SSPRK3 ? 5 : 3))
        return fail(ctx, MGRIT_EINVAL, "nx too small for the scheme");
    long long div = 1;
    for (int l = 0; l < levels - 1; ++l) div *= m;
    if (div > nt || nt % div) return fail(ctx, MGRIT_EINVAL, "nt must be divisible by m^(levels-1)");
    Launch ln64, ln32;
    const bool ok64 = choose_launch(nx, scheme, flux, 0, &ln64);
    const bool ok32 = choose_launch(nx, scheme, flux, 1, &ln32);
    if (!ok64 && !ok32)
        return fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the single-CTA slab limit", nx);

    ctx = new (std::nothrow) mgrit_ctx;
    if (!ctx) return fail(nullptr, MGRIT_ENOMEM, "host allocation failed");
    memset(ctx, 0, sizeof *ctx);
    ctx->nx = nx;
    ctx->nt = nt;
    ctx->m = m;
    ctx->L = levels;
    ctx->scheme = scheme;
    ctx->flux = flux;
    ctx->ln64 = ln64;
    ctx->ln32 = ln32;
    mgrit_default_params(&ctx->p);
    if (!ok64) ctx->p.precision = 32;   // only FP32 sweeps fit in one CTA
    long long n = nt;
    for (int l = 0; l < levels; ++l) {
        ctx->nt_l[l] = (int)n;
        ctx->nC_l[l] = (int)(n / m);
        n /= m;
    }
    set_level_steps(ctx);
    *out = ctx;
    return MGRIT_OK;
}

static void free_workspaces(mgrit_ctx *ctx)
{
    if (ctx->gA) cudaGraphExecDestroy(ctx->gA);
    if (ctx->gB) cudaGraphExecDestroy(ctx->gB);
    ctx->gA = ctx->gB = nullptr;
    for (int l = 0; l < MAXLEV; ++l) {
        cudaFree(ctx->u[l]);
        cudaFree(ctx->g[l]);
        cudaFree(ctx->newC[l]);
        cudaFree(ctx->phirow[l]);
        cudaFree(ctx->cstep[l]);
        ctx->u[l] = ctx->newC[l] = ctx->phirow[l] = ctx->cstep[l] = nullptr;
        ctx->g[l] = nullptr;
    }
    cudaFree(ctx->u32c);
    cudaFree(ctx->ser32);
    cudaFree(ctx->resid_rows);
    cudaFree(ctx->partials);
    cudaFree(ctx->d_norm);
    ctx->u32c = nullptr;
    ctx->ser32 = nullptr;
    ctx->resid_rows = ctx->partials = ctx->d_norm = nullptr;
    if (ctx->h_norm) cudaFreeHost(ctx->h_norm);
    ctx->h_norm = nullptr;
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    ctx->cap = nullptr;
    ctx->ev0 = ctx->ev1 = nullptr;
    ctx->alloc = ctx->prepared = ctx->have_state = false;
}

extern "C" int mgrit_set_params(mgrit_ctx *ctx, const mgrit_params *p)
{
    if (!ctx || !p) return fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st = check_params(ctx, p);
    if (st) return st;
    const bool same_graph = ctx->p.T == p->T && ctx->p.L == p->L && ctx->p.relax == p->relax &&
                            ctx->p.guess == p->guess && ctx->p.numflux == p->numflux &&
                            ctx->p.precision == p->precision;
    if (ctx->alloc && (p->precision == 32) != (ctx->f32 != 0)) free_workspaces(ctx);
    ctx->p = *p;
    set_level_steps(ctx);
    if (!same_graph) {
        if (ctx->gA) cudaGraphExecDestroy(ctx->gA);
        if (ctx->gB) cudaGraphExecDestroy(ctx->gB);
        ctx->gA = ctx->gB = nullptr;
        ctx->prepared = false;
    }
    return MGRIT_OK;
}

static int dalloc(mgrit_ctx *ctx, void **ptr, size_t rows, size_t elem)
{
    CK(cudaMalloc(ptr, elem * rows * (size_t)ctx->nx));
    return MGRIT_OK;
}

// is level l's u stored in FP32?
static bool level_f32(const mgrit_ctx *ctx, int l) { return ctx->f32 && l < ctx->L - 1; }

// Cluster size for sequential stepping: the largest power of two K <= 16
// leaving at least 256 cells per CTA, reduced until the device can co-schedule
// one cluster of that shape.  nx < 512 keeps the single-CTA kernel.
static void choose_cluster(mgrit_ctx *ctx, int f32, ClusterLaunch *lc)
{
    lc->fn = nullptr;
    const int nx = ctx->nx;
    int K = 1;
    while (K < CLUSTER_MAX && nx / (2 * K) >= 256) K *= 2;
    for (; K >= 2; K /= 2) {
        const int nmax = (nx + K - 1) / K;
        const int cpt = nmax <= MAX_THREADS ? 1 : 2;
        if (nmax > 2 * MAX_THREADS) break;
        const void *fn = f32 ? table().seqc32[ctx->scheme][ctx->flux][cpt - 1]
                             : table().seqc64[ctx->scheme][ctx->flux][cpt - 1];
        const size_t smem = f32 ? cluster_smem_bytes<float>(nx, K) : cluster_smem_bytes<double>(nx, K);
        const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
        if (K > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))
            continue;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(K);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = K;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        lc->fn = fn;
        lc->K = K;
        lc->threads = threads;
        lc->smem = smem;
        return;
    }
    cudaGetLastError();   // clear a refused attribute or occupancy query
}

// sequential stepping in the precision of `lc`/`ln` (cluster if available)
static cudaError_t launch_seq(const ClusterLaunch &lc, const Launch &ln, cudaStream_t s, void *a)
{
    if (!lc.fn) return ln.slab ? launch1(ln.slab, 1, ln, s, a) : cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(lc.K);
    cfg.blockDim = dim3(lc.threads);
    cfg.dynamicSmemBytes = lc.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = lc.K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {a};
    return cudaLaunchKernelExC(&cfg, lc.fn, args);
}

static int ensure_alloc(mgrit_ctx *ctx)
{
    if (ctx->alloc) return MGRIT_OK;
    CK(cudaGetDevice(&ctx->device));
    ctx->f32 = ctx->p.precision == 32;
    const int L = ctx->L;
    const size_t es = ctx->f32 ? sizeof(float) : sizeof(double);
    int st;
    for (int l = 0; l < L - 1; ++l) {
        if ((st = dalloc(ctx, &ctx->newC[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = dalloc(ctx, &ctx->phirow[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = dalloc(ctx, &ctx->cstep[l], ctx->nC_l[l], es))) return st;
    }
    for (int l = 1; l < L; ++l) {
        const size_t el = level_f32(ctx, l) ? sizeof(float) : sizeof(double);
        if ((st = dalloc(ctx, &ctx->u[l], ctx->nt_l[l] + 1, el))) return st;
        if ((st = dalloc(ctx, (void **)&ctx->g[l], ctx->nt_l[l] + 1, sizeof(double)))) return st;
    }
    if (ctx->f32) {
        if ((st = dalloc(ctx, (void **)&ctx->u32c, ctx->nt_l[L - 1] + 1, sizeof(float)))) return st;
        if ((st = dalloc(ctx, (void **)&ctx->ser32, 1, sizeof(float)))) return st;
    }
    ctx->nparts = restrict_blocks(ctx->nC_l[0], ctx->nx);
    CK(cudaMalloc((void **)&ctx->partials, sizeof(double) * ctx->nparts));
    CK(cudaMalloc((void **)&ctx->d_norm, sizeof(double)));
    CK(cudaMallocHost((void **)&ctx->h_norm, sizeof(double)));
    CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
    if (ctx->ln64.slab)
        CK(cudaFuncSetAttribute(ctx->ln64.slab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ctx->ln64.smem));
    if (ctx->ln32.slab)
        CK(cudaFuncSetAttribute(ctx->ln32.slab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ctx->ln32.smem));
    choose_cluster(ctx, 0, &ctx->lc64);
    if (ctx->f32) choose_cluster(ctx, 1, &ctx->lc32);
    if (!ctx->ln64.slab && !ctx->lc64.fn)
        return fail(ctx, MGRIT_EINVAL, "no FP64 slab or cluster fits nx = %d for the coarsest solve",
                    ctx->nx);
    ctx->alloc = true;
    return MGRIT_OK;
}

// ---- individual kernel launches -------------------------------------------

template <typename R>
static SlabArgs<R> base_args(const mgrit_ctx *ctx, int mode, int l)
{
    SlabArgs<R> a;
    memset(&a, 0, sizeof a);
    a.mode = mode;
    a.nx = ctx->nx;
    a.m = ctx->m;
    a.nC = ctx->nC_l[l];
    a.fcf = ctx->p.relax == MGRIT_RELAX_FCF;
    a.numflux = ctx->p.numflux;
    a.dxinv = (R)(ctx->nx / ctx->p.L);
    a.dt = (R)ctx->dt_l[l];
    a.dtc = (R)(l + 1 < ctx->L ? ctx->dt_l[l + 1] : 0.0);
    return a;
}

// the buffer (and its precision) holding the level-l C-points that the
// level-l relaxation reads
static const void *cpoint_source(const mgrit_ctx *ctx, int l)
{
    if (l == 0) return (ctx->L == 2 && ctx->f32) ? (const void *)ctx->u32c : ctx->u[1];
    return ctx->u[l];
}

template <typename R>
static cudaError_t enqueue_relax_t(mgrit_ctx *ctx, int l, cudaStream_t s, const Launch &ln)
{
    SlabArgs<R> a = base_args<R>(ctx, MODE_RELAX, l);
    a.uC = static_cast<const R *>(cpoint_source(ctx, l));
    a.strideC = (long long)(l == 0 ? 1 : ctx->m) * ctx->nx;
    a.g = l == 0 ? nullptr : ctx->g[l];
    a.newC = static_cast<R *>(ctx->newC[l]);
    a.phirow = static_cast<R *>(ctx->phirow[l]);
    a.cstep = static_cast<R *>(ctx->cstep[l]);
    a.nrows_uC = a.nrows_newC = a.nrows_phirow = a.nC + 1;
    a.nrows_cstep = a.nC;
    a.nrows_g = ctx->nt_l[l] + 1;
    return launch1(ln.slab, a.nC + 1, ln, s, &a);
}

static cudaError_t enqueue_relax(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    return ctx->f32 ? enqueue_relax_t<float>(ctx, l, s, ctx->ln32)
                    : enqueue_relax_t<double>(ctx, l, s, ctx->ln64);
}

static cudaError_t enqueue_restrict(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    RestrictArgs a;
    memset(&a, 0, sizeof a);
    a.newC = ctx->newC[l];
    a.phirow = ctx->phirow[l];
    a.cstep = ctx->cstep[l];
    a.g = l == 0 ? nullptr : ctx->g[l];
    a.gn = ctx->g[l + 1];
    a.un = ctx->u[l + 1];
    a.partials = l == 0 ? ctx->partials : nullptr;
    a.nrows_g = ctx->nt_l[l] + 1;
    a.nx = ctx->nx;
    a.m = ctx->m;
    a.nC = ctx->nC_l[l];
    a.guess = ctx->p.guess;
    a.state_f32 = ctx->f32;
    a.un_f32 = level_f32(ctx, l + 1);
    const int blocks = l == 0 ? ctx->nparts : restrict_blocks(a.nC, a.nx);
    return launch_restrict(a, blocks, s);
}

// coarsest level, always FP64; in FP32-sweep mode its rows are then mirrored
// in FP32 for the level above
static cudaError_t enqueue_coarse(mgrit_ctx *ctx, cudaStream_t s)
{
    const int l = ctx->L - 1;
    SlabArgs<double> a = base_args<double>(ctx, MODE_SEQ, l);
    a.src = ctx->g[l];
    a.g = ctx->g[l];
    a.rows = static_cast<double *>(ctx->u[l]);
    a.nsteps = ctx->nt_l[l];
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    cudaError_t e = launch_seq(ctx->lc64, ctx->ln64, s, &a);
    if (e != cudaSuccess || !ctx->f32) return e;
    return launch_convert(ctx->u[l], 0, ctx->u32c, 1, (long long)(ctx->nt_l[l] + 1) * ctx->nx, s);
}

template <typename R>
static cudaError_t enqueue_interp_t(mgrit_ctx *ctx, int l, cudaStream_t s, const Launch &ln)
{
    SlabArgs<R> a = base_args<R>(ctx, MODE_INTERP, l);
    const void *coarse = (l + 1 == ctx->L - 1 && ctx->f32) ? (const void *)ctx->u32c : ctx->u[l + 1];
    a.uC = static_cast<const R *>(coarse);
    a.g = ctx->g[l];
    a.rows = static_cast<R *>(ctx->u[l]);
    a.nrows_uC = a.nC + 1;
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    return launch1(ln.slab, a.nC, ln, s, &a);
}

static cudaError_t enqueue_interp(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    return ctx->f32 ? enqueue_interp_t<float>(ctx, l, s, ctx->ln32)
                    : enqueue_interp_t<double>(ctx, l, s, ctx->ln64);
}

static cudaError_t enqueue_part_a(mgrit_ctx *ctx, cudaStream_t s)
{
    cudaError_t e;
    if ((e = enqueue_relax(ctx, 0, s))) return e;
    if ((e = enqueue_restrict(ctx, 0, s))) return e;
    return launch_norm(ctx->partials, ctx->nparts, ctx->d_norm, s);
}

static cudaError_t enqueue_part_b(mgrit_ctx *ctx, cudaStream_t s)
{
    cudaError_t e;
    for (int l = 1; l < ctx->L - 1; ++l) {
        if ((e = enqueue_relax(ctx, l, s))) return e;
        if ((e = enqueue_restrict(ctx, l, s))) return e;
    }
    if ((e = enqueue_coarse(ctx, s))) return e;
    for (int l = ctx->L - 2; l >= 1; --l)
        if ((e = enqueue_interp(ctx, l, s))) return e;
    return cudaSuccess;
}

static int capture(mgrit_ctx *ctx, cudaError_t (*fn)(mgrit_ctx *, cudaStream_t),
                   cudaGraphExec_t *out)
{
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = fn(ctx, ctx->cap);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(ctx, MGRIT_ECUDA, "graph capture: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, MGRIT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MGRIT_OK;
}

static int ensure_graphs(mgrit_ctx *ctx)
{
    int st;
    if (!ctx->gA && (st = capture(ctx, enqueue_part_a, &ctx->gA))) return st;
    if (!ctx->gB && (st = capture(ctx, enqueue_part_b, &ctx->gB))) return st;
    return MGRIT_OK;
}

// initial iterate: every level-0 C-point = u0; row 0 of every u_l and g_l = u0
static int init_iterate(mgrit_ctx *ctx, const double *u0, cudaStream_t s)
{
    const int nx = ctx->nx;
    const void *c0 = cpoint_source(ctx, 0);
    const int c0_f32 = ctx->f32;   // u[1] (FP32 unless coarsest) or the FP32 mirror
    CK(launch_broadcast_row(u0, const_cast<void *>(c0), c0_f32, nx, (long long)ctx->nC_l[0] + 1, s));
    for (int l = 1; l < ctx->L; ++l) {
        CK(cudaMemcpyAsync(ctx->g[l], u0, sizeof(double) * nx, cudaMemcpyDeviceToDevice, s));
        if (ctx->u[l] != c0) CK(launch_broadcast_row(u0, ctx->u[l], level_f32(ctx, l), nx, 1, s));
    }
    return MGRIT_OK;
}

extern "C" double mgrit_cycle_cell_updates(const mgrit_ctx *ctx)
{
    if (!ctx) return 0.0;
    const double m = ctx->m;
    double steps = 0.0;
    for (int l = 0; l < ctx->L - 1; ++l) {
        const double nc = ctx->nC_l[l];
        const double relax = ctx->p.relax == MGRIT_RELAX_FCF ? nc * m + nc * m : nc * m;
        steps += relax + nc;                        // + the coarse step for the FAS term
        if (l >= 1) steps += nc * (m - 1);          // interpolation F-relaxation
    }
    steps += ctx->nt_l[ctx->L - 1];                 // coarsest sequential solve
    return steps * ctx->nx;
}

static int prepare(mgrit_ctx *ctx, const double *u0_dev, cudaStream_t s)
{
    if (!u0_dev) return fail(ctx, MGRIT_EINVAL, "u0_dev is NULL");
    int st;
    if ((st = ensure_alloc(ctx))) return st;
    if ((st = ensure_graphs(ctx))) return st;
    if ((st = init_iterate(ctx, u0_dev, s))) return st;
    ctx->prepared = true;
    return MGRIT_OK;
}

// level-0 C-points after the last relaxation (rows first..first+nrows-1 of newC[0]) -> FP64 out
static int copy_out(mgrit_ctx *ctx, double *out, int first, int nrows, cudaStream_t s)
{
    const size_t off = (size_t)first * ctx->nx;
    const long long n = (long long)nrows * ctx->nx;
    if (ctx->f32)
        CK(launch_convert(static_cast<float *>(ctx->newC[0]) + off, 1, out, 0, n, s));
    else
        CK(cudaMemcpyAsync(out, static_cast<double *>(ctx->newC[0]) + off, sizeof(double) * n,
                           cudaMemcpyDeviceToDevice, s));
    return MGRIT_OK;
}

extern "C" int mgrit_solve(mgrit_ctx *ctx, const double *u0_dev, double *uC_out_dev,
                           double *uT_out_dev, void *stream, mgrit_stats *stats)
{
    if (!ctx) return MGRIT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st = prepare(ctx, u0_dev, s);
    if (st) return st;
    if (stats) memset(stats, 0, sizeof *stats);
    CK(cudaEventRecord(ctx->ev0, s));
    double hist[256];
    double r0 = 0.0;
    int k = 0;
    int status = MGRIT_OK;
    int stagnated = 0;
    double updates = 0.0;
    const double cyc = mgrit_cycle_cell_updates(ctx);
    const double relax0 = (double)ctx->nx * ctx->nC_l[0] *
                          ((ctx->p.relax == MGRIT_RELAX_FCF ? 2.0 : 1.0) * ctx->m + 1.0);
    for (;; ++k) {
        CK(cudaGraphLaunch(ctx->gA, s));
        updates += relax0;
        CK(cudaMemcpyAsync(ctx->h_norm, ctx->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double rk = *ctx->h_norm;
        if (k < 256) hist[k] = rk;
        if (stats && k < 256) stats->res_hist[k] = rk;
        if (k == 0) r0 = rk;
        if (rk < ctx->p.tol) { status = MGRIT_OK; break; }
        if (!std::isfinite(rk) || rk > 1e8 * r0) { status = MGRIT_EDIVERGED; break; }
        // FP32 sweeps: the FP64 residual of an FP32 iteration levels off near
        // FP32 rounding; stop once two cycles gain less than 10 %
        if (ctx->f32 && k >= 2 && k < 256 && rk > 0.9 * hist[k - 2]) {
            status = MGRIT_OK;
            stagnated = 1;
            break;
        }
        if (k >= ctx->p.max_iter) { status = MGRIT_ENOTCONV; break; }
        CK(cudaGraphLaunch(ctx->gB, s));
        updates += cyc - relax0;
    }
    CK(cudaEventRecord(ctx->ev1, s));
    if (uC_out_dev && (st = copy_out(ctx, uC_out_dev, 0, ctx->nC_l[0] + 1, s))) return st;
    if (uT_out_dev && (st = copy_out(ctx, uT_out_dev, ctx->nC_l[0], 1, s))) return st;
    CK(cudaStreamSynchronize(s));
    ctx->have_state = true;
    if (stats) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        stats->iters = k;
        stats->status = status;
        stats->t_total_ms = ms;
        stats->cell_updates = updates;
        stats->stagnated = stagnated;
    }
    if (status == MGRIT_EDIVERGED) fail(ctx, status, "diverged at cycle %d", k);
    if (status == MGRIT_ENOTCONV) fail(ctx, status, "not converged after %d cycles", k);
    return status;
}

extern "C" int mgrit_run_cycles(mgrit_ctx *ctx, const double *u0_dev, int ncycles, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (ncycles < 0) return fail(ctx, MGRIT_EINVAL, "ncycles must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int st = prepare(ctx, u0_dev, s);
    if (st) return st;
    for (int k = 0; k < ncycles; ++k) {
        CK(cudaGraphLaunch(ctx->gA, s));
        CK(cudaGraphLaunch(ctx->gB, s));
    }
    ctx->have_state = ncycles > 0;
    return MGRIT_OK;
}

extern "C" int mgrit_copy_cpoints(mgrit_ctx *ctx, double *uC_out_dev, void *stream)
{
    if (!ctx || !uC_out_dev) return fail(ctx, MGRIT_EINVAL, "NULL argument");
    if (!ctx->have_state) return fail(ctx, MGRIT_EINVAL, "no solve has run on this context");
    return copy_out(ctx, uC_out_dev, 0, ctx->nC_l[0] + 1, (cudaStream_t)stream);
}

extern "C" int mgrit_serial_step(mgrit_ctx *ctx, const double *u0_dev, double *uT_dev, int nsteps,
                                 void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!u0_dev || !uT_dev || nsteps < 0) return fail(ctx, MGRIT_EINVAL, "bad arguments");
    int st;
    if ((st = ensure_alloc(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->f32) {
        SlabArgs<double> a = base_args<double>(ctx, MODE_SEQ, 0);
        a.src = u0_dev;
        a.out = uT_dev;
        a.nsteps = nsteps;
        CK(launch_seq(ctx->lc64, ctx->ln64, s, &a));
        return MGRIT_OK;
    }
    // FP32 sweeps: step an FP32 copy of u0 and widen the result
    CK(launch_convert(u0_dev, 0, ctx->ser32, 1, ctx->nx, s));
    SlabArgs<float> a = base_args<float>(ctx, MODE_SEQ, 0);
    a.src = ctx->ser32;
    a.out = ctx->ser32;
    a.nsteps = nsteps;
    CK(launch_seq(ctx->lc32, ctx->ln32, s, &a));
    CK(launch_convert(ctx->ser32, 1, uT_dev, 0, ctx->nx, s));
    return MGRIT_OK;
}

extern "C" int mgrit_residual(mgrit_ctx *ctx, const double *uC_dev, double *norm_out, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!uC_dev || !norm_out) return fail(ctx, MGRIT_EINVAL, "NULL argument");
    if (!ctx->ln64.slab) return fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP64 slab limit", ctx->nx);
    int st;
    if ((st = ensure_alloc(ctx))) return st;
    if (!ctx->resid_rows &&
        (st = dalloc(ctx, (void **)&ctx->resid_rows, ctx->nC_l[0] + 1, sizeof(double))))
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    // always the FP64 operator: the residual of the FP64 discrete system
    SlabArgs<double> a = base_args<double>(ctx, MODE_RELAX, 0);
    a.uC = uC_dev;
    a.strideC = ctx->nx;
    a.fcf = 0;
    a.phirow = ctx->resid_rows;
    a.nrows_uC = a.nrows_phirow = a.nC + 1;
    CK(launch1(ctx->ln64.slab, a.nC, ctx->ln64, s, &a));
    RestrictArgs r;
    memset(&r, 0, sizeof r);
    r.newC = uC_dev;
    r.phirow = ctx->resid_rows;
    r.partials = ctx->partials;
    r.nx = ctx->nx;
    r.m = ctx->m;
    r.nC = ctx->nC_l[0];
    CK(launch_restrict(r, ctx->nparts, s));
    CK(launch_norm(ctx->partials, ctx->nparts, ctx->d_norm, s));
    CK(cudaMemcpyAsync(ctx->h_norm, ctx->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *norm_out = *ctx->h_norm;
    return MGRIT_OK;
}

extern "C" int mgrit_launch_kernel(mgrit_ctx *ctx, int which, int level, int reps, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!ctx->prepared) return fail(ctx, MGRIT_EINVAL, "no solve has run on this context");
    if (reps < 0) return fail(ctx, MGRIT_EINVAL, "reps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ctx->L;
    for (int r = 0; r < reps; ++r) {
        switch (which) {
        case 0:
            if (level < 0 || level > L - 2) return fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_relax(ctx, level, s));
            break;
        case 1:
            if (level < 0 || level > L - 2) return fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_restrict(ctx, level, s));
            break;
        case 2:
            CK(enqueue_coarse(ctx, s));
            break;
        case 3:
            if (level < 1 || level > L - 2) return fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_interp(ctx, level, s));
            break;
        default:
            return fail(ctx, MGRIT_EINVAL, "unknown kernel id %d", which);
        }
    }
    return MGRIT_OK;
}

extern "C" int mgrit_query(const mgrit_ctx *ctx, int what)
{
    if (!ctx) return -1;
    const bool f32 = ctx->alloc ? ctx->f32 != 0 : ctx->p.precision == 32;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    const ClusterLaunch &lc = f32 ? ctx->lc32 : ctx->lc64;
    switch (what) {
    case 0: return ln.cpt;
    case 1: return ln.threads;
    case 2: return ctx->alloc ? (lc.fn ? lc.K : 1) : 0;
    default: return -1;
    }
}

extern "C" const char *mgrit_last_error(const mgrit_ctx *ctx)
{
    return ctx ? ctx->err : g_create_err;
}

extern "C" void mgrit_destroy(mgrit_ctx *ctx)
{
    if (!ctx) return;
    free_workspaces(ctx);
    delete ctx;
}
