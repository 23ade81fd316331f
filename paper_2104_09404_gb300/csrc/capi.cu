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

#include "ctx.cuh"
#include "kernel_table.cuh"
#include "restrict.cuh"

using namespace mgrit;

static char g_create_err[256] = "";

int mgrit_fail(mgrit_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

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

// smallest cells-per-thread giving at most MAX_THREADS threads per CTA; FP64
// WENO5 slabs start at 4, so that every shape forms the interface quads of
// split_flux_quad (and gives the same bits)
static bool choose_launch(int nx, int scheme, int flux, int f32, Launch *ln)
{
    memset(ln, 0, sizeof *ln);
    const int ncpt = f32 ? NCPT : NCPT64;
    for (int ci = !f32 && scheme == MGRIT_WENO5_SSPRK3 ? 2 : 0; ci < ncpt; ++ci) {
        const int cpt = CPT_VALUES[ci];
        const int need = (nx + cpt - 1) / cpt;
        if (need <= MAX_THREADS) {
            const int threads = ((need + 31) / 32) * 32;
            const size_t smem = f32 ? slab_smem_bytes<float>(nx, cpt, threads)
                                    : slab_smem_bytes<double>(nx, cpt, threads);
            if (smem > 227 * 1024) return false;
            ln->cpt = cpt;
            ln->threads = threads;
            ln->smem = smem;
            ln->slab = f32 ? table().slab32[scheme][flux][ci] : table().slab64[scheme][flux][ci];
            return ln->slab != nullptr;
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
    p->coarse = MGRIT_COARSE_REDISC;
    p->chunk_clusters = 1;
    p->seq_stepper = 0;
}

static int check_params(mgrit_ctx *ctx, const mgrit_params *p)
{
    if (!(p->T > 0) || !(p->L > 0) || !std::isfinite(p->T) || !std::isfinite(p->L))
        return mgrit_fail(ctx, MGRIT_EINVAL, "T and L must be positive and finite");
    if (p->relax != MGRIT_RELAX_F && p->relax != MGRIT_RELAX_FCF)
        return mgrit_fail(ctx, MGRIT_EINVAL, "relax must be F (0) or FCF (1)");
    if (p->cycle != MGRIT_CYCLE_V && p->cycle != MGRIT_CYCLE_F)
        return mgrit_fail(ctx, MGRIT_EINVAL, "cycle must be V (0) or F (1)");
    if (p->guess != MGRIT_GUESS_EQ17 && p->guess != MGRIT_GUESS_INJECT)
        return mgrit_fail(ctx, MGRIT_EINVAL, "guess must be 0 or 1");
    if (p->numflux != MGRIT_LF_SPLIT && p->numflux != MGRIT_LF_STATE && p->numflux != MGRIT_ROE)
        return mgrit_fail(ctx, MGRIT_EINVAL, "numflux must be 0, 1 or 2");
    if (!(p->tol >= 0)) return mgrit_fail(ctx, MGRIT_EINVAL, "tol must be >= 0");
    if (p->max_iter < 0 || p->max_iter > 254)
        return mgrit_fail(ctx, MGRIT_EINVAL, "max_iter must be in [0, 254]");
    if (p->precision != 64 && p->precision != 32)
        return mgrit_fail(ctx, MGRIT_EINVAL, "precision must be 64 or 32");
    if (p->coarse < MGRIT_COARSE_REDISC || p->coarse > MGRIT_COARSE_PSI1)
        return mgrit_fail(ctx, MGRIT_EINVAL, "coarse must be 0, 1 or 2");
    if (p->chunk_clusters != 0 && p->chunk_clusters != 1 && p->chunk_clusters != 2 && p->chunk_clusters != 4)
        return mgrit_fail(ctx, MGRIT_EINVAL, "chunk_clusters must be 0, 1, 2 or 4");
    if (p->seq_stepper < 0 || p->seq_stepper > 3)
        return mgrit_fail(ctx, MGRIT_EINVAL, "seq_stepper must be 0, 1, 2 or 3");
    if (ctx && p->coarse != MGRIT_COARSE_REDISC && ctx->scheme != MGRIT_LF_FE)
        return mgrit_fail(ctx, MGRIT_EINVAL, "matched coarse integrators need the MGRIT_LF_FE scheme");
    if (ctx && ctx->scheme == MGRIT_LF_FE && p->precision != 64)
        return mgrit_fail(ctx, MGRIT_EINVAL, "the MGRIT_LF_FE scheme runs in FP64 only");
    if (p->precision == 64 && !ctx->ln64.slab && !ctx->cluster64)
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP64 slab limit", ctx->nx);
    if (p->precision == 32 && !ctx->ln32.slab)
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP32 single-CTA slab limit", ctx->nx);
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
    if (!out) return mgrit_fail(ctx, MGRIT_EINVAL, "out is NULL");
    *out = nullptr;
    if (scheme != MGRIT_WENO5_SSPRK3 && scheme != MGRIT_FO_FE && scheme != MGRIT_LF_FE)
        return mgrit_fail(ctx, MGRIT_EINVAL, "unknown scheme %d", scheme);
    if (flux != MGRIT_BURGERS && flux != MGRIT_ADVECTION)
        return mgrit_fail(ctx, MGRIT_EINVAL, "unknown flux %d", flux);
    if (m < 2) return mgrit_fail(ctx, MGRIT_EINVAL, "m must be >= 2");
    if (levels < 2 || levels >= MAXLEV) return mgrit_fail(ctx, MGRIT_EINVAL, "levels must be in [2, 31]");
    if (nt < 1) return mgrit_fail(ctx, MGRIT_EINVAL, "nt must be >= 1");
    if (nx < (scheme == MGRIT_WENO5_SSPRK3 ? 5 : 3))
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx too small for the scheme");
    long long div = 1;
    for (int l = 0; l < levels - 1; ++l) div *= m;
    if (div > nt || nt % div) return mgrit_fail(ctx, MGRIT_EINVAL, "nt must be divisible by m^(levels-1)");
    Launch ln64, ln32;
    const bool ok64 = choose_launch(nx, scheme, flux, 0, &ln64);
    const bool ok32 = choose_launch(nx, scheme, flux, 1, &ln32);
    // FP64 slices beyond one CTA run on clusters of up to 16 CTAs with at most
    // 1024 cells each (the limit of the cluster coarsest solve)
    const bool cl64 = !ok64 && scheme != MGRIT_LF_FE && nx <= CLUSTER_MAX * 2 * MAX_THREADS;
    if (!ok64 && !ok32 && !cl64)
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the slab limit", nx);

    ctx = new (std::nothrow) mgrit_ctx;
    if (!ctx) return mgrit_fail(nullptr, MGRIT_ENOMEM, "host allocation failed");
    memset(ctx, 0, sizeof *ctx);
    ctx->nx = nx;
    ctx->nt = nt;
    ctx->m = m;
    ctx->L = levels;
    ctx->scheme = scheme;
    ctx->flux = flux;
    ctx->ln64 = ln64;
    ctx->ln32 = ln32;
    ctx->cluster64 = cl64;
    mgrit_default_params(&ctx->p);
    if (!ok64 && !cl64) ctx->p.precision = 32;   // only FP32 sweeps fit
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
    mgrit_adj_free(ctx);
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
    cudaFree(ctx->gbuf.part);
    cudaFree(ctx->gbuf.halo);
    cudaFree(ctx->gbuf.bar);
    cudaFree(ctx->gbuf.err);
    memset(&ctx->gbuf, 0, sizeof ctx->gbuf);
    memset(&ctx->lg64, 0, sizeof ctx->lg64);
    memset(&ctx->lg32, 0, sizeof ctx->lg32);
    ctx->seq64 = ctx->seq32 = 0;
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

static int choose_levels(mgrit_ctx *ctx);
template <typename R>
static SlabArgs<R> relax_args(const mgrit_ctx *ctx, int l);

extern "C" int mgrit_set_params(mgrit_ctx *ctx, const mgrit_params *p)
{
    if (!ctx || !p) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st = check_params(ctx, p);
    if (st) return st;
    // the captured graphs hold every parameter but the stopping rules
    const bool same_graph = ctx->p.T == p->T && ctx->p.L == p->L && ctx->p.relax == p->relax &&
                            ctx->p.cycle == p->cycle && ctx->p.guess == p->guess &&
                            ctx->p.numflux == p->numflux && ctx->p.precision == p->precision &&
                            ctx->p.coarse == p->coarse &&
                            ctx->p.chunk_clusters == p->chunk_clusters &&
                            ctx->p.seq_stepper == p->seq_stepper;
    const bool rechoose = ctx->alloc && (ctx->p.chunk_clusters != p->chunk_clusters ||
                                         ctx->p.numflux != p->numflux);
    if (ctx->alloc && (p->precision == 32) != (ctx->f32 != 0)) free_workspaces(ctx);
    ctx->p = *p;
    set_level_steps(ctx);
    if (rechoose && ctx->alloc && (st = choose_levels(ctx))) return st;
    if (!same_graph) {
        mgrit_adj_drop_graphs(ctx);
        if (ctx->gA) cudaGraphExecDestroy(ctx->gA);
        if (ctx->gB) cudaGraphExecDestroy(ctx->gB);
        ctx->gA = ctx->gB = nullptr;
        ctx->prepared = false;
    }
    return MGRIT_OK;
}

int mgrit_dalloc(mgrit_ctx *ctx, void **ptr, size_t rows, size_t elem)
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
    if (ctx->scheme == MGRIT_LF_FE) return;   // single-CTA kernel only
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
        if (!cluster_fits(fn, K, threads, smem)) continue;
        lc->fn = fn;
        lc->K = K;
        lc->cpt = cpt;
        lc->threads = threads;
        lc->smem = smem;
        return;
    }
}

// Cluster shape for the chunks of level l (relaxation: nC_l + 1 chunks,
// interpolation: nC_l).  With a one-CTA slab available, clusters are used only
// where the chunks alone leave SMs idle: the largest power of two K <= 16 with
// chunks x K <= SMs and at least 256 cells per CTA (a level of 17 chunks then
// runs on 136 CTAs instead of 17).  Without one (FP64 nx > 8192), the same
// K if there is one, else the smallest K whose blocks fit (at most 2048 cells
// per CTA): many chunks fill the SMs anyway, and fewer CTAs per chunk means
// less exchange.  Each candidate must be co-schedulable.
static void choose_level_cluster(const mgrit_ctx *ctx, int f32, int l, ClusterLaunch *lc)
{
    memset(lc, 0, sizeof *lc);
    if (ctx->scheme == MGRIT_LF_FE || l > ctx->L - 2) return;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    if (ln.slab && !ctx->p.chunk_clusters) return;
    const int nx = ctx->nx, items = ctx->nC_l[l] + 1;
    ClusterLaunch fill, any;   // largest K that fills the SMs; smallest K that fits
    memset(&fill, 0, sizeof fill);
    memset(&any, 0, sizeof any);
    for (int K = CLUSTER_MAX; K >= 2; K /= 2) {
        const int nmax = (nx + K - 1) / K;
        if (nmax > 4 * MAX_THREADS) break;   // smaller K would not fit either
        const bool fills = (long long)items * K <= ctx->nsm;
        if (ln.slab && (!fills || nmax < 256)) continue;
        const int cpt = nmax <= MAX_THREADS ? 1 : nmax <= 2 * MAX_THREADS ? 2 : 4;
        const int ci = cpt == 1 ? 0 : cpt == 2 ? 1 : 2;
        const void *fn = f32 ? table().relc32[ctx->scheme][ctx->flux][ci]
                             : table().relc64[ctx->scheme][ctx->flux][ci];
        const size_t smem = f32 ? cluster_smem_bytes<float>(nx, K) : cluster_smem_bytes<double>(nx, K);
        const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
        if (!fn) continue;
        if (!cluster_fits(fn, K, threads, smem)) continue;
        const ClusterLaunch c{fn, K, cpt, threads, smem};
        if (fills && !fill.fn) fill = c;
        any = c;
    }
    *lc = fill.fn ? fill : ln.slab ? ClusterLaunch{} : any;
}

// a level's chunks on clusters of run-major slabs instead of the shape above:
// where the timed choice took them (WENO5 split form), one-CTA chunks are
// allowed either way (chunk_clusters) or do not fit, and the level's chunks
// fill the SMs
static void apply_tl(const mgrit_ctx *ctx, int f32, int l, ClusterLaunch *lc)
{
    const int slot = ctx->p.chunk_clusters == 2 ? 1 : ctx->p.chunk_clusters == 4 ? 2 : 0;
    const ClusterLaunch &tl = f32 ? ctx->tl32[slot] : ctx->tl64[slot];
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    if (!tl.fn || ctx->scheme != MGRIT_WENO5_SSPRK3 || ctx->p.numflux != NF_SPLIT) return;
    if (ln.slab && !ctx->p.chunk_clusters) return;
    if ((long long)(ctx->nC_l[l] + 1) * tl.K < ctx->nsm && lc->fn) return;
    *lc = tl;
}

// the chunk launch shapes of every level below the coarsest, in the
// allocated precision and in FP64 (mgrit_residual's operator)
static int choose_levels(mgrit_ctx *ctx)
{
    for (int l = 0; l < ctx->L - 1; ++l) {
        choose_level_cluster(ctx, 0, l, &ctx->lr64[l]);
        apply_tl(ctx, 0, l, &ctx->lr64[l]);
        if (ctx->f32) {
            choose_level_cluster(ctx, 1, l, &ctx->lr32[l]);
            apply_tl(ctx, 1, l, &ctx->lr32[l]);
        } else {
            memset(&ctx->lr32[l], 0, sizeof ctx->lr32[l]);
        }
        const bool ok = ctx->f32 ? (ctx->ln32.slab || ctx->lr32[l].fn) : (ctx->ln64.slab || ctx->lr64[l].fn);
        if (!ok)
            return mgrit_fail(ctx, MGRIT_EINVAL, "no slab or cluster shape fits nx = %d at level %d",
                              ctx->nx, l);
    }
    return MGRIT_OK;
}

// `clusters` clusters of lc.K CTAs
static cudaError_t launch_clusters(const ClusterLaunch &lc, int clusters, cudaStream_t s, void *a)
{
    void *args[] = {a};
    return launch_in_clusters(lc.fn, lc.K, (long long)clusters * lc.K, lc.threads, lc.smem, s, args);
}

// `chunks` relaxation or interpolation chunks: one cluster each, else one CTA each
static cudaError_t launch_chunks(const ClusterLaunch &lc, const Launch &ln, int chunks,
                                 cudaStream_t s, void *a)
{
    if (chunks <= 0) return cudaSuccess;
    if (lc.fn) return launch_clusters(lc, chunks, s, a);
    return ln.slab ? launch1(ln.slab, chunks, ln, s, a) : cudaErrorInvalidConfiguration;
}

// the grid stepper: barrier counter zeroed, then a cooperative launch (all G
// CTAs co-resident, or the launch fails).  skip_cta >= 0 makes that CTA skip
// the first barrier (the bounded-wait test hook).
template <typename R>
static cudaError_t launch_grid(const GridLaunch &lg, const GridBufs &gb, const SlabArgs<R> &a,
                               cudaStream_t s, int skip_cta = -1)
{
    cudaError_t e = cudaMemsetAsync(gb.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    GridArgs<R> ga;
    memset(&ga, 0, sizeof ga);
    ga.a = a;
    ga.gb = gb;
    ga.skip_cta = skip_cta;
    void *args[] = {&ga};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(lg.G);
    cfg.blockDim = dim3(lg.threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, lg.fn, args);
}

// the sequential stepper a context uses in FP64 or FP32: 1 one CTA, 2 the
// cluster, 3 the grid (mgrit_params.seq_stepper where that fits, else the
// timed choice; the grid needs the split numerical flux)
static int seq_kind(const mgrit_ctx *ctx, bool f32)
{
    const GridLaunch &lg = f32 ? ctx->lg32 : ctx->lg64;
    const ClusterLaunch &lc = f32 ? ctx->lc32 : ctx->lc64;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    const bool grid_ok = lg.fn && ctx->p.numflux == MGRIT_LF_SPLIT;
    const int want = ctx->p.seq_stepper;
    if (want == 1 && ln.slab) return 1;
    if (want == 2 && lc.fn) return 2;
    if (want == 3 && grid_ok) return 3;
    int k = f32 ? ctx->seq32 : ctx->seq64;
    if (k == 3 && !grid_ok) k = 0;
    if (k == 1 && !ln.slab) k = 0;
    if (k == 2 && !lc.fn) k = 0;
    if (k == 0) k = lc.fn ? 2 : 1;
    return k;
}

// sequential stepping of a context in FP64 (f32 = 0) or FP32: the grid
// stepper where it was chosen and the split flux is in use, else the cluster
// or one-CTA stepper
template <typename R>
static cudaError_t launch_seq_ctx(const mgrit_ctx *ctx, const SlabArgs<R> &a, cudaStream_t s)
{
    const bool f32 = sizeof(R) == 4;
    const GridLaunch &lg = f32 ? ctx->lg32 : ctx->lg64;
    const ClusterLaunch &lc = f32 ? ctx->lc32 : ctx->lc64;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    const int kind = seq_kind(ctx, f32);
    SlabArgs<R> b = a;
    if (kind == 3) return launch_grid(lg, ctx->gbuf, a, s);
    if (kind == 1) return launch1(ln.slab, 1, ln, s, &b);
    return launch_clusters(lc, 1, s, &b);
}

// true (and the flag cleared) if a grid-stepper wait gave up since the
// last check; call after the stream's work has completed
static bool grid_timed_out(mgrit_ctx *ctx)
{
    if (!ctx->gbuf.err) return false;
    int err = 0;
    if (cudaMemcpy(&err, ctx->gbuf.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (err) cudaMemset(ctx->gbuf.err, 0, sizeof(int));
    return err != 0;
}

// Kernel of the sequential chains, chosen by timing 16 steps of each shape
// that fits on a zero state (the work does not depend on the data): one CTA,
// the cluster, and the grid stepper with G = SMs, SMs/2, SMs/4, ... CTAs (8
// to 127 cells each, a lane pair per interface, co-resident).  *kind gets
// the fastest (1 one CTA, 2 cluster, 3 grid) and *lg the fastest grid shape
// (null if none fits).  Grid: split numerical flux, WENO5 or first order,
// nx >= 512.
template <typename R>
static int choose_seq(mgrit_ctx *ctx, GridLaunch *lg, int *kind, R *row)
{
    memset(lg, 0, sizeof *lg);
    const bool f32 = sizeof(R) == 4;
    const ClusterLaunch &lc = f32 ? ctx->lc32 : ctx->lc64;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    *kind = lc.fn ? 2 : 1;
    if (!row) return MGRIT_OK;
    const int nx = ctx->nx;
    cudaStream_t s = ctx->cap;
    CK(cudaMemsetAsync(row, 0, sizeof(R) * nx, s));
    SlabArgs<R> a;
    memset(&a, 0, sizeof a);
    a.mode = MODE_SEQ;
    a.nx = nx;
    a.numflux = MGRIT_LF_SPLIT;
    a.dxinv = (R)(nx / ctx->p.L);
    a.dt = (R)ctx->dt_l[0];
    a.src = row;
    a.out = row;
    const int steps = 16;
    auto time_ms = [&](auto launch) -> float {
        a.nsteps = 2;
        if (launch() != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        a.nsteps = steps;
        cudaEventRecord(ctx->ev0, s);
        if (launch() != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        cudaEventRecord(ctx->ev1, s);
        if (cudaEventSynchronize(ctx->ev1) != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        float ms = -1.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        return ms;
    };
    float best = -1.f;
    auto consider = [&](float ms, int k) {
        if (ms > 0.f && (best < 0.f || ms < best)) {
            best = ms;
            *kind = k;
        }
    };
    if (ln.slab) consider(time_ms([&] {
        SlabArgs<R> b = a;
        return launch1(ln.slab, 1, ln, s, &b);
    }), 1);
    if (lc.fn) consider(time_ms([&] {
        SlabArgs<R> b = a;
        return launch_clusters(lc, 1, s, &b);
    }), 2);
    const void *fn = f32 ? table().grid32[ctx->scheme == MGRIT_LF_FE ? 0 : ctx->scheme][ctx->flux]
                         : table().grid64[ctx->scheme == MGRIT_LF_FE ? 0 : ctx->scheme][ctx->flux];
    if (ctx->scheme == MGRIT_LF_FE || nx < 512 || !fn) return MGRIT_OK;
    float gbest = -1.f;
    int nb = 0;
    for (int G = ctx->nsm < GRID_MAX ? ctx->nsm : GRID_MAX; G >= 8; G /= 2) {
        const int n = (nx + G - 1) / G;
        if (n < 8 || nx / G < 8) continue;
        const int threads = ((2 * (n + 1) + 31) / 32) * 32;   // a lane pair per interface
        if (threads > GRID_THREADS) break;   // fewer CTAs would only be larger
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess ||
            (long long)nb * ctx->nsm < G) {
            cudaGetLastError();
            continue;
        }
        const GridLaunch cand{fn, G, threads};
        const float ms = time_ms([&] { return launch_grid(cand, ctx->gbuf, a, s); });
        if (ms > 0.f && (gbest < 0.f || ms < gbest)) {
            gbest = ms;
            *lg = cand;
        }
    }
    consider(gbest, 3);
    // a wait that gave up during the choice would leave the error flag set
    int err = 0;
    CK(cudaMemcpy(&err, ctx->gbuf.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        memset(lg, 0, sizeof *lg);
        if (*kind == 3) *kind = lc.fn ? 2 : 1;
        CK(cudaMemset(ctx->gbuf.err, 0, sizeof(int)));
    }
    return MGRIT_OK;
}

// WENO5 slabs: the cells per thread of the one-CTA slab, chosen by timing
// the level-0 relaxation with 1x, 2x and 4x the smallest that fits (FP64:
// up to 16 cells per thread) on min(chunks, 2 x SMs) chunks of a zero state.
// Fewer, fuller threads let two CTAs share an SM and hide each other's
// barriers.  Every shape performs the same operations per cell, so the
// choice gives the same bits.
template <typename R>
static int tune_slab(mgrit_ctx *ctx)
{
    const bool f32 = sizeof(R) == 4;
    Launch &cur = f32 ? ctx->ln32 : ctx->ln64;
    if (ctx->scheme != MGRIT_WENO5_SSPRK3 || !cur.slab) return MGRIT_OK;
    const int ncpt = f32 ? NCPT : NCPT64;
    int ci0 = 0;
    while (ci0 < ncpt && CPT_VALUES[ci0] != cur.cpt) ++ci0;
    SlabArgs<R> a = relax_args<R>(ctx, 0);
    const int chunks = ctx->nC_l[0] + 1 < 2 * ctx->nsm ? ctx->nC_l[0] + 1 : 2 * ctx->nsm;
    cudaStream_t s = ctx->cap;
    CK(cudaMemsetAsync(const_cast<R *>(a.uC), 0, sizeof(R) * (size_t)ctx->nx * chunks, s));
    Launch best = cur;
    float best_ms = -1.f;
    for (int ci = ci0; ci < ncpt && ci <= ci0 + 2; ++ci) {
        const int cpt = CPT_VALUES[ci];
        const int need = (ctx->nx + cpt - 1) / cpt;
        Launch ln;
        ln.cpt = cpt;
        ln.threads = ((need + 31) / 32) * 32;
        ln.smem = slab_smem_bytes<R>(ctx->nx, cpt, ln.threads);
        ln.slab = f32 ? table().slab32[ctx->scheme][ctx->flux][ci] : table().slab64[ctx->scheme][ctx->flux][ci];
        if (!ln.slab || ln.smem > (size_t)SMEM_OPTIN) continue;
        CK(cudaFuncSetAttribute(ln.slab, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
        float ms = -1.f;
        for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
            CK(cudaEventRecord(ctx->ev0, s));
            CK(launch1(ln.slab, chunks, ln, s, &a));
            CK(cudaEventRecord(ctx->ev1, s));
            CK(cudaEventSynchronize(ctx->ev1));
            CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        }
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = ln;
        }
    }
    cur = best;
    return MGRIT_OK;
}

// Clusters of run-major slabs for the chunks of the WENO5 split form when nx
// > 8192 (one FP32 CTA would hold 32 cells per thread and spill; an FP64
// slice does not fit one CTA): K = 2 or 4 CTAs of 8 or 16 cells per thread,
// timed on the level-0 relaxation of min(chunks, 8 x SMs) chunks of a zero
// state against the level's current shape (the one-CTA slab or the cluster
// stepper's chunks); the fastest is kept.  The choice applies to the levels
// whose chunks fill the SMs (apply_tl).
// Slots 1 and 2 keep the first shape that fits with K = 2 and 4, for
// chunk_clusters = 2 and 4 (no timing).
template <typename R>
static int tune_tl(mgrit_ctx *ctx)
{
    const bool f32 = sizeof(R) == 4;
    ClusterLaunch *tls = f32 ? ctx->tl32 : ctx->tl64;
    ClusterLaunch &tl = tls[0];
    memset(tls, 0, 3 * sizeof(ClusterLaunch));
    if (ctx->scheme != MGRIT_WENO5_SSPRK3 || ctx->nx <= 8192) return MGRIT_OK;
    const Launch &ln = f32 ? ctx->ln32 : ctx->ln64;
    const ClusterLaunch cur = f32 ? ctx->lr32[0] : ctx->lr64[0];
    SlabArgs<R> a = relax_args<R>(ctx, 0);
    // enough chunks for several waves of every candidate (2 x SMs chunks
    // timed K = 2 ahead of a K = 4 that is faster on the whole level)
    const int chunks = ctx->nC_l[0] + 1 < 8 * ctx->nsm ? ctx->nC_l[0] + 1 : 8 * ctx->nsm;
    cudaStream_t s = ctx->cap;
    CK(cudaMemsetAsync(const_cast<R *>(a.uC), 0, sizeof(R) * (size_t)ctx->nx * chunks, s));
    auto time_shape = [&](const ClusterLaunch &lc, float *ms) -> int {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(launch_chunks(lc, ln, chunks, s, &a));   // warm-up
        CK(cudaEventRecord(e0, s));
        CK(launch_chunks(lc, ln, chunks, s, &a));
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return MGRIT_OK;
    };
    // the timing needs the split form and a shape to compare with
    const bool timed = ctx->p.numflux == NF_SPLIT && ctx->p.chunk_clusters == 1 && (cur.fn || ln.slab);
    float best_ms = -1.f;
    int st;
    if (timed && (st = time_shape(cur, &best_ms))) return st;
    for (int K = 2; K <= 4; K *= 2) {
        const int nmax = (ctx->nx + K - 1) / K;
        for (int ci = 1; ci >= 0; --ci) {
            const int cpt = ci ? 16 : 8;
            const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
            if (threads > MAX_THREADS) continue;
            const void *fn = f32 ? table().tlc32[ctx->flux][ci] : table().tlc64[ctx->flux][ci];
            const size_t smem = slab_cluster_smem_bytes<R>(nmax, cpt, threads);
            if (!fn || smem > (size_t)SMEM_OPTIN || !cluster_fits(fn, K, threads, smem)) continue;
            const ClusterLaunch c{fn, K, cpt, threads, smem};
            if (!tls[K / 2].fn) tls[K / 2] = c;
            if (!timed) continue;
            float ms = -1.f;
            if ((st = time_shape(c, &ms))) return st;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                tl = c;
            }
        }
    }
    return MGRIT_OK;
}

int mgrit_ensure_alloc(mgrit_ctx *ctx)
{
    if (ctx->alloc) return MGRIT_OK;
    CK(cudaGetDevice(&ctx->device));
    ctx->f32 = ctx->p.precision == 32;
    const int L = ctx->L;
    const size_t es = ctx->f32 ? sizeof(float) : sizeof(double);
    int st;
    for (int l = 0; l < L - 1; ++l) {
        if ((st = mgrit_dalloc(ctx, &ctx->newC[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = mgrit_dalloc(ctx, &ctx->phirow[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = mgrit_dalloc(ctx, &ctx->cstep[l], ctx->nC_l[l], es))) return st;
    }
    for (int l = 1; l < L; ++l) {
        const size_t el = level_f32(ctx, l) ? sizeof(float) : sizeof(double);
        if ((st = mgrit_dalloc(ctx, &ctx->u[l], ctx->nt_l[l] + 1, el))) return st;
        if ((st = mgrit_dalloc(ctx, (void **)&ctx->g[l], ctx->nt_l[l] + 1, sizeof(double)))) return st;
    }
    if (ctx->f32) {
        if ((st = mgrit_dalloc(ctx, (void **)&ctx->u32c, ctx->nt_l[L - 1] + 1, sizeof(float)))) return st;
        if ((st = mgrit_dalloc(ctx, (void **)&ctx->ser32, 1, sizeof(float)))) return st;
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
                                SMEM_OPTIN));
    if (ctx->ln32.slab)
        CK(cudaFuncSetAttribute(ctx->ln32.slab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_OPTIN));
    CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    choose_cluster(ctx, 0, &ctx->lc64);
    if (ctx->f32) choose_cluster(ctx, 1, &ctx->lc32);
    CK(cudaMalloc((void **)&ctx->gbuf.part, sizeof(double) * 2 * GRID_MAX));
    CK(cudaMalloc((void **)&ctx->gbuf.halo, sizeof(double) * 2 * GRID_MAX * 6));
    CK(cudaMalloc((void **)&ctx->gbuf.bar, sizeof(unsigned)));
    CK(cudaMalloc((void **)&ctx->gbuf.err, sizeof(int)));
    CK(cudaMemset(ctx->gbuf.err, 0, sizeof(int)));
    // the timed choices run on rows the solve overwrites later: the slab
    // shape (in the sweep precision) on the level-0 C-point source, the FP64
    // sequential stepper on the level-0 C-point row buffer (FP64 mode) or a
    // fresh FP64 row, the FP32 one on the FP32 serial row
    if (ctx->f32 ? (st = tune_slab<float>(ctx)) : (st = tune_slab<double>(ctx))) return st;
    if (!ctx->f32) {
        if ((st = choose_seq<double>(ctx, &ctx->lg64, &ctx->seq64, static_cast<double *>(ctx->newC[0]))))
            return st;
    } else {
        double *tmp = nullptr;
        CK(cudaMalloc((void **)&tmp, sizeof(double) * ctx->nx));
        st = choose_seq<double>(ctx, &ctx->lg64, &ctx->seq64, tmp);
        cudaFree(tmp);
        if (st) return st;
        if ((st = choose_seq<float>(ctx, &ctx->lg32, &ctx->seq32, ctx->ser32))) return st;
    }
    if (!ctx->ln64.slab && !ctx->lc64.fn)
        return mgrit_fail(ctx, MGRIT_EINVAL, "no FP64 slab or cluster fits nx = %d for the coarsest solve",
                    ctx->nx);
    int st2;
    memset(ctx->tl64, 0, sizeof ctx->tl64);
    memset(ctx->tl32, 0, sizeof ctx->tl32);
    if ((st2 = choose_levels(ctx))) return st2;
    // clusters of run-major slabs (nx > 8192), timed against the shapes
    // just chosen, on the same level-0 C-point source as tune_slab
    if (ctx->f32 ? (st2 = tune_tl<float>(ctx)) : (st2 = tune_tl<double>(ctx))) return st2;
    if ((st2 = choose_levels(ctx))) return st2;
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
    if (ctx->p.coarse != MGRIT_COARSE_REDISC) {
        // matched integrators on the coarse levels: level k integrates m^k fine steps
        int M = 1;
        for (int k = 0; k < l; ++k) M *= ctx->m;
        a.psiM = l == 0 ? 0 : M;
        a.psiMc = M * ctx->m;
        a.psiOrder = ctx->p.coarse == MGRIT_COARSE_PSI1 ? 1 : 0;
        a.psiDt = (R)ctx->dt_l[0];
    }
    return a;
}

// the buffer (and its precision) holding the level-l C-points that the
// level-l relaxation reads
static const void *cpoint_source(const mgrit_ctx *ctx, int l)
{
    if (l == 0) return (ctx->L == 2 && ctx->f32) ? (const void *)ctx->u32c : ctx->u[1];
    return ctx->u[l];
}

// argument blocks of the level kernels (shared by the single-instance graphs
// and the batched launches)
template <typename R>
static SlabArgs<R> relax_args(const mgrit_ctx *ctx, int l)
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
    return a;
}

static RestrictArgs restrict_args(const mgrit_ctx *ctx, int l)
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
    return a;
}

static SlabArgs<double> coarse_args(const mgrit_ctx *ctx)
{
    const int l = ctx->L - 1;
    SlabArgs<double> a = base_args<double>(ctx, MODE_SEQ, l);
    a.src = ctx->g[l];
    a.g = ctx->g[l];
    a.rows = static_cast<double *>(ctx->u[l]);
    a.nsteps = ctx->nt_l[l];
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    return a;
}

template <typename R>
static SlabArgs<R> interp_args(const mgrit_ctx *ctx, int l)
{
    SlabArgs<R> a = base_args<R>(ctx, MODE_INTERP, l);
    const void *coarse = (l + 1 == ctx->L - 1 && ctx->f32) ? (const void *)ctx->u32c : ctx->u[l + 1];
    a.uC = static_cast<const R *>(coarse);
    a.g = ctx->g[l];
    a.rows = static_cast<R *>(ctx->u[l]);
    a.nrows_uC = a.nC + 1;
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    return a;
}

template <typename R>
static cudaError_t enqueue_relax_t(mgrit_ctx *ctx, int l, cudaStream_t s, const Launch &ln,
                                   const ClusterLaunch &lc)
{
    SlabArgs<R> a = relax_args<R>(ctx, l);
    return launch_chunks(lc, ln, a.nC + 1, s, &a);
}

static cudaError_t enqueue_relax(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    return ctx->f32 ? enqueue_relax_t<float>(ctx, l, s, ctx->ln32, ctx->lr32[l])
                    : enqueue_relax_t<double>(ctx, l, s, ctx->ln64, ctx->lr64[l]);
}

static cudaError_t enqueue_restrict(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    RestrictArgs a = restrict_args(ctx, l);
    const int blocks = l == 0 ? ctx->nparts : restrict_blocks(a.nC, a.nx);
    return launch_restrict(a, blocks, s);
}

// coarsest level, always FP64; in FP32-sweep mode its rows are then mirrored
// in FP32 for the level above
static cudaError_t enqueue_coarse(mgrit_ctx *ctx, cudaStream_t s)
{
    const int l = ctx->L - 1;
    SlabArgs<double> a = coarse_args(ctx);
    cudaError_t e = launch_seq_ctx(ctx, a, s);
    if (e != cudaSuccess || !ctx->f32) return e;
    return launch_convert(ctx->u[l], 0, ctx->u32c, 1, (long long)(ctx->nt_l[l] + 1) * ctx->nx, s);
}

template <typename R>
static cudaError_t enqueue_interp_t(mgrit_ctx *ctx, int l, cudaStream_t s, const Launch &ln,
                                    const ClusterLaunch &lc)
{
    SlabArgs<R> a = interp_args<R>(ctx, l);
    return launch_chunks(lc, ln, a.nC, s, &a);
}

static cudaError_t enqueue_interp(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    return ctx->f32 ? enqueue_interp_t<float>(ctx, l, s, ctx->ln32, ctx->lr32[l])
                    : enqueue_interp_t<double>(ctx, l, s, ctx->ln64, ctx->lr64[l]);
}

static cudaError_t enqueue_part_a(mgrit_ctx *ctx, cudaStream_t s)
{
    cudaError_t e;
    if ((e = enqueue_relax(ctx, 0, s))) return e;
    if ((e = enqueue_restrict(ctx, 0, s))) return e;
    return launch_norm(ctx->partials, ctx->nparts, ctx->d_norm, s);
}

// Launch order below level 0: the V-cycle of Algorithm 1 (relax, restrict,
// recurse, interpolate) or the F-cycle (below each level an F-cycle, then
// one V-cycle), for any set of level operations
struct CycleOps {
    cudaError_t (*relax)(mgrit_ctx *, int, cudaStream_t);
    cudaError_t (*restrict_)(mgrit_ctx *, int, cudaStream_t);
    cudaError_t (*coarse)(mgrit_ctx *, cudaStream_t);
    cudaError_t (*interp)(mgrit_ctx *, int, cudaStream_t);
};

static cudaError_t emit_cycle(mgrit_ctx *ctx, const CycleOps &o, int l, bool fcycle, cudaStream_t s)
{
    if (l == ctx->L - 1) return o.coarse(ctx, s);
    cudaError_t e;
    if ((e = o.relax(ctx, l, s))) return e;
    if ((e = o.restrict_(ctx, l, s))) return e;
    if ((e = emit_cycle(ctx, o, l + 1, fcycle, s))) return e;
    if ((e = o.interp(ctx, l, s))) return e;
    if (!fcycle) return cudaSuccess;
    if ((e = o.relax(ctx, l, s))) return e;
    if ((e = o.restrict_(ctx, l, s))) return e;
    if ((e = emit_cycle(ctx, o, l + 1, false, s))) return e;
    return o.interp(ctx, l, s);
}

cudaError_t mgrit_emit_below_level0(mgrit_ctx *ctx, cudaError_t (*relax)(mgrit_ctx *, int, cudaStream_t),
                                    cudaError_t (*restrict_)(mgrit_ctx *, int, cudaStream_t),
                                    cudaError_t (*coarse)(mgrit_ctx *, cudaStream_t),
                                    cudaError_t (*interp)(mgrit_ctx *, int, cudaStream_t),
                                    cudaStream_t s)
{
    const CycleOps o{relax, restrict_, coarse, interp};
    return emit_cycle(ctx, o, 1, ctx->p.cycle == MGRIT_CYCLE_F, s);
}

static cudaError_t enqueue_part_b(mgrit_ctx *ctx, cudaStream_t s)
{
    return mgrit_emit_below_level0(ctx, enqueue_relax, enqueue_restrict, enqueue_coarse,
                                   enqueue_interp, s);
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
        return mgrit_fail(ctx, MGRIT_ECUDA, "graph capture: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return mgrit_fail(ctx, MGRIT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MGRIT_OK;
}

static int ensure_graphs(mgrit_ctx *ctx)
{
    int st;
    if (!ctx->gA && (st = capture(ctx, enqueue_part_a, &ctx->gA))) return st;
    if (!ctx->gB && (st = capture(ctx, enqueue_part_b, &ctx->gB))) {
        // a graph that the cooperative grid stepper cannot be captured into:
        // the coarsest solve falls back to the cluster / one-CTA stepper
        if (!ctx->lg64.fn) return st;
        cudaGetLastError();
        ctx->lg64.fn = nullptr;
        if (ctx->seq64 == 3) ctx->seq64 = 0;
        if ((st = capture(ctx, enqueue_part_b, &ctx->gB))) return st;
    }
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

// Phi applications below level l of one cycle (V or F), see emit_cycle
static double steps_below(const mgrit_ctx *ctx, int l, bool fcycle)
{
    if (l == ctx->L - 1) return ctx->nt_l[l];       // coarsest sequential solve
    const double m = ctx->m, nc = ctx->nC_l[l];
    // relaxation (F: m per chunk, FCF: 2m) + the coarse step for the FAS term
    const double relax = (ctx->p.relax == MGRIT_RELAX_FCF ? 2.0 : 1.0) * nc * m + nc;
    const double interp = nc * (m - 1);             // interpolation F-relaxation
    double steps = relax + steps_below(ctx, l + 1, fcycle) + interp;
    if (fcycle) steps += relax + steps_below(ctx, l + 1, false) + interp;
    return steps;
}

extern "C" double mgrit_cycle_cell_updates(const mgrit_ctx *ctx)
{
    if (!ctx) return 0.0;
    const double m = ctx->m, nc = ctx->nC_l[0];
    const double relax0 = (ctx->p.relax == MGRIT_RELAX_FCF ? 2.0 : 1.0) * nc * m + nc;
    return (relax0 + steps_below(ctx, 1, ctx->p.cycle == MGRIT_CYCLE_F)) * ctx->nx;
}

static int prepare(mgrit_ctx *ctx, const double *u0_dev, cudaStream_t s)
{
    if (!u0_dev) return mgrit_fail(ctx, MGRIT_EINVAL, "u0_dev is NULL");
    int st;
    if ((st = mgrit_ensure_alloc(ctx))) return st;
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
    // a grid-stepper wait that gave up (coarsest solve) makes the solve's
    // values meaningless: report it
    if (grid_timed_out(ctx)) status = MGRIT_ETIMEOUT;
    if (stats) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        stats->iters = k;
        stats->status = status;
        stats->t_total_ms = ms;
        stats->cell_updates = updates;
        stats->stagnated = stagnated;
    }
    if (status == MGRIT_ETIMEOUT) mgrit_fail(ctx, status, "a grid-stepper wait gave up");
    if (status == MGRIT_EDIVERGED) mgrit_fail(ctx, status, "diverged at cycle %d", k);
    if (status == MGRIT_ENOTCONV) mgrit_fail(ctx, status, "not converged after %d cycles", k);
    return status;
}

extern "C" int mgrit_run_cycles(mgrit_ctx *ctx, const double *u0_dev, int ncycles, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (ncycles < 0) return mgrit_fail(ctx, MGRIT_EINVAL, "ncycles must be >= 0");
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
    if (!ctx || !uC_out_dev) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    if (!ctx->have_state) return mgrit_fail(ctx, MGRIT_EINVAL, "no solve has run on this context");
    return copy_out(ctx, uC_out_dev, 0, ctx->nC_l[0] + 1, (cudaStream_t)stream);
}

extern "C" int mgrit_serial_step(mgrit_ctx *ctx, const double *u0_dev, double *uT_dev, int nsteps,
                                 void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!u0_dev || !uT_dev || nsteps < 0) return mgrit_fail(ctx, MGRIT_EINVAL, "bad arguments");
    int st;
    if ((st = mgrit_ensure_alloc(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->f32) {
        SlabArgs<double> a = base_args<double>(ctx, MODE_SEQ, 0);
        a.src = u0_dev;
        a.out = uT_dev;
        a.nsteps = nsteps;
        CK(launch_seq_ctx(ctx, a, s));
        return MGRIT_OK;
    }
    // FP32 sweeps: step an FP32 copy of u0 and widen the result
    CK(launch_convert(u0_dev, 0, ctx->ser32, 1, ctx->nx, s));
    SlabArgs<float> a = base_args<float>(ctx, MODE_SEQ, 0);
    a.src = ctx->ser32;
    a.out = ctx->ser32;
    a.nsteps = nsteps;
    CK(launch_seq_ctx(ctx, a, s));
    CK(launch_convert(ctx->ser32, 1, uT_dev, 0, ctx->nx, s));
    return MGRIT_OK;
}

extern "C" int mgrit_sync_status(mgrit_ctx *ctx, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (grid_timed_out(ctx))
        return mgrit_fail(ctx, MGRIT_ETIMEOUT, "a grid-stepper wait gave up");
    return MGRIT_OK;
}

extern "C" int mgrit_test_grid_timeout(mgrit_ctx *ctx, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    int st;
    if ((st = mgrit_ensure_alloc(ctx))) return st;
    if (!ctx->lg64.fn) return mgrit_fail(ctx, MGRIT_EINVAL, "this context steps without the grid stepper");
    cudaStream_t s = (cudaStream_t)stream;
    SlabArgs<double> a = base_args<double>(ctx, MODE_SEQ, 0);
    a.src = static_cast<const double *>(ctx->newC[0]);
    a.out = nullptr;
    a.nsteps = 1;
    CK(launch_grid(ctx->lg64, ctx->gbuf, a, s, 0));
    return mgrit_sync_status(ctx, stream);
}

extern "C" int mgrit_residual(mgrit_ctx *ctx, const double *uC_dev, double *norm_out, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!uC_dev || !norm_out) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st;
    if ((st = mgrit_ensure_alloc(ctx))) return st;
    if (!ctx->ln64.slab && !ctx->lr64[0].fn)
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the FP64 slab limit", ctx->nx);
    if (!ctx->resid_rows &&
        (st = mgrit_dalloc(ctx, (void **)&ctx->resid_rows, ctx->nC_l[0] + 1, sizeof(double))))
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    // always the FP64 operator: the residual of the FP64 discrete system
    SlabArgs<double> a = base_args<double>(ctx, MODE_RELAX, 0);
    a.uC = uC_dev;
    a.strideC = ctx->nx;
    a.fcf = 0;
    a.phirow = ctx->resid_rows;
    a.nrows_uC = a.nrows_phirow = a.nC + 1;
    CK(launch_chunks(ctx->lr64[0], ctx->ln64, a.nC, s, &a));
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
    if (!ctx->prepared) return mgrit_fail(ctx, MGRIT_EINVAL, "no solve has run on this context");
    if (reps < 0) return mgrit_fail(ctx, MGRIT_EINVAL, "reps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ctx->L;
    for (int r = 0; r < reps; ++r) {
        switch (which) {
        case 0:
            if (level < 0 || level > L - 2) return mgrit_fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_relax(ctx, level, s));
            break;
        case 1:
            if (level < 0 || level > L - 2) return mgrit_fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_restrict(ctx, level, s));
            break;
        case 2:
            CK(enqueue_coarse(ctx, s));
            break;
        case 3:
            if (level < 1 || level > L - 2) return mgrit_fail(ctx, MGRIT_EINVAL, "bad level");
            CK(enqueue_interp(ctx, level, s));
            break;
        default:
            return mgrit_fail(ctx, MGRIT_EINVAL, "unknown kernel id %d", which);
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
    case 2:     // CTAs of the cluster the sequential chains use (1: one CTA; 0: the grid stepper)
    case 3: {   // CTAs of the grid stepper the sequential chains use (0: not used)
        if (!ctx->alloc) return 0;
        const int kind = seq_kind(ctx, f32);
        if (what == 3) return kind == 3 ? (f32 ? ctx->lg32.G : ctx->lg64.G) : 0;
        return kind == 3 ? 0 : kind == 1 ? 1 : lc.K;
    }
    default:
        if (what >= 100 && what < 100 + ctx->L - 1) {   // level what-100 relaxation / interpolation
            if (!ctx->alloc) return 0;
            const ClusterLaunch &lr = f32 ? ctx->lr32[what - 100] : ctx->lr64[what - 100];
            return lr.fn ? lr.K : 1;
        }
        if (what >= 200 && what < 200 + ctx->L - 1) {   // level what-200 on run-major cluster slabs?
            if (!ctx->alloc) return 0;
            const ClusterLaunch &lr = f32 ? ctx->lr32[what - 200] : ctx->lr64[what - 200];
            const ClusterLaunch *tl = f32 ? ctx->tl32 : ctx->tl64;
            return lr.fn && (lr.fn == tl[0].fn || lr.fn == tl[1].fn || lr.fn == tl[2].fn) ? 1 : 0;
        }
        return -1;
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

// ===========================================================================
// Batches: many independent instances (uneven nx, nt, levels, flux) advanced
// together.  Each instance keeps its own level workspaces (an mgrit_ctx);
// every phase of a cycle is one batched launch per launch class, with a
// block map telling each CTA its instance and chunk.  V-cycle phases are
// ordered by level depth: relaxation + restriction of depth d for every
// instance that has a level d below its coarsest, then every coarsest solve,
// then the interpolations from the deepest depth up.  F-cycle phases merge
// the instances' own launch orders (emit_merged_cycle).  A device-side mask
// lets converged instances skip all work while the others continue.
// ===========================================================================

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "batch_table.cuh"

namespace {

struct BLaunch {
    int kind;           // 0 slab kernel, 1 restriction, 2 norm, 3 FP64 -> FP32 conversion,
                        // 4 cluster sequential kernel (un_f32 holds the cluster size)
    const void *fn;     // slab kernel instance
    int threads;
    size_t smem;
    int nblocks;
    int state_f32, un_f32;
    void *d_args;
    BatchItem *d_map;
};

const BatchTable &btable()
{
    static BatchTable t = [] {
        BatchTable k;
        memset(&k, 0, sizeof k);
        fill_batch_f32_burgers(k);
        fill_batch_f32_advection(k);
        fill_batch_f64_burgers(k);
        fill_batch_f64_advection(k);
        return k;
    }();
    return t;
}

int cpt_index(int cpt)
{
    for (int i = 0; i < NCPT; ++i)
        if (CPT_VALUES[i] == cpt) return i;
    return -1;
}

}  // namespace

struct mgrit_batch {
    int n;
    mgrit_params p;
    std::vector<mgrit_ctx *> ctx;
    std::vector<int> cpt;        // cells per thread of the sweep kernels, per instance
    std::vector<int> cpt64;      // cells per thread of the FP64 coarsest solve, per instance
    std::vector<int> ck;         // coarsest solve: cluster size per instance (1: one CTA)
    int maxL;
    int *d_active;
    int *h_active;
    double *d_norms;
    double *h_norms;
    std::vector<BLaunch> A, B;
    std::vector<void *> tables;  // device launch tables
    cudaGraphExec_t gA, gB;
    cudaStream_t cap;
    char err[256];
};

static int bfail(mgrit_batch *b, int code, const char *fmt, ...)
{
    char *buf = b ? b->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define BCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? MGRIT_ENOMEM : MGRIT_ECUDA, \
                         "%s: %s", #call, cudaGetErrorString(e_));                       \
    } while (0)

static int threads_for(int nx, int cpt) { return (((nx + cpt - 1) / cpt + 31) / 32) * 32; }

static void batch_free_tables(mgrit_batch *b)
{
    if (b->gA) cudaGraphExecDestroy(b->gA);
    if (b->gB) cudaGraphExecDestroy(b->gB);
    b->gA = b->gB = nullptr;
    for (void *p : b->tables) cudaFree(p);
    b->tables.clear();
    b->A.clear();
    b->B.clear();
}

template <typename T>
static int upload(mgrit_batch *b, const std::vector<T> &v, T **out)
{
    BCK(cudaMalloc((void **)out, sizeof(T) * std::max<size_t>(v.size(), 1)));
    b->tables.push_back(*out);
    if (!v.empty()) BCK(cudaMemcpy(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return MGRIT_OK;
}

// one launch per (flux, cells per thread, threads) class of slab work items
template <typename R>
struct SlabGroups {
    struct G {
        std::vector<SlabArgs<R>> args;
        std::vector<BatchItem> map;
        int nx_max = 0;
    };
    std::map<std::tuple<int, int, int>, G> g;

    void add(int inst, int flux, int cpt, const SlabArgs<R> &a, int nitems)
    {
        G &grp = g[std::make_tuple(flux, cpt, threads_for(a.nx, cpt))];
        const int ai = (int)grp.args.size();
        grp.args.push_back(a);
        for (int j = 0; j < nitems; ++j) grp.map.push_back(BatchItem{ai, j, inst, 0});
        grp.nx_max = std::max(grp.nx_max, a.nx);
    }

    int emit(mgrit_batch *b, std::vector<BLaunch> &out)
    {
        for (auto &kv : g) {
            const int flux = std::get<0>(kv.first), cpt = std::get<1>(kv.first);
            G &grp = kv.second;
            BLaunch L;
            memset(&L, 0, sizeof L);
            L.kind = 0;
            L.fn = sizeof(R) == 4 ? btable().slab32[flux][cpt_index(cpt)]
                                  : btable().slab64[flux][cpt_index(cpt)];
            L.threads = std::get<2>(kv.first);
            L.smem = slab_smem_bytes<R>(grp.nx_max, cpt, L.threads);
            L.nblocks = (int)grp.map.size();
            SlabArgs<R> *da;
            int st;
            if ((st = upload(b, grp.args, &da))) return st;
            if ((st = upload(b, grp.map, &L.d_map))) return st;
            L.d_args = da;
            BCK(cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
            out.push_back(L);
        }
        return MGRIT_OK;
    }
};

// (instance, level) pairs of one batched phase
typedef std::vector<std::pair<int, int>> InstLevels;

static InstLevels at_depth(const mgrit_batch *b, int depth, int lo_margin, int hi_margin,
                           const std::vector<int> *only = nullptr)
{
    // every instance with lo_margin <= depth <= L - hi_margin
    InstLevels il;
    for (int i = 0; i < b->n; ++i) {
        if (depth < lo_margin || depth > b->ctx[i]->L - hi_margin) continue;
        if (only && std::find(only->begin(), only->end(), i) == only->end()) continue;
        il.push_back(std::make_pair(i, depth));
    }
    return il;
}

static int emit_restrict_at(mgrit_batch *b, const InstLevels &il, std::vector<BLaunch> &out)
{
    std::map<std::pair<int, int>, std::pair<std::vector<RestrictBatchArgs>, std::vector<BatchItem>>> grp;
    for (const auto &x : il) {
        const int i = x.first, l = x.second;
        mgrit_ctx *c = b->ctx[i];
        RestrictBatchArgs ra;
        ra.r = restrict_args(c, l);
        ra.nblocks = l == 0 ? c->nparts : restrict_blocks(ra.r.nC, ra.r.nx);
        auto &e = grp[std::make_pair(ra.r.state_f32, ra.r.un_f32)];
        const int ai = (int)e.first.size();
        e.first.push_back(ra);
        for (int k = 0; k < ra.nblocks; ++k) e.second.push_back(BatchItem{ai, 0, i, k});
    }
    for (auto &kv : grp) {
        BLaunch L;
        memset(&L, 0, sizeof L);
        L.kind = 1;
        L.state_f32 = kv.first.first;
        L.un_f32 = kv.first.second;
        L.nblocks = (int)kv.second.second.size();
        RestrictBatchArgs *da;
        int st;
        if ((st = upload(b, kv.second.first, &da))) return st;
        if ((st = upload(b, kv.second.second, &L.d_map))) return st;
        L.d_args = da;
        out.push_back(L);
    }
    return MGRIT_OK;
}

static int emit_restrict(mgrit_batch *b, int depth, std::vector<BLaunch> &out)
{
    return emit_restrict_at(b, at_depth(b, depth, 0, 2), out);
}

template <typename R>
static int emit_relax_at(mgrit_batch *b, const InstLevels &il, std::vector<BLaunch> &out)
{
    SlabGroups<R> sg;
    for (const auto &x : il) {
        mgrit_ctx *c = b->ctx[x.first];
        SlabArgs<R> a = relax_args<R>(c, x.second);
        sg.add(x.first, c->flux, b->cpt[x.first], a, a.nC + 1);
    }
    return sg.emit(b, out);
}

template <typename R>
static int emit_relax(mgrit_batch *b, int depth, std::vector<BLaunch> &out,
                      const std::vector<int> *only = nullptr)
{
    return emit_relax_at<R>(b, at_depth(b, depth, 0, 2, only), out);
}

template <typename R>
static int emit_interp_at(mgrit_batch *b, const InstLevels &il, std::vector<BLaunch> &out)
{
    SlabGroups<R> sg;
    for (const auto &x : il) {
        mgrit_ctx *c = b->ctx[x.first];
        SlabArgs<R> a = interp_args<R>(c, x.second);
        sg.add(x.first, c->flux, b->cpt[x.first], a, a.nC);
    }
    return sg.emit(b, out);
}

template <typename R>
static int emit_interp(mgrit_batch *b, int depth, std::vector<BLaunch> &out)
{
    return emit_interp_at<R>(b, at_depth(b, depth, 1, 2), out);
}

// launch shape of the batched FP64 coarsest solve of one nx on a cluster of K
// CTAs (cells per thread 1 or 2); false if K does not fit or cannot be
// co-scheduled
static bool batch_cluster_shape(int nx, int flux, int K, ClusterLaunch *lc)
{
    memset(lc, 0, sizeof *lc);
    if (K < 2 || K > CLUSTER_MAX) return false;
    const int nmax = (nx + K - 1) / K;
    if (nmax > 2 * MAX_THREADS || nmax < 2 * GHOST) return false;
    const int cpt = nmax <= MAX_THREADS ? 1 : 2;
    const void *fn = btable().seqc64[flux][cpt - 1];
    const size_t smem = cluster_smem_bytes<double>(nx, K);
    const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
    if (!cluster_fits(fn, K, threads, smem)) return false;
    lc->fn = fn;
    lc->K = K;
    lc->cpt = cpt;
    lc->threads = threads;
    lc->smem = smem;
    return true;
}

static int emit_coarse(mgrit_batch *b, std::vector<BLaunch> &out,
                       const std::vector<int> *only = nullptr)
{
    SlabGroups<double> sg;
    // cluster launches grouped by (flux, cells per thread, cluster size, threads)
    std::map<std::tuple<int, int, int, int>, std::pair<std::vector<SlabArgs<double>>, std::vector<BatchItem>>> cg;
    std::map<std::tuple<int, int, int, int>, size_t> csmem;
    std::vector<ConvertBatchArgs> cv;
    std::vector<BatchItem> cmap;
    for (int i = 0; i < b->n; ++i) {
        mgrit_ctx *c = b->ctx[i];
        if (only && std::find(only->begin(), only->end(), i) == only->end()) continue;
        ClusterLaunch lc;
        if (b->ck[i] >= 2 && batch_cluster_shape(c->nx, c->flux, b->ck[i], &lc)) {
            const auto key = std::make_tuple(c->flux, lc.cpt, lc.K, lc.threads);
            auto &e = cg[key];
            const int ai = (int)e.first.size();
            e.first.push_back(coarse_args(c));
            e.second.push_back(BatchItem{ai, 0, i, 0});
            csmem[key] = std::max(csmem[key], lc.smem);
        } else {
            sg.add(i, c->flux, b->cpt64[i], coarse_args(c), 1);
        }
        if (c->f32) {
            const long long n = (long long)(c->nt_l[c->L - 1] + 1) * c->nx;
            const int nb = (int)std::min<long long>((n + 255) / 256, 64);
            const int ai = (int)cv.size();
            cv.push_back(ConvertBatchArgs{static_cast<const double *>(c->u[c->L - 1]), c->u32c, n});
            for (int k = 0; k < nb; ++k) cmap.push_back(BatchItem{ai, nb, i, k});
        }
    }
    int st;
    if ((st = sg.emit(b, out))) return st;
    for (auto &kv : cg) {
        BLaunch L;
        memset(&L, 0, sizeof L);
        L.kind = 4;
        L.fn = btable().seqc64[std::get<0>(kv.first)][std::get<1>(kv.first) - 1];
        L.un_f32 = std::get<2>(kv.first);   // cluster size
        L.threads = std::get<3>(kv.first);
        L.smem = csmem[kv.first];
        L.nblocks = (int)kv.second.second.size() * L.un_f32;
        SlabArgs<double> *da;
        if ((st = upload(b, kv.second.first, &da))) return st;
        if ((st = upload(b, kv.second.second, &L.d_map))) return st;
        L.d_args = da;
        if (L.un_f32 > 8) BCK(cudaFuncSetAttribute(L.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        BCK(cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
        out.push_back(L);
    }
    if (!cv.empty()) {
        BLaunch L;
        memset(&L, 0, sizeof L);
        L.kind = 3;
        L.nblocks = (int)cmap.size();
        ConvertBatchArgs *da;
        if ((st = upload(b, cv, &da))) return st;
        if ((st = upload(b, cmap, &L.d_map))) return st;
        L.d_args = da;
        out.push_back(L);
    }
    return MGRIT_OK;
}

static int emit_norm(mgrit_batch *b, std::vector<BLaunch> &out)
{
    std::vector<NormBatchArgs> na;
    for (int i = 0; i < b->n; ++i)
        na.push_back(NormBatchArgs{b->ctx[i]->partials, b->ctx[i]->nparts, b->d_norms + i});
    BLaunch L;
    memset(&L, 0, sizeof L);
    L.kind = 2;
    L.nblocks = b->n;
    NormBatchArgs *da;
    int st;
    if ((st = upload(b, na, &da))) return st;
    L.d_args = da;
    out.push_back(L);
    return MGRIT_OK;
}

static cudaError_t enqueue_blaunch(const mgrit_batch *b, const BLaunch &L, cudaStream_t s)
{
    switch (L.kind) {
    case 0: {
        const int *act = b->d_active;
        void *d_args = L.d_args;
        BatchItem *d_map = L.d_map;
        void *args[] = {&d_args, &d_map, (void *)&act};
        return cudaLaunchKernel(L.fn, dim3(L.nblocks), dim3(L.threads), args, L.smem, s);
    }
    case 1:
        return launch_restrict_batch(static_cast<const RestrictBatchArgs *>(L.d_args), L.d_map,
                                     L.nblocks, L.state_f32, L.un_f32, b->d_active, s);
    case 2:
        return launch_norm_batch(static_cast<const NormBatchArgs *>(L.d_args), L.nblocks,
                                 b->d_active, s);
    case 3:
        return launch_convert_batch(static_cast<const ConvertBatchArgs *>(L.d_args), L.d_map,
                                    L.nblocks, b->d_active, s);
    default: {   // one cluster of L.un_f32 CTAs per item
        const int *act = b->d_active;
        void *d_args = L.d_args;
        BatchItem *d_map = L.d_map;
        void *args[] = {&d_args, &d_map, (void *)&act};
        return launch_in_clusters(L.fn, L.un_f32, L.nblocks, L.threads, L.smem, s, args);
    }
    }
}

static int batch_capture(mgrit_batch *b, const std::vector<BLaunch> &ls, cudaGraphExec_t *out)
{
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (const BLaunch &L : ls)
        if ((e = enqueue_blaunch(b, L, b->cap)) != cudaSuccess) break;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(b, MGRIT_ECUDA, "batch graph capture: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, MGRIT_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    return MGRIT_OK;
}

// One operation of an instance's cycle below level 0 at level l (kind 0
// relaxation, 1 restriction, 2 coarsest solve, 3 interpolation), in the
// order emit_cycle launches them for a single instance
struct BOp {
    int kind, l;
};

static void cycle_ops(const mgrit_ctx *c, int l, bool fcycle, std::vector<BOp> &out)
{
    if (l == c->L - 1) {
        out.push_back(BOp{2, l});
        return;
    }
    for (int pass = 0; pass < (fcycle ? 2 : 1); ++pass) {
        out.push_back(BOp{0, l});
        out.push_back(BOp{1, l});
        cycle_ops(c, l + 1, fcycle && pass == 0, out);   // F-cycle, then one V-cycle
        out.push_back(BOp{3, l});
    }
}

// Graph B from each instance's own launch order.  The F-cycle's order depends
// on the instance's depth, so instances are not aligned by level: each phase
// takes the operation kind that most instances have next (ties: the lower
// kind) and advances every instance whose next operation is of that kind, at
// that instance's own level.  Instances are independent, so any interleaving
// that keeps each instance's order computes what the single-instance graphs do.
static int emit_merged_cycle(mgrit_batch *b, bool fcycle, std::vector<BLaunch> &out)
{
    const bool f32 = b->p.precision == 32;
    std::vector<std::vector<BOp>> ops(b->n);
    for (int i = 0; i < b->n; ++i) cycle_ops(b->ctx[i], 1, fcycle, ops[i]);
    std::vector<size_t> pos(b->n, 0);
    for (;;) {
        int cnt[4] = {0, 0, 0, 0};
        for (int i = 0; i < b->n; ++i)
            if (pos[i] < ops[i].size()) ++cnt[ops[i][pos[i]].kind];
        int k = 0;
        for (int q = 1; q < 4; ++q)
            if (cnt[q] > cnt[k]) k = q;
        if (cnt[k] == 0) return MGRIT_OK;
        InstLevels il;
        std::vector<int> inst;
        for (int i = 0; i < b->n; ++i) {
            if (pos[i] >= ops[i].size() || ops[i][pos[i]].kind != k) continue;
            il.push_back(std::make_pair(i, ops[i][pos[i]].l));
            inst.push_back(i);
            ++pos[i];
        }
        int st;
        switch (k) {
        case 0: st = f32 ? emit_relax_at<float>(b, il, out) : emit_relax_at<double>(b, il, out); break;
        case 1: st = emit_restrict_at(b, il, out); break;
        case 2: st = emit_coarse(b, out, &inst); break;
        default: st = f32 ? emit_interp_at<float>(b, il, out) : emit_interp_at<double>(b, il, out); break;
        }
        if (st) return st;
    }
}

static int batch_build(mgrit_batch *b)
{
    batch_free_tables(b);
    const bool f32 = b->p.precision == 32;
    int st;
    // graph A: level-0 relaxation, restriction to level 1, norms
    if ((st = f32 ? emit_relax<float>(b, 0, b->A) : emit_relax<double>(b, 0, b->A))) return st;
    if ((st = emit_restrict(b, 0, b->A))) return st;
    if ((st = emit_norm(b, b->A))) return st;
    // graph B: deeper levels, coarsest solves, interpolation
    if (b->p.cycle == MGRIT_CYCLE_F) {
        if ((st = emit_merged_cycle(b, true, b->B))) return st;
        if ((st = batch_capture(b, b->A, &b->gA))) return st;
        return batch_capture(b, b->B, &b->gB);
    }
    for (int d = 1; d <= b->maxL - 2; ++d) {
        if ((st = f32 ? emit_relax<float>(b, d, b->B) : emit_relax<double>(b, d, b->B))) return st;
        if ((st = emit_restrict(b, d, b->B))) return st;
    }
    if ((st = emit_coarse(b, b->B))) return st;
    for (int d = b->maxL - 2; d >= 1; --d)
        if ((st = f32 ? emit_interp<float>(b, d, b->B) : emit_interp<double>(b, d, b->B))) return st;
    if ((st = batch_capture(b, b->A, &b->gA))) return st;
    return batch_capture(b, b->B, &b->gB);
}

extern "C" int mgrit_batch_create(mgrit_batch **out, const mgrit_instance *inst, int n,
                                  const mgrit_params *params)
{
    mgrit_batch *b = nullptr;
    if (!out || !inst || n < 1) return bfail(b, MGRIT_EINVAL, "bad batch arguments");
    *out = nullptr;
    mgrit_params p;
    if (params) p = *params; else mgrit_default_params(&p);
    b = new (std::nothrow) mgrit_batch();
    if (!b) return bfail(nullptr, MGRIT_ENOMEM, "host allocation failed");
    b->n = n;
    b->p = p;
    b->maxL = 0;
    b->d_active = nullptr;
    b->h_active = nullptr;
    b->d_norms = nullptr;
    b->h_norms = nullptr;
    b->gA = b->gB = nullptr;
    b->cap = nullptr;
    b->err[0] = 0;
    int st = MGRIT_OK;
    for (int i = 0; i < n && st == MGRIT_OK; ++i) {
        const mgrit_instance &d = inst[i];
        if (d.scheme != MGRIT_WENO5_SSPRK3) {
            st = bfail(b, MGRIT_EINVAL, "instance %d: batches run WENO5/SSPRK3 only", i);
            break;
        }
        mgrit_ctx *c = nullptr;
        st = mgrit_create(&c, d.nx, d.nt, d.m, d.levels, d.scheme, d.flux);
        if (st) {
            bfail(b, st, "instance %d: %s", i, mgrit_last_error(nullptr));
            break;
        }
        b->ctx.push_back(c);
        mgrit_params pi = p;
        pi.T = d.T;
        if ((st = mgrit_set_params(c, &pi))) {
            bfail(b, st, "instance %d: %s", i, c->err);
            break;
        }
        const Launch &ln = p.precision == 32 ? c->ln32 : c->ln64;
        if (cpt_index(ln.cpt) < 0 || cpt_index(ln.cpt) > 4 || !c->ln64.slab) {
            st = bfail(b, MGRIT_EINVAL, "instance %d: nx = %d exceeds the batched slab limit", i, d.nx);
            break;
        }
        b->cpt.push_back(ln.cpt);
        b->cpt64.push_back(c->ln64.cpt);
        b->ck.push_back(1);   // set from the occupancy rule once the context has allocated
        b->maxL = std::max(b->maxL, d.levels);
        if ((st = mgrit_ensure_alloc(c))) {
            bfail(b, st, "instance %d: %s", i, c->err);
            break;
        }
        b->ck.back() = c->lc64.fn ? c->lc64.K : 1;
    }
    mgrit_batch *bb = b;
    auto cleanup = [&]() { mgrit_batch_destroy(bb); };
    if (st) {
        // keep the message for mgrit_last_error(NULL)
        snprintf(g_create_err, sizeof g_create_err, "%s", b->err);
        cleanup();
        return st;
    }
    cudaError_t e;
    if ((e = cudaMalloc((void **)&b->d_active, sizeof(int) * n)) ||
        (e = cudaMallocHost((void **)&b->h_active, sizeof(int) * n)) ||
        (e = cudaMalloc((void **)&b->d_norms, sizeof(double) * n)) ||
        (e = cudaMallocHost((void **)&b->h_norms, sizeof(double) * n)) ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking))) {
        snprintf(g_create_err, sizeof g_create_err, "batch allocation: %s", cudaGetErrorString(e));
        cleanup();
        return MGRIT_ENOMEM;
    }
    if ((st = batch_build(b))) {
        snprintf(g_create_err, sizeof g_create_err, "%s", b->err);
        cleanup();
        return st;
    }
    *out = b;
    return MGRIT_OK;
}

static int batch_init(mgrit_batch *b, const double *const *u0_dev, cudaStream_t s)
{
    if (!u0_dev) return bfail(b, MGRIT_EINVAL, "u0_dev is NULL");
    for (int i = 0; i < b->n; ++i) {
        if (!u0_dev[i]) return bfail(b, MGRIT_EINVAL, "u0_dev[%d] is NULL", i);
        int st = init_iterate(b->ctx[i], u0_dev[i], s);
        if (st) return bfail(b, st, "instance %d: %s", i, b->ctx[i]->err);
        b->ctx[i]->prepared = true;
        b->h_active[i] = 1;
    }
    BCK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * b->n, cudaMemcpyHostToDevice, s));
    return MGRIT_OK;
}

extern "C" int mgrit_batch_run_cycles(mgrit_batch *b, const double *const *u0_dev, int ncycles,
                                      void *stream)
{
    if (!b) return MGRIT_EINVAL;
    if (ncycles < 0) return bfail(b, MGRIT_EINVAL, "ncycles must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int st = batch_init(b, u0_dev, s);
    if (st) return st;
    for (int k = 0; k < ncycles; ++k) {
        BCK(cudaGraphLaunch(b->gA, s));
        BCK(cudaGraphLaunch(b->gB, s));
    }
    for (int i = 0; i < b->n; ++i) b->ctx[i]->have_state = ncycles > 0;
    return MGRIT_OK;
}

extern "C" int mgrit_batch_solve(mgrit_batch *b, const double *const *u0_dev, double *const *uT_dev,
                                 int *status, int *iters, double *final_res, void *stream)
{
    if (!b) return MGRIT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st = batch_init(b, u0_dev, s);
    if (st) return st;
    const int n = b->n;
    std::vector<double> r0(n, 0.0), rm1(n, 0.0), rm2(n, 0.0);
    std::vector<int> stat(n, MGRIT_ENOTCONV), it(n, 0);
    int remaining = n;
    for (int k = 0; remaining > 0; ++k) {
        BCK(cudaGraphLaunch(b->gA, s));
        BCK(cudaMemcpyAsync(b->h_norms, b->d_norms, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) {
            if (!b->h_active[i]) continue;
            const double rk = b->h_norms[i];
            if (k == 0) r0[i] = rk;
            int done = 0;
            if (rk < b->p.tol) { stat[i] = MGRIT_OK; done = 1; }
            else if (!std::isfinite(rk) || rk > 1e8 * r0[i]) { stat[i] = MGRIT_EDIVERGED; done = 1; }
            else if (b->p.precision == 32 && k >= 2 && rk > 0.9 * rm2[i]) { stat[i] = MGRIT_OK; done = 1; }
            else if (k >= b->p.max_iter) { stat[i] = MGRIT_ENOTCONV; done = 1; }
            rm2[i] = rm1[i];
            rm1[i] = rk;
            it[i] = k;
            if (final_res) final_res[i] = rk;
            if (done) {
                b->h_active[i] = 0;
                --remaining;
            }
        }
        if (remaining == 0) break;
        BCK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
        BCK(cudaGraphLaunch(b->gB, s));
    }
    for (int i = 0; i < n; ++i) {
        b->ctx[i]->have_state = true;
        if (uT_dev && uT_dev[i] && (st = copy_out(b->ctx[i], uT_dev[i], b->ctx[i]->nC_l[0], 1, s)))
            return bfail(b, st, "instance %d: %s", i, b->ctx[i]->err);
        if (status) status[i] = stat[i];
        if (iters) iters[i] = it[i];
    }
    BCK(cudaStreamSynchronize(s));
    return MGRIT_OK;
}

// time `reps` replays of a list of launches (after one warm-up replay)
static int time_launches(mgrit_batch *b, const std::vector<BLaunch> &ls, int reps, cudaStream_t s,
                         cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    for (const BLaunch &L : ls) BCK(enqueue_blaunch(b, L, s));
    BCK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
        for (const BLaunch &L : ls) BCK(enqueue_blaunch(b, L, s));
    BCK(cudaEventRecord(e1, s));
    BCK(cudaEventSynchronize(e1));
    BCK(cudaEventElapsedTime(ms, e0, e1));
    return MGRIT_OK;
}

static void drop_tables(mgrit_batch *b, size_t keep)
{
    for (size_t t = keep; t < b->tables.size(); ++t) cudaFree(b->tables[t]);
    b->tables.resize(keep);
}

// Autotuner.  (1) For every group of instances with the same (flux, nx), time
// the level-0 relaxation with 1x, 2x and 4x the minimal cells per thread
// (fewer, fuller threads) and keep the fastest.  (2) The cluster policy of the
// coarsest solves, timed on the whole coarsest phase (timed one group at a
// time, the largest clusters win, but all groups run together and 16-CTA
// clusters cannot all be resident at once).  (3) Whole cycles with the tuned
// and the rule cluster policy, the faster kept.  Then rebuild the graphs.
extern "C" int mgrit_batch_autotune(mgrit_batch *b, const double *const *u0_dev, int reps,
                                    void *stream)
{
    if (!b) return MGRIT_EINVAL;
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    int st = batch_init(b, u0_dev, s);
    if (st) return st;
    const bool f32 = b->p.precision == 32;
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (int i = 0; i < b->n; ++i) groups[std::make_pair(b->ctx[i]->flux, b->ctx[i]->nx)].push_back(i);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (auto &kv : groups) {
        const std::vector<int> &ids = kv.second;
        const int base = b->cpt[ids[0]];
        int best = base;
        float best_ms = 1e30f;
        for (int mul = 1; mul <= 4; mul *= 2) {
            const int cpt = base * mul;
            if (cpt_index(cpt) < 0 || cpt_index(cpt) > 4) break;
            for (int i : ids) b->cpt[i] = cpt;
            std::vector<BLaunch> mine;   // the level-0 relaxation of this group only
            const size_t keep = b->tables.size();
            if ((st = f32 ? emit_relax<float>(b, 0, mine, &ids) : emit_relax<double>(b, 0, mine, &ids)))
                break;
            for (const BLaunch &L : mine) BCK(enqueue_blaunch(b, L, s));   // warm-up
            BCK(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r)
                for (const BLaunch &L : mine) BCK(enqueue_blaunch(b, L, s));
            BCK(cudaEventRecord(e1, s));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            for (size_t t = keep; t < b->tables.size(); ++t) cudaFree(b->tables[t]);
            b->tables.resize(keep);
            if (ms < best_ms) {
                best_ms = ms;
                best = cpt;
            }
        }
        if (st) break;
        for (int i : ids) b->cpt[i] = best;
    }
    // (2) The coarsest solves of all instances run together (one launch per
    // shape class), so the cluster policy is timed on the whole phase:
    // the single-instance occupancy rule K0, K0 / 2, 2 K0 (at most 16) and one
    // CTA for every instance; a size that does not fit falls back to one CTA
    if (!st) {
        std::vector<int> rule(b->n);
        for (int i = 0; i < b->n; ++i) rule[i] = b->ctx[i]->lc64.fn ? b->ctx[i]->lc64.K : 1;
        int best_policy = 0;
        float best_ms = 1e30f;
        for (int policy = 0; policy < 4 && !st; ++policy) {
            for (int i = 0; i < b->n; ++i) {
                int K = rule[i];
                if (K >= 2) K = policy == 0 ? K : policy == 1 ? K / 2 : policy == 2 ? std::min(2 * K, CLUSTER_MAX) : 1;
                ClusterLaunch lc;
                b->ck[i] = (K >= 2 && batch_cluster_shape(b->ctx[i]->nx, b->ctx[i]->flux, K, &lc)) ? K : 1;
            }
            std::vector<BLaunch> mine;
            const size_t keep = b->tables.size();
            float ms = 0.f;
            if ((st = emit_coarse(b, mine)) == MGRIT_OK) st = time_launches(b, mine, reps, s, e0, e1, &ms);
            drop_tables(b, keep);
            if (!st && ms < best_ms) {
                best_ms = ms;
                best_policy = policy;
            }
        }
        for (int i = 0; i < b->n; ++i) {
            int K = rule[i];
            if (K >= 2)
                K = best_policy == 0 ? K : best_policy == 1 ? K / 2
                  : best_policy == 2 ? std::min(2 * K, CLUSTER_MAX) : 1;
            ClusterLaunch lc;
            b->ck[i] = (K >= 2 && batch_cluster_shape(b->ctx[i]->nx, b->ctx[i]->flux, K, &lc)) ? K : 1;
        }
    }
    // (3) End to end: stage 2 timed the coarsest phase alone; whole cycles
    // (graphs A and B) with the tuned and the rule policy decide
    if (!st) {
        const std::vector<int> tuned_ck = b->ck;
        std::vector<int> rule_ck(b->n);
        for (int i = 0; i < b->n; ++i) rule_ck[i] = b->ctx[i]->lc64.fn ? b->ctx[i]->lc64.K : 1;
        int best = 0;
        float best_ms = 1e30f;
        for (int combo = 0; combo < 2 && !st; ++combo) {
            b->ck = combo ? rule_ck : tuned_ck;
            if ((st = batch_build(b))) break;
            float ms = 0.f;
            BCK(cudaGraphLaunch(b->gA, s));   // warm-up
            BCK(cudaGraphLaunch(b->gB, s));
            BCK(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) {
                BCK(cudaGraphLaunch(b->gA, s));
                BCK(cudaGraphLaunch(b->gB, s));
            }
            BCK(cudaEventRecord(e1, s));
            BCK(cudaEventSynchronize(e1));
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = combo;
            }
        }
        b->ck = best ? rule_ck : tuned_ck;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    return batch_build(b);
}

// Profiling hook: the batched level-0 relaxation phase, `reps` times, from
// launch tables of its own (dropped once the launches have finished).
extern "C" int mgrit_batch_launch_relax(mgrit_batch *b, int reps, void *stream)
{
    if (!b) return MGRIT_EINVAL;
    if (reps < 1) return bfail(b, MGRIT_EINVAL, "reps must be at least 1");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BLaunch> ls;
    const size_t keep = b->tables.size();
    int st = b->p.precision == 32 ? emit_relax<float>(b, 0, ls) : emit_relax<double>(b, 0, ls);
    for (int r = 0; r < reps && !st; ++r)
        for (const BLaunch &L : ls)
            if (enqueue_blaunch(b, L, s) != cudaSuccess) {
                st = bfail(b, MGRIT_ECUDA, "launch: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
    if (cudaStreamSynchronize(s) != cudaSuccess && !st)
        st = bfail(b, MGRIT_ECUDA, "synchronise: %s", cudaGetErrorString(cudaGetLastError()));
    drop_tables(b, keep);
    return st;
}

extern "C" double mgrit_batch_cycle_cell_updates(const mgrit_batch *b)
{
    if (!b) return 0.0;
    double s = 0.0;
    for (const mgrit_ctx *c : b->ctx) s += mgrit_cycle_cell_updates(c);
    return s;
}

extern "C" int mgrit_batch_query(const mgrit_batch *b, int instance, int what)
{
    if (!b || instance < 0 || instance >= b->n) return -1;
    switch (what) {
    case 0: return b->cpt[instance];
    case 1: return threads_for(b->ctx[instance]->nx, b->cpt[instance]);
    case 2: return b->ctx[instance]->L;
    case 3: return 1;   // one work item (slab) per CTA
    case 4: return b->ck[instance];
    default: return -1;
    }
}

extern "C" int mgrit_batch_copy_cpoints(mgrit_batch *b, int instance, double *uC_out_dev, void *stream)
{
    if (!b || instance < 0 || instance >= b->n) return MGRIT_EINVAL;
    return mgrit_copy_cpoints(b->ctx[instance], uC_out_dev, stream);
}

extern "C" const char *mgrit_batch_last_error(const mgrit_batch *b)
{
    return b ? b->err : g_create_err;
}

extern "C" void mgrit_batch_destroy(mgrit_batch *b)
{
    if (!b) return;
    batch_free_tables(b);
    for (mgrit_ctx *c : b->ctx) mgrit_destroy(c);
    cudaFree(b->d_active);
    cudaFree(b->d_norms);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_norms) cudaFreeHost(b->h_norms);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}
