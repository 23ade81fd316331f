// Adjoint entry points of the C ABI (declared in include/mgrit.h):
// mgrit_step_vjp, mgrit_adjoint_serial and mgrit_adjoint.
//
// Adjoint MGRIT data in HBM, all FP64, mirroring the forward solver's layout
// with the time axis reversed (row k of a level = reversed point k, i.e.
// forward point N_l - k):
//   traj        forward fine states u^0..u^{N-1}, regenerated from the
//               forward C-point checkpoints by one launch (chunk j from uC_j)
//   level 0     C-points live in u[1]; newC[0], phirow[0], cstep[0]
//   0 < l < L-1 u[l], g[l] ((N_l+1) rows), newC/phirow/cstep[l]
//   l = L-1     u[L-1], g[L-1]
//   scratch     one row per relaxation CTA (the stage state u1 of a VJP)
//   cps         nt/m forward checkpoints of the serial adjoint
// One cycle = graph A (level-0 relaxation, residual + restriction, norm) and
// graph B (coarser levels, coarsest solve, interpolation), as forward.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "adj_table.cuh"
#include "ctx.cuh"
#include "restrict.cuh"

using namespace mgrit;

namespace mgrit {

struct AdjWork {
    const void *fn;      // k_adjoint instance for (scheme, flux, cells per thread)
    int threads, cpt;
    size_t smem;
    // sequential chains (coarsest adjoint solve, serial adjoint) on a cluster:
    // k_adjoint_cluster instance, null if nx < 512 or no cluster fits
    const void *cfn;
    int cK, cthreads;
    size_t csmem, cfwd;
    // chunks of level l (relaxation, interpolation, trajectory at level 0,
    // the single VJP) on clusters: k_adjoint_cluster_chunk instance, null for
    // one CTA per chunk; chosen for the chunk_clusters value in lr_cc
    struct Shape {
        const void *fn;
        int K, threads;
        size_t smem, fwd;
    } lr[MAXLEV];
    int lr_cc;
    double *traj;
    double *u[MAXLEV], *g[MAXLEV];
    double *newC[MAXLEV], *phirow[MAXLEV], *cstep[MAXLEV];
    double *scratch;
    double *cps;
    double *partials;
    int nparts;
    double *d_norm;
    cudaGraphExec_t gA, gB;
};

}  // namespace mgrit

static const AdjTable &adj_table()
{
    static AdjTable t = [] {
        AdjTable k;
        memset(&k, 0, sizeof k);
        fill_adj_all(k);
        return k;
    }();
    return t;
}

void mgrit_adj_drop_graphs(mgrit_ctx *ctx)
{
    AdjWork *w = ctx->adj;
    if (!w) return;
    if (w->gA) cudaGraphExecDestroy(w->gA);
    if (w->gB) cudaGraphExecDestroy(w->gB);
    w->gA = w->gB = nullptr;
}

void mgrit_adj_free(mgrit_ctx *ctx)
{
    AdjWork *w = ctx->adj;
    if (!w) return;
    if (w->gA) cudaGraphExecDestroy(w->gA);
    if (w->gB) cudaGraphExecDestroy(w->gB);
    for (int l = 0; l < MAXLEV; ++l) {
        cudaFree(w->u[l]);
        cudaFree(w->g[l]);
        cudaFree(w->newC[l]);
        cudaFree(w->phirow[l]);
        cudaFree(w->cstep[l]);
    }
    cudaFree(w->traj);
    cudaFree(w->scratch);
    cudaFree(w->cps);
    cudaFree(w->partials);
    cudaFree(w->d_norm);
    delete w;
    ctx->adj = nullptr;
}

// smallest cells-per-thread giving at most 512 threads per CTA, if the
// adjoint slab's shared memory fits
static bool adj_choose(const mgrit_ctx *ctx, AdjWork *w)
{
    if (ctx->scheme != MGRIT_WENO5_SSPRK3 && ctx->scheme != MGRIT_FO_FE) return false;
    const size_t smem = adj_smem_bytes<double>(ctx->nx);
    if (smem > 227 * 1024) return false;
    static const int cpts[NCPT_ADJ] = {1, 2, 4, 8};
    for (int ci = 0; ci < NCPT_ADJ; ++ci) {
        const int need = (ctx->nx + cpts[ci] - 1) / cpts[ci];
        if (need <= 512) {
            w->cpt = cpts[ci];
            w->threads = ((need + 31) / 32) * 32;
            w->smem = smem;
            w->fn = adj_table().k[ctx->scheme][ctx->flux][ci];
            return w->fn != nullptr;
        }
    }
    return false;
}

static int adj_check(mgrit_ctx *ctx)
{
    if (ctx->scheme == MGRIT_LF_FE)
        return mgrit_fail(ctx, MGRIT_EINVAL, "the adjoint covers the WENO5 and first-order schemes");
    if (ctx->p.numflux != MGRIT_LF_SPLIT)
        return mgrit_fail(ctx, MGRIT_EINVAL, "the adjoint differentiates the split numerical flux only");
    AdjWork probe;
    memset(&probe, 0, sizeof probe);
    // one CTA holds up to 4096 cells; wider slices run on clusters of up to
    // 16 CTAs x 1024 cells
    if (!adj_choose(ctx, &probe) && ctx->nx > CLUSTER_MAX * 1024)
        return mgrit_fail(ctx, MGRIT_EINVAL, "nx = %d exceeds the adjoint limit (16384)", ctx->nx);
    return MGRIT_OK;
}

static int adj_alloc(mgrit_ctx *ctx, AdjWork *w)
{
    int st;
    const int L = ctx->L;
    const size_t es = sizeof(double);
    if ((st = mgrit_dalloc(ctx, (void **)&w->traj, ctx->nt, es))) return st;
    for (int l = 1; l < L; ++l) {
        if ((st = mgrit_dalloc(ctx, (void **)&w->u[l], ctx->nt_l[l] + 1, es))) return st;
        if ((st = mgrit_dalloc(ctx, (void **)&w->g[l], ctx->nt_l[l] + 1, es))) return st;
    }
    for (int l = 0; l < L - 1; ++l) {
        if ((st = mgrit_dalloc(ctx, (void **)&w->newC[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = mgrit_dalloc(ctx, (void **)&w->phirow[l], ctx->nC_l[l] + 1, es))) return st;
        if ((st = mgrit_dalloc(ctx, (void **)&w->cstep[l], ctx->nC_l[l], es))) return st;
    }
    const int srows = ctx->nC_l[0] + 1 > 1 + ctx->m ? ctx->nC_l[0] + 1 : 1 + ctx->m;
    if ((st = mgrit_dalloc(ctx, (void **)&w->scratch, srows, es))) return st;
    if ((st = mgrit_dalloc(ctx, (void **)&w->cps, ctx->nC_l[0], es))) return st;
    w->nparts = restrict_blocks(ctx->nC_l[0], ctx->nx);
    CK(cudaMalloc((void **)&w->partials, sizeof(double) * w->nparts));
    CK(cudaMalloc((void **)&w->d_norm, sizeof(double)));
    if (w->fn) CK(cudaFuncSetAttribute(w->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN));
    return MGRIT_OK;
}

// One cluster shape for the sequential adjoint chains: K CTAs of at most 1024
// and at least 64 cells each (1 or 2 cells per thread), if it can be
// co-scheduled.
static bool adj_cluster_shape(const mgrit_ctx *ctx, int K, AdjWork *w)
{
    const int nx = ctx->nx;
    const int nmax = (nx + K - 1) / K;
    if (K < 2 || K > CLUSTER_MAX || nmax > 1024 || nmax < 64) return false;
    const int cpt = nmax <= 512 ? 1 : 2;
    const void *fn = adj_table().kc[ctx->scheme][ctx->flux][cpt - 1];
    const size_t fwd = cluster_smem_bytes<double>(nx, K);
    const size_t smem = fwd + cluster_adj_extra_bytes<double>(nx, K);
    const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
    if (!fn || !cluster_fits(fn, K, threads, smem)) return false;
    w->cfn = fn;
    w->cK = K;
    w->cthreads = threads;
    w->csmem = smem;
    w->cfwd = fwd;
    return true;
}

static AdjArgs adj_base(const mgrit_ctx *ctx, int mode, int l);
static cudaError_t adj_launch_seq(const mgrit_ctx *ctx, cudaStream_t s, AdjArgs *a);

// Cluster for the sequential adjoint chains.  The forward stepper's rule
// gives K0: the largest power of two K <= 16 leaving at least 256 cells per
// CTA, reduced until one cluster of that shape can be co-scheduled (nx < 512:
// none, one CTA).  A transposed step is latency-bound on its cluster (four
// cluster barriers per stage), so K0, 2 K0 and 4 K0 (at most 16, at least 64
// cells per CTA) are timed on 8 steps of the coarsest adjoint solve on zero
// data, and the fastest is kept.
static int adj_choose_cluster(mgrit_ctx *ctx, AdjWork *w)
{
    w->cfn = nullptr;
    const int nx = ctx->nx;
    int K = 1;
    while (K < CLUSTER_MAX && nx / (2 * K) >= 256) K *= 2;
    for (; K >= 2; K /= 2)
        if (adj_cluster_shape(ctx, K, w)) break;
    if (!w->cfn) return MGRIT_OK;
    const int K0 = w->cK;
    const int l = ctx->L - 1;
    AdjArgs a = adj_base(ctx, ADJ_SEQ, l);
    a.src = w->g[l];
    a.g = w->g[l];
    a.rows = w->u[l];
    a.nsteps = ctx->nt_l[l] < 8 ? ctx->nt_l[l] : 8;
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    cudaStream_t s = ctx->cap;
    CK(cudaMemsetAsync(w->traj, 0, sizeof(double) * (size_t)ctx->nt * nx, s));
    CK(cudaMemsetAsync(w->g[l], 0, sizeof(double) * (size_t)(ctx->nt_l[l] + 1) * nx, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int bestK = K0;
    float best = -1.f;
    for (int k = K0; k <= 4 * K0 && k <= CLUSTER_MAX; k *= 2) {
        if (!adj_cluster_shape(ctx, k, w)) continue;
        float ms = 0.f;
        CK(adj_launch_seq(ctx, s, &a));   // warm-up
        CK(cudaEventRecord(e0, s));
        CK(adj_launch_seq(ctx, s, &a));
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best < 0.f || ms < best) {
            best = ms;
            bestK = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    adj_cluster_shape(ctx, bestK, w);
    return MGRIT_OK;
}

// Cluster shape for the adjoint chunks of level l, by the forward rule: with a
// one-CTA adjoint slab, the largest K in {16, 8, 4, 2} with chunks x K <= SMs
// and 256..1024 cells per CTA, else none; without one (nx > 4096), that K if
// it exists, else the smallest K with at most 1024 cells per CTA.
static void adj_choose_level(const mgrit_ctx *ctx, AdjWork *w, int l)
{
    AdjWork::Shape fill, any;   // largest K that fills the SMs; smallest K that fits
    memset(&fill, 0, sizeof fill);
    memset(&any, 0, sizeof any);
    memset(&w->lr[l], 0, sizeof w->lr[l]);
    if (w->fn && !ctx->p.chunk_clusters) return;
    const int nx = ctx->nx, items = ctx->nC_l[l] + 1;
    for (int K = CLUSTER_MAX; K >= 2; K /= 2) {
        const int nmax = (nx + K - 1) / K;
        if (nmax > 1024) break;   // smaller K would not fit either
        const bool fills = (long long)items * K <= ctx->nsm;
        if (w->fn && (!fills || nmax < 256)) continue;
        const int cpt = nmax <= 512 ? 1 : 2;
        const void *fn = adj_table().kcc[ctx->scheme][ctx->flux][cpt - 1];
        const size_t fwd = cluster_smem_bytes<double>(nx, K);
        const size_t smem = fwd + cluster_adj_extra_bytes<double>(nx, K);
        const int threads = (((nmax + cpt - 1) / cpt + 31) / 32) * 32;
        if (!fn || smem > (size_t)SMEM_OPTIN) continue;
        if (!cluster_fits(fn, K, threads, smem)) continue;
        const AdjWork::Shape c{fn, K, threads, smem, fwd};
        if (fills && !fill.fn) fill = c;
        any = c;
    }
    if (fill.fn) w->lr[l] = fill;
    else if (!w->fn) w->lr[l] = any;
}

static int adj_choose_levels(mgrit_ctx *ctx, AdjWork *w)
{
    for (int l = 0; l < ctx->L - 1; ++l) {
        adj_choose_level(ctx, w, l);
        if (!w->fn && !w->lr[l].fn)
            return mgrit_fail(ctx, MGRIT_EINVAL, "no adjoint slab or cluster fits nx = %d", ctx->nx);
    }
    w->lr_cc = ctx->p.chunk_clusters;
    return MGRIT_OK;
}

// adjoint workspaces on first use; a failed allocation leaves none behind
static int adj_ensure(mgrit_ctx *ctx)
{
    int st;
    if ((st = adj_check(ctx))) return st;
    if ((st = mgrit_ensure_alloc(ctx))) return st;
    if (ctx->adj) {
        // chunk shapes follow chunk_clusters (set_params dropped the graphs)
        if (ctx->adj->lr_cc != ctx->p.chunk_clusters) return adj_choose_levels(ctx, ctx->adj);
        return MGRIT_OK;
    }
    AdjWork *w = new (std::nothrow) AdjWork;
    if (!w) return mgrit_fail(ctx, MGRIT_ENOMEM, "host allocation failed");
    memset(w, 0, sizeof *w);
    ctx->adj = w;
    adj_choose(ctx, w);
    if ((st = adj_alloc(ctx, w))) {
        mgrit_adj_free(ctx);
        return st;
    }
    if ((st = adj_choose_cluster(ctx, w))) {
        mgrit_adj_free(ctx);
        return st;
    }
    if (!w->fn && !w->cfn) {
        mgrit_adj_free(ctx);
        return mgrit_fail(ctx, MGRIT_EINVAL, "no adjoint cluster fits nx = %d", ctx->nx);
    }
    if ((st = adj_choose_levels(ctx, w))) {
        mgrit_adj_free(ctx);
        return st;
    }
    return MGRIT_OK;
}

static AdjArgs adj_base(const mgrit_ctx *ctx, int mode, int l)
{
    const AdjWork *w = ctx->adj;
    AdjArgs a;
    memset(&a, 0, sizeof a);
    a.mode = mode;
    a.nx = ctx->nx;
    a.m = ctx->m;
    a.nC = ctx->nC_l[l];
    a.fcf = ctx->p.relax == MGRIT_RELAX_FCF;
    a.dxinv = ctx->nx / ctx->p.L;
    a.dt = ctx->dt_l[l];
    a.dtc = l + 1 < ctx->L ? ctx->dt_l[l + 1] : 0.0;
    a.N = ctx->nt;
    long long s = 1;
    for (int k = 0; k < l; ++k) s *= ctx->m;
    a.s = s;
    a.sc = s * ctx->m;
    a.traj = w->traj;
    a.nrows_traj = ctx->nt;
    a.scratch = w->scratch;
    return a;
}

static cudaError_t adj_launch(const mgrit_ctx *ctx, int grid, cudaStream_t s, AdjArgs *a)
{
    const AdjWork *w = ctx->adj;
    void *args[] = {a};
    return cudaLaunchKernel(w->fn, dim3(grid), dim3(w->threads), args, w->smem, s);
}

// `chunks` chunks of level l (ADJ_RELAX, ADJ_INTERP, ADJ_TRAJ, ADJ_VJP): one
// cluster each if chosen, else one CTA each
static cudaError_t adj_launch_chunks(const mgrit_ctx *ctx, int l, int chunks, cudaStream_t s, AdjArgs *a)
{
    const AdjWork *w = ctx->adj;
    const AdjWork::Shape &c = w->lr[l];
    if (chunks <= 0) return cudaSuccess;
    if (!c.fn) return w->fn ? adj_launch(ctx, chunks, s, a) : cudaErrorInvalidConfiguration;
    unsigned long long fwd = c.fwd;
    void *args[] = {a, &fwd};
    return launch_in_clusters(c.fn, c.K, (long long)chunks * c.K, c.threads, c.smem, s, args);
}

// a sequential chain (ADJ_SEQ, ADJ_SERIAL): one cluster if chosen, else one CTA
static cudaError_t adj_launch_seq(const mgrit_ctx *ctx, cudaStream_t s, AdjArgs *a)
{
    const AdjWork *w = ctx->adj;
    if (!w->cfn) return adj_launch(ctx, 1, s, a);
    unsigned long long fwd = w->cfwd;
    void *args[] = {a, &fwd};
    return launch_in_clusters(w->cfn, w->cK, w->cK, w->cthreads, w->csmem, s, args);
}

static cudaError_t adj_relax(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    AdjWork *w = ctx->adj;
    AdjArgs a = adj_base(ctx, ADJ_RELAX, l);
    a.uC = l == 0 ? w->u[1] : w->u[l];
    a.strideC = (long long)(l == 0 ? 1 : ctx->m) * ctx->nx;
    a.g = l == 0 ? nullptr : w->g[l];
    a.newC = w->newC[l];
    a.phirow = w->phirow[l];
    a.cstep = w->cstep[l];
    a.nrows_uC = a.nrows_newC = a.nrows_phirow = a.nC + 1;
    a.nrows_cstep = a.nC;
    a.nrows_g = ctx->nt_l[l] + 1;
    return adj_launch_chunks(ctx, l, a.nC + 1, s, &a);
}

static cudaError_t adj_restrict(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    AdjWork *w = ctx->adj;
    RestrictArgs r;
    memset(&r, 0, sizeof r);
    r.newC = w->newC[l];
    r.phirow = w->phirow[l];
    r.cstep = w->cstep[l];
    r.g = l == 0 ? nullptr : w->g[l];
    r.gn = w->g[l + 1];
    r.un = w->u[l + 1];
    r.partials = l == 0 ? w->partials : nullptr;
    r.nrows_g = ctx->nt_l[l] + 1;
    r.nx = ctx->nx;
    r.m = ctx->m;
    r.nC = ctx->nC_l[l];
    r.guess = ctx->p.guess;
    return launch_restrict(r, l == 0 ? w->nparts : restrict_blocks(r.nC, r.nx), s);
}

static cudaError_t adj_coarse(mgrit_ctx *ctx, cudaStream_t s)
{
    AdjWork *w = ctx->adj;
    const int l = ctx->L - 1;
    AdjArgs a = adj_base(ctx, ADJ_SEQ, l);
    a.src = w->g[l];
    a.g = w->g[l];
    a.rows = w->u[l];
    a.nsteps = ctx->nt_l[l];
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    return adj_launch_seq(ctx, s, &a);
}

static cudaError_t adj_interp(mgrit_ctx *ctx, int l, cudaStream_t s)
{
    AdjWork *w = ctx->adj;
    AdjArgs a = adj_base(ctx, ADJ_INTERP, l);
    a.uC = w->u[l + 1];
    a.g = w->g[l];
    a.rows = w->u[l];
    a.nrows_uC = a.nC + 1;
    a.nrows_g = a.nrows_rows = ctx->nt_l[l] + 1;
    return adj_launch_chunks(ctx, l, a.nC, s, &a);
}

static cudaError_t adj_part_a(mgrit_ctx *ctx, cudaStream_t s)
{
    cudaError_t e;
    if ((e = adj_relax(ctx, 0, s))) return e;
    if ((e = adj_restrict(ctx, 0, s))) return e;
    return launch_norm(ctx->adj->partials, ctx->adj->nparts, ctx->adj->d_norm, s);
}

static cudaError_t adj_part_b(mgrit_ctx *ctx, cudaStream_t s)
{
    return mgrit_emit_below_level0(ctx, adj_relax, adj_restrict, adj_coarse, adj_interp, s);
}

static int adj_capture(mgrit_ctx *ctx, cudaError_t (*fn)(mgrit_ctx *, cudaStream_t),
                       cudaGraphExec_t *out)
{
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = fn(ctx, ctx->cap);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return mgrit_fail(ctx, MGRIT_ECUDA, "adjoint graph capture: %s",
                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return mgrit_fail(ctx, MGRIT_ECUDA, "adjoint graph instantiate: %s", cudaGetErrorString(e));
    return MGRIT_OK;
}

extern "C" int mgrit_step_vjp(mgrit_ctx *ctx, const double *u_dev, const double *lam_dev,
                              double *out_dev, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!u_dev || !lam_dev || !out_dev) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st;
    if ((st = adj_ensure(ctx))) return st;
    AdjArgs a = adj_base(ctx, ADJ_VJP, 0);
    a.src = u_dev;
    a.uC = lam_dev;
    a.out = out_dev;
    CK(adj_launch_chunks(ctx, 0, 1, (cudaStream_t)stream, &a));
    return MGRIT_OK;
}

extern "C" int mgrit_adjoint_serial(mgrit_ctx *ctx, const double *u0_dev, const double *lamT_dev,
                                    double *lam0_dev, void *stream)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!u0_dev || !lamT_dev || !lam0_dev) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st;
    if ((st = adj_ensure(ctx))) return st;
    AdjWork *w = ctx->adj;
    AdjArgs a = adj_base(ctx, ADJ_SERIAL, 0);
    a.src = u0_dev;
    a.uC = lamT_dev;
    a.out = lam0_dev;
    a.rows = w->cps;
    a.nrows_rows = ctx->nC_l[0];
    CK(adj_launch_seq(ctx, (cudaStream_t)stream, &a));   // a cluster whenever no one-CTA slab fits
    return MGRIT_OK;
}

extern "C" int mgrit_adjoint(mgrit_ctx *ctx, const double *uC_dev, const double *lamT_dev,
                             double *lam0_dev, double *lamC_dev, void *stream, mgrit_stats *stats)
{
    if (!ctx) return MGRIT_EINVAL;
    if (!uC_dev || !lamT_dev) return mgrit_fail(ctx, MGRIT_EINVAL, "NULL argument");
    int st;
    if ((st = adj_ensure(ctx))) return st;
    AdjWork *w = ctx->adj;
    if (!w->gA && (st = adj_capture(ctx, adj_part_a, &w->gA))) return st;
    if (!w->gB && (st = adj_capture(ctx, adj_part_b, &w->gB))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = ctx->nx, nC = ctx->nC_l[0];
    if (stats) memset(stats, 0, sizeof *stats);
    CK(cudaEventRecord(ctx->ev0, s));
    // forward fine states from the C-point checkpoints
    AdjArgs t = adj_base(ctx, ADJ_TRAJ, 0);
    t.uC = uC_dev;
    t.rows = w->traj;
    t.nrows_uC = nC + 1;
    CK(adj_launch_chunks(ctx, 0, nC, s, &t));
    // initial iterate: every level-0 C-point = lamT; row 0 of every u_l, g_l = lamT
    CK(launch_broadcast_row(lamT_dev, w->u[1], 0, nx, (long long)nC + 1, s));
    for (int l = 1; l < ctx->L; ++l) {
        CK(cudaMemcpyAsync(w->g[l], lamT_dev, sizeof(double) * nx, cudaMemcpyDeviceToDevice, s));
        if (l > 1)
            CK(cudaMemcpyAsync(w->u[l], lamT_dev, sizeof(double) * nx, cudaMemcpyDeviceToDevice, s));
    }
    const double cyc = mgrit_cycle_cell_updates(ctx);
    const double relax0 = (double)nx * nC *
                          ((ctx->p.relax == MGRIT_RELAX_FCF ? 2.0 : 1.0) * ctx->m + 1.0);
    double updates = (double)nx * nC * (ctx->m - 1);   // trajectory regeneration
    double r0 = 0.0;
    int k = 0, status = MGRIT_OK;
    for (;; ++k) {
        CK(cudaGraphLaunch(w->gA, s));
        updates += relax0;
        CK(cudaMemcpyAsync(ctx->h_norm, w->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double rk = *ctx->h_norm;
        if (stats && k < 256) stats->res_hist[k] = rk;
        if (k == 0) r0 = rk;
        if (rk < ctx->p.tol) { status = MGRIT_OK; break; }
        if (!std::isfinite(rk) || rk > 1e8 * r0) { status = MGRIT_EDIVERGED; break; }
        if (k >= ctx->p.max_iter) { status = MGRIT_ENOTCONV; break; }
        CK(cudaGraphLaunch(w->gB, s));
        updates += cyc - relax0;
    }
    CK(cudaEventRecord(ctx->ev1, s));
    // reversed point nt (= forward point 0) is the last level-0 C-point
    if (lam0_dev)
        CK(cudaMemcpyAsync(lam0_dev, w->newC[0] + (size_t)nC * nx, sizeof(double) * nx,
                           cudaMemcpyDeviceToDevice, s));
    if (lamC_dev) CK(launch_reverse_rows(w->newC[0], lamC_dev, (long long)nC + 1, nx, s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        stats->iters = k;
        stats->status = status;
        stats->t_total_ms = ms;
        stats->cell_updates = updates;
    }
    if (status == MGRIT_EDIVERGED) mgrit_fail(ctx, status, "adjoint diverged at cycle %d", k);
    if (status == MGRIT_ENOTCONV) mgrit_fail(ctx, status, "adjoint not converged after %d cycles", k);
    return status;
}

extern "C" int mgrit_adjoint_query(const mgrit_ctx *ctx, int what)
{
    if (!ctx) return -1;
    AdjWork w;
    memset(&w, 0, sizeof w);
    const bool ok = ctx->p.numflux == MGRIT_LF_SPLIT && adj_choose(ctx, &w);
    switch (what) {
    case 0: return ok ? w.cpt : 0;
    case 1: return ok ? w.threads : 0;
    case 2: return ctx->adj ? (ctx->adj->cfn ? ctx->adj->cK : 1) : 0;
    default:
        if (what >= 100 && what < 100 + ctx->L - 1) {   // level what-100 chunks
            if (!ctx->adj) return 0;
            const AdjWork::Shape &c = ctx->adj->lr[what - 100];
            return c.fn ? c.K : 1;
        }
        return -1;
    }
}
