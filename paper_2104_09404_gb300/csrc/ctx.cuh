// Private host-side definitions shared by the C-ABI translation units
// (capi.cu: forward solver and batches; capi_adjoint.cu: the adjoint).
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "../../include/mgrit.h"
#include "grid_seq.cuh"

namespace mgrit {

constexpr int MAXLEV = 32;

// Every kernel's dynamic shared-memory limit is raised to the opt-in maximum
// (227 KB per CTA) once, not to the size one launch needs: kernel instances
// are shared between contexts of different nx, and a later, smaller setting
// would make an earlier context's launches fail.
constexpr int SMEM_OPTIN = 227 * 1024;

struct Launch {
    const void *slab;   // k_slab instance for (precision, scheme, flux, cells per thread); null: unsupported
    int threads;
    int cpt;
    size_t smem;
};

// stepping on thread-block clusters: the sequential chain (coarsest solve,
// serial stepper) or one cluster per chunk (relaxation, interpolation)
struct ClusterLaunch {
    const void *fn;     // k_seq_cluster / k_slab_cluster instance; null: one-CTA k_slab
    int K;              // CTAs in the cluster
    int cpt;            // cells per thread (1 or 2)
    int threads;
    size_t smem;
};

// sequential stepping on a cooperative grid of G CTAs (k_seq_grid)
struct GridLaunch {
    const void *fn;     // null: not used (cluster or one-CTA stepper instead)
    int G;              // CTAs
    int threads;
};

struct AdjWork;   // adjoint workspaces (capi_adjoint.cu), allocated on first use

// Raise fn's cluster-size (K > 8) and shared-memory limits and report whether
// one cluster of K CTAs x `threads` with `smem` dynamic bytes can be
// co-scheduled on the device.  A refused attribute or query leaves no error.
inline bool cluster_fits(const void *fn, int K, int threads, size_t smem)
{
    if ((K > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OPTIN) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
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
        return false;
    }
    return true;
}

// nblocks CTAs of fn (a multiple of K) in clusters of K; args as for cudaLaunchKernel
inline cudaError_t launch_in_clusters(const void *fn, int K, long long nblocks, int threads, size_t smem,
                                      cudaStream_t s, void **args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace mgrit

struct mgrit_ctx {
    int nx, nt, m, L, scheme, flux;
    mgrit_params p;
    int nt_l[mgrit::MAXLEV], nC_l[mgrit::MAXLEV];
    double dt_l[mgrit::MAXLEV];
    mgrit::Launch ln64, ln32;
    mgrit::ClusterLaunch lc64, lc32;
    // grid-wide sequential stepping, chosen by timing against the cluster
    // stepper when the workspaces are allocated (fn null: cluster / one CTA)
    mgrit::GridLaunch lg64, lg32;   // fastest grid shape (fn null: none fits)
    int seq64, seq32;               // the fastest sequential stepper timed (1 one CTA, 2 cluster, 3 grid)
    mgrit::GridBufs gbuf;
    // relaxation / interpolation of level l on clusters (fn null: one CTA per
    // chunk), chosen when the workspaces are allocated
    mgrit::ClusterLaunch lr64[mgrit::MAXLEV], lr32[mgrit::MAXLEV];
    // WENO5 split form, nx > 8192: clusters of run-major slabs (k_slab_tlc)
    // for the levels whose chunks fill the SMs.  [0]: the shape timed faster
    // than the one-CTA slab or the cluster stepper's chunks (fn null: those
    // were faster); [1], [2]: the first shape that fits with K = 2 and 4
    // (chunk_clusters = 2 and 4)
    mgrit::ClusterLaunch tl64[3], tl32[3];
    bool cluster64;      // FP64 slices only fit on clusters (nx > 8192)
    int nsm;             // SMs of the device
    int f32;             // precision the workspaces were allocated for (1: FP32 sweeps)
    bool alloc;
    bool prepared;       // workspaces, graphs and an initial iterate exist
    bool have_state;     // a level-0 relaxation has produced newC[0]
    int device;
    void *u[mgrit::MAXLEV];
    double *g[mgrit::MAXLEV];
    void *newC[mgrit::MAXLEV], *phirow[mgrit::MAXLEV], *cstep[mgrit::MAXLEV];
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
    mgrit::AdjWork *adj;
    char err[256];
};

// record a one-line error (ctx may be null: the creation error) and return code
int mgrit_fail(mgrit_ctx *c, int code, const char *fmt, ...);
// device rows x nx elements of `elem` bytes
int mgrit_dalloc(mgrit_ctx *ctx, void **ptr, size_t rows, size_t elem);
// level workspaces, events and the capture stream of the forward solver
int mgrit_ensure_alloc(mgrit_ctx *ctx);
// release the adjoint workspaces (no-op if none)
void mgrit_adj_free(mgrit_ctx *ctx);
// drop the adjoint's captured graphs (parameters changed); no-op if none
void mgrit_adj_drop_graphs(mgrit_ctx *ctx);
// enqueue the part of one cycle below level 0 (V- or F-cycle by ctx->p.cycle)
// from the given level operations
cudaError_t mgrit_emit_below_level0(mgrit_ctx *ctx, cudaError_t (*relax)(mgrit_ctx *, int, cudaStream_t),
                                    cudaError_t (*restrict_)(mgrit_ctx *, int, cudaStream_t),
                                    cudaError_t (*coarse)(mgrit_ctx *, cudaStream_t),
                                    cudaError_t (*interp)(mgrit_ctx *, int, cudaStream_t),
                                    cudaStream_t s);

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return mgrit_fail(ctx, e_ == cudaErrorMemoryAllocation ? MGRIT_ENOMEM : MGRIT_ECUDA, \
                              "%s: %s", #call, cudaGetErrorString(e_));                \
    } while (0)
