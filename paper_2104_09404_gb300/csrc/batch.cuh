// Batched launches: many independent MGRIT instances (uneven nx and nt) in
// one launch per phase of the V-cycle.  Every CTA reads its work item from a
// block map: the instance's argument block, the chunk index within the
// instance's level, and the instance id (for the convergence mask).  All
// items of one launch share the CTA shape (threads x cells per thread) of
// their launch class; the slab code is the single-instance code.
#pragma once
#include "cluster_seq.cuh"
#include "restrict.cuh"

namespace mgrit {

struct BatchItem {
    int args;       // index into the launch's argument array
    int chunk;      // chunk j (relaxation/interpolation) or 0 (sequential)
    int instance;   // instance id (convergence mask)
    int block;      // block index within the item (restriction) or 0
};

// One CTA per work item of the block map (instance argument block, chunk,
// instance id).  A persistent variant, CTAs looping over items with 1-8
// slabs per CTA chosen by the autotuner, was measured slower at every
// setting: 122 vs 91 ms per batch cycle even at one item per CTA, because
// inside the item loop the slab code takes more registers (121 instead of
// 64 at 4 cells per thread; out of line, the call boundary still costs 90).
// `active` (may be null): instances whose entry is 0 have converged and skip all work
template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_slab_batch(const SlabArgs<R> *__restrict__ args,
                                                    const BatchItem *__restrict__ map,
                                                    const int *__restrict__ active)
{
    const BatchItem it = map[blockIdx.x];
    if (active && !active[it.instance]) return;
    const SlabArgs<R> a = args[it.args];
    extern __shared__ __align__(16) unsigned char smem[];
    Slab<R, SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv, a.numflux);
    S.pair_div = a.mode != MODE_SEQ;
    if (a.mode == MODE_RELAX)
        relax_chunk(S, a, it.chunk);
    else if (a.mode == MODE_INTERP)
        interp_chunk(S, a, it.chunk);
    else
        seq_march(S, a);
}

// Sequential solves of many items, one thread-block cluster per item (all
// items of a launch share the cluster size): the batched coarsest solves.
template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_seq_cluster_batch(const SlabArgs<R> *__restrict__ args,
                                                           const BatchItem *__restrict__ map,
                                                           const int *__restrict__ active)
{
    cg::cluster_group cl = cg::this_cluster();
    const BatchItem it = map[blockIdx.x / cl.num_blocks()];
    if (active && !active[it.instance]) return;   // uniform over the cluster
    const SlabArgs<R> a = args[it.args];
    extern __shared__ __align__(16) unsigned char smem[];
    ClusterSlab<R, SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv, a.numflux);
    R u[CPT];
    int stage = 0;
    S.load(u, a.src);
    for (int i = 1; i <= a.nsteps; ++i) {
        S.step(u, a.dt, stage);
        if (a.g) S.add(u, rowp(a.g, i, a.nx, a.nrows_g));
        if (a.rows) S.store(u, rowp(a.rows, i, a.nx, a.nrows_rows));
    }
    if (a.out) S.store(u, a.out);
    S.cl.sync();
}

struct RestrictBatchArgs {
    RestrictArgs r;   // the single-instance arguments
    int nblocks;      // blocks given to this item
};

// Residual + FAS restriction of many items; the blocks of an item walk its
// rows and columns as k_restrict's do, so every partial sum is reproducible.
template <typename S, typename U>
__global__ void __launch_bounds__(RESTRICT_THREADS)
    k_restrict_batch(const RestrictBatchArgs *__restrict__ args, const BatchItem *__restrict__ map,
                     const int *__restrict__ active)
{
    __shared__ double red[RESTRICT_THREADS / 32];
    const BatchItem it = map[blockIdx.x];
    if (active && !active[it.instance]) return;
    const RestrictBatchArgs &ba = args[it.args];
    const RestrictArgs &a = ba.r;
    double acc = restrict_block<S, U>(a, it.block, ba.nblocks);
    if (a.partials) {
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < RESTRICT_THREADS / 32; ++w) s += red[w];
            a.partials[it.block] = s;
        }
    }
}

// norms[i] = sqrt(sum of partials of instance i), one block per instance
struct NormBatchArgs {
    const double *partials;
    int n;
    double *out;
};

// FP64 -> FP32 row copies of many items (coarsest-level mirrors)
struct ConvertBatchArgs {
    const double *src;
    float *dst;
    long long n;
};

}  // namespace mgrit
