// Relaxation and interpolation chunks on thread-block clusters.
//
// The F-/FCF-relaxation (Sec. 3.2) and the ideal interpolation (Eq.
// interpolation) of one C-interval are a short chain of Phi applications on
// one slice.  k_slab gives each chunk one CTA, which leaves SMs idle on the
// coarse levels (a level with 17 chunks fills 17 of 152 SMs) and cannot hold
// an FP64 slice beyond 8192 cells.  Here each chunk runs on a cluster of K
// CTAs with the DSMEM stepper of cluster_seq.cuh (contiguous cell blocks,
// ghosts and the LF alpha exchanged through distributed shared memory):
// cluster c = blockIdx.x / K relaxes or interpolates chunk c, with exactly the
// chunk logic of the one-CTA kernel (relax_chunk / interp_chunk).
#pragma once
#include "cluster_seq.cuh"

namespace mgrit {

// ClusterSlab with its own stage counter, in the interface relax_chunk and
// interp_chunk expect
template <typename R, int SCHEME, int FLUX, int CPT>
struct ClusterChunkSlab {
    static constexpr int kScheme = SCHEME, kCpt = CPT;
    ClusterSlab<R, SCHEME, FLUX, CPT> &C;
    int stage;
    int psiM;   // unused: the classical LF scheme has no cluster kernels

    __device__ __forceinline__ ClusterChunkSlab(ClusterSlab<R, SCHEME, FLUX, CPT> &c)
        : C(c), stage(0), psiM(0) {}
    __device__ __forceinline__ void step(R (&u)[CPT], R dt) { C.step(u, dt, stage); }
    __device__ __forceinline__ void load(R (&u)[CPT], const R *row) const { C.load(u, row); }
    __device__ __forceinline__ void store(const R (&u)[CPT], R *row) const { C.store(u, row); }
    __device__ __forceinline__ void add(R (&u)[CPT], const double *row) const { C.add(u, row); }
};

// MODE_RELAX (grid (nC + 1) x K) or MODE_INTERP (grid nC x K); cluster size K
// is the launch's cluster dimension.  Every CTA of a cluster takes the same
// branches (they depend on the chunk index and the arguments only), so all of
// them reach every cluster barrier.
template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_slab_cluster(SlabArgs<R> a)
{
    static_assert(SCHEME != SCH_LF_FE, "the classical LF scheme runs on one-CTA slabs");
    extern __shared__ __align__(16) unsigned char smem[];
    ClusterSlab<R, SCHEME, FLUX, CPT> C(smem, a.nx, a.dxinv, a.numflux);
    ClusterChunkSlab<R, SCHEME, FLUX, CPT> S(C);
    const int j = (int)(blockIdx.x / C.cl.num_blocks());
    if (a.mode == MODE_RELAX)
        relax_chunk(S, a, j);
    else
        interp_chunk(S, a, j);
    C.cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

// The same chunks on clusters of run-major slabs (Slab with CLUSTER; WENO5
// split form): each CTA holds a contiguous block of the slice in the one-CTA
// slab's layout and arithmetic, with alpha and the ghost cells exchanged
// through distributed shared memory, one cluster barrier per stage.  Slices
// too wide for one CTA's registers (FP32 beyond 8192 cells, FP64 beyond 8192)
// then run at 8 or 16 cells per thread (timed at allocation) with the
// sliding windows.
template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_slab_tlc(SlabArgs<R> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Slab<R, SCHEME, FLUX, CPT, false, true> S(smem, a.nx, a.dxinv, a.numflux);
    S.pair_div = true;
    const int j = (int)(blockIdx.x / cg::this_cluster().num_blocks());
    if (a.mode == MODE_RELAX)
        relax_chunk(S, a, j);
    else
        interp_chunk(S, a, j);
    cg::this_cluster().sync();   // no CTA leaves while a neighbour may still read its shared memory
}

}  // namespace mgrit
