// Instances of the batched slab kernel, indexed by [flux][cells-per-thread]
// (WENO5-JS + SSPRK3 only).
#pragma once
#include "batch.cuh"
#include "kernel_table.cuh"

namespace mgrit {

struct BatchTable {
    const void *slab32[2][NCPT];
    const void *slab64[2][NCPT];
    const void *seqc64[2][2];   // k_seq_cluster_batch (FP64), cells per thread 1 or 2
};

template <typename R, int F>
void fill_batch(const void *(&t)[2][NCPT])
{
    t[F][0] = (const void *)&k_slab_batch<R, SCH_WENO5_SSPRK3, F, 1>;
    t[F][1] = (const void *)&k_slab_batch<R, SCH_WENO5_SSPRK3, F, 2>;
    t[F][2] = (const void *)&k_slab_batch<R, SCH_WENO5_SSPRK3, F, 4>;
    t[F][3] = (const void *)&k_slab_batch<R, SCH_WENO5_SSPRK3, F, 8>;
    t[F][4] = (const void *)&k_slab_batch<R, SCH_WENO5_SSPRK3, F, 16>;
}

template <int F>
void fill_batch_cluster(const void *(&t)[2][2])
{
    t[F][0] = (const void *)&k_seq_cluster_batch<double, SCH_WENO5_SSPRK3, F, 1>;
    t[F][1] = (const void *)&k_seq_cluster_batch<double, SCH_WENO5_SSPRK3, F, 2>;
}

// one translation unit per (precision, flux), compiled in parallel
void fill_batch_f32_burgers(BatchTable &t);
void fill_batch_f32_advection(BatchTable &t);
void fill_batch_f64_burgers(BatchTable &t);
void fill_batch_f64_advection(BatchTable &t);

// batched restriction / norm / conversion launchers (batch_ops.cu)
cudaError_t launch_restrict_batch(const RestrictBatchArgs *args, const BatchItem *map, int nblocks,
                                  int state_f32, int un_f32, const int *active, cudaStream_t s);
cudaError_t launch_norm_batch(const NormBatchArgs *args, int n, const int *active, cudaStream_t s);
cudaError_t launch_convert_batch(const ConvertBatchArgs *args, const BatchItem *map, int nblocks,
                                 const int *active, cudaStream_t s);

}  // namespace mgrit
