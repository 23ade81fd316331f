// Batched FP64 WENO5-JS + SSPRK3 kernels, linear advection flux.
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f64_advection(BatchTable &t)
{
    fill_batch<double, FLX_ADVECTION>(t.slab64);
    fill_batch_cluster<FLX_ADVECTION>(t.seqc64);
}
}  // namespace mgrit
