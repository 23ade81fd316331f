// Batched FP64 WENO5-JS + SSPRK3 slab kernels (Burgers and advection).
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f64(BatchTable &t)
{
    fill_batch<double, FLX_BURGERS>(t.slab64);
    fill_batch<double, FLX_ADVECTION>(t.slab64);
    fill_batch_cluster<FLX_BURGERS>(t.seqc64);
    fill_batch_cluster<FLX_ADVECTION>(t.seqc64);
}
}  // namespace mgrit
