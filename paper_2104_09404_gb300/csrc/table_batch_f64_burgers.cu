// Batched FP64 WENO5-JS + SSPRK3 kernels, Burgers flux.
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f64_burgers(BatchTable &t)
{
    fill_batch<double, FLX_BURGERS>(t.slab64);
    fill_batch_cluster<FLX_BURGERS>(t.seqc64);
}
}  // namespace mgrit
