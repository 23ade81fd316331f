// Batched FP32 WENO5-JS + SSPRK3 kernels, linear advection flux.
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f32_advection(BatchTable &t)
{
    fill_batch<float, FLX_ADVECTION>(t.slab32);
}
}  // namespace mgrit
