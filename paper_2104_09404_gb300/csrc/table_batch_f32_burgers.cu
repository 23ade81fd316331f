// Batched FP32 WENO5-JS + SSPRK3 kernels, Burgers flux.
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f32_burgers(BatchTable &t)
{
    fill_batch<float, FLX_BURGERS>(t.slab32);
}
}  // namespace mgrit
