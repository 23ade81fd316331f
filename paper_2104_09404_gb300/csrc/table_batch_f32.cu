// Batched FP32 WENO5-JS + SSPRK3 slab kernels (Burgers and advection).
#include "batch_table.cuh"
namespace mgrit {
void fill_batch_f32(BatchTable &t)
{
    fill_batch<float, FLX_BURGERS>(t.slab32);
    fill_batch<float, FLX_ADVECTION>(t.slab32);
}
}  // namespace mgrit
