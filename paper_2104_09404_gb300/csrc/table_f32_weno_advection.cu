// FP32 WENO5-JS + SSPRK3, linear advection flux.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f32_weno_advection(KernelTable &t)
{
    fill_sf32<SCH_WENO5_SSPRK3, FLX_ADVECTION>(t.slab32);
}
}  // namespace mgrit
