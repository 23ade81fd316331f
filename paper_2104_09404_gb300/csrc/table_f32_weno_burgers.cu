// FP32 WENO5-JS + SSPRK3, Burgers flux.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f32_weno_burgers(KernelTable &t)
{
    fill_sf32<SCH_WENO5_SSPRK3, FLX_BURGERS>(t.slab32);
}
}  // namespace mgrit
