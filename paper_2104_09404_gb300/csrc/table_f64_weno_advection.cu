// FP64 WENO5-JS + SSPRK3, linear advection flux.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_weno_advection(KernelTable &t)
{
    fill_sf<double, SCH_WENO5_SSPRK3, FLX_ADVECTION>(t.slab64);
}
}  // namespace mgrit
