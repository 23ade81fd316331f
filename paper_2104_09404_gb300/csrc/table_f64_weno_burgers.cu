// FP64 WENO5-JS + SSPRK3, Burgers flux.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_weno_burgers(KernelTable &t)
{
    fill_sf<double, SCH_WENO5_SSPRK3, FLX_BURGERS>(t.slab64);
}
}  // namespace mgrit
