// FP64 classical Lax-Friedrichs + forward Euler (Eq. fineLF) with the matched
// coarse integrators, both fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_lf(KernelTable &t)
{
    fill_sf<double, SCH_LF_FE, FLX_BURGERS>(t.slab64);
    fill_sf<double, SCH_LF_FE, FLX_ADVECTION>(t.slab64);
}
}  // namespace mgrit
