// FP64 first-order reconstruction + forward Euler, both fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_fo(KernelTable &t)
{
    fill_sf<double, SCH_FO_FE, FLX_BURGERS>(t.slab64);
    fill_sf<double, SCH_FO_FE, FLX_ADVECTION>(t.slab64);
    fill_cluster<double, SCH_FO_FE, FLX_BURGERS>(t.seqc64);
    fill_cluster<double, SCH_FO_FE, FLX_ADVECTION>(t.seqc64);
}
}  // namespace mgrit
