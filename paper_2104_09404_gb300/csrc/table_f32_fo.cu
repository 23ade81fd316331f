// FP32 first-order reconstruction + forward Euler, both fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f32_fo(KernelTable &t)
{
    fill_sf32<SCH_FO_FE, FLX_BURGERS>(t.slab32);
    fill_sf32<SCH_FO_FE, FLX_ADVECTION>(t.slab32);
    fill_cluster<float, SCH_FO_FE, FLX_BURGERS>(t.seqc32);
    fill_cluster<float, SCH_FO_FE, FLX_ADVECTION>(t.seqc32);
}
}  // namespace mgrit
