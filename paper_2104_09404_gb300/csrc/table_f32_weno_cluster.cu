// F32 WENO5-JS + SSPRK3 cluster (DSMEM) sequential kernels, both fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f32_weno_cluster(KernelTable &t)
{
    fill_cluster<float, SCH_WENO5_SSPRK3, FLX_BURGERS>(t.seqc32);
    fill_cluster<float, SCH_WENO5_SSPRK3, FLX_ADVECTION>(t.seqc32);
}
}  // namespace mgrit
