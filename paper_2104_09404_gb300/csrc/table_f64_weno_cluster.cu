// F64 WENO5-JS + SSPRK3 cluster (DSMEM) sequential kernels, both fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_weno_cluster(KernelTable &t)
{
    fill_cluster<double, SCH_WENO5_SSPRK3, FLX_BURGERS>(t.seqc64);
    fill_cluster<double, SCH_WENO5_SSPRK3, FLX_ADVECTION>(t.seqc64);
}
}  // namespace mgrit
