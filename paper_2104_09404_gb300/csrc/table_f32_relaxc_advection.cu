// F32 relaxation/interpolation chunks on thread-block clusters
// (k_slab_cluster), advection flux: WENO5-JS + SSPRK3 and first order + FE.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f32_relaxc_advection(KernelTable &t)
{
    fill_cluster_relax<float, SCH_WENO5_SSPRK3, FLX_ADVECTION>(t.relc32);
    fill_cluster_relax<float, SCH_FO_FE, FLX_ADVECTION>(t.relc32);
}
}  // namespace mgrit
