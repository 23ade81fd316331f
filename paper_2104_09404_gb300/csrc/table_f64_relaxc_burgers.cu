// F64 relaxation/interpolation chunks on thread-block clusters
// (k_slab_cluster), burgers flux: WENO5-JS + SSPRK3 and first order + FE.
#include "kernel_table.cuh"
namespace mgrit {
void fill_f64_relaxc_burgers(KernelTable &t)
{
    fill_cluster_relax<double, SCH_WENO5_SSPRK3, FLX_BURGERS>(t.relc64);
    fill_cluster_relax<double, SCH_FO_FE, FLX_BURGERS>(t.relc64);
}
}  // namespace mgrit
