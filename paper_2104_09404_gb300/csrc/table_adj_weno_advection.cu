// Adjoint kernels: WENO5-JS + SSPRK3, linear advection.
#include "adj_table.cuh"
namespace mgrit {
void fill_adj_weno_advection(AdjTable &t) { fill_adj_sf<SCH_WENO5_SSPRK3, FLX_ADVECTION>(t); }
}  // namespace mgrit
