// Adjoint kernels: WENO5-JS + SSPRK3, Burgers flux.
#include "adj_table.cuh"
namespace mgrit {
void fill_adj_weno_burgers(AdjTable &t) { fill_adj_sf<SCH_WENO5_SSPRK3, FLX_BURGERS>(t); }
}  // namespace mgrit
