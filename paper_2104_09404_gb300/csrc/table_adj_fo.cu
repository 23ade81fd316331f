// Adjoint kernels: first-order reconstruction + forward Euler, both fluxes.
#include "adj_table.cuh"
namespace mgrit {
void fill_adj_fo(AdjTable &t)
{
    fill_adj_sf<SCH_FO_FE, FLX_BURGERS>(t);
    fill_adj_sf<SCH_FO_FE, FLX_ADVECTION>(t);
}
}  // namespace mgrit
