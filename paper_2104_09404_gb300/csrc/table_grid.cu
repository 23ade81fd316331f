// Grid-wide sequential steppers (k_seq_grid), FP64 and FP32, both schemes and fluxes.
#include "kernel_table.cuh"
namespace mgrit {
void fill_grid(KernelTable &t)
{
    t.grid64[0][0] = (const void *)&k_seq_grid<double, SCH_WENO5_SSPRK3, FLX_BURGERS>;
    t.grid64[0][1] = (const void *)&k_seq_grid<double, SCH_WENO5_SSPRK3, FLX_ADVECTION>;
    t.grid64[1][0] = (const void *)&k_seq_grid<double, SCH_FO_FE, FLX_BURGERS>;
    t.grid64[1][1] = (const void *)&k_seq_grid<double, SCH_FO_FE, FLX_ADVECTION>;
    t.grid32[0][0] = (const void *)&k_seq_grid<float, SCH_WENO5_SSPRK3, FLX_BURGERS>;
    t.grid32[0][1] = (const void *)&k_seq_grid<float, SCH_WENO5_SSPRK3, FLX_ADVECTION>;
    t.grid32[1][0] = (const void *)&k_seq_grid<float, SCH_FO_FE, FLX_BURGERS>;
    t.grid32[1][1] = (const void *)&k_seq_grid<float, SCH_FO_FE, FLX_ADVECTION>;
}
}  // namespace mgrit
