// F32 WENO5-JS + SSPRK3 relaxation / interpolation chunks on clusters of
// run-major slabs (k_slab_tlc), burgers flux, 8 and 16 cells per thread.
#include "kernel_table.cuh"
namespace mgrit {
void fill_tlc_f32_burgers(KernelTable &t) { fill_tlc<float, FLX_BURGERS>(t.tlc32); }
}  // namespace mgrit
