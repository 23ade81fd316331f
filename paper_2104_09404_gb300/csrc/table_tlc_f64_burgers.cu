// F64 WENO5-JS + SSPRK3 relaxation / interpolation chunks on clusters of
// run-major slabs (k_slab_tlc), burgers flux, 8 and 16 cells per thread.
#include "kernel_table.cuh"
namespace mgrit {
void fill_tlc_f64_burgers(KernelTable &t) { fill_tlc<double, FLX_BURGERS>(t.tlc64); }
}  // namespace mgrit
