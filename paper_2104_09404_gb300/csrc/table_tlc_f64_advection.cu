// F64 WENO5-JS + SSPRK3 relaxation / interpolation chunks on clusters of
// run-major slabs (k_slab_tlc), advection flux, 8 and 16 cells per thread.
#include "kernel_table.cuh"
namespace mgrit {
void fill_tlc_f64_advection(KernelTable &t) { fill_tlc<double, FLX_ADVECTION>(t.tlc64); }
}  // namespace mgrit
