// Residual / FAS restriction at C-points, the deterministic norm, and row
// conversions between the sweep precision and FP64.
#pragma once
#include <cuda_runtime.h>

namespace mgrit {

struct RestrictArgs {
    const void *newC;      // level-l C-points after relaxation, rows 0..nC (sweep precision)
    const void *phirow;    // rows 1..nC: Phi_l(u^{mi-1}) (sweep precision)
    const void *cstep;     // rows 0..nC-1: Phi_{l+1}(u^{m(i-1)}), or null (residual only)
    const double *g;       // level-l g rows (nt_l+1) x nx, or null (level 0)
    double *gn;            // level-(l+1) g rows, or null
    void *un;              // level-(l+1) u rows, or null
    double *partials;      // per-block sums of r^2, or null
    long long nrows_g;     // rows of g (checked by MGRIT_DEBUG builds)
    int nx, m, nC, guess;
    int state_f32;         // newC/phirow/cstep hold float
    int un_f32;            // un holds float
};

constexpr int RESTRICT_THREADS = 256;

// number of blocks used for nC x nx elements (fixed per problem size, so the
// norm's summation order is fixed)
int restrict_blocks(int nC, int nx);

cudaError_t launch_restrict(const RestrictArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_norm(const double *partials, int n, double *out, cudaStream_t s);
// rows [0, nrows) of dst (float if dst_f32, else double) = src (one FP64 row)
cudaError_t launch_broadcast_row(const double *src, void *dst, int dst_f32, int nx,
                                 long long nrows, cudaStream_t s);
// dst[0..n) = src[0..n) with a precision conversion (either side float or double)
cudaError_t launch_convert(const void *src, int src_f32, void *dst, int dst_f32, long long n,
                           cudaStream_t s);

}  // namespace mgrit
