// Residual and FAS restriction at the C-points of a level (Sec. 3.2):
//   r^i       = Phi_l(u^{mi-1}) + g_l^{mi} - u_l^{mi}
//   g_{l+1}^i = g_l^{mi} + Phi_l(u^{mi-1}) - Phi_{l+1}(u_l^{m(i-1)})   (Eq. restriction::rhs)
//   u_{l+1}^i = Phi_l(u^{mi-1}) + g_l^{mi}                            (Eq. restriction::u)
//             or u_l^{mi} (injection, Eq. restrictionOperator)
// for i = 1..nC.  The Phi values were produced by the relaxation kernel, so
// this pass is a pure stream over rows (HBM-bound).  The squared residual is
// summed per block in a fixed order; k_norm adds the partials in a fixed
// order, so the norm is bitwise reproducible from run to run.
#include "restrict.cuh"

#ifdef MGRIT_DEBUG
#include <cstdio>
#endif

namespace mgrit {

__global__ void __launch_bounds__(RESTRICT_THREADS) k_restrict(RestrictArgs a)
{
    __shared__ double red[RESTRICT_THREADS / 32];
    const long long n = (long long)a.nC * a.nx;
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = 1 + e / a.nx;
        const long long c = e - (i - 1) * a.nx;
        const long long at = i * a.nx + c;
#ifdef MGRIT_DEBUG
        if (a.g && (long long)a.m * i >= a.nrows_g) {
            printf("MGRIT_DEBUG restrict g row %lld of %lld\n", (long long)a.m * i, a.nrows_g);
            continue;
        }
#endif
        const double gl = a.g ? a.g[(long long)a.m * i * a.nx + c] : 0.0;
        const double phi = a.phirow[at];
        const double uc = a.newC[at];
        const double r = phi + gl - uc;
        acc += r * r;
        if (a.cstep) {
            a.gn[at] = gl + phi - a.cstep[(i - 1) * a.nx + c];
            a.un[at] = a.guess == 0 ? phi + gl : uc;
        }
    }
    if (a.partials) {
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < RESTRICT_THREADS / 32; ++w) s += red[w];
            a.partials[blockIdx.x] = s;
        }
    }
}

// out = sqrt(sum of partials[0..n)), fixed summation order, one block
__global__ void __launch_bounds__(256) k_norm(const double *partials, int n, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s += partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// rows [0, nrows) of dst = src
__global__ void k_broadcast_row(const double *src, double *dst, int nx, long long nrows)
{
    const long long n = nrows * nx;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e % nx];
}

int restrict_blocks(int nC, int nx)
{
    const long long n = (long long)nC * nx;
    long long b = (n + RESTRICT_THREADS * 4 - 1) / (RESTRICT_THREADS * 4);
    const long long cap = 152 * 8;   // 8 resident blocks on each of the 152 SMs
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_restrict(const RestrictArgs &a, int blocks, cudaStream_t s)
{
    k_restrict<<<blocks, RESTRICT_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_norm(const double *partials, int n, double *out, cudaStream_t s)
{
    k_norm<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

cudaError_t launch_broadcast_row(const double *src, double *dst, int nx, long long nrows,
                                 cudaStream_t s)
{
    long long n = nrows * nx;
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    k_broadcast_row<<<(int)b, 256, 0, s>>>(src, dst, nx, nrows);
    return cudaGetLastError();
}

}  // namespace mgrit
