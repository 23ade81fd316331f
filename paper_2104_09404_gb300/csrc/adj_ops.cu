// Row reversal for the adjoint outputs (reversed-time rows -> forward order).
#include "adj_table.cuh"

namespace mgrit {

__global__ void k_reverse_rows(const double *__restrict__ src, double *__restrict__ dst,
                               long long nrows, int nx)
{
    const long long n = nrows * nx;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / nx;
        const long long c = e - r * nx;
        dst[(nrows - 1 - r) * nx + c] = src[e];
    }
}

cudaError_t launch_reverse_rows(const double *src, double *dst, long long nrows, int nx,
                                cudaStream_t s)
{
    const long long n = nrows * nx;
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_reverse_rows<<<(unsigned)blocks, 256, 0, s>>>(src, dst, nrows, nx);
    return cudaGetLastError();
}

}  // namespace mgrit
