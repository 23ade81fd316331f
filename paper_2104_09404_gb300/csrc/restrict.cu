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

// S: precision of the relaxation outputs; U: precision of the next level's
// state rows.  Every sum is formed in FP64 (the tau-correction of the FAS
// right-hand side, the residual and its norm stay FP64 in FP32-sweep mode).
template <typename S, typename U>
__global__ void __launch_bounds__(RESTRICT_THREADS) k_restrict(RestrictArgs a)
{
    __shared__ double red[RESTRICT_THREADS / 32];
    double acc = restrict_block<S, U>(a, (int)blockIdx.x, (int)gridDim.x);
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

// rows [0, nrows) of dst = src (one FP64 row), converted to T
template <typename T>
__global__ void k_broadcast_row(const double *src, T *dst, int nx, long long nrows)
{
    const long long n = nrows * nx;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = (T)src[e % nx];
}

template <typename A, typename B>
__global__ void k_convert(const A *src, B *dst, long long n)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = (B)src[e];
}

static int stream_blocks(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

int restrict_blocks(int nC, int nx)
{
    const int gx = (nx + 2 * RESTRICT_THREADS - 1) / (2 * RESTRICT_THREADS);
    const int cap = 152 * 8;   // 8 resident blocks on each of the 152 SMs
    int gy = cap / gx;
    if (gy > nC) gy = nC;
    if (gy < 1) gy = 1;
    return gx * gy;
}

cudaError_t launch_restrict(const RestrictArgs &a, int blocks, cudaStream_t s)
{
    if (!a.state_f32)
        k_restrict<double, double><<<blocks, RESTRICT_THREADS, 0, s>>>(a);
    else if (a.un_f32)
        k_restrict<float, float><<<blocks, RESTRICT_THREADS, 0, s>>>(a);
    else
        k_restrict<float, double><<<blocks, RESTRICT_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_norm(const double *partials, int n, double *out, cudaStream_t s)
{
    k_norm<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

cudaError_t launch_broadcast_row(const double *src, void *dst, int dst_f32, int nx,
                                 long long nrows, cudaStream_t s)
{
    const int b = stream_blocks(nrows * nx);
    if (dst_f32)
        k_broadcast_row<float><<<b, 256, 0, s>>>(src, static_cast<float *>(dst), nx, nrows);
    else
        k_broadcast_row<double><<<b, 256, 0, s>>>(src, static_cast<double *>(dst), nx, nrows);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void *src, int src_f32, void *dst, int dst_f32, long long n,
                           cudaStream_t s)
{
    const int b = stream_blocks(n);
    if (src_f32 && dst_f32)
        k_convert<float, float><<<b, 256, 0, s>>>(static_cast<const float *>(src),
                                                  static_cast<float *>(dst), n);
    else if (src_f32)
        k_convert<float, double><<<b, 256, 0, s>>>(static_cast<const float *>(src),
                                                   static_cast<double *>(dst), n);
    else if (dst_f32)
        k_convert<double, float><<<b, 256, 0, s>>>(static_cast<const double *>(src),
                                                   static_cast<float *>(dst), n);
    else
        k_convert<double, double><<<b, 256, 0, s>>>(static_cast<const double *>(src),
                                                    static_cast<double *>(dst), n);
    return cudaGetLastError();
}

}  // namespace mgrit
