// Launchers of the batched restriction, norm and conversion kernels.
#include "batch_table.cuh"

namespace mgrit {

__global__ void __launch_bounds__(256) k_norm_batch(const NormBatchArgs *__restrict__ args,
                                                    const int *__restrict__ active)
{
    __shared__ double red[256];
    const NormBatchArgs a = args[blockIdx.x];
    if (active && !active[blockIdx.x]) return;
    double s = 0.0;
    for (int k = threadIdx.x; k < a.n; k += 256) s += a.partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.out = sqrt(red[0]);
}

__global__ void k_convert_batch(const ConvertBatchArgs *__restrict__ args,
                                const BatchItem *__restrict__ map, const int *__restrict__ active)
{
    const BatchItem it = map[blockIdx.x];
    if (active && !active[it.instance]) return;
    const ConvertBatchArgs a = args[it.args];
    const long long stride = (long long)it.chunk * blockDim.x;   // chunk holds the item's block count
    for (long long e = (long long)it.block * blockDim.x + threadIdx.x; e < a.n; e += stride)
        a.dst[e] = (float)a.src[e];
}

cudaError_t launch_restrict_batch(const RestrictBatchArgs *args, const BatchItem *map, int nblocks,
                                  int state_f32, int un_f32, const int *active, cudaStream_t s)
{
    if (!state_f32)
        k_restrict_batch<double, double><<<nblocks, RESTRICT_THREADS, 0, s>>>(args, map, active);
    else if (un_f32)
        k_restrict_batch<float, float><<<nblocks, RESTRICT_THREADS, 0, s>>>(args, map, active);
    else
        k_restrict_batch<float, double><<<nblocks, RESTRICT_THREADS, 0, s>>>(args, map, active);
    return cudaGetLastError();
}

cudaError_t launch_norm_batch(const NormBatchArgs *args, int n, const int *active, cudaStream_t s)
{
    k_norm_batch<<<n, 256, 0, s>>>(args, active);
    return cudaGetLastError();
}

cudaError_t launch_convert_batch(const ConvertBatchArgs *args, const BatchItem *map, int nblocks,
                                 const int *active, cudaStream_t s)
{
    k_convert_batch<<<nblocks, 256, 0, s>>>(args, map, active);
    return cudaGetLastError();
}

}  // namespace mgrit
