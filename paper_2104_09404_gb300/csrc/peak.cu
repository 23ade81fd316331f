// Arithmetic-throughput probes of the SIMT pipes the sweeps run on: the
// roofline denominators of the ALU-bound kernels (the relaxation, the
// sequential steppers and the adjoint are bound by FP64 or FP32 multiply-add
// issue, not by memory).  Every thread runs CHAINS independent multiply-add
// recurrences x <- x * a + b, so that the pipe, not the dependency latency,
// sets the rate; the chains are summed and written only if the sum is NaN
// (never, for the values below), which keeps the loop alive without memory
// traffic.  One multiply-add counts as 2 flops.
#include <cuda_runtime.h>

#include "../../include/mgrit.h"
#include "slab.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int PROBE_THREADS = 256;

// written only when a chain sum is NaN (never for the values used); a
// file-scope device variable keeps the store in range without an allocation
__device__ double g_probe_sink;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_f64(int iters, double a, double b)
{
    double x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s != s) g_probe_sink = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_f32(int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = 1.0f + 1e-3f * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = __fmaf_rn(x[k], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s != s) g_probe_sink = s;
}

// packed pairs: one instruction performs two FP32 multiply-adds
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_f32x2(int iters, float a, float b)
{
    float2 x[CHAINS];
    const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        x[k] = make_float2(1.0f + 1e-3f * (threadIdx.x + k), 1.0f - 1e-3f * (threadIdx.x + k));
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = __ffma2_rn(x[k], av, bv);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k].x + x[k].y;
    if (s != s) g_probe_sink = s;
}

}  // namespace

extern "C" int mgrit_fma_probe(int kind, int iters, int blocks_per_sm, double *flops_out, void *stream)
{
    if (!flops_out || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || kind < 0 || kind > 2)
        return MGRIT_EINVAL;
    *flops_out = 0.0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MGRIT_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = nsm * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MGRIT_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MGRIT_ECUDA;
    }
    // a = 1 - 2^-20, b = 2^-20: the recurrences converge to 1 and never overflow
    const double a = 1.0 - 0x1p-20, b = 0x1p-20;
    cudaEventRecord(e0, s);
    if (kind == 0)
        k_probe_f64<<<blocks, PROBE_THREADS, 0, s>>>(iters, a, b);
    else if (kind == 1)
        k_probe_f32<<<blocks, PROBE_THREADS, 0, s>>>(iters, (float)a, (float)b);
    else
        k_probe_f32x2<<<blocks, PROBE_THREADS, 0, s>>>(iters, (float)a, (float)b);
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.f)) return MGRIT_ECUDA;
    const double fmas = (double)blocks * PROBE_THREADS * CHAINS * 8.0 * iters * (kind == 2 ? 2.0 : 1.0);
    *flops_out = 2.0 * fmas / (ms * 1e-3);
    return MGRIT_OK;
}
