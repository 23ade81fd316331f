// Residual / FAS restriction at C-points, the deterministic norm, and row
// conversions between the sweep precision and FP64.
#pragma once
#include <cuda_runtime.h>

#ifdef MGRIT_DEBUG
#include <cstdio>
#endif

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
// norm's summation order is fixed): a grid of gx x gy blocks, gx =
// ceil(nx / (2 RESTRICT_THREADS)) over the columns (two per thread) and gy
// over the rows
int restrict_blocks(int nC, int nx);

// aligned for a load or store of two consecutive elements of T
template <typename T>
__device__ __forceinline__ bool pair_aligned(const T *p)
{
    return p == nullptr || ((unsigned long long)p & (2 * sizeof(T) - 1)) == 0;
}

template <typename T>
__device__ __forceinline__ void ld2(const T *p, bool vec, bool two, double &x, double &y)
{
    if (vec) {
        if constexpr (sizeof(T) == 8) {
            const double2 v = *reinterpret_cast<const double2 *>(p);
            x = v.x;
            y = v.y;
        } else {
            const float2 v = *reinterpret_cast<const float2 *>(p);
            x = (double)v.x;
            y = (double)v.y;
        }
    } else {
        x = (double)p[0];
        y = two ? (double)p[1] : 0.0;
    }
}

template <typename T>
__device__ __forceinline__ void st2(T *p, bool vec, bool two, double x, double y)
{
    if (vec) {
        if constexpr (sizeof(T) == 8)
            *reinterpret_cast<double2 *>(p) = make_double2(x, y);
        else
            *reinterpret_cast<float2 *>(p) = make_float2((float)x, (float)y);
    } else {
        p[0] = (T)x;
        if (two) p[1] = (T)y;
    }
}

// The residual and restriction of block b of the nblocks = gx x gy blocks
// of restrict_blocks: rows 1 + by, 1 + by + gy, ... at the two columns c, c + 1
// of this thread (c = 2 (bx RESTRICT_THREADS + t)); returns the thread's sum
// of r^2 in that fixed order.  Pairs move as one 16- (FP64) or 8-byte (FP32)
// access where nx is even and every row array is aligned for it.
template <typename S, typename U>
__device__ __forceinline__ double restrict_block(const RestrictArgs &a, int b, int nblocks)
{
    const int nx = a.nx;
    const int gx = (nx + 2 * RESTRICT_THREADS - 1) / (2 * RESTRICT_THREADS);
    const int gy = nblocks / gx;
    const int bx = b % gx, by = b / gx;
    const int c = 2 * (bx * RESTRICT_THREADS + (int)threadIdx.x);
    if (c >= nx || by >= gy) return 0.0;
    const S *newC = static_cast<const S *>(a.newC);
    const S *phirow = static_cast<const S *>(a.phirow);
    const S *cstep = static_cast<const S *>(a.cstep);
    U *un = static_cast<U *>(a.un);
    const bool two = c + 1 < nx;
    const bool vec = (nx & 1) == 0 && pair_aligned(newC) && pair_aligned(phirow) && pair_aligned(cstep) &&
                     pair_aligned(a.g) && pair_aligned(a.gn) && pair_aligned(un);
    double acc = 0.0;
#pragma unroll 2
    for (long long i = 1 + by; i <= a.nC; i += gy) {
        const long long at = i * nx + c;
#ifdef MGRIT_DEBUG
        if (a.g && (long long)a.m * i >= a.nrows_g) {
            printf("MGRIT_DEBUG restrict g row %lld of %lld\n", (long long)a.m * i, a.nrows_g);
            continue;
        }
#endif
        double g0 = 0.0, g1 = 0.0, p0, p1, u0, u1;
        if (a.g) ld2(a.g + (long long)a.m * i * nx + c, vec, two, g0, g1);
        ld2(phirow + at, vec, two, p0, p1);
        ld2(newC + at, vec, two, u0, u1);
        const double r0 = p0 + g0 - u0, r1 = p1 + g1 - u1;
        acc += r0 * r0;
        if (two) acc += r1 * r1;
        if (cstep) {
            double c0, c1;
            ld2(cstep + (i - 1) * nx + c, vec, two, c0, c1);
            st2(a.gn + at, vec, two, g0 + p0 - c0, g1 + p1 - c1);
            if (a.guess == 0)
                st2(un + at, vec, two, p0 + g0, p1 + g1);
            else
                st2(un + at, vec, two, u0, u1);
        }
    }
    return acc;
}

cudaError_t launch_restrict(const RestrictArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_norm(const double *partials, int n, double *out, cudaStream_t s);
// rows [0, nrows) of dst (float if dst_f32, else double) = src (one FP64 row)
cudaError_t launch_broadcast_row(const double *src, void *dst, int dst_f32, int nx,
                                 long long nrows, cudaStream_t s);
// dst[0..n) = src[0..n) with a precision conversion (either side float or double)
cudaError_t launch_convert(const void *src, int src_f32, void *dst, int dst_f32, long long n,
                           cudaStream_t s);

}  // namespace mgrit
