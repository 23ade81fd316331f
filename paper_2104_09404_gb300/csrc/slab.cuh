// Slab engine: one CTA owns one spatial slice u^n (nx cells) and applies the
// time-stepper Phi of Sec. 2.2 to it, keeping u^n in registers and the
// stage fluxes in shared memory for every step of a C-interval.
//
// Cell ownership is interleaved: thread t owns cells t + c*blockDim.x,
// c = 0..CPT-1 (cells >= nx are idle).  Consecutive lanes touch
// consecutive cells, so shared-memory traffic is conflict-free and global
// row loads/stores are coalesced.
//
// Shared memory: three arrays of nx + 6 values (the split fluxes f^+ and f^-
// with 3 periodic ghost cells on each side -- the WENO5 half-stencil -- and
// the interface fluxes) plus NWARP_MAX values for the block max reduction of
// the global Lax-Friedrichs alpha.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#ifdef MGRIT_DEBUG
#include <cstdio>
#endif

namespace mgrit {

enum { SCH_WENO5_SSPRK3 = 0, SCH_FO_FE = 1, SCH_LF_FE = 2 };
enum { FLX_BURGERS = 0, FLX_ADVECTION = 1 };
enum { NF_SPLIT = 0, NF_STATE = 1, NF_ROE = 2 };

constexpr int GHOST = 3;
constexpr int NWARP_MAX = 32;

// MGRIT_DEBUG builds check every shared-memory index and every global row
// index against its array's extent; a violation is printed once per thread
// and the access is skipped (shared reads then see element 0), so a bad
// index is reported instead of faulting.
#ifdef MGRIT_DEBUG
#define MGRIT_SH(arr, idx, lim)                                                              \
    (*((unsigned)(idx) < (unsigned)(lim)                                                       \
           ? &(arr)[(idx)]                                                                     \
           : (printf("MGRIT_DEBUG smem %s[%d] limit %d block %d thread %d\n", #arr, (int)(idx), \
                     (int)(lim), (int)blockIdx.x, (int)threadIdx.x),                           \
              &(arr)[0])))
#else
#define MGRIT_SH(arr, idx, lim) ((arr)[(idx)])
#endif

// Physical flux (Sec. 2, Eq. burgers) and |eigenvalue| of its Jacobian.
template <int FLUX, typename R>
__device__ __forceinline__ R phys_flux(R u)
{
    return FLUX == FLX_BURGERS ? R(0.5) * u * u : u;
}
template <int FLUX, typename R>
__device__ __forceinline__ R phys_speed(R u)
{
    return FLUX == FLX_BURGERS ? fabs(u) : R(1);
}

// WENO5-JS value left of the interface i+1/2 from (a..e) = q_{i-2..i+2}
// (Sec. 2.1.1, k = 2).  Candidate values P_r (times 6), smoothness
// indicators in the expanded form 13/12 (2nd difference)^2 + 1/4 (1st
// difference)^2 (equal to the quadratic forms B_r of the paper), weights
// alpha_r = d_r / (eps + beta_r)^2 with d = (1, 6, 3)/10 for the stencils
// ending at i, i+1, i+2.  The weight normalisation is done over a common
// denominator: multiplying numerator and denominator of
// sum_r alpha_r p_r / sum_r alpha_r by prod_r (eps + beta_r)^2 leaves a
// single division per reconstruction (the 1/10 of d_r cancels).
template <typename R>
__device__ __forceinline__ void weno5_left_nd(R a, R b, R c, R d, R e, R &num, R &den);

template <typename R>
__device__ __forceinline__ R weno5_left(R a, R b, R c, R d, R e)
{
    R num, den;
    weno5_left_nd(a, b, c, d, e, num, den);
    // FP32 sweeps divide with the fast intrinsic (2 ulp; den lies in
    // [6e-24, 1e30] for |q| <= 1e3, inside its range); FP64 divides exactly
    if (sizeof(R) == 4) return R(__fdividef(float(num), float(den)));
    return num / den;
}

// weno5_left as the fraction num / den (the common-denominator form below)
template <typename R>
__device__ __forceinline__ void weno5_left_nd(R a, R b, R c, R d, R e, R &num, R &den)
{
    const R eps = R(1e-6);
    const R k13 = R(13.0 / 12.0);
    const R P0 = R(2) * a - R(7) * b + R(11) * c;   // stencil {i-2, i-1, i}
    const R P1 = -b + R(5) * c + R(2) * d;          // stencil {i-1, i, i+1}
    const R P2 = R(2) * c + R(5) * d - e;           // stencil {i, i+1, i+2}
    const R x0 = a - R(2) * b + c, y0 = a - R(4) * b + R(3) * c;
    const R x1 = b - R(2) * c + d, y1 = b - d;
    const R x2 = c - R(2) * d + e, y2 = R(3) * c - R(4) * d + e;
    R s0 = eps + k13 * x0 * x0 + R(0.25) * y0 * y0;
    R s1 = eps + k13 * x1 * x1 + R(0.25) * y1 * y1;
    R s2 = eps + k13 * x2 * x2 + R(0.25) * y2 * y2;
    s0 *= s0;
    s1 *= s1;
    s2 *= s2;
    const R t0 = s1 * s2;              // d_0 = 1  (x 1/10)
    const R t1 = R(6) * (s0 * s2);     // d_1 = 6
    const R t2 = R(3) * (s0 * s1);     // d_2 = 3
    num = P0 * t0 + P1 * t1 + P2 * t2;
    den = R(6) * (t0 + t1 + t2);
}

// FP32: the same fraction with every multiply-add explicit, in the order of
// the packed-pair version below (weno5_left_x2), so that an FP32
// reconstruction gives the same bits whether it runs alone or in a pair
template <>
__device__ __forceinline__ void weno5_left_nd<float>(float a, float b, float c, float d, float e,
                                                     float &num, float &den)
{
    const float P0 = __fmaf_rn(2.f, a, __fmaf_rn(-7.f, b, __fmul_rn(11.f, c)));
    const float P1 = __fmaf_rn(-1.f, b, __fmaf_rn(5.f, c, __fmul_rn(2.f, d)));
    const float P2 = __fmaf_rn(2.f, c, __fmaf_rn(5.f, d, __fmul_rn(-1.f, e)));
    const float x0 = __fmaf_rn(-2.f, b, __fadd_rn(a, c));
    const float y0 = __fmaf_rn(-4.f, b, __fmaf_rn(3.f, c, a));
    const float x1 = __fmaf_rn(-2.f, c, __fadd_rn(b, d));
    const float y1 = __fmaf_rn(-1.f, d, b);
    const float x2 = __fmaf_rn(-2.f, d, __fadd_rn(c, e));
    const float y2 = __fmaf_rn(-4.f, d, __fmaf_rn(3.f, c, e));
    const float k13 = 13.f / 12.f, q = 0.25f, eps = 1e-6f;
    float s0 = __fmaf_rn(__fmul_rn(k13, x0), x0, __fmaf_rn(__fmul_rn(q, y0), y0, eps));
    float s1 = __fmaf_rn(__fmul_rn(k13, x1), x1, __fmaf_rn(__fmul_rn(q, y1), y1, eps));
    float s2 = __fmaf_rn(__fmul_rn(k13, x2), x2, __fmaf_rn(__fmul_rn(q, y2), y2, eps));
    s0 = __fmul_rn(s0, s0);
    s1 = __fmul_rn(s1, s1);
    s2 = __fmul_rn(s2, s2);
    const float t0 = __fmul_rn(s1, s2);
    const float t1 = __fmul_rn(6.f, __fmul_rn(s0, s2));
    const float t2 = __fmul_rn(3.f, __fmul_rn(s0, s1));
    num = __fmaf_rn(P0, t0, __fmaf_rn(P1, t1, __fmul_rn(P2, t2)));
    den = __fmul_rn(6.f, __fadd_rn(t0, __fadd_rn(t1, t2)));
}

// Roe flux of a scalar law from the reconstructed states a = u^-, b = u^+
// (Sec. 2.1.2, Eq. roeflux): Roe speed lam = (u^+ + u^-)/2 for Burgers, 1 for
// advection; eigenvalues at the states lam^-/+ = f'(u^-/+); Harten-Hyman fix
//   delta = max(0, lam - lam^-, lam^+ - lam),
//   q = (lam^2/delta + delta)/2 if |lam| < delta, else |lam|;
//   F = (f(u^-) + f(u^+))/2 - q (u^+ - u^-)/2.
template <int FLUX, typename R>
__device__ __forceinline__ R roe_flux(R a, R b)
{
    const R lam = FLUX == FLX_BURGERS ? R(0.5) * (b + a) : R(1);
    const R lm = FLUX == FLX_BURGERS ? a : R(1);
    const R lp = FLUX == FLX_BURGERS ? b : R(1);
    R delta = R(0);
    if (lam - lm > delta) delta = lam - lm;
    if (lp - lam > delta) delta = lp - lam;
    const R q = fabs(lam) < delta ? R(0.5) * (lam * lam / delta + delta) : fabs(lam);
    return R(0.5) * (phys_flux<FLUX>(a) + phys_flux<FLUX>(b)) - R(0.5) * q * (b - a);
}

template <typename R>
__device__ __forceinline__ R warp_max(R v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// |x| as an ordered integer: for non-negative IEEE values integer order of
// the bit patterns is numeric order, so the global max |f'| of the LF alpha
// is taken on the integer pipes (the FP64 pipe is this kernel's bottleneck);
// the result is the same value bit for bit, and a NaN (whose magnitude bits
// exceed every finite value) propagates into alpha.
__device__ __forceinline__ long long mag_key(double x)
{
    return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}
__device__ __forceinline__ int mag_key(float x) { return __float_as_int(x) & 0x7fffffff; }
__device__ __forceinline__ double key_value(long long k) { return __longlong_as_double(k); }
__device__ __forceinline__ float key_value(int k) { return __int_as_float(k); }

// Block-wide max of magnitude keys; every thread returns it.  One barrier.
// `red` (NWARP_MAX values of R) holds the per-warp partials.
template <typename R, typename K>
__device__ __forceinline__ K block_max_key(K v, R *red)
{
    static_assert(sizeof(K) == sizeof(R), "key and value sizes differ");
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const K u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    K *kred = reinterpret_cast<K *>(red);
    if ((threadIdx.x & 31) == 0) MGRIT_SH(kred, threadIdx.x >> 5, NWARP_MAX) = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    K r = kred[0];
    for (int k = 1; k < nw; ++k) {
        const K u = MGRIT_SH(kred, k, NWARP_MAX);
        r = u > r ? u : r;
    }
    return r;
}

// Block-wide max; every thread returns the result.  Contains one barrier.
template <typename R>
__device__ __forceinline__ R block_max(R v, R *red)
{
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) MGRIT_SH(red, threadIdx.x >> 5, NWARP_MAX) = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    R r = red[0];
    for (int k = 1; k < nw; ++k) r = fmax(r, MGRIT_SH(red, k, NWARP_MAX));
    return r;
}

// Two WENO5 reconstructions at once on packed FP32 pairs: the operations of
// weno5_left_nd<float> in the same order, each a single packed instruction
// for both lanes (FP32 slabs are bound by instruction issue, not by the FMA
// pipe).  Lane k reconstructs from the k-th components of a..e.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 weno5_left_x2(float2 a, float2 b, float2 c, float2 d, float2 e)
{
    const float2 P0 = __ffma2_rn(f2(2.f), a, __ffma2_rn(f2(-7.f), b, __fmul2_rn(f2(11.f), c)));
    const float2 P1 = __ffma2_rn(f2(-1.f), b, __ffma2_rn(f2(5.f), c, __fmul2_rn(f2(2.f), d)));
    const float2 P2 = __ffma2_rn(f2(2.f), c, __ffma2_rn(f2(5.f), d, __fmul2_rn(f2(-1.f), e)));
    const float2 x0 = __ffma2_rn(f2(-2.f), b, __fadd2_rn(a, c));
    const float2 y0 = __ffma2_rn(f2(-4.f), b, __ffma2_rn(f2(3.f), c, a));
    const float2 x1 = __ffma2_rn(f2(-2.f), c, __fadd2_rn(b, d));
    const float2 y1 = __ffma2_rn(f2(-1.f), d, b);
    const float2 x2 = __ffma2_rn(f2(-2.f), d, __fadd2_rn(c, e));
    const float2 y2 = __ffma2_rn(f2(-4.f), d, __ffma2_rn(f2(3.f), c, e));
    const float2 k13 = f2(13.f / 12.f), q = f2(0.25f), eps = f2(1e-6f);
    float2 s0 = __ffma2_rn(__fmul2_rn(k13, x0), x0, __ffma2_rn(__fmul2_rn(q, y0), y0, eps));
    float2 s1 = __ffma2_rn(__fmul2_rn(k13, x1), x1, __ffma2_rn(__fmul2_rn(q, y1), y1, eps));
    float2 s2 = __ffma2_rn(__fmul2_rn(k13, x2), x2, __ffma2_rn(__fmul2_rn(q, y2), y2, eps));
    s0 = __fmul2_rn(s0, s0);
    s1 = __fmul2_rn(s1, s1);
    s2 = __fmul2_rn(s2, s2);
    const float2 t0 = __fmul2_rn(s1, s2);                          // d_0 = 1  (x 1/10)
    const float2 t1 = __fmul2_rn(f2(6.f), __fmul2_rn(s0, s2));     // d_1 = 6
    const float2 t2 = __fmul2_rn(f2(3.f), __fmul2_rn(s0, s1));     // d_2 = 3
    const float2 num = __ffma2_rn(P0, t0, __ffma2_rn(P1, t1, __fmul2_rn(P2, t2)));
    const float2 den = __fmul2_rn(f2(6.f), __fadd2_rn(t0, __fadd2_rn(t1, t2)));
    // the fast division as in weno5_left (den in [6e-24, 1e30] for |q| <= 1e3)
    return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

template <typename R, int SCHEME, int FLUX, int CPT>
struct Slab {
    R *qa;        // nx + 6: f^+ (split form) or the stage state (state form)
    R *qb;        // nx + 6: f^- (split form)
    R *qf;        // nx + 1: interface fluxes, qf[i+1] = F_{i+1/2}, qf[0] = F_{-1/2}
    R *red;       // NWARP_MAX
    int nx;
    int numflux;
    R dxinv;
    // SCH_LF_FE only: the integrator of the current level.  psiM = 0: the fine
    // scheme Eq. (fineLF) with the step passed to step(); psiM = M >= 1: the
    // matched integrator for M fine steps of size psiDt, zeroth order
    // (psiOrder 0, Eq. coarseLFord0) or first order (1, Eq. coarseLFord1)
    int psiM, psiOrder;
    R psiDt;
    static constexpr int kScheme = SCHEME, kCpt = CPT;

    __device__ __forceinline__ Slab(unsigned char *smem, int nx_, R dxinv_, int numflux_)
        : nx(nx_), numflux(numflux_), dxinv(dxinv_), psiM(0), psiOrder(0), psiDt(R(0))
    {
        qa = reinterpret_cast<R *>(smem);
        qb = qa + (nx + 2 * GHOST);
        qf = qb + (nx + 2 * GHOST);
        red = qf + (nx + 2 * GHOST);
    }

    static constexpr int RECON_UNROLL = sizeof(R) == 4 ? 1 : CPT;

    __device__ __forceinline__ int cell(int c) const { return threadIdx.x + c * blockDim.x; }
    __device__ __forceinline__ int lim() const { return nx + 2 * GHOST; }   // extent of qa, qb, qf

    // store cell i (and its periodic ghost copy) into slot i + GHOST
    __device__ __forceinline__ void put(R *arr, int i, R v) const
    {
        MGRIT_SH(arr, i + GHOST, lim()) = v;
        if (i < GHOST) MGRIT_SH(arr, i + GHOST + nx, lim()) = v;
        if (i >= nx - GHOST) MGRIT_SH(arr, i + GHOST - nx, lim()) = v;
    }

    // left-biased reconstruction at i+1/2 from slots around s = i + GHOST
    __device__ __forceinline__ R rec_minus(const R *q, int s) const
    {
        if (SCHEME == SCH_FO_FE) return MGRIT_SH(q, s, lim());
        return weno5_left<R>(MGRIT_SH(q, s - 2, lim()), MGRIT_SH(q, s - 1, lim()), MGRIT_SH(q, s, lim()),
                             MGRIT_SH(q, s + 1, lim()), MGRIT_SH(q, s + 2, lim()));
    }
    // right-biased reconstruction at i+1/2: the mirrored stencil
    __device__ __forceinline__ R rec_plus(const R *q, int s) const
    {
        if (SCHEME == SCH_FO_FE) return MGRIT_SH(q, s + 1, lim());
        return weno5_left<R>(MGRIT_SH(q, s + 3, lim()), MGRIT_SH(q, s + 2, lim()), MGRIT_SH(q, s + 1, lim()),
                             MGRIT_SH(q, s, lim()), MGRIT_SH(q, s - 1, lim()));
    }

    // F_{i+1/2} = W^-(f^+) + W^+(f^-) of the split form.  With WENO5 in FP64
    // the two fractions share one division, n1/d1 + n2/d2 = (n1 d2 + n2 d1) /
    // (d1 d2) (each d lies in [6e-24, 1e30] for |q| <= 1e3): the FP64 pipe is
    // this kernel's bottleneck and an IEEE division is a long sequence on it
    __device__ __forceinline__ R split_flux(int s) const
    {
        if (SCHEME == SCH_FO_FE || sizeof(R) == 4) return rec_minus(qa, s) + rec_plus(qb, s);
        const int L = lim();
        R n1, d1, n2, d2;
        weno5_left_nd<R>(MGRIT_SH(qa, s - 2, L), MGRIT_SH(qa, s - 1, L), MGRIT_SH(qa, s, L),
                         MGRIT_SH(qa, s + 1, L), MGRIT_SH(qa, s + 2, L), n1, d1);
        weno5_left_nd<R>(MGRIT_SH(qb, s + 3, L), MGRIT_SH(qb, s + 2, L), MGRIT_SH(qb, s + 1, L),
                         MGRIT_SH(qb, s, L), MGRIT_SH(qb, s - 1, L), n2, d2);
        return (n1 * d2 + n2 * d1) / (d1 * d2);
    }

    // FP32 WENO5 split fluxes of the owned interfaces two at a time (cells
    // c and c+1 of this thread) on packed pairs; a cell beyond nx reads slot
    // GHOST instead (in range) and its result is dropped
    __device__ __forceinline__ void split_fluxes_x2() const
    {
        const int L = lim();
#pragma unroll 1
        for (int c = 0; c < CPT; c += 2) {
            const int i0 = cell(c), i1 = c + 1 < CPT ? cell(c + 1) : nx;
            if (i0 >= nx) break;   // cells grow with c
            const int s0 = i0 + GHOST, s1 = (i1 < nx ? i1 : 0) + GHOST;
            const float2 m = weno5_left_x2(
                make_float2(MGRIT_SH(qa, s0 - 2, L), MGRIT_SH(qa, s1 - 2, L)),
                make_float2(MGRIT_SH(qa, s0 - 1, L), MGRIT_SH(qa, s1 - 1, L)),
                make_float2(MGRIT_SH(qa, s0, L), MGRIT_SH(qa, s1, L)),
                make_float2(MGRIT_SH(qa, s0 + 1, L), MGRIT_SH(qa, s1 + 1, L)),
                make_float2(MGRIT_SH(qa, s0 + 2, L), MGRIT_SH(qa, s1 + 2, L)));
            const float2 p = weno5_left_x2(
                make_float2(MGRIT_SH(qb, s0 + 3, L), MGRIT_SH(qb, s1 + 3, L)),
                make_float2(MGRIT_SH(qb, s0 + 2, L), MGRIT_SH(qb, s1 + 2, L)),
                make_float2(MGRIT_SH(qb, s0 + 1, L), MGRIT_SH(qb, s1 + 1, L)),
                make_float2(MGRIT_SH(qb, s0, L), MGRIT_SH(qb, s1, L)),
                make_float2(MGRIT_SH(qb, s0 - 1, L), MGRIT_SH(qb, s1 - 1, L)));
            put_flux(i0, m.x + p.x);
            if (i1 < nx) put_flux(i1, m.y + p.y);
        }
    }

    __device__ __forceinline__ void put_flux(int i, R F) const
    {
        MGRIT_SH(qf, i + 1, nx + 1) = F;
        if (i == nx - 1) qf[0] = F;
    }

    // Interface fluxes F_{i+1/2} of the stage input w into qf (Sec. 2.1.2).
    // Ends with a barrier after which qf is complete.
    __device__ __forceinline__ void fluxes(const R (&w)[CPT])
    {
        __syncthreads();   // previous readers of qa/qb/qf/red are done
        if (numflux == NF_SPLIT) {
            R alpha = R(1);
            if (FLUX == FLX_BURGERS) {   // alpha = max_j |u_j|
                decltype(mag_key(R(0))) v = 0;
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (cell(c) < nx) {
                        const auto k = mag_key(w[c]);
                        v = k > v ? k : v;
                    }
                alpha = key_value(block_max_key(v, red));
            }
            // f^+/- = f(u)/2 +/- (alpha/2) u, as one multiply-add on f/2
            const R h = R(0.5) * alpha;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const R p = R(0.5) * phys_flux<FLUX>(w[c]);
                    put(qa, i, fma(h, w[c], p));
                    put(qb, i, fma(-h, w[c], p));
                }
            }
            __syncthreads();
            // (beyond 8 cells per thread the pairs' live registers spill)
            if constexpr (sizeof(R) == 4 && SCHEME == SCH_WENO5_SSPRK3 && CPT <= 8) {
                split_fluxes_x2();
            } else {
            // this loop touches no register array, so FP32 slabs keep it rolled
            // (fewer live registers for 16-32 cells per thread); FP64 unrolls it
#pragma unroll(RECON_UNROLL)
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) put_flux(i, split_flux(i + GHOST));
            }
            }
        } else if (numflux == NF_ROE) {
            // local per interface: no global speed, no reduction
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) put(qa, i, w[c]);
            }
            __syncthreads();
#pragma unroll(RECON_UNROLL)
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx)
                    put_flux(i, roe_flux<FLUX>(rec_minus(qa, i + GHOST), rec_plus(qa, i + GHOST)));
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) put(qa, i, w[c]);
            }
            __syncthreads();
            // u^-_{i+1/2} parked in qb[i], u^+_{i+1/2} in qf[i+1]; each thread
            // reads back only its own slots, then overwrites qf[i+1] with F
            decltype(mag_key(R(0))) v = 0;   // max |u^-|, |u^+| (Burgers)
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const R um = rec_minus(qa, i + GHOST);
                    const R up = rec_plus(qa, i + GHOST);
                    MGRIT_SH(qb, i, nx) = um;
                    MGRIT_SH(qf, i + 1, nx + 1) = up;
                    const auto km = mag_key(um), kp = mag_key(up);
                    const auto k = km > kp ? km : kp;
                    v = k > v ? k : v;
                }
            }
            R alpha = R(1);
            if (FLUX == FLX_BURGERS) alpha = key_value(block_max_key(v, red));
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const R um = MGRIT_SH(qb, i, nx), up = MGRIT_SH(qf, i + 1, nx + 1);
                    put_flux(i, R(0.5) * (phys_flux<FLUX>(up) + phys_flux<FLUX>(um)) -
                                    R(0.5) * alpha * (up - um));
                }
            }
        }
        __syncthreads();
    }

    // A_i(w) = -(F_{i+1/2} - F_{i-1/2}) / dx for owned slot c (Eq. spaceDisc);
    // valid after fluxes().
    __device__ __forceinline__ R A(int c) const
    {
        const int i = cell(c);
        return -(MGRIT_SH(qf, i + 1, nx + 1) - MGRIT_SH(qf, i, nx + 1)) * dxinv;
    }

    // Eq. (fineLF): u <- E u - dt D f(u), (E v)_i = (v_{i+1} + v_{i-1})/2,
    // (D v)_i = (v_{i+1} - v_{i-1})/(2 dx); or, with psiM = M >= 1, the
    // matched integrators of Sec. 3.3 for M fine steps of size psiDt:
    //   zeroth order  E^M u - M psiDt D f(u)
    //   first order   E^M u - psiDt sum_{i=1..M} E^{i-1} D f(E^{M-i} u),
    // the sum formed by Horner's rule: acc_M = D f(u), then for k = 1..M-1
    // acc <- D f(E^k u) + E acc, so acc ends as the sum.
    __device__ __forceinline__ void lf_step(R (&u)[CPT], R dt)
    {
        const R hd = R(0.5) * dxinv;
        R v[CPT], acc[CPT];
        const bool first = psiM >= 1 && psiOrder == 1;
        const int M = psiM >= 1 ? psiM : 1;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            v[c] = u[c];
            acc[c] = R(0);
        }
        for (int k = 0; k < M; ++k) {
            __syncthreads();   // earlier readers of qa/qb/qf are done
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    put(qa, i, v[c]);
                    if (k == 0 || first) put(qb, i, phys_flux<FLUX>(v[c]));
                    if (first && k > 0) put(qf, i, acc[c]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const int s = i + GHOST;
                    const R Df = (MGRIT_SH(qb, s + 1, lim()) - MGRIT_SH(qb, s - 1, lim())) * hd;
                    if (first)
                        acc[c] = k == 0 ? Df
                                        : Df + R(0.5) * (MGRIT_SH(qf, s + 1, lim()) + MGRIT_SH(qf, s - 1, lim()));
                    else if (k == 0)
                        acc[c] = Df;   // D f(u)
                    v[c] = R(0.5) * (MGRIT_SH(qa, s + 1, lim()) + MGRIT_SH(qa, s - 1, lim()));
                }
            }
        }
        // v = E^M u; acc = D f(u) (fine, zeroth order) or the first-order sum
        const R h = psiM >= 1 ? (first ? psiDt : R(M) * psiDt) : dt;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < nx) u[c] = v[c] - h * acc[c];
    }

    // u <- Phi(u) with step dt: SSPRK3 (Eq. SSPRK3), forward Euler (Eq. SSPRK1)
    // or Eq. (fineLF) and its matched integrators (lf_step)
    __device__ __forceinline__ void step(R (&u)[CPT], R dt)
    {
        if (SCHEME == SCH_LF_FE) {
            lf_step(u, dt);
            return;
        }
        if (SCHEME == SCH_FO_FE) {
            fluxes(u);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (cell(c) < nx) u[c] = u[c] + dt * A(c);
            return;
        }
        R w[CPT];
        fluxes(u);
#pragma unroll
        for (int c = 0; c < CPT; ++c) w[c] = (cell(c) < nx) ? u[c] + dt * A(c) : R(0);
        fluxes(w);
        const R q = R(0.25) * dt;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < nx) w[c] = R(0.75) * u[c] + R(0.25) * w[c] + q * A(c);
        fluxes(w);
        const R t = R(2.0 / 3.0) * dt;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < nx) u[c] = R(1.0 / 3.0) * u[c] + R(2.0 / 3.0) * w[c] + t * A(c);
    }

    __device__ __forceinline__ void load(R (&u)[CPT], const R *__restrict__ row) const
    {
#ifdef MGRIT_DEBUG
        if (!row) return;
#endif
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            u[c] = (i < nx) ? row[i] : R(0);
        }
    }
    __device__ __forceinline__ void store(const R (&u)[CPT], R *__restrict__ row) const
    {
#ifdef MGRIT_DEBUG
        if (!row) return;
#endif
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            if (i < nx) row[i] = u[c];
        }
    }
    // u += g row; g is kept in FP64 (the FAS tau term), so an FP32 sweep adds
    // in FP64 and rounds the sum once
    __device__ __forceinline__ void add(R (&u)[CPT], const double *__restrict__ row) const
    {
#ifdef MGRIT_DEBUG
        if (!row) return;
#endif
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            if (i < nx) u[c] = R((double)u[c] + row[i]);
        }
    }
};

// shared-memory bytes of one slab
template <typename R>
inline size_t slab_smem_bytes(int nx)
{
    return sizeof(R) * (3 * (size_t)(nx + 2 * GHOST) + NWARP_MAX);
}

}  // namespace mgrit
