// Slab engine: one CTA owns one spatial slice u^n (nx cells) and applies the
// time-stepper Phi of Sec. 2.2 to it, keeping u^n in registers and the
// stage fluxes in shared memory for every step of a C-interval.
//
// Cell ownership is interleaved: thread t owns cells t + c*blockDim.x,
// c = 0..CPT-1 (cells >= nx are idle), so global row loads and stores are
// coalesced.  The interface fluxes are computed in contiguous runs instead:
// thread t takes the interfaces t*CPT .. t*CPT + CPT - 1 and slides a window
// of first differences along them (WenoWin below).
//
// Shared memory: three arrays (the half split fluxes q^+ and q^- with 3
// periodic ghost cells on each side -- the WENO5 half-stencil -- and the
// interface fluxes; at 2 or more cells per thread in the run-major layout
// of Slab) plus NWARP_MAX values for the block max reduction of the global
// Lax-Friedrichs alpha.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#ifdef MGRIT_DEBUG
#include <cstdio>
#endif

namespace mgrit {

namespace cg = cooperative_groups;

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

// FP32: the same fraction with every multiply-add explicit (used by the
// state-form and Roe fluxes, whose reconstructions act on the state), so
// that an FP32 reconstruction gives the same bits in every kernel that
// evaluates it
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

// ---------------------------------------------------------------------------
// Windowed WENO5-JS for the split form (Sec. 2.1.1, k = 2; Sec. 2.1.2).
//
// The arrays hold q = f^{+/-}/2 (a power-of-two scaling, exact).  With the
// first differences e_j = q_{j+1} - q_j, every quantity of Eqs. (C), (B) and
// (omega) at the interface i+1/2 is a short expression in e_{i-2..i+1}:
//   candidates   p_r = f_i + g_r / 6 (in units of f), g = 2 (5e_{i-1} - 2e_{i-2},
//                e_{i-1} + 2e_i, 4e_i - e_{i+1}) in units of q;
//   indicators   beta_r = (13/3) z_r^2 + y_r^2 with the second differences
//                z = e_j - e_{j-1} of the three 3-cell windows j = i-1, i, i+1
//                and y = (3e_{i-1} - e_{i-2}, e_{i-1} + e_i, e_{i+1} - 3e_i)
//                (the quadratic forms B_r of the paper, scaled by q = f/2);
//   weights      alpha_r = d_r / (eps + beta_r)^2, d = (1, 6, 3)/10,
//                normalised over a common denominator.
// The term Z_j = eps + (13/3) z_j^2 of window j is used by three
// neighbouring interfaces, and e_j by four, so a thread that owns a run of
// consecutive interfaces slides a window along them and forms each e_j and
// Z_j once.  The right-biased reconstruction of f^- is the same expression on
// the mirrored stencil, i.e. on (e_{i+2}, e_{i+1}, e_i, e_{i-1}) and
// (Z_{i+2}, Z_{i+1}, Z_i), with g and y negated.
//
// Every operation has explicit rounding, so each e_j, Z_j and interface
// flux is the same bit pattern whichever thread or CTA shape computes it
// (FP32 also on packed pairs, one instruction for two lanes).

template <typename V> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double k(double c) { return c; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double neg(double a) { return -a; }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float k(double c) { return (float)c; }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    // the fast division (2 ulp; the denominators stay inside [1e-24, 1e30])
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
};
template <> struct Ar<float2> {
    static __device__ __forceinline__ float2 k(double c) { return make_float2((float)c, (float)c); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b rounded once, as __fsub_rn
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, k(-1.0), a); }
    static __device__ __forceinline__ float2 div(float2 a, float2 b)
    {
        return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
    }
    static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
};

// Z of a 3-cell window from its two first differences (e_j, e_{j-1})
template <typename V>
__device__ __forceinline__ V weno_z(V ej, V ejm)
{
    using A = Ar<V>;
    const V z = A::sub(ej, ejm);
    return A::fma(A::mul(A::k(13.0 / 3.0), z), z, A::k(1e-6));
}

// Numerator N and denominator D of sum_r omega_r g_r = N / D for the
// stencil direction with first differences E0..E3 (e_{i-2..i+1} for the
// left-biased value) and window terms Z0..Z2 (Z_{i-1}, Z_i, Z_{i+1}):
//   N = g0 S1 S2 + 6 g1 S0 S2 + 3 g2 S0 S1,  D = S1 S2 + 6 S0 S2 + 3 S0 S1,
// S_r = (eps + beta_r)^2; the reconstructed value is q_i + N / (6 D).
template <typename V>
__device__ __forceinline__ void weno_nd_win(V E0, V E1, V E2, V E3, V Z0, V Z1, V Z2, V &N, V &D)
{
    using A = Ar<V>;
    const V y0 = A::fma(A::k(3.0), E1, A::neg(E0));
    const V y1 = A::add(E1, E2);
    const V y2 = A::fma(A::k(-3.0), E2, E3);
    const V g0 = A::fma(A::k(2.0), y0, A::neg(E1));   // 5 e_{i-1} - 2 e_{i-2}
    const V g1 = A::add(y1, E2);                                   // e_{i-1} + 2 e_i
    const V g2 = A::sub(E2, y2);                                   // 4 e_i - e_{i+1}
    V s0 = A::fma(y0, y0, Z0);
    V s1 = A::fma(y1, y1, Z1);
    V s2 = A::fma(y2, y2, Z2);
    s0 = A::mul(s0, s0);
    s1 = A::mul(s1, s1);
    s2 = A::mul(s2, s2);
    const V t = A::mul(s1, s2);                 // d_0 = 1  (x 1/10)
    const V a = A::mul(A::k(3.0), s1);          // d_2 = 3
    const V b = A::mul(A::k(6.0), s2);          // d_1 = 6
    D = A::fma(s0, A::add(a, b), t);
    N = A::fma(g0, t, A::mul(s0, A::fma(g1, b, A::mul(g2, a))));
}

// the window of one array along a run of interfaces (see above):
// f^+ (left-biased at i+1/2): e = (e_{i-2}, e_{i-1}, e_i, e_{i+1}),
//     z = (Z_{i-1}, Z_i, Z_{i+1}), last = q_{i+2};
// f^- (right-biased at i+1/2): e = (e_{i-1}, e_i, e_{i+1}, e_{i+2}),
//     z = (Z_i, Z_{i+1}, Z_{i+2}), last = q_{i+3}.
// The base values (q^+_i, q^-_{i+1}) are read from shared memory when needed,
// which keeps the window at eight registers (sixteen in FP64) per array.
template <typename V>
struct WenoWin {
    V last, e0, e1, e2, e3, z0, z1, z2;
    // from the values v0..v4 at five consecutive cells of the stencil
    __device__ __forceinline__ void init(V v0, V v1, V v2, V v3, V v4)
    {
        using A = Ar<V>;
        last = v4;
        e0 = A::sub(v1, v0);
        e1 = A::sub(v2, v1);
        e2 = A::sub(v3, v2);
        e3 = A::sub(v4, v3);
        z0 = weno_z(e1, e0);
        z1 = weno_z(e2, e1);
        z2 = weno_z(e3, e2);
    }
    // one interface to the right, given the next cell value
    __device__ __forceinline__ void advance(V v)
    {
        using A = Ar<V>;
        const V en = A::sub(v, last);
        const V zn = weno_z(en, e3);
        last = v;
        e0 = e1;
        e1 = e2;
        e2 = e3;
        e3 = en;
        z0 = z1;
        z1 = z2;
        z2 = zn;
    }
    __device__ __forceinline__ void left(V &N, V &D) const { weno_nd_win(e0, e1, e2, e3, z0, z1, z2, N, D); }
    // mirrored stencil: N carries the sign of the negated g
    __device__ __forceinline__ void right(V &N, V &D) const { weno_nd_win(e3, e2, e1, e0, z2, z1, z0, N, D); }
};

// interface flux F = W^-(f^+) + W^+(f^-) from the two windows and the base
// values qp = q^+_i, qm = q^-_{i+1} (Burgers), returned as G = 3F:
//   G = 6 (q^+_i + q^-_{i+1}) + (N^+ D^- - N^- D^+) / (D^+ D^-)
// (the factor 1/3 of the reconstructions is applied with dt/dx in the stage
// update, see RK), with one division in FP64 (each D lies in [1e-23, 1e33]
// for |q| <= 1e3, so the product stays far inside the FP64 range) and two in
// FP32
template <typename V>
__device__ __forceinline__ V split_flux_combine(V Np, V Dp, V Nm, V Dm, V qp, V qm)
{
    using A = Ar<V>;
    const V base = A::add(qp, qm);
    if constexpr (std::is_same<V, double>::value) {
        const V num = A::fma(Np, Dm, A::neg(A::mul(Nm, Dp)));
        return A::fma(A::k(6.0), base, A::div(num, A::mul(Dp, Dm)));
    } else {
        return A::fma(A::k(6.0), base, A::sub(A::div(Np, Dp), A::div(Nm, Dm)));
    }
}

// FP64: the numerator and denominator of split_flux_combine's fraction, and
// its base term, for an interface whose division is shared with others
// (split_flux_pair, split_flux_quad)
struct SplitParts {
    double num, den, base;
};
__device__ __forceinline__ SplitParts split_flux_parts(double Np, double Dp, double Nm, double Dm, double qp,
                                                       double qm)
{
    using A = Ar<double>;
    SplitParts r;
    r.base = A::add(qp, qm);
    r.num = A::fma(Np, Dm, A::neg(A::mul(Nm, Dp)));
    r.den = A::mul(Dp, Dm);
    return r;
}
// G of two interfaces from one reciprocal: with d = den0 den1 and i = 1/d
// (correctly rounded), num0/den0 = num0 (den1 i) and num1/den1 =
// num1 (den0 i), each quotient within three roundings.  Each D lies in
// [1e-23, 1e33] for |q| <= 1e3, so d lies in [1e-92, 1e132]; where d falls
// outside [2^-996, 2^997] (tested on its exponent bits, on the integer pipe)
// the two plain divisions are taken instead.
__device__ __forceinline__ void split_flux_pair(const SplitParts &a, const SplitParts &b, double &Ga, double &Gb)
{
    using A = Ar<double>;
    const double d = A::mul(a.den, b.den);
    const unsigned e = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;   // biased exponent (sign: d > 0)
    if (e - 27u <= 1993u) {
        const double inv = __drcp_rn(d);
        Ga = A::fma(6.0, a.base, A::mul(a.num, A::mul(b.den, inv)));
        Gb = A::fma(6.0, b.base, A::mul(b.num, A::mul(a.den, inv)));
    } else {
        Ga = A::fma(6.0, a.base, A::div(a.num, a.den));
        Gb = A::fma(6.0, b.base, A::div(b.num, b.den));
    }
}

// G of four interfaces from one reciprocal of the product of their
// denominators: r = 1/(d0 d1 d2 d3), 1/(d0 d1) = r d2 d3 and 1/(d2 d3) =
// r d0 d1, then each quotient as in split_flux_pair.  The product lies in
// [1e-184, 1e264] for |q| <= 1e3; outside [2^-996, 2^997] the two pairs are
// formed instead (each with its own range test).
__device__ __forceinline__ void split_flux_quad(const SplitParts (&x)[4], double (&G)[4])
{
    using A = Ar<double>;
    const double p01 = A::mul(x[0].den, x[1].den), p23 = A::mul(x[2].den, x[3].den);
    const double p = A::mul(p01, p23);
    const unsigned e = ((unsigned)__double2hiint(p) >> 20) & 0x7ffu;
    if (e - 27u <= 1993u) {
        const double r = __drcp_rn(p);
        const double i01 = A::mul(r, p23), i23 = A::mul(r, p01);   // 1/(d0 d1), 1/(d2 d3)
        G[0] = A::fma(6.0, x[0].base, A::mul(x[0].num, A::mul(x[1].den, i01)));
        G[1] = A::fma(6.0, x[1].base, A::mul(x[1].num, A::mul(x[0].den, i01)));
        G[2] = A::fma(6.0, x[2].base, A::mul(x[2].num, A::mul(x[3].den, i23)));
        G[3] = A::fma(6.0, x[3].base, A::mul(x[3].num, A::mul(x[2].den, i23)));
    } else {
        split_flux_pair(x[0], x[1], G[0], G[1]);
        split_flux_pair(x[2], x[3], G[2], G[3]);
    }
}

template <typename V>
__device__ __forceinline__ V split_flux_win(const WenoWin<V> &P, const WenoWin<V> &M, V qp, V qm)
{
    V Np, Dp, Nm, Dm;
    P.left(Np, Dp);
    M.right(Nm, Dm);
    return split_flux_combine(Np, Dp, Nm, Dm, qp, qm);
}

// advection (alpha = 1): f^- = (u - u)/2 is zero, so its reconstruction is
// exactly zero and G = 3 W^-(f^+) = 6 q^+_i + N^+ / D^+
template <typename V>
__device__ __forceinline__ V split_flux_win_adv(const WenoWin<V> &P, V qp)
{
    using A = Ar<V>;
    V Np, Dp;
    P.left(Np, Dp);
    return A::fma(A::k(6.0), qp, A::div(Np, Dp));
}

// The split fluxes of Burgers' flux in the scaled form the windows take,
// q^+/- = f^+/-/2 = u (u/8 +/- alpha/4) (Eq. LFflux with f = u^2/2), a4 =
// alpha/4.  FP64 forms q^- from q^+ as q^+ - (alpha/2) u, one multiply-add
// instead of two operations (the FP64 sweeps are bound by their FP64
// instruction count); FP32 keeps both products.  Every kernel forms them
// here, so the steppers agree bit for bit.
template <typename R>
__device__ __forceinline__ void burgers_q(R x, R a4, R &qp, R &qm)
{
    qp = Ar<R>::mul(Ar<R>::fma(R(0.125), x, a4), x);
    if constexpr (sizeof(R) == 8)
        qm = Ar<R>::fma(R(-2) * a4, x, qp);   // -2 a4 = -alpha/2 exactly
    else
        qm = Ar<R>::mul(Ar<R>::fma(R(0.125), x, -a4), x);
}

// Runge-Kutta stage updates of Eq. (SSPRK3) and forward Euler (Eq. SSPRK1)
// from the difference dG = G_{i+1/2} - G_{i-1/2} of a cell's interface
// values G = F / s (s = 1/3 for the WENO5 split form, whose G is 3F; s = 1
// otherwise), so that dt A_i = k1 dG with k1 = -(dt/dx) s (Eq. spaceDisc).
// The coefficients are formed once per step (coef), and every stepper (the
// one-CTA slab, the cluster stepper, the grid stepper) performs the same
// operations, so a chain of steps gives the same bits on each of them.
//  - FP64: the Shu-Osher combinations as written, 3/4 u + 1/4 w + 1/4 dt A
//    and 1/3 u + 2/3 w + 2/3 dt A (closest to the oracle's operation order);
//  - FP32: the same combinations in increment form, u + 1/4 ((w - u) + dt A)
//    and u + 2/3 ((w - u) + dt A), which round the state once per stage
//    (w - u and the increment are small and nearly exact): over the 65536
//    steps of the largest workload this halves the drift from FP64 stepping.
template <typename R>
struct RK {
    using A_ = Ar<R>;
    static constexpr bool INC = sizeof(R) == 4;
    struct Coef {
        R k1;   // -(dt/dx) s: dt A = k1 dG
        R k2;   // k1 / 4 (FP64 stage 2)
        R k3;   // 2/3 k1 (FP64 stage 3)
    };
    static __device__ __forceinline__ Coef coef(R dt, R dxinv, R s)
    {
        Coef c;
        c.k1 = A_::mul(A_::mul(A_::neg(dt), dxinv), s);
        c.k2 = A_::mul(R(0.25), c.k1);
        c.k3 = A_::mul(R(2.0 / 3.0), c.k1);
        return c;
    }
    // u + dt A (forward Euler; the first SSPRK3 stage)
    static __device__ __forceinline__ R euler(R u, const Coef &c, R dG) { return A_::fma(c.k1, dG, u); }
    // 3/4 u + 1/4 w + 1/4 dt A
    static __device__ __forceinline__ R stage2(R u, R w, const Coef &c, R dG)
    {
        if (INC) return A_::fma(R(0.25), A_::fma(c.k1, dG, A_::sub(w, u)), u);
        return A_::fma(R(0.75), u, A_::fma(R(0.25), w, A_::mul(c.k2, dG)));
    }
    // 1/3 u + 2/3 w + 2/3 dt A
    static __device__ __forceinline__ R stage3(R u, R w, const Coef &c, R dG)
    {
        if (INC) return A_::fma(R(2.0 / 3.0), A_::fma(c.k1, dG, A_::sub(w, u)), u);
        return A_::fma(R(1.0 / 3.0), u, A_::fma(R(2.0 / 3.0), w, A_::mul(c.k3, dG)));
    }
};

// s of RK: the WENO5 split form stores G = 3F (split_flux_combine)
template <typename R>
__device__ __forceinline__ R flux_scale(bool weno_split)
{
    return weno_split ? R(1.0 / 3.0) : R(1);
}

// Run stride of the run-major layout of Slab below for a CTA of `threads`
// threads: the runs 0 .. threads + RO + 1 (RO runs of left ghosts, the
// threads' runs, the right ghosts), rounded up so that the interleaved writes
// of 32 consecutive cells hit distinct banks: P = 32/CPT (mod 32) for FP32
// (one word per bank), P = 16/CPT (mod 16) for FP64 (a double spans two
// banks, and a warp's doubles are served in two halves).  FP32 sizes it for
// the largest CTA (512 threads), so that it is a compile-time constant of
// the CTA shape; FP64 sizes it for the launch, whose slab is twice as large.
template <typename R>
__host__ __device__ constexpr int slab_run_stride(int cpt, int threads)
{
    const int ro = cpt >= 4 ? 1 : 2;
    const int p0 = (sizeof(R) == 4 ? 512 : threads) + ro + 2;
    const int bank = sizeof(R) == 4 ? 32 : 16;
    const int r0 = cpt <= bank ? (bank / cpt) % bank : 0;
    return p0 + ((r0 - p0 % bank) % bank + bank) % bank;
}

// FLAT: keep every cell at slot i + GHOST whatever CPT (the adjoint slab,
// which overlays its own arrays on that layout).
// CLUSTER: one of the K CTAs of a thread-block cluster that share one slice
// (WENO5 split form only): CTA r holds the contiguous cells [lo, lo + nx) of
// it in the same run-major layout, and fluxes_cluster() exchanges the
// Lax-Friedrichs alpha and the 3 + 3 ghost cells through distributed shared
// memory instead of the periodic copies.
template <typename R, int SCHEME, int FLUX, int CPT, bool FLAT = false, bool CLUSTER = false>
struct Slab {
    R *qa;        // slots of cells -3..nx+2: f^+ / 2 (WENO5 split form), f^+ (first
                  // order), or the stage state (state form, Roe)
    R *qb;        // the same slots: f^- / 2 or f^-
    R *qf;        // slots 0..nx: interface fluxes, qf[i+1] = F_{i+1/2}, qf[0] = F_{-1/2}
    R *red;       // NWARP_MAX
    R *ck;        // [2] CLUSTER: this CTA's alpha key, by stage parity
    R *gw;        // [2][6] CLUSTER: stage inputs of the ghost cells -3..-1, nx..nx+2,
                  // written by the neighbours, by stage parity
    int nx;       // cells of this slab (CLUSTER: of this CTA's block)
    int lo;       // first cell of the block in the slice (0 unless CLUSTER)
    int rank, K;  // CLUSTER: block rank and cluster size
    int par;      // CLUSTER: stage parity
    int numflux;
    R dxinv;
    // SCH_LF_FE only: the integrator of the current level.  psiM = 0: the fine
    // scheme Eq. (fineLF) with the step passed to step(); psiM = M >= 1: the
    // matched integrator for M fine steps of size psiDt, zeroth order
    // (psiOrder 0, Eq. coarseLFord0) or first order (1, Eq. coarseLFord1)
    int psiM, psiOrder;
    R psiDt;
    // FP64 WENO5 split form: interfaces in quads share one reciprocal
    // (split_flux_quad).  Set by the relaxation and interpolation sweeps; the
    // sequential chains keep one division per interface, the operations of
    // the cluster and grid steppers.
    bool pair_div;
    static constexpr int kScheme = SCHEME, kCpt = CPT;

    // Shared-array layout.  Slabs with CPT >= 2 use a run-major layout: the
    // window pass gives thread t the run of interfaces t*CPT .. t*CPT + CPT - 1,
    // and cell i sits at slot k * P + r with r = (i + RO*CPT) / CPT (its run,
    // after RO runs of left ghosts) and k = (i + RO*CPT) mod CPT.  Lanes
    // reading element k of consecutive runs then touch consecutive slots, a
    // window step is a constant offset, and the run stride P
    // (slab_run_stride) keeps the interleaved writes of 32 consecutive cells
    // free of bank conflicts too.  CPT = 1 slabs (and FLAT ones) keep cell i
    // (i = -3 .. nx+2) at slot i + GHOST.  The interface flux F_{i+1/2} is
    // kept at cell i of qf (F_{-1/2} at cell -1).
    static constexpr bool TL = !FLAT && CPT >= 2;
    static_assert(!CLUSTER || (TL && SCHEME == SCH_WENO5_SSPRK3), "cluster slabs: run-major WENO5 only");
    static constexpr int LOG = CPT >= 32 ? 5 : CPT >= 16 ? 4 : CPT >= 8 ? 3 : CPT >= 4 ? 2 : CPT >= 2 ? 1 : 0;
    static constexpr int RO = CPT >= 4 ? 1 : 2;
    // FP32: the run stride as a compile-time constant
    static constexpr int P32 = slab_run_stride<float>(CPT, 512);
    // elements of each of qa, qb, qf
    static __host__ __device__ __forceinline__ int extent(int nx, int threads)
    {
        return TL ? CPT * slab_run_stride<R>(CPT, threads) : nx + 2 * GHOST;
    }

    int E;        // elements per array
    int pstride;  // slot distance between a thread's consecutive interleaved cells
    int prun;     // run stride (FP64; FP32 uses P32)

    __device__ __forceinline__ int P() const { return sizeof(R) == 4 ? P32 : prun; }

    __device__ __forceinline__ Slab(unsigned char *smem, int nx_, R dxinv_, int numflux_)
        : nx(nx_), lo(0), rank(0), K(1), par(0), numflux(numflux_), dxinv(dxinv_), psiM(0), psiOrder(0),
          psiDt(R(0)), pair_div(false)
    {
        const int T = (int)blockDim.x;
        if constexpr (CLUSTER) {
            cg::cluster_group cl = cg::this_cluster();
            K = (int)cl.num_blocks();
            rank = (int)cl.block_rank();
            lo = (int)((long long)rank * nx_ / K);
            nx = (int)((long long)(rank + 1) * nx_ / K) - lo;
        }
        E = extent(nx, T);
        prun = slab_run_stride<R>(CPT, T);
        // blockDim.x is a multiple of 32, hence of CPT: cell t + c*T + o sits at
        // sl(t + o) + c * pstride
        pstride = TL ? T / CPT : T;
        qa = reinterpret_cast<R *>(smem);
        qb = qa + E;
        qf = qb + E;
        red = qf + E;
        ck = red + NWARP_MAX;
        gw = ck + 2;
    }

    __device__ __forceinline__ int cell(int c) const { return threadIdx.x + c * blockDim.x; }
    __device__ __forceinline__ int lim() const { return E; }   // extent of qa, qb, qf

    // slot of cell i
    __device__ __forceinline__ int sl(int i) const
    {
        if (!TL) return i + GHOST;
        const int v = i + RO * CPT;
        return (v & (CPT - 1)) * P() + (v >> LOG);
    }
    __device__ __forceinline__ R &ce(R *arr, int i) const { return MGRIT_SH(arr, sl(i), lim()); }
    __device__ __forceinline__ R ce(const R *arr, int i) const { return MGRIT_SH(arr, sl(i), lim()); }

    // store cell i (and its periodic ghost copy)
    __device__ __forceinline__ void put(R *arr, int i, R v) const
    {
        ce(arr, i) = v;
        if (i < GHOST) ce(arr, i + nx) = v;
        if (i >= nx - GHOST) ce(arr, i - nx) = v;
    }
    // interfaces i0 .. i0 + run() - 1 (i0 = t * CPT) of this thread's contiguous run
    __device__ __forceinline__ int run() const
    {
        const int r = nx - (int)threadIdx.x * CPT;
        return r < 0 ? 0 : (r < CPT ? r : CPT);
    }
    // slot of cell(c) + o (affine in c, see pstride)
    __device__ __forceinline__ int pc(int c, int o) const { return sl((int)threadIdx.x + o) + c * pstride; }
    // put() for this thread's owned cell c (c a constant once unrolled; a
    // CTA has at least 32 threads, so only c = 0 can hold cells 0..2)
    __device__ __forceinline__ void put_c(R *arr, int c, R v) const
    {
        const int i = cell(c);
        MGRIT_SH(arr, pc(c, 0), lim()) = v;
        if constexpr (CLUSTER) return;   // ghosts come from the neighbours
        if (c == 0 && i < GHOST) ce(arr, i + nx) = v;
        if (i >= nx - GHOST) ce(arr, i - nx) = v;
    }
    // slot of cell i0 + m of this thread's run (i0 = t * CPT), m a constant
    // in -CPT*RO .. 2*CPT - 1 once the loops below are unrolled
    __device__ __forceinline__ int rs(int m) const
    {
        if (!TL) return (int)threadIdx.x * CPT + m + GHOST;
        const int mm = m + RO * CPT;   // >= 0
        return (mm & (CPT - 1)) * P() + (int)threadIdx.x + (mm >> LOG);
    }

    // left-biased reconstruction at i+1/2 from the cells around i
    __device__ __forceinline__ R rec_minus(const R *q, int i) const
    {
        if (SCHEME == SCH_FO_FE) return ce(q, i);
        return weno5_left<R>(ce(q, i - 2), ce(q, i - 1), ce(q, i), ce(q, i + 1), ce(q, i + 2));
    }
    // right-biased reconstruction at i+1/2: the mirrored stencil
    __device__ __forceinline__ R rec_plus(const R *q, int i) const
    {
        if (SCHEME == SCH_FO_FE) return ce(q, i + 1);
        return weno5_left<R>(ce(q, i + 3), ce(q, i + 2), ce(q, i + 1), ce(q, i), ce(q, i - 1));
    }

    // F_{i+1/2} into cell i of qf (and F_{-1/2} = F_{nx-1/2} into cell -1)
    __device__ __forceinline__ void put_flux(int i, R F) const
    {
        ce(qf, i) = F;
        if (i == nx - 1) ce(qf, -1) = F;
    }

    // WENO5 split fluxes of the interfaces i0 .. i0 + CPT - 1 (i0 = t * CPT)
    // from qa = f^+/2 and qb = f^-/2, one sliding window per array (see
    // WenoWin), stored as G = 3F.  Reads cells i0 - 2 .. i0 + n + 2, all inside
    // the arrays for every interface i < nx.  FP64: a rolled loop (the window
    // shifts by register moves; unrolled, the slabs spill), four interfaces
    // per iteration (then pairs) with pair_div; FP32: unrolled, so every slot is
    // the thread's base plus a constant.
    __device__ __forceinline__ void split_fluxes_win() const
    {
        const int i0 = threadIdx.x * CPT;
        if (i0 >= nx) return;
        const int n = nx - i0 < CPT ? nx - i0 : CPT;
        auto A_ = [&](int m) { return MGRIT_SH(qa, rs(m), lim()); };
        auto B_ = [&](int m) { return MGRIT_SH(qb, rs(m), lim()); };
        WenoWin<R> P, M;
        P.init(A_(-2), A_(-1), A_(0), A_(1), A_(2));
        if (FLUX == FLX_BURGERS) M.init(B_(-1), B_(0), B_(1), B_(2), B_(3));
        if constexpr (sizeof(R) == 8 && FLUX == FLX_BURGERS && CPT >= 2) {
            if (pair_div) {
                // interfaces in quads (k .. k+3, k a multiple of 4), then the
                // rest in pairs and a last one alone: i0 is a multiple of 4
                // (FP64 WENO5 slabs have at least 4 cells per thread), so every
                // CTA shape forms the same global quads [4j, 4j+3] and the
                // same tail
                int k0 = 0;
#pragma unroll 1
                for (; k0 + 3 < n; k0 += 4) {
                    SplitParts x[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        R Np, Dp, Nm, Dm;
                        P.left(Np, Dp);
                        M.right(Nm, Dm);
                        x[q] = split_flux_parts(Np, Dp, Nm, Dm, A_(k0 + q), B_(k0 + q + 1));
                        if (k0 + q + 1 < n) {
                            P.advance(A_(k0 + q + 3));
                            M.advance(B_(k0 + q + 4));
                        }
                    }
                    R G[4];
                    split_flux_quad(x, G);
#pragma unroll
                    for (int q = 0; q < 4; ++q) MGRIT_SH(qf, rs(k0 + q), lim()) = G[q];
                }
#pragma unroll 1
                for (int k = k0; k < n; k += 2) {
                    R Np, Dp, Nm, Dm;
                    P.left(Np, Dp);
                    M.right(Nm, Dm);
                    const SplitParts x = split_flux_parts(Np, Dp, Nm, Dm, A_(k), B_(k + 1));
                    if (k + 1 >= n) {
                        MGRIT_SH(qf, rs(k), lim()) = Ar<R>::fma(6.0, x.base, Ar<R>::div(x.num, x.den));
                        break;
                    }
                    P.advance(A_(k + 3));
                    M.advance(B_(k + 4));
                    P.left(Np, Dp);
                    M.right(Nm, Dm);
                    const SplitParts y = split_flux_parts(Np, Dp, Nm, Dm, A_(k + 1), B_(k + 2));
                    R G0, G1;
                    split_flux_pair(x, y, G0, G1);
                    MGRIT_SH(qf, rs(k), lim()) = G0;
                    MGRIT_SH(qf, rs(k + 1), lim()) = G1;
                    if (k + 2 < n) {
                        P.advance(A_(k + 4));
                        M.advance(B_(k + 5));
                    }
                }
                if (!CLUSTER && i0 + n == nx) ce(qf, -1) = MGRIT_SH(qf, rs(n - 1), lim());
                return;
            }
        }
#pragma unroll(sizeof(R) == 4 ? CPT : 1)
        for (int k = 0; k < CPT; ++k) {
            if (k >= n) break;
            const R qp = A_(k);
            const R F = FLUX == FLX_BURGERS ? split_flux_win(P, M, qp, B_(k + 1)) : split_flux_win_adv(P, qp);
            MGRIT_SH(qf, rs(k), lim()) = F;
            if (k + 1 < n) {
                P.advance(A_(k + 3));
                if (FLUX == FLX_BURGERS) M.advance(B_(k + 4));
            }
        }
        // G_{-1/2} = G_{nx-1/2}, from the thread whose run ends at nx - 1 (a
        // cluster slab forms it from its ghosts instead)
        if (!CLUSTER && i0 + n == nx) ce(qf, -1) = MGRIT_SH(qf, rs(n - 1), lim());
    }

    // FP32: the same windows on packed pairs.  Lane x of the pair walks
    // interfaces i0 .. i0 + CPT/2 - 1, lane y i0 + CPT/2 .. i0 + CPT - 1;
    // each lane performs the scalar window's operations, so the bits do not
    // depend on the pairing.  Where lane y's interfaces run past nx its cells
    // still lie inside the arrays (the run stride leaves two runs to the
    // right of the last thread's); those results are dropped.
    __device__ __forceinline__ void split_fluxes_win2() const
    {
        static_assert(sizeof(R) == 4 && CPT >= 2, "packed windows are FP32 with CPT >= 2");
        constexpr int H = CPT / 2;
        const int i0 = threadIdx.x * CPT;
        if (i0 >= nx) return;
        const int n = nx - i0 < CPT ? nx - i0 : CPT;
        auto ld = [&](const R *q, int m) {
            return make_float2(MGRIT_SH(q, rs(m), lim()), MGRIT_SH(q, rs(m + H), lim()));
        };
        WenoWin<float2> P, M;
        P.init(ld(qa, -2), ld(qa, -1), ld(qa, 0), ld(qa, 1), ld(qa, 2));
        if (FLUX == FLX_BURGERS) M.init(ld(qb, -1), ld(qb, 0), ld(qb, 1), ld(qb, 2), ld(qb, 3));
#pragma unroll
        for (int k = 0; k < H; ++k) {
            if (k >= n) break;
            const float2 qp = ld(qa, k);
            const float2 F = FLUX == FLX_BURGERS ? split_flux_win(P, M, qp, ld(qb, k + 1))
                                                 : split_flux_win_adv(P, qp);
            MGRIT_SH(qf, rs(k), lim()) = F.x;
            if (H + k < n) MGRIT_SH(qf, rs(H + k), lim()) = F.y;
            if (k + 1 < H) {
                P.advance(ld(qa, k + 3));
                if (FLUX == FLX_BURGERS) M.advance(ld(qb, k + 4));
            }
        }
        // F_{-1/2} = F_{nx-1/2}, from the thread whose run ends at nx - 1 (its
        // own store of that interface precedes this read in program order; a
        // cluster slab forms it from its ghosts instead)
        if (!CLUSTER && i0 + n == nx) ce(qf, -1) = MGRIT_SH(qf, rs(n - 1), lim());
    }

    // Interface fluxes F_{i+1/2} of the stage input w into qf (Sec. 2.1.2).
    // Ends with a barrier after which qf is complete.
    // CLUSTER: the split-form interface values of this CTA's block.  Per stage
    // one cluster barrier: before it, each CTA publishes its alpha key and
    // writes the stage inputs of its three first and three last cells into
    // the ghost slots of its neighbours (double-buffered by stage parity: a
    // CTA writes buffer p of stage s + 2 only after the barrier of stage
    // s + 1, which no CTA passes before every CTA has read stage s's values);
    // after it, alpha is the maximum of the K keys, and each CTA forms q of
    // its own and its ghost cells.  G_{-1/2} is formed from the left ghosts
    // by one thread, with the windows of the other interfaces' operations.
    __device__ __forceinline__ void fluxes_cluster(const R (&w)[CPT])
    {
        using KT = decltype(mag_key(R(0)));
        cg::cluster_group cl = cg::this_cluster();
        __syncthreads();   // previous readers of qa/qb/qf/red are done
        const int p = par;
        par ^= 1;
        KT v = 0;
        if (FLUX == FLX_BURGERS) {
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (cell(c) < nx) {
                    const KT k = mag_key(w[c]);
                    v = k > v ? k : v;
                }
            v = block_max_key(v, red);
            if (threadIdx.x == 0) reinterpret_cast<KT *>(ck)[p] = v;
        }
        {
            const unsigned right = (unsigned)((rank + 1) % K), left = (unsigned)((rank + K - 1) % K);
            R *gr = cl.map_shared_rank(gw, right), *gl = cl.map_shared_rank(gw, left);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx && i >= nx - GHOST) gr[6 * p + i - (nx - GHOST)] = w[c];   // its cells -3..-1
                if (c == 0 && i < GHOST) gl[6 * p + GHOST + i] = w[c];             // its cells n..n+2
            }
        }
        cl.sync();
        R alpha = R(1);
        if (FLUX == FLX_BURGERS) {
            KT m = 0;
            for (int r = 0; r < K; ++r) {
                const KT k = reinterpret_cast<const KT *>(cl.map_shared_rank(ck, (unsigned)r))[p];
                m = k > m ? k : m;
            }
            alpha = key_value(m);
        }
        const R a4 = R(0.25) * alpha;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < nx) {
                if (FLUX == FLX_BURGERS) {
                    R qpv, qmv;
                    burgers_q(w[c], a4, qpv, qmv);
                    MGRIT_SH(qa, pc(c, 0), lim()) = qpv;
                    MGRIT_SH(qb, pc(c, 0), lim()) = qmv;
                } else {
                    MGRIT_SH(qa, pc(c, 0), lim()) = R(0.5) * w[c];
                }
            }
        if (threadIdx.x < 2 * GHOST) {
            const int t = (int)threadIdx.x;
            const int i = t < GHOST ? t - GHOST : nx + t - GHOST;
            const R x = gw[6 * p + t];
            if (FLUX == FLX_BURGERS) {
                R qpv, qmv;
                burgers_q(x, a4, qpv, qmv);
                ce(qa, i) = qpv;
                ce(qb, i) = qmv;
            } else {
                ce(qa, i) = R(0.5) * x;
            }
        }
        __syncthreads();
        if constexpr (sizeof(R) == 4 && CPT <= 16)
            split_fluxes_win2();
        else
            split_fluxes_win();
        if (threadIdx.x == blockDim.x - 1) {   // G_{-1/2} from cells -3..2
            WenoWin<R> P;
            P.init(ce(qa, -3), ce(qa, -2), ce(qa, -1), ce(qa, 0), ce(qa, 1));
            R G;
            if (FLUX == FLX_BURGERS) {
                WenoWin<R> M;
                M.init(ce(qb, -2), ce(qb, -1), ce(qb, 0), ce(qb, 1), ce(qb, 2));
                G = split_flux_win(P, M, ce(qa, -1), ce(qb, 0));
            } else {
                G = split_flux_win_adv(P, ce(qa, -1));
            }
            ce(qf, -1) = G;
        }
        __syncthreads();
    }

    __device__ __forceinline__ void fluxes(const R (&w)[CPT])
    {
        if constexpr (CLUSTER) {
            fluxes_cluster(w);
            return;
        }
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
            if (SCHEME == SCH_WENO5_SSPRK3) {
                // q^+/- = f^+/-/2 = u (u/8 +/- alpha/4) (Burgers), u/2 and 0 (advection)
                const R a4 = R(0.25) * alpha;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int i = cell(c);
                    if (i < nx) {
                        if (FLUX == FLX_BURGERS) {
                            R qpv, qmv;
                            burgers_q(w[c], a4, qpv, qmv);
                            put_c(qa, c, qpv);
                            put_c(qb, c, qmv);
                        } else {
                            put_c(qa, c, R(0.5) * w[c]);
                        }
                    }
                }
                __syncthreads();
                // (packed FP32 windows beyond 16 cells per thread would spill)
                if constexpr (sizeof(R) == 4 && CPT >= 2 && CPT <= 16)
                    split_fluxes_win2();
                else
                    split_fluxes_win();
            } else {
                // first order: f^+/- = f(u)/2 +/- (alpha/2) u, one multiply-add on f/2
                const R h = R(0.5) * alpha;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int i = cell(c);
                    if (i < nx) {
                        const R p = R(0.5) * phys_flux<FLUX>(w[c]);
                        put_c(qa, c, fma(h, w[c], p));
                        put_c(qb, c, fma(-h, w[c], p));
                    }
                }
                __syncthreads();
                const int i0 = threadIdx.x * CPT, n = run();
#pragma unroll 1
                for (int k = 0; k < n; ++k)
                    put_flux(i0 + k, rec_minus(qa, i0 + k) + rec_plus(qb, i0 + k));
            }
        } else if (numflux == NF_ROE) {
            // local per interface: no global speed, no reduction
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) put_c(qa, c, w[c]);
            }
            __syncthreads();
            const int i0 = threadIdx.x * CPT, n = run();
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                put_flux(i0 + k, roe_flux<FLUX>(rec_minus(qa, i0 + k), rec_plus(qa, i0 + k)));
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) put_c(qa, c, w[c]);
            }
            __syncthreads();
            // u^-_{i+1/2} parked in qb cell i, u^+_{i+1/2} in qf cell i for this
            // thread's run of interfaces; each thread reads back only its own
            // cells, then overwrites qf cell i with F
            const int i0 = threadIdx.x * CPT, n = run();
            decltype(mag_key(R(0))) v = 0;   // max |u^-|, |u^+| (Burgers)
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                const int i = i0 + k;
                const R um = rec_minus(qa, i);
                const R up = rec_plus(qa, i);
                ce(qb, i) = um;
                ce(qf, i) = up;
                const auto km = mag_key(um), kp = mag_key(up);
                const auto kk = km > kp ? km : kp;
                v = kk > v ? kk : v;
            }
            R alpha = R(1);
            if (FLUX == FLX_BURGERS) alpha = key_value(block_max_key(v, red));
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                const int i = i0 + k;
                const R um = ce(qb, i), up = ce(qf, i);
                put_flux(i, R(0.5) * (phys_flux<FLUX>(up) + phys_flux<FLUX>(um)) - R(0.5) * alpha * (up - um));
            }
        }
        __syncthreads();
    }

    // dG_i = G_{i+1/2} - G_{i-1/2} for owned slot c, valid after fluxes():
    // dt A_i(w) = k1 dG_i (Eq. spaceDisc; RK)
    __device__ __forceinline__ R df(int c) const
    {
        return Ar<R>::sub(MGRIT_SH(qf, pc(c, 0), lim()), MGRIT_SH(qf, pc(c, -1), lim()));
    }
    // the stage coefficients of a step of size dt
    __device__ __forceinline__ typename RK<R>::Coef coef(R dt) const
    {
        return RK<R>::coef(dt, dxinv, flux_scale<R>(SCHEME == SCH_WENO5_SSPRK3 && numflux == NF_SPLIT));
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
                    const R Df = (ce(qb, i + 1) - ce(qb, i - 1)) * hd;
                    if (first)
                        acc[c] = k == 0 ? Df
                                        : Df + R(0.5) * (ce(qf, i + 1) + ce(qf, i - 1));
                    else if (k == 0)
                        acc[c] = Df;   // D f(u)
                    v[c] = R(0.5) * (ce(qa, i + 1) + ce(qa, i - 1));
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
        const typename RK<R>::Coef K = coef(dt);
        if (SCHEME == SCH_FO_FE) {
            fluxes(u);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (cell(c) < nx) u[c] = RK<R>::euler(u[c], K, df(c));
            return;
        }
        // the three stages as one rolled loop, so that the flux pass is
        // compiled once per call site of step() (the unrolled window code is
        // large, and several copies of it miss in the instruction cache)
        R w[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) w[c] = u[c];
#pragma unroll 1
        for (int st = 0; st < 3; ++st) {
            fluxes(w);
            if (st == 0) {
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (cell(c) < nx) w[c] = RK<R>::euler(u[c], K, df(c));
            } else if (st == 1) {
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (cell(c) < nx) w[c] = RK<R>::stage2(u[c], w[c], K, df(c));
            } else {
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (cell(c) < nx) w[c] = RK<R>::stage3(u[c], w[c], K, df(c));
            }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) u[c] = w[c];
    }

    __device__ __forceinline__ void load(R (&u)[CPT], const R *__restrict__ row) const
    {
#ifdef MGRIT_DEBUG
        if (!row) return;
#endif
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            u[c] = (i < nx) ? row[lo + i] : R(0);
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
            if (i < nx) row[lo + i] = u[c];
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
            if (i < nx) u[c] = R((double)u[c] + row[lo + i]);
        }
    }
};

// shared-memory bytes of one slab of nx cells on `threads` threads with cpt
// cells per thread (the layout of Slab above)
template <typename R>
inline size_t slab_smem_bytes(int nx, int cpt, int threads)
{
    const size_t e = cpt >= 2 ? (size_t)cpt * slab_run_stride<R>(cpt, threads) : (size_t)nx + 2 * GHOST;
    return sizeof(R) * (3 * e + NWARP_MAX);
}
// the same for one CTA of a cluster slab (its block of at most nmax cells;
// the layout does not depend on nmax), with the alpha keys and ghost inputs
template <typename R>
inline size_t slab_cluster_smem_bytes(int nmax, int cpt, int threads)
{
    return slab_smem_bytes<R>(nmax, cpt, threads) + sizeof(R) * (2 + 12);
}

}  // namespace mgrit
