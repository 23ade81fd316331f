// Discrete adjoint of the time-stepper, lam <- Phi'(u)^T lam, and the adjoint
// MGRIT kernels (Algorithm 1 run backward in time on lam^n = Phi'(u^n)^T lam^{n+1}).
//
// The paper has no adjoint; this differentiates the scheme the forward
// kernels implement (WENO5-JS or first order, global Lax-Friedrichs
// splitting with alpha = max|f'|, SSPRK3 or forward Euler; split numerical
// flux only).  One VJP step:
//   forward: recompute the SSPRK3 stage states u1, u2 from u;
//   backward through Eq. (SSPRK3) stage by stage, each stage needing
//   mu -> A'(w)^T mu at its stage state w:
//     muF_i  = (mu_{i+1} - mu_i) / dx              (Eq. spaceDisc, F_i = F_{i+1/2})
//     mu_f+  = sum over interfaces of muF_i dW/dq  (left-biased stencils of f+)
//     mu_f-  = the same over the mirrored stencils of f-
//     out_j += mu_f+_j (f'(w_j) + alpha)/2 + mu_f-_j (f'(w_j) - alpha)/2
//     out_k* += sign(w_k*) sum_j w_j (mu_f+_j - mu_f-_j)/2   (k* = first maximiser of |f'|)
// The scatter from interfaces to cells is done as a gather over five shared
// arrays (one per stencil position), so every sum has a fixed order and the
// result is reproducible bit for bit.
//
// Adjoint MGRIT in reversed time k = N - n: v^k = Phi'(u^{N-k})^T v^{k-1},
// v^0 = lam^N.  The propagator of the step ending at point i of level l is
// the transposed linearisation of Phi_l (step dt_l) at the forward fine
// state of index N - i s_l, s_l = m^l: the fine states for level 0 and the
// injected forward C-states for the coarse levels.  The relaxation,
// interpolation and coarsest kernels below have the structure of the
// forward ones (kernels.cuh) with that propagator; the FAS residual and
// restriction kernel is shared (it only combines rows).
#pragma once
#include "kernels.cuh"

namespace mgrit {

// d W / d(a..e) of weno5_left(a..e):
//   W = sum_r w_r p_r, w_r = alpha_r / sum alpha, alpha_r = d_r / s_r^2, s_r = eps + beta_r
//   dW = sum_r w_r dp_r + sum_r (p_r - W) dalpha_r / sum alpha,
//   dalpha_r = -2 alpha_r / s_r dbeta_r,
//   beta_r = 13/12 x_r^2 + 1/4 y_r^2  ->  dbeta_r = 13/6 x_r dx_r + 1/2 y_r dy_r.
// Two divisions: 1/s_r = (product of the other two s) / (s_0 s_1 s_2), and
// 1 / sum alpha (each s_r >= eps = 1e-6, so the product stays normal).
template <typename R>
__device__ __forceinline__ void weno5_left_grad(R a, R b, R c, R d, R e, R (&g)[5])
{
    const R eps = R(1e-6);
    const R sixth = R(1.0 / 6.0);
    const R p0 = (R(2) * a - R(7) * b + R(11) * c) * sixth;   // stencil {i-2, i-1, i}, d = 1/10
    const R p1 = (-b + R(5) * c + R(2) * d) * sixth;         // stencil {i-1, i, i+1}, d = 6/10
    const R p2 = (R(2) * c + R(5) * d - e) * sixth;          // stencil {i, i+1, i+2}, d = 3/10
    const R x0 = a - R(2) * b + c, y0 = a - R(4) * b + R(3) * c;
    const R x1 = b - R(2) * c + d, y1 = b - d;
    const R x2 = c - R(2) * d + e, y2 = R(3) * c - R(4) * d + e;
    const R s0 = eps + R(13.0 / 12.0) * x0 * x0 + R(0.25) * y0 * y0;
    const R s1 = eps + R(13.0 / 12.0) * x1 * x1 + R(0.25) * y1 * y1;
    const R s2 = eps + R(13.0 / 12.0) * x2 * x2 + R(0.25) * y2 * y2;
    // With P_r the product of the two other s and S = s0 s1 s2, the weights
    // are w_r = d_r P_r^2 / Q with Q = sum_r d_r P_r^2, and 1/s_r = P_r / S:
    // both quotients come from one reciprocal X = 1 / (Q S) (1/Q = S X,
    // 1/S = Q X).  Q S ~ s^7 stays inside the FP64 range for s <= 1e40.
    const R P0 = s1 * s2, P1 = s0 * s2, P2 = s0 * s1;
    const R S = s0 * P0;
    const R t0 = R(0.1) * P0 * P0, t1 = R(0.6) * P1 * P1, t2 = R(0.3) * P2 * P2;
    const R Q = t0 + t1 + t2;
    const R X = R(1) / (Q * S);
    const R iQ = S * X, iS = Q * X;
    const R r0 = P0 * iS, r1 = P1 * iS, r2 = P2 * iS;   // 1 / s_r
    const R w0 = t0 * iQ, w1 = t1 * iQ, w2 = t2 * iQ;
    const R W = w0 * p0 + w1 * p1 + w2 * p2;
    // (p_r - W) (dalpha_r / dbeta_r) / sum alpha = (p_r - W) (-2 w_r / s_r)
    const R k0 = (p0 - W) * (R(-2) * w0 * r0);
    const R k1 = (p1 - W) * (R(-2) * w1 * r1);
    const R k2 = (p2 - W) * (R(-2) * w2 * r2);
    // dbeta_r/dq = 13/6 x_r dx_r/dq + 1/2 y_r dy_r/dq with
    //   x0: (1,-2,1,0,0)  y0: (1,-4,3,0,0)
    //   x1: (0,1,-2,1,0)  y1: (0,1,0,-1,0)
    //   x2: (0,0,1,-2,1)  y2: (0,0,3,-4,1)
    const R bx0 = R(13.0 / 6.0) * x0, by0 = R(0.5) * y0;
    const R bx1 = R(13.0 / 6.0) * x1, by1 = R(0.5) * y1;
    const R bx2 = R(13.0 / 6.0) * x2, by2 = R(0.5) * y2;
    g[0] = w0 * R(2.0 / 6.0) + k0 * (bx0 + by0);
    g[1] = w0 * R(-7.0 / 6.0) + w1 * R(-1.0 / 6.0) + k0 * (R(-2) * bx0 - R(4) * by0) +
           k1 * (bx1 + by1);
    g[2] = w0 * R(11.0 / 6.0) + w1 * R(5.0 / 6.0) + w2 * R(2.0 / 6.0) +
           k0 * (bx0 + R(3) * by0) + k1 * (R(-2) * bx1) + k2 * (bx2 + R(3) * by2);
    g[3] = w1 * R(2.0 / 6.0) + w2 * R(5.0 / 6.0) + k1 * (bx1 - by1) +
           k2 * (R(-2) * bx2 - R(4) * by2);
    g[4] = w2 * R(-1.0 / 6.0) + k2 * (bx2 + by2);
}

// Shared memory of one adjoint slab (units of R, then NWARP_MAX ints):
//   [0, nx+6)            qa   (forward slab: f+ / the split flux being differentiated)
//   [nx+6, 6nx+6)        cg   5 x nx interface contributions, overlapping the
//                             forward slab's qb, qf and red (not live together)
//   [6nx+6, 7nx+8)       mu   the cotangent with one periodic ghost each side
//   [7nx+8, 7nx+40)      sred block-sum / argmax partials
//   then NWARP_MAX ints  ired argmax indices
template <typename R>
inline size_t adj_smem_bytes(int nx)
{
    return sizeof(R) * (7 * (size_t)nx + 8 + NWARP_MAX) + sizeof(int) * NWARP_MAX;
}

template <typename R, int SCHEME, int FLUX, int CPT>
struct AdjSlab {
    Slab<R, SCHEME, FLUX, CPT, true> F;   // forward stage recomputation (flat layout)
    R *cg, *mu, *sred;
    int *ired;
    int nx;
    R dxinv;
    static constexpr int kCpt = CPT;

    __device__ __forceinline__ AdjSlab(unsigned char *smem, int nx_, R dxinv_)
        : F(smem, nx_, dxinv_, NF_SPLIT), nx(nx_), dxinv(dxinv_)
    {
        R *base = reinterpret_cast<R *>(smem);
        cg = base + (nx + 2 * GHOST);
        mu = base + (6 * nx + 2 * GHOST);
        sred = base + (7 * nx + 8);
        ired = reinterpret_cast<int *>(sred + NWARP_MAX);
    }

    __device__ __forceinline__ int cell(int c) const { return threadIdx.x + c * blockDim.x; }
    __device__ __forceinline__ int wrap(int i) const { return i < 0 ? i + nx : (i >= nx ? i - nx : i); }
    __device__ __forceinline__ R &CG(int p, int i) const { return MGRIT_SH(cg, p * nx + i, 5 * nx); }
    __device__ __forceinline__ R &MU(int i) const { return MGRIT_SH(mu, i, nx + 2); }

    // block-wide sum in a fixed order (warp tree, then the warps in order)
    __device__ __forceinline__ R block_sum(R v)
    {
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) MGRIT_SH(sred, threadIdx.x >> 5, NWARP_MAX) = v;
        __syncthreads();
        R s = R(0);
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += MGRIT_SH(sred, k, NWARP_MAX);
        return s;
    }

    // alpha = max_j |f'(w_j)| and its first maximiser; contains one barrier
    __device__ __forceinline__ R alpha_argmax(const R (&w)[CPT], int &kstar)
    {
        R v = R(-1);
        int idx = 0x7fffffff;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            if (i < nx) {
                const R s = phys_speed<FLUX>(w[c]);
                if (s > v) { v = s; idx = i; }   // cells of a thread ascend with c
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const R ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if ((threadIdx.x & 31) == 0) {
            MGRIT_SH(sred, threadIdx.x >> 5, NWARP_MAX) = v;
            MGRIT_SH(ired, threadIdx.x >> 5, NWARP_MAX) = idx;
        }
        __syncthreads();
        R best = sred[0];
        int bi = ired[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            const R ov = MGRIT_SH(sred, k, NWARP_MAX);
            const int oi = MGRIT_SH(ired, k, NWARP_MAX);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        kstar = bi;
        return best;
    }

    // out += A'(w)^T (scale m) for the owned cells.  m and out may be the
    // same array: m is read into shared memory before out is written.
    __device__ __forceinline__ void adjA(const R (&w)[CPT], const R (&m)[CPT], R scale, R (&out)[CPT])
    {
        __syncthreads();   // earlier readers of the shared arrays are done
        int kstar = -1;
        R alpha = R(1);
        if (FLUX == FLX_BURGERS) alpha = alpha_argmax(w, kstar);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int i = cell(c);
            if (i < nx) {
                const R v = scale * m[c];
                MU(i + 1) = v;
                if (i == nx - 1) MU(0) = v;
                if (i == 0) MU(nx + 1) = v;
                if (SCHEME != SCH_FO_FE) F.put(F.qa, i, R(0.5) * (phys_flux<FLUX>(w[c]) + alpha * w[c]));
            }
        }
        __syncthreads();
        R loc = R(0);
        if (SCHEME == SCH_FO_FE) {
            // F_i = f+_i + f-_{i+1}: mu_f+_j = muF_j, mu_f-_j = muF_{j-1}
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < nx) {
                    const R fprime = FLUX == FLX_BURGERS ? w[c] : R(1);
                    const R mp = (MU(j + 2) - MU(j + 1)) * dxinv;
                    const R mm = (MU(j + 1) - MU(j)) * dxinv;
                    out[c] += mp * R(0.5) * (fprime + alpha) + mm * R(0.5) * (fprime - alpha);
                    loc += R(0.5) * w[c] * (mp - mm);
                }
            }
        } else {
            // f+: interface i reads f+_{i-2..i+2}; position p is cell i-2+p
#pragma unroll(1)
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const R muF = (MU(i + 2) - MU(i + 1)) * dxinv;
                    const int s = i + GHOST;
                    const int L = F.lim();
                    R g[5];
                    weno5_left_grad<R>(MGRIT_SH(F.qa, s - 2, L), MGRIT_SH(F.qa, s - 1, L),
                                       MGRIT_SH(F.qa, s, L), MGRIT_SH(F.qa, s + 1, L),
                                       MGRIT_SH(F.qa, s + 2, L), g);
#pragma unroll
                    for (int p = 0; p < 5; ++p) CG(p, i) = muF * g[p];
                }
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < nx) {
                    R acc = R(0);
#pragma unroll
                    for (int p = 0; p < 5; ++p) acc += CG(p, wrap(j + 2 - p));
                    const R fprime = FLUX == FLX_BURGERS ? w[c] : R(1);
                    out[c] += acc * R(0.5) * (fprime + alpha);
                    loc += R(0.5) * w[c] * acc;
                }
            }
            __syncthreads();
            // f-: interface i reads (f-_{i+3}, f-_{i+2}, f-_{i+1}, f-_i, f-_{i-1});
            // position p is cell i+3-p
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) F.put(F.qa, i, R(0.5) * (phys_flux<FLUX>(w[c]) - alpha * w[c]));
            }
            __syncthreads();
#pragma unroll(1)
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < nx) {
                    const R muF = (MU(i + 2) - MU(i + 1)) * dxinv;
                    const int s = i + GHOST;
                    const int L = F.lim();
                    R g[5];
                    weno5_left_grad<R>(MGRIT_SH(F.qa, s + 3, L), MGRIT_SH(F.qa, s + 2, L),
                                       MGRIT_SH(F.qa, s + 1, L), MGRIT_SH(F.qa, s, L),
                                       MGRIT_SH(F.qa, s - 1, L), g);
#pragma unroll
                    for (int p = 0; p < 5; ++p) CG(p, i) = muF * g[p];
                }
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < nx) {
                    R acc = R(0);
#pragma unroll
                    for (int p = 0; p < 5; ++p) acc += CG(p, wrap(j - 3 + p));
                    const R fprime = FLUX == FLX_BURGERS ? w[c] : R(1);
                    out[c] += acc * R(0.5) * (fprime - alpha);
                    loc -= R(0.5) * w[c] * acc;
                }
            }
        }
        if (FLUX == FLX_BURGERS) {
            const R mualpha = block_sum(loc);   // every thread takes part (one barrier)
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (cell(c) == kstar && w[c] != R(0)) out[c] += w[c] > R(0) ? mualpha : -mualpha;
        }
    }

    // lam <- Phi'(u)^T lam for one step dt at the forward state in row urow.
    // st: one global row of scratch (the stage state u1, own cells only).
    __device__ __noinline__ void vjp(const R *__restrict__ urow, R *__restrict__ st,
                                        R (&lam)[CPT], R dt)
    {
        R v[CPT], out[CPT];
        F.load(v, urow);
        if (SCHEME == SCH_FO_FE) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) out[c] = lam[c];
            adjA(v, lam, dt, out);
#pragma unroll
            for (int c = 0; c < CPT; ++c) lam[c] = out[c];
            return;
        }
        // forward stages of Eq. (SSPRK3): u1 = u + dt A(u) (kept in st),
        // u2 = 3/4 u + 1/4 u1 + 1/4 dt A(u1) (kept in v)
        {
            R w[CPT];
            const typename RK<R>::Coef K = F.coef(dt);
            F.fluxes(v);
#pragma unroll
            for (int c = 0; c < CPT; ++c) w[c] = (cell(c) < nx) ? RK<R>::euler(v[c], K, F.df(c)) : R(0);
            F.store(w, st);
            F.fluxes(w);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                v[c] = (cell(c) < nx) ? RK<R>::stage2(v[c], w[c], K, F.df(c)) : R(0);
        }
        // stage 3: out = 1/3 u + 2/3 u2 + 2/3 dt A(u2)
        //   lam_u += 1/3 lam;  l2 = 2/3 lam + A'(u2)^T (dt l2_0), l2_0 = 2/3 lam
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            out[c] = R(1.0 / 3.0) * lam[c];
            lam[c] = R(2.0 / 3.0) * lam[c];
        }
        adjA(v, lam, dt, lam);
        // stage 2: u2 = 3/4 u + 1/4 u1 + 1/4 dt A(u1)
        //   lam_u += 3/4 l2;  l1 = 1/4 l2 + A'(u1)^T (dt l1_0), l1_0 = 1/4 l2
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            out[c] += R(0.75) * lam[c];
            lam[c] = R(0.25) * lam[c];
        }
        F.load(v, st);
        adjA(v, lam, dt, lam);
        // stage 1: u1 = u + dt A(u):  lam_u += l1 + A'(u)^T (dt l1)
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[c] += lam[c];
        F.load(v, urow);
        adjA(v, lam, dt, out);
#pragma unroll
        for (int c = 0; c < CPT; ++c) lam[c] = out[c];
    }
};

enum { ADJ_RELAX = 0, ADJ_INTERP = 1, ADJ_SEQ = 2, ADJ_TRAJ = 3, ADJ_VJP = 4, ADJ_SERIAL = 5 };

struct AdjArgs {
    int mode;
    int nx, m, nC, fcf, nsteps;
    double dxinv, dt, dtc;
    long long N;            // fine steps
    long long s, sc;        // fine steps per step of this level and of the next coarser level
    const double *traj;     // forward fine states, rows 0..N-1
    // ADJ_RELAX: as SlabArgs (C-point sources uC, newC, phirow, cstep, g)
    const double *uC;
    long long strideC;
    double *newC, *phirow, *cstep;
    const double *g;
    // ADJ_SEQ: start src, rows 1..nsteps into rows; ADJ_INTERP: fine rows into rows;
    // ADJ_TRAJ: forward C-points uC -> rows (the trajectory); ADJ_VJP: out = Phi'(src)^T uC;
    // ADJ_SERIAL: forward from src with checkpoints into rows, lam^N = uC, lam^0 -> out
    const double *src;
    double *rows;
    double *out;
    double *scratch;        // per CTA: 1 row (stage state); ADJ_SERIAL: 1 + m rows
    long long nrows_uC, nrows_newC, nrows_phirow, nrows_cstep, nrows_g, nrows_rows, nrows_traj;
};

// forward state at which the step ending at point i (stride s) is linearised
__device__ __forceinline__ const double *adj_fwd(const AdjArgs &a, long long i, long long s)
{
    return rowp(a.traj, a.N - i * s, a.nx, a.nrows_traj);
}

// adj_relax_chunk and adj_interp_chunk take any adjoint slab
// with S.F.load/store/add/step, S.vjp and the constant kCpt: the one-CTA
// AdjSlab, or one spread over a thread-block cluster (cluster_adjoint.cuh)
template <typename SL>
__device__ __forceinline__ void adj_relax_chunk(SL &S, const AdjArgs &a, const int j, double *st)
{
    constexpr int CPT = SL::kCpt;
    // CTA j = 0..nC, as relax_chunk: FCF recomputes C_j from the old
    // C_{j-1}; then the F-relaxation of chunk j, the coarse step of the FAS
    // term from the new C_j, and the fine step into the next C-point.
    const int nx = a.nx, m = a.m;
    double v[CPT];
    if (j == 0 || !a.fcf) {
        S.F.load(v, rowp(a.uC, j, (int)a.strideC, a.nrows_uC));
    } else {
        S.F.load(v, rowp(a.uC, j - 1, (int)a.strideC, a.nrows_uC));
        for (int r = 1; r <= m; ++r) {
            const long long i = (long long)m * (j - 1) + r;
            S.vjp(adj_fwd(a, i, a.s), st, v, a.dt);
            if (a.g) S.F.add(v, rowp(a.g, i, nx, a.nrows_g));
        }
    }
    if (a.newC) S.F.store(v, rowp(a.newC, j, nx, a.nrows_newC));
    if (j == a.nC) return;
    if (a.cstep) {
        S.vjp(adj_fwd(a, j + 1, a.sc), st, v, a.dtc);
        S.F.store(v, rowp(a.cstep, j, nx, a.nrows_cstep));
        S.F.load(v, rowp(a.newC, j, nx, a.nrows_newC));
    }
    for (int r = 1; r < m; ++r) {
        const long long i = (long long)m * j + r;
        S.vjp(adj_fwd(a, i, a.s), st, v, a.dt);
        if (a.g) S.F.add(v, rowp(a.g, i, nx, a.nrows_g));
    }
    S.vjp(adj_fwd(a, (long long)m * (j + 1), a.s), st, v, a.dt);
    S.F.store(v, rowp(a.phirow, j + 1, nx, a.nrows_phirow));
}

template <typename SL>
__device__ __forceinline__ void adj_interp_chunk(SL &S, const AdjArgs &a, const int j, double *st)
{
    constexpr int CPT = SL::kCpt;
    const int nx = a.nx, m = a.m;
    double v[CPT];
    S.F.load(v, rowp(a.uC, j, nx, a.nrows_uC));
    S.F.store(v, rowp(a.rows, (long long)m * j, nx, a.nrows_rows));
    for (int r = 1; r < m; ++r) {
        const long long i = (long long)m * j + r;
        S.vjp(adj_fwd(a, i, a.s), st, v, a.dt);
        S.F.add(v, rowp(a.g, i, nx, a.nrows_g));
        S.F.store(v, rowp(a.rows, i, nx, a.nrows_rows));
    }
    if (j == a.nC - 1) {
        S.F.load(v, rowp(a.uC, a.nC, nx, a.nrows_uC));
        S.F.store(v, rowp(a.rows, (long long)m * a.nC, nx, a.nrows_rows));
    }
}

template <int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_adjoint(AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    AdjSlab<double, SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv);
    const int nx = a.nx;
    double *st = a.scratch ? a.scratch + (long long)blockIdx.x * nx : nullptr;
    double v[CPT];
    switch (a.mode) {
    case ADJ_RELAX:
        adj_relax_chunk(S, a, (int)blockIdx.x, st);
        break;
    case ADJ_INTERP:
        adj_interp_chunk(S, a, (int)blockIdx.x, st);
        break;
    case ADJ_SEQ:
        // coarsest level: v^i = Phi'(U_i)^T v^{i-1} + g^i, i = 1..nsteps
        S.F.load(v, a.src);
        for (int i = 1; i <= a.nsteps; ++i) {
            S.vjp(adj_fwd(a, i, a.s), st, v, a.dt);
            S.F.add(v, rowp(a.g, i, nx, a.nrows_g));
            S.F.store(v, rowp(a.rows, i, nx, a.nrows_rows));
        }
        break;
    case ADJ_TRAJ: {
        // forward fine states of chunk j from its C-point: u^{mj+r} = Phi^r(uC_j)
        const int j = (int)blockIdx.x;
        S.F.load(v, rowp(a.uC, j, nx, a.nrows_uC));
        S.F.store(v, rowp(a.rows, (long long)a.m * j, nx, a.nrows_traj));
        for (int r = 1; r < a.m; ++r) {
            S.F.step(v, a.dt);
            S.F.store(v, rowp(a.rows, (long long)a.m * j + r, nx, a.nrows_traj));
        }
        break;
    }
    case ADJ_VJP:
        S.F.load(v, a.uC);
        S.vjp(a.src, st, v, a.dt);
        S.F.store(v, a.out);
        break;
    case ADJ_SERIAL: {
        // serial adjoint with C-point checkpointing: forward nsteps = nC m
        // steps keeping u^{mj} (rows j = 0..nC-1), then chunk by chunk from
        // the last: recompute the chunk's m states from its checkpoint into
        // scratch rows 1..m, and apply their m VJPs backward
        double *states = st + nx;
        S.F.load(v, a.src);
        for (int j = 0; j < a.nC; ++j) {
            S.F.store(v, rowp(a.rows, j, nx, a.nrows_rows));
            for (int r = 0; r < a.m; ++r) S.F.step(v, a.dt);
        }
        double lam[CPT];
        S.F.load(lam, a.uC);
        for (int j = a.nC - 1; j >= 0; --j) {
            S.F.load(v, rowp(a.rows, j, nx, a.nrows_rows));
            S.F.store(v, states);
            for (int r = 1; r < a.m; ++r) {
                S.F.step(v, a.dt);
                S.F.store(v, states + (long long)r * nx);
            }
            for (int r = a.m - 1; r >= 0; --r) S.vjp(states + (long long)r * nx, st, lam, a.dt);
        }
        S.F.store(lam, a.out);
        break;
    }
    default:
        break;
    }
}

}  // namespace mgrit
