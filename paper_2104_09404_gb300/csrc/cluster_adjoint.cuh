// Transposed steps on a thread-block cluster: the sequential adjoint chains
// (the coarsest adjoint solve and the serial adjoint) spread one slab over K
// CTAs (contiguous blocks of cells), as the forward cluster stepper does.
//
// One transposed stage mu -> A'(w)^T mu (see adjoint.cuh for the algebra):
//   S0  alpha = max|f'(w)| and its first maximiser: per-CTA (value, index),
//       cluster barrier, every CTA reduces the K partials in rank order
//       (Burgers only; alpha = 1 for advection)
//   S1  f+, f- and mu of the own cells; cluster barrier; 3 ghost cells of
//       f+/- and 1 of mu on each side read from the neighbours (DSMEM)
//   S2  the five gradient contributions of every own interface for f+ and
//       f-; cluster barrier; each cell gathers its entries, the ones of the
//       two (f+) or three/one (f-) interfaces beyond the block edge from the
//       neighbours' shared memory
//   S3  the alpha term: per-CTA partial of sum w (mu_f+ - mu_f-)/2, cluster
//       barrier, sum of the K partials in rank order (Burgers only)
// Every array a neighbour reads is written again only after a later cluster
// barrier of the same stage sequence, and all CTAs run the same control
// flow, so the barriers always match.
#pragma once
#include "adjoint.cuh"
#include "cluster_seq.cuh"

namespace mgrit {

template <int SCHEME, int FLUX, int CPT>
struct ClusterAdj {
    using R = double;
    ClusterSlab<R, SCHEME, FLUX, CPT> F;   // forward stage recomputation
    R *fp, *fm;   // nmax + 6: f+ / f- of the own cells at local + GHOST, 3 ghosts per side
    R *mu;        // nmax + 2: mu of local cell j at j + 1, one ghost per side
    R *cgp, *cgm; // 5 x nmax: interface contributions (f+, f-)
    R *pv, *ps, *bcv, *bcs, *sred;
    int *pi, *bci, *ired;

    __device__ __forceinline__ ClusterAdj(unsigned char *smem, int nx, R dxinv, size_t fwd_bytes)
        : F(smem, nx, dxinv, NF_SPLIT)
    {
        const int nm = F.nmax;
        R *b = reinterpret_cast<R *>(smem + fwd_bytes);
        fp = b;
        fm = fp + (nm + 2 * GHOST);
        mu = fm + (nm + 2 * GHOST);
        cgp = mu + (nm + 2);
        cgm = cgp + 5 * nm;
        pv = cgm + 5 * nm;
        ps = pv + 1;
        bcv = ps + 1;
        bcs = bcv + 1;
        sred = bcs + 1;
        pi = reinterpret_cast<int *>(sred + NWARP_MAX);
        bci = pi + 1;
        ired = bci + 1;
    }

    __device__ __forceinline__ int cell(int c) const { return threadIdx.x + c * blockDim.x; }
    __device__ __forceinline__ int nloc(int r) const
    {
        return (int)((long long)(r + 1) * F.nx / F.K) - (int)((long long)r * F.nx / F.K);
    }
    __device__ __forceinline__ int lim() const { return F.nmax + 2 * GHOST; }

    // contribution p of interface i (local index, -3 <= i <= n) from array base
    // (cgp or cgm), from this CTA or a neighbour
    __device__ __forceinline__ R cg_at(R *base, int p, int i)
    {
        const int n = F.n, nm = F.nmax;
        if (i >= 0 && i < n) return MGRIT_SH(base, p * nm + i, 5 * nm);
        if (i < 0) {
            const int left = (F.rank + F.K - 1) % F.K;
            const R *src = F.cl.map_shared_rank(base, (unsigned)left);
            return MGRIT_SH(src, p * nm + nloc(left) + i, 5 * nm);
        }
        const int right = (F.rank + 1) % F.K;
        const R *src = F.cl.map_shared_rank(base, (unsigned)right);
        return MGRIT_SH(src, p * nm + (i - n), 5 * nm);
    }

    // out += A'(w)^T (scale m) for the own cells (m and out may alias)
    __device__ __forceinline__ void adjA(const R (&w)[CPT], const R (&m)[CPT], R scale, R (&out)[CPT])
    {
        const int n = F.n, lo = F.lo, K = F.K;
        const R dxinv = F.dxinv;
        R alpha = R(1);
        int kstar = -1;
        __syncthreads();   // this CTA's earlier readers of the shared arrays are done
        if (FLUX == FLX_BURGERS) {
            // S0: first maximiser of |f'| over the cluster
            R v = R(-1);
            int idx = 0x7fffffff;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < n) {
                    const R s = phys_speed<FLUX>(w[c]);
                    if (s > v) { v = s; idx = lo + j; }
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
            if (threadIdx.x == 0) {
                R best = sred[0];
                int bi = ired[0];
                for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                    const R ov = MGRIT_SH(sred, k, NWARP_MAX);
                    const int oi = MGRIT_SH(ired, k, NWARP_MAX);
                    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                }
                *pv = best;
                *pi = bi;
            }
            F.cl.sync();
            if (threadIdx.x == 0) {
                R best = R(-1);
                int bi = 0x7fffffff;
                for (int r = 0; r < K; ++r) {
                    const R ov = *F.cl.map_shared_rank(pv, (unsigned)r);
                    const int oi = *F.cl.map_shared_rank(pi, (unsigned)r);
                    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                }
                *bcv = best;
                *bci = bi;
            }
            __syncthreads();
            alpha = *bcv;
            kstar = *bci;
        }
        // S1: f+/- and mu of the own cells, then the ghosts
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int j = cell(c);
            if (j < n) {
                const R f = phys_flux<FLUX>(w[c]);
                MGRIT_SH(fp, j + GHOST, lim()) = R(0.5) * (f + alpha * w[c]);
                MGRIT_SH(fm, j + GHOST, lim()) = R(0.5) * (f - alpha * w[c]);
                MGRIT_SH(mu, j + 1, F.nmax + 2) = scale * m[c];
            }
        }
        F.cl.sync();
        {
            const int t = threadIdx.x;
            const int left = (F.rank + K - 1) % K, right = (F.rank + 1) % K;
            const int nl = nloc(left);
            if (t < 12) {
                R *arr = t < 6 ? fp : fm;
                const int k = t % 6;
                if (k < GHOST) {   // slot k <- left neighbour's local cell nl - 3 + k
                    const R *src = F.cl.map_shared_rank(arr, (unsigned)left);
                    MGRIT_SH(arr, k, lim()) = MGRIT_SH(src, nl - GHOST + k + GHOST, lim());
                } else {           // slot n + k <- right neighbour's local cell k - 3
                    const R *src = F.cl.map_shared_rank(arr, (unsigned)right);
                    MGRIT_SH(arr, n + k, lim()) = MGRIT_SH(src, k - GHOST + GHOST, lim());
                }
            } else if (t == 12) {
                const R *src = F.cl.map_shared_rank(mu, (unsigned)left);
                mu[0] = MGRIT_SH(src, nl, F.nmax + 2);
            } else if (t == 13) {
                const R *src = F.cl.map_shared_rank(mu, (unsigned)right);
                MGRIT_SH(mu, n + 1, F.nmax + 2) = src[1];
            }
        }
        __syncthreads();
        R loc = R(0);
        if (SCHEME == SCH_FO_FE) {
            // F_i = f+_i + f-_{i+1}: mu_f+_j = muF_j, mu_f-_j = muF_{j-1}
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < n) {
                    const R fprime = FLUX == FLX_BURGERS ? w[c] : R(1);
                    const R mp = (MGRIT_SH(mu, j + 2, F.nmax + 2) - MGRIT_SH(mu, j + 1, F.nmax + 2)) * dxinv;
                    const R mm = (MGRIT_SH(mu, j + 1, F.nmax + 2) - MGRIT_SH(mu, j, F.nmax + 2)) * dxinv;
                    out[c] += mp * R(0.5) * (fprime + alpha) + mm * R(0.5) * (fprime - alpha);
                    loc += R(0.5) * w[c] * (mp - mm);
                }
            }
        } else {
            // S2: contributions of the own interfaces i (between local cells i, i+1)
            const int nm = F.nmax;
#pragma unroll(1)
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) {
                    const R muF = (MGRIT_SH(mu, i + 2, nm + 2) - MGRIT_SH(mu, i + 1, nm + 2)) * dxinv;
                    const int s = i + GHOST, L = lim();
                    R g[5];
                    weno5_left_grad<R>(MGRIT_SH(fp, s - 2, L), MGRIT_SH(fp, s - 1, L), MGRIT_SH(fp, s, L),
                                       MGRIT_SH(fp, s + 1, L), MGRIT_SH(fp, s + 2, L), g);
#pragma unroll
                    for (int p = 0; p < 5; ++p) MGRIT_SH(cgp, p * nm + i, 5 * nm) = muF * g[p];
                    weno5_left_grad<R>(MGRIT_SH(fm, s + 3, L), MGRIT_SH(fm, s + 2, L), MGRIT_SH(fm, s + 1, L),
                                       MGRIT_SH(fm, s, L), MGRIT_SH(fm, s - 1, L), g);
#pragma unroll
                    for (int p = 0; p < 5; ++p) MGRIT_SH(cgm, p * nm + i, 5 * nm) = muF * g[p];
                }
            }
            F.cl.sync();
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = cell(c);
                if (j < n) {
                    R ap = R(0), am = R(0);
#pragma unroll
                    for (int p = 0; p < 5; ++p) ap += cg_at(cgp, p, j + 2 - p);
#pragma unroll
                    for (int p = 0; p < 5; ++p) am += cg_at(cgm, p, j - 3 + p);
                    const R fprime = FLUX == FLX_BURGERS ? w[c] : R(1);
                    out[c] += ap * R(0.5) * (fprime + alpha);
                    loc += R(0.5) * w[c] * ap;
                    out[c] += am * R(0.5) * (fprime - alpha);
                    loc -= R(0.5) * w[c] * am;
                }
            }
        }
        if (FLUX == FLX_BURGERS) {
            // S3: mu_alpha = sum over the cluster, partials added in rank order
#pragma unroll
            for (int o = 16; o; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
            if ((threadIdx.x & 31) == 0) MGRIT_SH(sred, threadIdx.x >> 5, NWARP_MAX) = loc;
            __syncthreads();
            if (threadIdx.x == 0) {
                R sacc = R(0);
                for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sacc += MGRIT_SH(sred, k, NWARP_MAX);
                *ps = sacc;
            }
            F.cl.sync();
            if (threadIdx.x == 0) {
                R tot = R(0);
                for (int r = 0; r < K; ++r) tot += *F.cl.map_shared_rank(ps, (unsigned)r);
                *bcs = tot;
            }
            __syncthreads();
            const R mualpha = *bcs;
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (lo + cell(c) == kstar && cell(c) < n && w[c] != R(0))
                    out[c] += w[c] > R(0) ? mualpha : -mualpha;
        }
        // neighbours read this CTA's f+/- and mu ghosts after S1; S2 (WENO) or
        // S3 (Burgers) separates those reads from the next stage's writes, and
        // first-order advection, which has neither, takes one barrier here
        if (SCHEME == SCH_FO_FE && FLUX != FLX_BURGERS) F.cl.sync();
    }

    // lam <- Phi'(u)^T lam at the forward state in row urow (st: stage-state row)
    __device__ __forceinline__ void vjp(const R *__restrict__ urow, R *__restrict__ st, R (&lam)[CPT],
                                        R dt, int &stage)
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
        {
            R w[CPT];
            const typename RK<R>::Coef K = F.coef(dt);
            F.fluxes(v, (stage++) & 1);
#pragma unroll
            for (int c = 0; c < CPT; ++c) w[c] = (cell(c) < F.n) ? RK<R>::euler(v[c], K, F.df(c)) : R(0);
            F.store(w, st);
            F.fluxes(w, (stage++) & 1);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                v[c] = (cell(c) < F.n) ? RK<R>::stage2(v[c], w[c], K, F.df(c)) : R(0);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            out[c] = R(1.0 / 3.0) * lam[c];
            lam[c] = R(2.0 / 3.0) * lam[c];
        }
        adjA(v, lam, dt, lam);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            out[c] += R(0.75) * lam[c];
            lam[c] = R(0.25) * lam[c];
        }
        F.load(v, st);
        adjA(v, lam, dt, lam);
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[c] += lam[c];
        F.load(v, urow);
        adjA(v, lam, dt, out);
#pragma unroll
        for (int c = 0; c < CPT; ++c) lam[c] = out[c];
    }
};

template <typename R>
inline size_t cluster_adj_extra_bytes(int nx, int K)
{
    const size_t nm = (size_t)((nx + K - 1) / K);
    return sizeof(R) * (2 * (nm + 2 * GHOST) + (nm + 2) + 10 * nm + 4 + NWARP_MAX) +
           sizeof(int) * (2 + NWARP_MAX);
}

// ADJ_SEQ / ADJ_SERIAL on one cluster (grid = one cluster of K CTAs); the
// forward stepper's part of the shared memory (cluster_smem_bytes<double>(nx,
// K) bytes) comes first, the adjoint arrays after it
template <int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_adjoint_cluster(AdjArgs a, unsigned long long fwd_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ClusterAdj<SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv, (size_t)fwd_bytes);
    const int nx = a.nx;
    double *st = a.scratch;
    double v[CPT];
    int stage = 0;
    if (a.mode == ADJ_SEQ) {
        S.F.load(v, a.src);
        for (int i = 1; i <= a.nsteps; ++i) {
            S.vjp(adj_fwd(a, i, a.s), st, v, a.dt, stage);
            S.F.add(v, rowp(a.g, i, nx, a.nrows_g));
            S.F.store(v, rowp(a.rows, i, nx, a.nrows_rows));
        }
    } else if (a.mode == ADJ_SERIAL) {
        double *states = st + nx;
        S.F.load(v, a.src);
        for (int j = 0; j < a.nC; ++j) {
            S.F.store(v, rowp(a.rows, j, nx, a.nrows_rows));
            for (int r = 0; r < a.m; ++r) S.F.step(v, a.dt, stage);
        }
        double lam[CPT];
        S.F.load(lam, a.uC);
        for (int j = a.nC - 1; j >= 0; --j) {
            S.F.load(v, rowp(a.rows, j, nx, a.nrows_rows));
            S.F.store(v, states);
            for (int r = 1; r < a.m; ++r) {
                S.F.step(v, a.dt, stage);
                S.F.store(v, states + (long long)r * nx);
            }
            for (int r = a.m - 1; r >= 0; --r) S.vjp(states + (long long)r * nx, st, lam, a.dt, stage);
        }
        S.F.store(lam, a.out);
    }
    S.F.cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

// ClusterAdj with its own stage counter, in the interface adj_relax_chunk,
// adj_interp_chunk and adj_traj_chunk expect.  The transposed step is one
// out-of-line function, as in the one-CTA kernel: inlined at every call site
// of the chunk functions it would multiply the compile time.
template <int SCHEME, int FLUX, int CPT>
struct ClusterAdjChunk {
    static constexpr int kCpt = CPT;
    struct Fwd {
        ClusterSlab<double, SCHEME, FLUX, CPT> &C;
        int &stage;
        __device__ __forceinline__ void load(double (&u)[CPT], const double *row) const { C.load(u, row); }
        __device__ __forceinline__ void store(const double (&u)[CPT], double *row) const { C.store(u, row); }
        __device__ __forceinline__ void add(double (&u)[CPT], const double *row) const { C.add(u, row); }
        __device__ __forceinline__ void step(double (&u)[CPT], double dt) { C.step(u, dt, stage); }
    };
    ClusterAdj<SCHEME, FLUX, CPT> &A;
    int stage;
    Fwd F;

    __device__ __forceinline__ ClusterAdjChunk(ClusterAdj<SCHEME, FLUX, CPT> &adj)
        : A(adj), stage(0), F{adj.F, stage} {}
    __device__ __noinline__ void vjp(const double *__restrict__ urow, double *__restrict__ st,
                                     double (&lam)[CPT], double dt)
    {
        A.vjp(urow, st, lam, dt, stage);
    }
};

// forward fine states of chunk j from its C-point, u^{mj+r} = Phi^r(uC_j)
// (the ADJ_TRAJ case of k_adjoint)
template <typename SL>
__device__ __forceinline__ void adj_traj_chunk(SL &S, const AdjArgs &a, const int j)
{
    double v[SL::kCpt];
    S.F.load(v, rowp(a.uC, j, a.nx, a.nrows_uC));
    S.F.store(v, rowp(a.rows, (long long)a.m * j, a.nx, a.nrows_traj));
    for (int r = 1; r < a.m; ++r) {
        S.F.step(v, a.dt);
        S.F.store(v, rowp(a.rows, (long long)a.m * j + r, a.nx, a.nrows_traj));
    }
}

// ADJ_RELAX / ADJ_INTERP / ADJ_TRAJ (grid chunks x K) and ADJ_VJP (one
// cluster) with one cluster of K CTAs per chunk: cluster c = blockIdx / K
// takes chunk c, with the one-CTA kernel's chunk logic and one scratch row per
// chunk.  Shared memory as k_adjoint_cluster.  Every CTA of a cluster takes
// the same branches, so all of them reach every cluster barrier.
template <int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_adjoint_cluster_chunk(AdjArgs a, unsigned long long fwd_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ClusterAdj<SCHEME, FLUX, CPT> A(smem, a.nx, a.dxinv, (size_t)fwd_bytes);
    ClusterAdjChunk<SCHEME, FLUX, CPT> S(A);
    const int j = (int)(blockIdx.x / A.F.cl.num_blocks());
    double *st = a.scratch ? a.scratch + (long long)j * a.nx : nullptr;
    switch (a.mode) {
    case ADJ_RELAX:
        adj_relax_chunk(S, a, j, st);
        break;
    case ADJ_INTERP:
        adj_interp_chunk(S, a, j, st);
        break;
    case ADJ_TRAJ:
        adj_traj_chunk(S, a, j);
        break;
    case ADJ_VJP: {
        double v[CPT];
        S.F.load(v, a.uC);
        S.vjp(a.src, st, v, a.dt);
        S.F.store(v, a.out);
        break;
    }
    default:
        break;
    }
    A.F.cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

}  // namespace mgrit
