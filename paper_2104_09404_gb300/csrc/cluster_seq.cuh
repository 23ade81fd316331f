// Sequential time-stepping of one slab spread over a thread-block cluster.
//
// The coarsest-level solve (Eq. coarseCorr) and the serial fine stepper are
// a chain of Phi applications on a single spatial slice, so one CTA would
// leave all but one SM idle.  Here the nx cells are split into K contiguous
// blocks, one per CTA of a cluster (K <= 16).  Every RK stage:
//   1. each CTA reduces max|f'| over its cells and publishes the partial in
//      its shared memory; cluster barrier; every CTA reads the K partials
//      through distributed shared memory (DSMEM) -> the global LF alpha;
//   2. each CTA writes f^+/- (split form) or the stage state (state form, Roe) of
//      its cells; cluster barrier; three ghost cells on each side are read
//      from the neighbouring CTAs' shared memory (periodic: rank 0's left
//      neighbour is rank K-1);
//   3. interface fluxes of the CTA's cells, plus the left boundary interface
//      (recomputed locally instead of fetched, saving a barrier), then the
//      flux difference and the RK combination in registers.
// The exchanged arrays are double-buffered by stage parity, so a CTA never
// overwrites values a neighbour may still be reading: two cluster barriers
// per stage (one for advection, whose alpha is 1).  The state form needs
// alpha after the reconstructions, so its barriers sit after step 3's
// reconstructions instead.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace mgrit {

namespace cg = cooperative_groups;

constexpr int CLUSTER_MAX = 16;

template <typename R, int SCHEME, int FLUX, int CPT>
struct ClusterSlab {
    // shared layout: ex[2][2][n+6] (split: f^+, f^-; state: w, unused), qf[n+2],
    // um[n+1] (state form), part[2] (alpha partials), bcast[1], red[NWARP_MAX]
    R *ex;
    R *qf;
    R *um;
    R *part;
    R *bcast;
    R *red;
    int nx, lo, n, nmax, rank, K, numflux;
    R dxinv;
    cg::cluster_group cl;

    __device__ __forceinline__ ClusterSlab(unsigned char *smem, int nx_, R dxinv_, int numflux_)
        : nx(nx_), numflux(numflux_), dxinv(dxinv_), cl(cg::this_cluster())
    {
        K = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
        lo = (int)((long long)rank * nx / K);
        const int hi = (int)((long long)(rank + 1) * nx / K);
        n = hi - lo;
        nmax = (nx + K - 1) / K;
        ex = reinterpret_cast<R *>(smem);
        qf = ex + 4 * (nmax + 2 * GHOST);
        um = qf + (nmax + 2);
        part = um + (nmax + 1);
        bcast = part + 2;
        red = bcast + 1;
    }

    __device__ __forceinline__ int lim() const { return nmax + 2 * GHOST; }
    __device__ __forceinline__ R *arr(int buf, int which) const
    {
        return ex + (2 * buf + which) * (nmax + 2 * GHOST);
    }
    __device__ __forceinline__ int cell(int c) const { return threadIdx.x + c * blockDim.x; }

    __device__ __forceinline__ R rec_minus(const R *q, int s) const
    {
        if (SCHEME == SCH_FO_FE) return MGRIT_SH(q, s, lim());
        return weno5_left<R>(MGRIT_SH(q, s - 2, lim()), MGRIT_SH(q, s - 1, lim()), MGRIT_SH(q, s, lim()),
                             MGRIT_SH(q, s + 1, lim()), MGRIT_SH(q, s + 2, lim()));
    }
    __device__ __forceinline__ R rec_plus(const R *q, int s) const
    {
        if (SCHEME == SCH_FO_FE) return MGRIT_SH(q, s + 1, lim());
        return weno5_left<R>(MGRIT_SH(q, s + 3, lim()), MGRIT_SH(q, s + 2, lim()), MGRIT_SH(q, s + 1, lim()),
                             MGRIT_SH(q, s, lim()), MGRIT_SH(q, s - 1, lim()));
    }

    // F_{i+1/2} of the split form at local slot s = i + GHOST: the windowed
    // WENO5 expressions of slab.cuh (one window per interface), or first order
    __device__ __forceinline__ R split_flux(const R *fp, const R *fm, int s) const
    {
        if (SCHEME == SCH_FO_FE) return MGRIT_SH(fp, s, lim()) + MGRIT_SH(fm, s + 1, lim());
        const int L = lim();
        WenoWin<R> P;
        P.init(MGRIT_SH(fp, s - 2, L), MGRIT_SH(fp, s - 1, L), MGRIT_SH(fp, s, L), MGRIT_SH(fp, s + 1, L),
               MGRIT_SH(fp, s + 2, L));
        if (FLUX == FLX_ADVECTION) return split_flux_win_adv(P, MGRIT_SH(fp, s, L));
        WenoWin<R> M;
        M.init(MGRIT_SH(fm, s - 1, L), MGRIT_SH(fm, s, L), MGRIT_SH(fm, s + 1, L), MGRIT_SH(fm, s + 2, L),
               MGRIT_SH(fm, s + 3, L));
        return split_flux_win(P, M, MGRIT_SH(fp, s, L), MGRIT_SH(fm, s + 1, L));
    }

    // global max of v over the cluster (publishes this CTA's partial in part[buf])
    __device__ __forceinline__ R cluster_max(R v, int buf)
    {
        v = block_max(v, red);
        if (threadIdx.x == 0) part[buf] = v;
        cl.sync();
        if (threadIdx.x < 32) {
            R x = R(0);
            if ((int)threadIdx.x < K) x = *cl.map_shared_rank(&part[buf], (unsigned)threadIdx.x);
            x = warp_max(x);
            if (threadIdx.x == 0) *bcast = x;
        }
        __syncthreads();
        return *bcast;
    }

    // copy 3 ghost cells on each side of arrays `which` (0, and 1 if both) of
    // buffer buf from the neighbouring CTAs (after a cluster barrier)
    __device__ __forceinline__ void ghosts(int buf, int nwhich)
    {
        const int t = threadIdx.x;
        if (t < 6 * nwhich) {
            const int which = t / 6, k = t % 6;
            R *mine = arr(buf, which);
            const int left = (rank + K - 1) % K, right = (rank + 1) % K;
            const int nl = (int)((long long)(left + 1) * nx / K) - (int)((long long)left * nx / K);
            if (k < GHOST) {   // slot k <- left neighbour's local cell nl - 3 + k
                const R *src = cl.map_shared_rank(arr(buf, which), (unsigned)left);
                mine[k] = src[nl - GHOST + k + GHOST];
            } else {           // slot n + 3 + (k-3) <- right neighbour's local cell k-3
                const R *src = cl.map_shared_rank(arr(buf, which), (unsigned)right);
                mine[n + k] = src[k - GHOST + GHOST];
            }
        }
        __syncthreads();
    }

    // interface fluxes of the stage input w: qf[j+1] = F at the right edge of
    // local cell j, qf[0] = F at the left edge of local cell 0
    __device__ __forceinline__ void fluxes(const R (&w)[CPT], int buf)
    {
        __syncthreads();   // previous readers of qf/um/red are done
        if (numflux == NF_SPLIT) {
            R alpha = R(1);
            if (FLUX == FLX_BURGERS) {
                R v = R(0);
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (cell(c) < n) v = fmax(v, phys_speed<FLUX>(w[c]));
                alpha = cluster_max(v, buf);
            }
            R *fp = arr(buf, 0), *fm = arr(buf, 1);
            // the one-CTA slab's split fluxes, formed the same way: WENO5 on
            // q = f^{+/-}/2 (q^- = 0 for advection), first order on f^{+/-}
            const R a4 = R(0.25) * alpha, h = R(0.5) * alpha;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) {
                    const R x = w[c];
                    R p, q;
                    if (SCHEME == SCH_WENO5_SSPRK3) {
                        if (FLUX == FLX_BURGERS) {
                            burgers_q(x, a4, p, q);
                        } else {
                            p = R(0.5) * x;
                            q = R(0);
                        }
                    } else {
                        const R f2 = R(0.5) * phys_flux<FLUX>(x);
                        p = fma(h, x, f2);
                        q = fma(-h, x, f2);
                    }
                    MGRIT_SH(fp, i + GHOST, lim()) = p;
                    MGRIT_SH(fm, i + GHOST, lim()) = q;
                }
            }
            cl.sync();
            ghosts(buf, 2);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) MGRIT_SH(qf, i + 1, nmax + 2) = split_flux(fp, fm, i + GHOST);
            }
            if (threadIdx.x == blockDim.x - 1)   // left boundary interface
                qf[0] = split_flux(fp, fm, GHOST - 1);
        } else if (numflux == NF_ROE) {
            // local per interface: one cluster barrier per stage, as for advection
            R *wa = arr(buf, 0);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) MGRIT_SH(wa, i + GHOST, lim()) = w[c];
            }
            cl.sync();
            ghosts(buf, 1);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n)
                    MGRIT_SH(qf, i + 1, nmax + 2) =
                        roe_flux<FLUX>(rec_minus(wa, i + GHOST), rec_plus(wa, i + GHOST));
            }
            if (threadIdx.x == blockDim.x - 1)
                qf[0] = roe_flux<FLUX>(rec_minus(wa, GHOST - 1), rec_plus(wa, GHOST - 1));
        } else {
            R *wa = arr(buf, 0);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) MGRIT_SH(wa, i + GHOST, lim()) = w[c];
            }
            cl.sync();
            ghosts(buf, 1);
            R v = R(0);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int i = cell(c);
                if (i < n) {
                    const R a = rec_minus(wa, i + GHOST), b = rec_plus(wa, i + GHOST);
                    MGRIT_SH(um, i + 1, nmax + 1) = a;
                    MGRIT_SH(qf, i + 1, nmax + 2) = b;
                    v = fmax(v, fmax(phys_speed<FLUX>(a), phys_speed<FLUX>(b)));
                }
            }
            if (threadIdx.x == blockDim.x - 1) {
                const R a = rec_minus(wa, GHOST - 1), b = rec_plus(wa, GHOST - 1);
                um[0] = a;
                qf[0] = b;
                v = fmax(v, fmax(phys_speed<FLUX>(a), phys_speed<FLUX>(b)));
            }
            R alpha = R(1);
            if (FLUX == FLX_BURGERS) alpha = cluster_max(v, buf);
            else __syncthreads();
            for (int j = threadIdx.x; j <= n; j += blockDim.x) {
                const R a = um[j], b = qf[j];
                qf[j] = R(0.5) * (phys_flux<FLUX>(b) + phys_flux<FLUX>(a)) - R(0.5) * alpha * (b - a);
            }
        }
        __syncthreads();
    }

    // dG of owned slot c (see RK) and the stage coefficients of a step
    __device__ __forceinline__ R df(int c) const
    {
        const int i = cell(c);
        return Ar<R>::sub(MGRIT_SH(qf, i + 1, nmax + 2), MGRIT_SH(qf, i, nmax + 2));
    }
    __device__ __forceinline__ typename RK<R>::Coef coef(R dt) const
    {
        return RK<R>::coef(dt, dxinv, flux_scale<R>(SCHEME == SCH_WENO5_SSPRK3 && numflux == NF_SPLIT));
    }

    // u <- Phi(u); stage buffers alternate with the global stage counter
    __device__ __forceinline__ void step(R (&u)[CPT], R dt, int &stage)
    {
        const typename RK<R>::Coef K = coef(dt);
        if (SCHEME == SCH_FO_FE) {
            fluxes(u, (stage++) & 1);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (cell(c) < n) u[c] = RK<R>::euler(u[c], K, df(c));
            return;
        }
        R w[CPT];
        fluxes(u, (stage++) & 1);
#pragma unroll
        for (int c = 0; c < CPT; ++c) w[c] = (cell(c) < n) ? RK<R>::euler(u[c], K, df(c)) : R(0);
        fluxes(w, (stage++) & 1);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < n) w[c] = RK<R>::stage2(u[c], w[c], K, df(c));
        fluxes(w, (stage++) & 1);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < n) u[c] = RK<R>::stage3(u[c], w[c], K, df(c));
    }

    __device__ __forceinline__ void load(R (&u)[CPT], const R *row) const
    {
#pragma unroll
        for (int c = 0; c < CPT; ++c) u[c] = (cell(c) < n) ? row[lo + cell(c)] : R(0);
    }
    __device__ __forceinline__ void store(const R (&u)[CPT], R *row) const
    {
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < n) row[lo + cell(c)] = u[c];
    }
    __device__ __forceinline__ void add(R (&u)[CPT], const double *row) const
    {
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (cell(c) < n) u[c] = R((double)u[c] + row[lo + cell(c)]);
    }
};

template <typename R>
inline size_t cluster_smem_bytes(int nx, int K)
{
    const int nmax = (nx + K - 1) / K;
    return sizeof(R) * (4 * (size_t)(nmax + 2 * GHOST) + (nmax + 2) + (nmax + 1) + 3 + NWARP_MAX);
}

// MODE_SEQ on a cluster: u^i = Phi(u^{i-1}) + g^i, i = 1..nsteps (grid = one cluster)
template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_seq_cluster(SlabArgs<R> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ClusterSlab<R, SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv, a.numflux);
    R u[CPT];
    int stage = 0;
    S.load(u, a.src);
    for (int i = 1; i <= a.nsteps; ++i) {
        S.step(u, a.dt, stage);
        if (a.g) S.add(u, rowp(a.g, i, a.nx, a.nrows_g));
        if (a.rows) S.store(u, rowp(a.rows, i, a.nx, a.nrows_rows));
    }
    if (a.out) S.store(u, a.out);
    S.cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

}  // namespace mgrit
