// MGRIT slab kernel (Sec. 3.2, Algorithm 1): one launch-time mode selects
//   MODE_RELAX   F- or FCF-relaxation of every C-interval of one level, plus the
//                two extra steps the FAS restriction needs (one CTA per chunk)
//   MODE_INTERP  ideal interpolation: injection + F-relaxation (Eq. interpolation)
//   MODE_SEQ     sequential stepping in one CTA: the coarsest solve (Eq.
//                coarseCorr) or the serial fine stepper
// The residual/restriction and norm kernels live in restrict.cu.
#pragma once
#include "slab.cuh"

namespace mgrit {

enum { MODE_RELAX = 0, MODE_INTERP = 1, MODE_SEQ = 2 };

// Row r of a [rows][nx] array with `nrows` rows; MGRIT_DEBUG builds check r
// and return null (the access is then skipped) when it is out of range.
template <typename T>
__device__ __forceinline__ T *rowp(T *base, long long r, int nx, long long nrows)
{
#ifdef MGRIT_DEBUG
    if (r < 0 || r >= nrows) {
        printf("MGRIT_DEBUG row %lld of %lld block %d thread %d\n", r, nrows, (int)blockIdx.x,
               (int)threadIdx.x);
        return nullptr;
    }
#endif
    return base + r * (long long)nx;
}

template <typename R>
struct SlabArgs {
    int mode;
    int nx, m, nC, fcf, numflux;
    int nsteps;           // MODE_SEQ
    R dxinv, dt, dtc;
    // MODE_RELAX
    const R *uC;          // C-point sources: C_j at uC + j * strideC (MODE_INTERP: coarse rows)
    long long strideC;
    R *newC;              // relaxed C-points, rows 0..nC (null: not stored)
    R *phirow;            // row j+1 = Phi_l(u^{m(j+1)-1})
    R *cstep;             // row j = Phi_{l+1}(newC_j), j < nC (null: skipped; needs newC)
    const double *g;      // level right-hand side rows (FP64 in every precision), or null (zero)
    // MODE_SEQ: start state src, rows 1..nsteps out in rows (optional), final in out
    // MODE_INTERP: fine rows out in rows
    const R *src;
    R *rows;
    R *out;
    // row extents of the arrays above (checked by MGRIT_DEBUG builds)
    long long nrows_uC, nrows_newC, nrows_phirow, nrows_cstep, nrows_g, nrows_rows;
    // SCH_LF_FE only: matched integrator of this level (psiM) and of the next
    // coarser one (psiMc) for psiM/psiMc fine steps of size psiDt; 0 = the
    // fine scheme with the level's step (rediscretisation)
    int psiM, psiMc, psiOrder;
    R psiDt;
};

// relax_chunk and interp_chunk take any slab type with load/store/add/step
// and the constants kScheme and kCpt: the one-CTA Slab, or a slab spread over
// a thread-block cluster (cluster_relax.cuh)
template <typename SL, typename R>
__device__ __forceinline__ void relax_chunk(SL &S, const SlabArgs<R> &a, const int j)
{
    constexpr int SCHEME = SL::kScheme, CPT = SL::kCpt;
    // CTA j = 0..nC.  FCF: new C_j = (Phi_l + g) applied m times from the old
    // C_{j-1} (F- then C-relaxation of chunk j-1); F: C_j kept.  Then the
    // F-relaxation of chunk j from the new C_j.  Chunks are independent
    // (block-diagonal A_FF, Eq. AFF): no grid-wide synchronisation.
    //
    // The steps run as one loop with a single call of S.step (each call site
    // compiles the whole time-stepper):
    //   r = 0 .. nF-1        C-relaxation prefix from C_{j-1} (FCF, j > 0),
    //                        then newC_j is stored;
    //   r = nF (if cstep)    the coarse step Phi_{l+1}(newC_j) of the FAS
    //                        term, then u is re-read from newC_j;
    //   the next m steps     the F-relaxation of chunk j; the m-th gives
    //                        Phi_l(u^{m(j+1)-1}) for the residual.
    const int nx = a.nx, m = a.m;
    const int nF = (j > 0 && a.fcf) ? m : 0;
    const bool coarse = a.cstep && j < a.nC;
    const int total = nF + (j < a.nC ? (coarse ? 1 : 0) + m : 0);
    R u[CPT];
    S.load(u, rowp(a.uC, nF ? j - 1 : j, (int)a.strideC, a.nrows_uC));
    if (!nF && a.newC) S.store(u, rowp(a.newC, j, nx, a.nrows_newC));
#pragma unroll 1
    for (int r = 0; r < total; ++r) {
        const bool is_coarse = coarse && r == nF;
        if (SCHEME == SCH_LF_FE) S.psiM = is_coarse ? a.psiMc : a.psiM;
        S.step(u, is_coarse ? a.dtc : a.dt);
        if (r < nF) {                                   // C-relaxation prefix
            if (a.g) S.add(u, rowp(a.g, (long long)m * (j - 1) + r + 1, nx, a.nrows_g));
            if (r + 1 == nF && a.newC) S.store(u, rowp(a.newC, j, nx, a.nrows_newC));
        } else if (is_coarse) {                         // coarse step of the FAS term
            // u is then re-read from the row this thread just stored (its
            // own cells), which saves CPT registers
            S.store(u, rowp(a.cstep, j, nx, a.nrows_cstep));
            S.load(u, rowp(a.newC, j, nx, a.nrows_newC));
        } else {                                        // F-relaxation step q of chunk j
            const int q = r - nF - (coarse ? 1 : 0) + 1;
            if (q < m) {
                if (a.g) S.add(u, rowp(a.g, (long long)m * j + q, nx, a.nrows_g));
            } else {
                S.store(u, rowp(a.phirow, j + 1, nx, a.nrows_phirow));
            }
        }
    }
    if (SCHEME == SCH_LF_FE) S.psiM = a.psiM;
}

template <typename SL, typename R>
__device__ __forceinline__ void interp_chunk(SL &S, const SlabArgs<R> &a, const int j)
{
    constexpr int CPT = SL::kCpt;
    // Eq. (interpolation): u_l^{mj} = u_{l+1}^j, u_l^{mj+r} = Phi_l(u_l^{mj+r-1}) + g_l^{mj+r}
    const int nx = a.nx, m = a.m;
    R u[CPT];
    S.load(u, rowp(a.uC, j, nx, a.nrows_uC));
    S.store(u, rowp(a.rows, (long long)m * j, nx, a.nrows_rows));
    for (int r = 1; r < m; ++r) {
        S.step(u, a.dt);
        S.add(u, rowp(a.g, (long long)m * j + r, nx, a.nrows_g));
        S.store(u, rowp(a.rows, (long long)m * j + r, nx, a.nrows_rows));
    }
    if (j == a.nC - 1) {   // the last C-point of the level
        S.load(u, rowp(a.uC, a.nC, nx, a.nrows_uC));
        S.store(u, rowp(a.rows, (long long)m * a.nC, nx, a.nrows_rows));
    }
}

template <typename R, int SCHEME, int FLUX, int CPT>
__device__ __forceinline__ void seq_march(Slab<R, SCHEME, FLUX, CPT> &S, const SlabArgs<R> &a)
{
    // u^i = Phi(u^{i-1}) + g^i, i = 1..nsteps, in one CTA
    const int nx = a.nx;
    R u[CPT];
    S.load(u, a.src);
    for (int i = 1; i <= a.nsteps; ++i) {
        S.step(u, a.dt);
        if (a.g) S.add(u, rowp(a.g, i, nx, a.nrows_g));
        if (a.rows) S.store(u, rowp(a.rows, i, nx, a.nrows_rows));
    }
    if (a.out) S.store(u, a.out);
}

template <typename R, int SCHEME, int FLUX, int CPT>
__global__ void __launch_bounds__(512) k_slab(SlabArgs<R> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Slab<R, SCHEME, FLUX, CPT> S(smem, a.nx, a.dxinv, a.numflux);
    S.pair_div = a.mode != MODE_SEQ;
    if (SCHEME == SCH_LF_FE) {
        S.psiM = a.psiM;
        S.psiOrder = a.psiOrder;
        S.psiDt = a.psiDt;
    }
    if (a.mode == MODE_RELAX)
        relax_chunk(S, a, (int)blockIdx.x);
    else if (a.mode == MODE_INTERP)
        interp_chunk(S, a, (int)blockIdx.x);
    else
        seq_march(S, a);
}

}  // namespace mgrit
