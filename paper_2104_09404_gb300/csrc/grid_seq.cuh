// Sequential time-stepping of one slice spread over a whole grid of CTAs.
//
// The coarsest-level solve (Eq. coarseCorr) and the serial fine stepper are a
// chain u^i = Phi(u^{i-1}) + g^i; inside one step the nx cells are
// independent except for the global Lax-Friedrichs alpha and the three ghost
// cells of each side of the WENO5 stencil.  A thread-block cluster holds at
// most 16 SMs; here the slice is split over G CTAs (up to one per SM, all
// co-resident: a cooperative launch), each holding a contiguous block of n
// cells.  Every RK stage:
//   1. each CTA publishes, in global memory, the maximum of |f'| over its
//      cells and the stage input of its three leftmost and three rightmost
//      cells;
//   2. one grid barrier: a counter with one arrival per CTA;
//   3. it reads the partial maxima (-> alpha) and its neighbours' boundary
//      cells, forms q = f^{+/-}/2 of its own and its ghost cells and computes the
//      n + 1 interface fluxes of its block, each by a pair of lanes (the
//      f^+ and the f^- reconstruction of slab.cuh, combined over a shuffle),
//      then the RK update.
// The published values are double-buffered by stage parity: a CTA writes the
// buffer of stage s + 2 only after the barrier of stage s + 1, which every CTA
// reaches only once it has read stage s's values.  (Tags per CTA, waited on
// only where needed, were measured slower: with Burgers every CTA needs every
// other's partial maximum, and polling 152 tags costs more than one counter.)
//
// Every wait is bounded: a CTA that waits longer than GRID_WAIT_NS sets the
// error flag and returns, and so does every CTA that waits for it, so the
// kernel always ends; the host reports MGRIT_ETIMEOUT.
#pragma once
#include "kernels.cuh"

namespace mgrit {

constexpr int GRID_MAX = 256;                       // CTAs of one grid stepper
constexpr int GRID_THREADS = 256;                   // at most, per CTA
constexpr unsigned long long GRID_WAIT_NS = 500000000ull;   // 0.5 s

// global buffers of one grid stepper (device memory owned by the context)
struct GridBufs {
    double *part;        // [2][GRID_MAX] per-CTA partial max |f'|
    double *halo;        // [2][GRID_MAX][6] boundary stage inputs (left 3, right 3)
    unsigned *bar;       // barrier counter (zeroed before each launch)
    int *err;            // set to 1 when a wait gave up
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number k (0, 1, ...) of a launch of G CTAs: one counter
// in global memory, one arrival per CTA.  Returns false on every thread of
// the CTA if the wait gave up (the error flag is then set).  skip: this CTA
// does not arrive (the test hook), so every wait on this barrier runs out.
__device__ __forceinline__ bool grid_barrier(const GridBufs &g, unsigned G, unsigned k, bool skip,
                                             int *abort_flag)
{
    __syncthreads();   // the CTA's published values are written
    if (threadIdx.x == 0) {
        int ok = 1;
        if (!skip) {
            __threadfence();
            atomicAdd(g.bar, 1u);
        }
        const unsigned target = G * (k + 1);
        const unsigned long long t0 = global_ns();
        // poll with short pauses: the wait is normally a few microseconds
        while (ld_acquire(g.bar) < target) {
            if (global_ns() - t0 > GRID_WAIT_NS) {
                atomicExch(g.err, 1);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        *abort_flag = ok ? 0 : 1;
    }
    __syncthreads();
    return *abort_flag == 0;
}

template <typename R>
struct GridArgs {
    SlabArgs<R> a;       // nx, dt, dxinv, nsteps, src, g, rows, out (MODE_SEQ fields)
    GridBufs gb;
    int skip_cta;        // test hook: this CTA never arrives at barrier 0 (-1: none)
};

// One step chain on G CTAs of T threads; CTA b owns cells [lo, hi), n = hi -
// lo <= T/2 - 1.  Thread j < n holds cell lo + j; the lane pair (2j, 2j+1)
// computes the interface lo - 1/2 + j, j = 0..n.  Split numerical flux only.
template <typename R, int SCHEME, int FLUX>
__global__ void __launch_bounds__(GRID_THREADS) k_seq_grid(GridArgs<R> ga)
{
    const SlabArgs<R> &a = ga.a;
    const GridBufs &gb = ga.gb;
    const int G = (int)gridDim.x, b = (int)blockIdx.x, t = (int)threadIdx.x;
    const int nx = a.nx;
    const int lo = (int)((long long)b * nx / G), hi = (int)((long long)(b + 1) * nx / G);
    const int n = hi - lo;
    constexpr int NS = GRID_THREADS / 2;
    // shared: q^+ and q^- of cells lo-3 .. hi+2, the n+1 interface fluxes,
    // the broadcast alpha and the abort flag
    __shared__ R qa[NS + 6], qb[NS + 6], qf[NS + 1], red[GRID_THREADS / 32];
    __shared__ R s_alpha;
    __shared__ int s_abort;
    using AR = Ar<R>;
    const bool own = t < n;
    const int bl = (b + G - 1) % G, br = (b + 1) % G;
    R u = own ? a.src[lo + t] : R(0);
    unsigned k = 0;   // stages done
    if (t == 0) s_abort = 0;

    // F_{lo-1/2+j} of the lane pair (2j, 2j+1) from the cells j-3..j+2 (local
    // slot = cell + 3).  Both lanes run the same instructions, so the pair
    // costs one reconstruction's time: the even lane reconstructs f^+ from
    // the left, the odd lane f^- from the right as a left-biased
    // reconstruction of the mirrored stencil.  The mirrored first
    // differences are the exact negatives of the forward ones, so the odd
    // lane obtains exactly -N and D of the right-biased expression (round to
    // nearest is symmetric), and the combined flux has the bits of slab.cuh's.
    auto interface = [&](int j, bool odd) -> R {
        const int s = j - 1 + GHOST;   // the interface's left cell
        if (SCHEME == SCH_FO_FE) return qa[s] + qb[s + 1];   // f^+_i + f^-_{i+1}
        WenoWin<R> P;
        if (FLUX == FLX_ADVECTION) {   // f^- = 0: one reconstruction, on both lanes
            P.init(qa[s - 2], qa[s - 1], qa[s], qa[s + 1], qa[s + 2]);
            return split_flux_win_adv(P, qa[s]);
        }
        const R *q = odd ? qb : qa;
        const int s0 = odd ? s + 3 : s - 2, d = odd ? -1 : 1;
        P.init(q[s0], q[s0 + d], q[s0 + 2 * d], q[s0 + 3 * d], q[s0 + 4 * d]);
        R N, D;
        P.left(N, D);
        const R No = __shfl_xor_sync(0xffffffffu, N, 1), Do = __shfl_xor_sync(0xffffffffu, D, 1);
        // even lane: (N^+, D^+) = (N, D), (N^-, D^-) = (-No, Do); the odd lane's result is dropped
        return split_flux_combine(N, D, AR::neg(No), Do, qa[s], qb[s + 1]);
    };

    // stage input w -> interface fluxes in qf; false if a wait gave up
    auto fluxes = [&](R w) -> bool {
        const int par = (int)(k & 1u);
        // 1. publish the partial max |f'| and the boundary inputs
        if (FLUX == FLX_BURGERS) {
            R v = own ? fabs(w) : R(0);
            v = warp_max(v);
            if ((t & 31) == 0) red[t >> 5] = v;
            __syncthreads();
            if (t == 0) {
                R m = red[0];
                for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
                gb.part[par * GRID_MAX + b] = (double)m;
            }
        }
        if (own && t < GHOST) gb.halo[(par * GRID_MAX + b) * 6 + t] = (double)w;
        if (own && t >= n - GHOST) gb.halo[(par * GRID_MAX + b) * 6 + GHOST + t - (n - GHOST)] = (double)w;
        // 2. grid barrier
        if (!grid_barrier(gb, (unsigned)G, k, b == ga.skip_cta && k == 0, &s_abort)) return false;
        ++k;
        // the ghost inputs (threads 0..5) are loaded while the last warp
        // reduces the partial maxima, so that the two global reads overlap
        R ghost = R(0);
        if (t < GHOST) ghost = (R)gb.halo[(par * GRID_MAX + bl) * 6 + GHOST + t];
        else if (t < 2 * GHOST) ghost = (R)gb.halo[(par * GRID_MAX + br) * 6 + (t - GHOST)];
        if (FLUX == FLX_BURGERS) {
            const int w0 = (int)blockDim.x - 32;
            if (t >= w0) {
                R m = R(0);
                for (int q = t - w0; q < G; q += 32) m = fmax(m, (R)gb.part[par * GRID_MAX + q]);
                m = warp_max(m);
                if (t == w0) s_alpha = m;
            }
            __syncthreads();
        }
        // 3. own and ghost q, interface fluxes
        const R alpha = FLUX == FLX_BURGERS ? s_alpha : R(1);
        auto put_q = [&](int slot, R x) {
            if (SCHEME == SCH_FO_FE) {
                // first order: f^+/- = f(x)/2 +/- (alpha/2) x
                const R p = R(0.5) * phys_flux<FLUX>(x), h = R(0.5) * alpha;
                qa[slot] = fma(h, x, p);
                qb[slot] = fma(-h, x, p);
            } else if (FLUX == FLX_BURGERS) {
                const R a4 = R(0.25) * alpha;
                R p, q;
                burgers_q(x, a4, p, q);
                qa[slot] = p;
                qb[slot] = q;
            } else {
                qa[slot] = R(0.5) * x;
            }
        };
        if (own) put_q(t + GHOST, w);
        if (t < GHOST) put_q(t, ghost);
        else if (t < 2 * GHOST) put_q(n + t, ghost);
        __syncthreads();
        // lane pairs: all lanes of a warp take part in the shuffle; pairs past
        // interface n read slots below n + 6 and drop the result
        {
            const int j = t >> 1;
            const int jj = j <= n ? j : n;
            const R F = interface(jj, (t & 1) != 0);
            if (j <= n && !(t & 1)) qf[j] = F;
        }
        __syncthreads();
        return true;
    };

    // dG of the own cell and the stage coefficients (see RK): the WENO5
    // split form stores G = 3F
    auto df = [&]() -> R { return AR::sub(qf[t + 1], qf[t]); };
    const typename RK<R>::Coef K = RK<R>::coef(a.dt, a.dxinv, flux_scale<R>(SCHEME == SCH_WENO5_SSPRK3));

    bool alive = true;
    for (int i = 1; i <= a.nsteps && alive; ++i) {
        if (SCHEME == SCH_FO_FE) {
            if (!(alive = fluxes(u))) break;
            if (own) u = RK<R>::euler(u, K, df());
        } else {
            if (!(alive = fluxes(u))) break;
            R w = own ? RK<R>::euler(u, K, df()) : R(0);
            if (!(alive = fluxes(w))) break;
            if (own) w = RK<R>::stage2(u, w, K, df());
            if (!(alive = fluxes(w))) break;
            if (own) u = RK<R>::stage3(u, w, K, df());
        }
        if (own && a.g) u = R((double)u + a.g[(long long)i * nx + lo + t]);
        if (own && a.rows) a.rows[(long long)i * nx + lo + t] = u;
    }
    if (alive && own && a.out) a.out[lo + t] = u;
}

}  // namespace mgrit
