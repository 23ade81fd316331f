// Table of kernel instances, indexed by [scheme][flux][cells-per-thread].
#pragma once
#include "cluster_relax.cuh"
#include "grid_seq.cuh"

namespace mgrit {

constexpr int NCPT = 6;
constexpr int CPT_VALUES[NCPT] = {1, 2, 4, 8, 16, 32};
constexpr int NCPT64 = 5;          // FP64 slabs stop at 16 cells per thread (nx <= 8192)
constexpr int MAX_THREADS = 512;   // matches __launch_bounds__ of k_slab

constexpr int NSCHEME = 3;         // WENO5 + SSPRK3, first order + FE, classical LF + FE

constexpr int NCPT_RELAXC = 3;     // k_slab_cluster: 1, 2 or 4 cells per thread

// scheme 2 (classical Lax-Friedrichs + forward Euler) exists in FP64 slabs
// only; the cluster kernels cover schemes 0 and 1
struct KernelTable {
    const void *slab64[NSCHEME][2][NCPT];
    const void *slab32[NSCHEME][2][NCPT];
    const void *seqc64[2][2][2];   // k_seq_cluster, cells per thread 1 or 2
    const void *seqc32[2][2][2];
    const void *relc64[2][2][NCPT_RELAXC];   // k_slab_cluster, cells per thread 1, 2, 4
    const void *relc32[2][2][NCPT_RELAXC];
    const void *grid64[2][2];   // k_seq_grid [scheme][flux] (WENO5 / first order, split flux)
    const void *grid32[2][2];
    const void *tlc64[2][2];    // k_slab_tlc [flux][0: 8, 1: 16 cells per thread] (WENO5 split form)
    const void *tlc32[2][2];
};

template <typename R, int F>
void fill_tlc(const void *(&t)[2][2])
{
    t[F][0] = (const void *)&k_slab_tlc<R, SCH_WENO5_SSPRK3, F, 8>;
    t[F][1] = (const void *)&k_slab_tlc<R, SCH_WENO5_SSPRK3, F, 16>;
}

template <typename R, int S, int F>
void fill_sf(const void *(&t)[NSCHEME][2][NCPT])
{
    t[S][F][0] = (const void *)&k_slab<R, S, F, 1>;
    t[S][F][1] = (const void *)&k_slab<R, S, F, 2>;
    t[S][F][2] = (const void *)&k_slab<R, S, F, 4>;
    t[S][F][3] = (const void *)&k_slab<R, S, F, 8>;
    t[S][F][4] = (const void *)&k_slab<R, S, F, 16>;
}

template <int S, int F>
void fill_sf32(const void *(&t)[NSCHEME][2][NCPT])
{
    fill_sf<float, S, F>(t);
    t[S][F][5] = (const void *)&k_slab<float, S, F, 32>;
}

template <typename R, int S, int F>
void fill_cluster(const void *(&t)[2][2][2])
{
    t[S][F][0] = (const void *)&k_seq_cluster<R, S, F, 1>;
    t[S][F][1] = (const void *)&k_seq_cluster<R, S, F, 2>;
}

template <typename R, int S, int F>
void fill_cluster_relax(const void *(&t)[2][2][NCPT_RELAXC])
{
    t[S][F][0] = (const void *)&k_slab_cluster<R, S, F, 1>;
    t[S][F][1] = (const void *)&k_slab_cluster<R, S, F, 2>;
    t[S][F][2] = (const void *)&k_slab_cluster<R, S, F, 4>;
}

// one translation unit per (precision, scheme, flux) and kind (slab or
// cluster kernels), compiled in parallel
void fill_f64_weno_burgers(KernelTable &t);
void fill_f64_weno_advection(KernelTable &t);
void fill_f64_weno_cluster(KernelTable &t);
void fill_f64_fo(KernelTable &t);
void fill_f64_lf(KernelTable &t);
void fill_f32_weno_burgers(KernelTable &t);
void fill_f32_weno_advection(KernelTable &t);
void fill_f32_weno_cluster(KernelTable &t);
void fill_f32_fo(KernelTable &t);
void fill_f64_relaxc_burgers(KernelTable &t);
void fill_f64_relaxc_advection(KernelTable &t);
void fill_f32_relaxc_burgers(KernelTable &t);
void fill_f32_relaxc_advection(KernelTable &t);
void fill_grid(KernelTable &t);
void fill_tlc_f64_burgers(KernelTable &t);
void fill_tlc_f64_advection(KernelTable &t);
void fill_tlc_f32_burgers(KernelTable &t);
void fill_tlc_f32_advection(KernelTable &t);

inline void fill_all(KernelTable &t)
{
    fill_grid(t);
    fill_tlc_f64_burgers(t);
    fill_tlc_f64_advection(t);
    fill_tlc_f32_burgers(t);
    fill_tlc_f32_advection(t);
    fill_f64_weno_burgers(t);
    fill_f64_weno_advection(t);
    fill_f64_weno_cluster(t);
    fill_f64_fo(t);
    fill_f64_lf(t);
    fill_f32_weno_burgers(t);
    fill_f32_weno_advection(t);
    fill_f32_weno_cluster(t);
    fill_f32_fo(t);
    fill_f64_relaxc_burgers(t);
    fill_f64_relaxc_advection(t);
    fill_f32_relaxc_burgers(t);
    fill_f32_relaxc_advection(t);
}

}  // namespace mgrit
