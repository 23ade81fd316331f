// Table of adjoint kernel instances (FP64), indexed by [scheme][flux][cells-per-thread].
#pragma once
#include "cluster_adjoint.cuh"

namespace mgrit {

constexpr int NCPT_ADJ = 4;   // 1, 2, 4, 8 cells per thread: one-CTA slabs up to nx = 4096

struct AdjTable {
    const void *k[2][2][NCPT_ADJ];
    const void *kc[2][2][2];   // k_adjoint_cluster, cells per thread 1 or 2
    const void *kcc[2][2][2];  // k_adjoint_cluster_chunk, cells per thread 1 or 2
};

template <int S, int F>
void fill_adj_sf(AdjTable &t)
{
    t.k[S][F][0] = (const void *)&k_adjoint<S, F, 1>;
    t.k[S][F][1] = (const void *)&k_adjoint<S, F, 2>;
    t.k[S][F][2] = (const void *)&k_adjoint<S, F, 4>;
    t.k[S][F][3] = (const void *)&k_adjoint<S, F, 8>;
    t.kc[S][F][0] = (const void *)&k_adjoint_cluster<S, F, 1>;
    t.kc[S][F][1] = (const void *)&k_adjoint_cluster<S, F, 2>;
    t.kcc[S][F][0] = (const void *)&k_adjoint_cluster_chunk<S, F, 1>;
    t.kcc[S][F][1] = (const void *)&k_adjoint_cluster_chunk<S, F, 2>;
}

// one translation unit per (scheme, flux) group, compiled in parallel
void fill_adj_weno_burgers(AdjTable &t);
void fill_adj_weno_advection(AdjTable &t);
void fill_adj_fo(AdjTable &t);

// dst row (nrows-1-r) = src row r, r = 0..nrows-1 (dst must not alias src)
cudaError_t launch_reverse_rows(const double *src, double *dst, long long nrows, int nx,
                                cudaStream_t s);

inline void fill_adj_all(AdjTable &t)
{
    fill_adj_weno_burgers(t);
    fill_adj_weno_advection(t);
    fill_adj_fo(t);
}

}  // namespace mgrit
