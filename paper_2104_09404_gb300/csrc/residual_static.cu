// mgrit_residual_static: the level-0 residual norm without any device
// allocation, for callers that cannot call cudaMalloc.
//
// It runs the same kernels as mgrit_residual (k_slab in relaxation mode for
// the Phi^m rows, k_restrict for the squared residual partials, k_norm for
// the sum), but their scratch lives in one file-scope device array instead
// of context buffers.  The array is part of this library's device image, so
// every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mgrit.h"
#include "kernel_table.cuh"
#include "restrict.cuh"

using namespace mgrit;

namespace {

// Phi^m rows: (nt/m + 1) x nx doubles at most; then the norm partials.
constexpr size_t ROWS_MAX = (size_t)MGRIT_STATIC_SCRATCH_DOUBLES;
constexpr size_t PARTIALS_MAX = 2048;
constexpr int MGRIT_NSCHEME_STATIC = 2;   // WENO5 + SSPRK3, first order + FE

static __device__ __align__(256) double g_static_scratch[ROWS_MAX + PARTIALS_MAX];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
// per device: the device address of g_static_scratch, and the kernel
// instances whose shared-memory limit this file has raised
struct DeviceSetup {
    double *scratch;
    const void *raised[MGRIT_NSCHEME_STATIC][2][NCPT64];
};
DeviceSetup g_dev[MAX_DEVICES];

const KernelTable &kernels()
{
    static const KernelTable t = [] {
        KernelTable k;
        memset(&k, 0, sizeof k);
        fill_all(k);
        return k;
    }();
    return t;
}

// Device address of the scratch array for the current device.  Host code may
// not use &g_static_scratch (that is a host-side stand-in); the address is
// looked up with the device current, on every call, so that a context
// re-created after a device reset (which loads the module, and the array,
// anew) gets its new address.  The per-device record of raised kernel
// attributes is dropped when the address changes.
cudaError_t scratch_address(double **out, int *dev_out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_dev[dev];
    if (static_cast<double *>(p) != d.scratch) {
        memset(&d, 0, sizeof d);
        d.scratch = static_cast<double *>(p);
    }
    *out = d.scratch;
    *dev_out = dev;
    return cudaSuccess;
}

// the FP64 one-CTA slab for (scheme, flux, nx): the smallest cells per
// thread giving at most MAX_THREADS threads (at least 4 for WENO5, as in the
// solver contexts, so that both form the same interface quads)
const void *select_slab(int nx, int scheme, int flux, int *threads, int *cpt, int *ci_out)
{
    for (int ci = scheme == MGRIT_WENO5_SSPRK3 ? 2 : 0; ci < NCPT64; ++ci) {
        const int need = (nx + CPT_VALUES[ci] - 1) / CPT_VALUES[ci];
        if (need <= MAX_THREADS) {
            *threads = ((need + 31) / 32) * 32;
            *cpt = CPT_VALUES[ci];
            *ci_out = ci;
            return kernels().slab64[scheme][flux][ci];
        }
    }
    return nullptr;
}

// raise the kernel's dynamic shared-memory limit to the opt-in maximum once
// per device (not to this launch's size: the kernel instance is shared with
// solver contexts whose slices may be wider)
cudaError_t raise_smem_once(int dev, int scheme, int flux, int ci, const void *slab)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const void *&done = g_dev[dev].raised[scheme][flux][ci];
    if (done == slab) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(slab, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess) done = slab;
    return e;
}

}  // namespace

extern "C" int mgrit_residual_static(int nx, int nt, int m, int scheme, int flux, int numflux,
                                     double T, double L, const double *uC_dev, double *norm_dev,
                                     void *stream)
{
    if (!uC_dev || !norm_dev) return MGRIT_EINVAL;
    if (scheme != MGRIT_WENO5_SSPRK3 && scheme != MGRIT_FO_FE) return MGRIT_EINVAL;
    if (flux != MGRIT_BURGERS && flux != MGRIT_ADVECTION) return MGRIT_EINVAL;
    if (numflux != MGRIT_LF_SPLIT && numflux != MGRIT_LF_STATE && numflux != MGRIT_ROE)
        return MGRIT_EINVAL;
    if (m < 2 || nt < m || nt % m) return MGRIT_EINVAL;
    if (nx < (scheme == MGRIT_WENO5_SSPRK3 ? 5 : 3)) return MGRIT_EINVAL;
    if (!(T > 0) || !(L > 0) || !std::isfinite(T) || !std::isfinite(L)) return MGRIT_EINVAL;
    const int nC = nt / m;
    if ((size_t)(nC + 1) * (size_t)nx > ROWS_MAX) return MGRIT_EINVAL;   // beyond the scratch
    int threads = 0, cpt = 0, ci = 0;
    const void *slab = select_slab(nx, scheme, flux, &threads, &cpt, &ci);
    if (!slab) return MGRIT_EINVAL;
    const size_t smem = slab_smem_bytes<double>(nx, cpt, threads);
    if (smem > 227 * 1024) return MGRIT_EINVAL;
    const int blocks = restrict_blocks(nC, nx);
    if ((size_t)blocks > PARTIALS_MAX) return MGRIT_EINVAL;

    cudaStream_t s = (cudaStream_t)stream;
    double *scratch = nullptr;
    int dev = 0;
    if (scratch_address(&scratch, &dev) != cudaSuccess) return MGRIT_ECUDA;
    double *rows = scratch;
    double *partials = scratch + ROWS_MAX;
    if (raise_smem_once(dev, scheme, flux, ci, slab) != cudaSuccess) return MGRIT_ECUDA;

    // rows 1..nC <- Phi_0^m(uC row j-1); every row and partial read below is
    // written first by this call, so nothing needs clearing
    SlabArgs<double> a;
    memset(&a, 0, sizeof a);
    a.mode = MODE_RELAX;
    a.nx = nx;
    a.m = m;
    a.nC = nC;
    a.fcf = 0;
    a.numflux = numflux;
    a.dxinv = nx / L;
    a.dt = T / nt;
    a.uC = uC_dev;
    a.strideC = nx;
    a.phirow = rows;
    a.nrows_uC = a.nrows_phirow = nC + 1;
    void *args[] = {&a};
    cudaError_t le = cudaLaunchKernel(slab, dim3(nC), dim3(threads), args, smem, s);
    if (le == cudaErrorInvalidValue && smem > 48 * 1024) {
        // the limit raised earlier no longer holds (a device reset that
        // kept the array's address): raise it again and retry once
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lock(g_setup_mutex);
            g_dev[dev].raised[scheme][flux][ci] = nullptr;
        }
        if (raise_smem_once(dev, scheme, flux, ci, slab) != cudaSuccess) return MGRIT_ECUDA;
        le = cudaLaunchKernel(slab, dim3(nC), dim3(threads), args, smem, s);
    }
    if (le != cudaSuccess) return MGRIT_ECUDA;

    RestrictArgs r;
    memset(&r, 0, sizeof r);
    r.newC = uC_dev;
    r.phirow = rows;
    r.partials = partials;
    r.nx = nx;
    r.m = m;
    r.nC = nC;
    if (launch_restrict(r, blocks, s) != cudaSuccess) return MGRIT_ECUDA;
    if (launch_norm(partials, blocks, norm_dev, s) != cudaSuccess) return MGRIT_ECUDA;
    return MGRIT_OK;
}
