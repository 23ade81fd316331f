"""The allocation-free residual entry point (mgrit_residual_static).

It serves callers that cannot call cudaMalloc (an application that owns all
device memory through its own pool, or a loop that must not trigger the
allocator's device synchronisation).  Its scratch is a static device array,
so this checks it through the C ABI against the allocating mgrit_residual,
on two calls in a row (the second must not see the first's leftovers).
This file sorts last so that a run stopping at the first failure has run
everything else first.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2104_09404_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_09404_gb300 import build as B, mgrit
    B.build()
    mgrit.load()
    return mgrit


def static_residual(M, uC, nt, m, T, scheme=0, flux=0, numflux=0):
    lib = M.load()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    nx = uC.shape[1]
    st = lib.mgrit_residual_static(nx, nt, m, scheme, flux, numflux, T, 1.0,
                                   ctypes.c_void_p(uC.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, float(out.item())


@pytest.mark.parametrize("nx,nt,m,scheme,flux,numflux", [
    (256, 128, 4, 0, 0, 0), (1000, 64, 8, 0, 1, 0), (64, 96, 2, 1, 0, 0),
    (300, 64, 4, 0, 0, 1),     # state-reconstruction Lax-Friedrichs flux
    (200, 64, 4, 0, 0, 2),     # Roe flux with the entropy fix
    (128, 64, 2, 1, 1, 2),
])
def test_static_residual_matches_allocating_entry_point(M, nx, nt, m, scheme, flux, numflux):
    T = 0.02
    u0 = inputs.fourier_ic(nx, seed=nx)
    traj = O.serial(u0, T / nt, nt, scheme, flux, numflux, store_all=True)
    s = M.Solver(nx, nt, m, 2, scheme, flux, T=T, numflux=numflux)
    rng = np.random.default_rng(1)
    for call in range(2):   # two calls in a row, different data
        uC = traj[::m].copy()
        uC[1:] += (10.0 ** (-3 - 2 * call)) * rng.standard_normal(uC[1:].shape)
        d = torch.as_tensor(uC, device="cuda")
        st, got = static_residual(M, d, nt, m, T, scheme, flux, numflux)
        assert st == M.OK
        ref = s.residual(d)
        assert got == pytest.approx(ref, rel=1e-10)
        assert got == pytest.approx(O.residual(uC, nt, m, T, scheme, flux, numflux), rel=1e-10)


def test_static_residual_refuses_what_it_does_not_cover(M):
    # the classical Lax-Friedrichs scheme and slices wider than one FP64 CTA
    d = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    assert static_residual(M, d, 16, 4, 0.1, scheme=2)[0] == M.EINVAL
    w = torch.zeros((3, 8200), dtype=torch.float64, device="cuda")
    assert static_residual(M, w, 8, 4, 0.1)[0] == M.EINVAL


def test_static_residual_rejects_sizes_beyond_its_scratch(M):
    nx, m = 4096, 4
    nt = m * ((1 << 21) // nx)          # (nt/m + 1) * nx just above the limit
    d = torch.zeros((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st, val = static_residual(M, d, nt, m, 0.1)
    assert st == M.EINVAL and val == -1.0   # nothing launched
    st, val = static_residual(M, d[:-1], nt - m, m, 0.1)   # exactly at the limit
    assert st == M.OK and val == 0.0     # Phi(0) = 0: the residual of zeros is exactly 0
