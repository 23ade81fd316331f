"""Transposed steps on thread-block clusters: adjoint chunks of levels whose
chunks alone would leave SMs idle, and slices beyond the one-CTA adjoint slab
(4096 < nx <= 16384), where every adjoint launch runs on clusters.  Same bar
as the one-CTA adjoint: the oracle's cycle count, residual history to
rtol 1e-9, and lambda within 1e-11 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_09404_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-11


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_09404_gb300 import build as B, mgrit
    B.build()
    mgrit.load()
    return mgrit


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(got, ref):
    return np.abs(np.asarray(got) - ref).max() / max(np.abs(ref).max(), 1e-300)


def nsm():
    return torch.cuda.get_device_properties(0).multi_processor_count


def expected_k(nx, chunks, one_cta_fits):
    """The host rule for adjoint chunks: with a one-CTA adjoint slab, the
    largest K in {16, 8, 4, 2} with chunks x K <= SMs and 256..1024 cells per
    CTA (else 1); without one, that K if it exists, else the smallest K with
    at most 1024 cells per CTA."""
    fit = [K for K in (16, 8, 4, 2) if -(-nx // K) <= 1024]
    fill = [K for K in fit if chunks * K <= nsm() and (not one_cta_fits or -(-nx // K) >= 256)]
    if fill:
        return fill[0]
    return 1 if one_cta_fits else fit[-1]


@pytest.mark.parametrize("nx,flux", [(6000, O.FLUX_BURGERS), (8192, O.FLUX_ADVECTION),
                                     (16384, O.FLUX_BURGERS)])
def test_wide_step_vjp_parity(M, nx, flux):
    u = inputs.fourier_ic(nx, seed=nx)
    lam = np.random.default_rng(nx).standard_normal(nx)
    dt = 0.4 / nx / max(np.abs(u).max(), 1.0)
    S = M.Solver(nx, 16, 4, 2, flux=flux, T=16 * dt)
    got = S.step_vjp(dev(u), dev(lam)).cpu().numpy()
    assert S.adjoint_query(0) == 0 and S.adjoint_query(100) > 1
    assert relerr(got, O.step_vjp(u, lam, dt, flux=flux)) <= RTOL


@pytest.mark.parametrize("nx,nt,m,scheme", [(8192, 32, 4, O.SCHEME_WENO5_SSPRK3),
                                            (12000, 16, 4, O.SCHEME_FO_FE)])
def test_wide_adjoint_serial_parity(M, nx, nt, m, scheme):
    u0 = inputs.fourier_ic(nx, seed=13)
    lamT = np.random.default_rng(14).standard_normal(nx)
    T = 0.3 * nt / (nx * np.abs(u0).max())
    S = M.Solver(nx, nt, m, 2, scheme, T=T)
    got = S.adjoint_serial(dev(u0), dev(lamT)).cpu().numpy()
    assert S.adjoint_query(2) == 16
    ref = O.adjoint_serial(u0, lamT, T / nt, nt, scheme=scheme)
    assert relerr(got, ref) <= RTOL


CASES = [
    # name, nx, nt, m, L, coarsest CFL, scheme, flux, params
    ("chunks-1024-L3", 1024, 64, 4, 3, 0.4, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, {}),
    ("chunks-2048-F-inject", 2048, 256, 4, 4, 0.4, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS,
     dict(relax=0, guess=1)),
    ("chunks-fo-advection", 3000, 64, 4, 3, 0.5, O.SCHEME_FO_FE, O.FLUX_ADVECTION, {}),
    ("chunks-fcycle", 1536, 128, 2, 4, 0.4, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS,
     dict(cycle=1)),
    ("wide-6000", 6000, 64, 4, 3, 0.4, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, {}),
    ("wide-16384-advection", 16384, 32, 2, 3, 0.5, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, {}),
]


@pytest.mark.parametrize("name,nx,nt,m,L,cfl,scheme,flux,kw", CASES, ids=[c[0] for c in CASES])
def test_cluster_adjoint_mgrit_parity(M, name, nx, nt, m, L, cfl, scheme, flux, kw):
    u0 = inputs.fourier_ic(nx, seed=41)
    speed = np.abs(u0).max() if flux == O.FLUX_BURGERS else 1.0
    T = cfl * nt / (nx * speed * m ** (L - 1))
    relax, guess, cycle = kw.get("relax", O.RELAX_FCF), kw.get("guess", O.GUESS_EQ17), kw.get("cycle", 0)
    fwd = O.mgrit(u0, nt, m, L, T, scheme=scheme, flux=flux, tol=1e-12, max_iter=80,
                  relax=relax, guess=guess)
    assert fwd["status"] == O.OK
    uC = fwd["uC"]
    lamT = np.random.default_rng(42).standard_normal(nx)
    ref = O.adjoint_mgrit(uC, lamT, nt, m, L, T, scheme=scheme, flux=flux, relax=relax,
                          guess=guess, tol=1e-10, max_iter=60, cycle=cycle)
    assert ref["status"] == O.OK
    S = M.Solver(nx, nt, m, L, scheme, flux, T=T, tol=1e-10, max_iter=60, **kw)
    st, lam0, lamC, stats = S.adjoint(dev(uC), dev(lamT), want_lamC=True)
    ks = [S.adjoint_query(100 + l) for l in range(L - 1)]
    assert ks == [expected_k(nx, nt // m ** (l + 1) + 1, nx <= 4096) for l in range(L - 1)], ks
    assert max(ks) > 1
    assert st == M.OK and stats.iters == ref["iters"]
    hist = np.array(stats.res_hist[:stats.iters + 1])
    np.testing.assert_allclose(hist, ref["res_hist"], rtol=1e-9, atol=1e-12 * ref["res_hist"][0])
    assert relerr(lam0.cpu().numpy(), ref["lam0"]) <= RTOL
    assert relerr(lamC.cpu().numpy(), ref["lamC"]) <= RTOL


def test_cluster_adjoint_is_deterministic_and_follows_chunk_clusters(M):
    nx, nt, m, L = 2048, 256, 4, 4
    u0 = inputs.fourier_ic(nx, seed=43)
    T = 0.4 * nt / (nx * np.abs(u0).max() * m ** (L - 1))
    S = M.Solver(nx, nt, m, L, T=T, tol=1e-10)
    st, _, uC, _ = S.solve(dev(u0))
    lamT = dev(np.random.default_rng(44).standard_normal(nx))
    a = S.adjoint(uC, lamT, want_lamC=True)
    b = S.adjoint(uC, lamT, want_lamC=True)
    assert max(S.adjoint_query(100 + l) for l in range(L - 1)) > 1
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    # one CTA per chunk on request: the same gradient to rounding
    S.set_params(chunk_clusters=0)
    c = S.adjoint(uC, lamT, want_lamC=True)
    assert [S.adjoint_query(100 + l) for l in range(L - 1)] == [1] * (L - 1)
    assert a[3].iters == c[3].iters
    assert relerr(c[1].cpu().numpy(), a[1].cpu().numpy()) <= RTOL
