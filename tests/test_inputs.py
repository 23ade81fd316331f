"""The seeded input generators (paper_2104_09404_gb300/inputs.py) against
their stated recipes: exact cell averages of the analytic initial conditions
(Sec. 2.1's finite-volume unknowns), the level rule, and the uneven batch."""
import numpy as np
import pytest

from paper_2104_09404_gb300 import inputs


def gauss_cell_averages(f, nx, Lx=1.0, order=12):
    """Cell averages of f by Gauss-Legendre quadrature in every cell."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    dx = Lx / nx
    left = np.arange(nx) * dx
    pts = left[:, None] + 0.5 * dx * (xg[None, :] + 1.0)
    return 0.5 * (f(pts) * wg[None, :]).sum(axis=1)


@pytest.mark.parametrize("nx", [5, 64, 777])
def test_sine_averages_are_exact(nx):
    got = inputs.sine_ic(nx, offset=0.5, amp=1.0)
    ref = gauss_cell_averages(lambda x: 0.5 + np.sin(2 * np.pi * x), nx)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    assert got.mean() == pytest.approx(0.5, abs=1e-14)   # the sine integrates to zero


@pytest.mark.parametrize("nx,seed", [(16, 0), (300, 3), (4096, 7)])
def test_fourier_averages_are_exact(nx, seed):
    a, phi = inputs.fourier_coeffs(seed)
    k = np.arange(1, 9)
    assert np.all(np.abs(a * k ** 2) < 10)   # N(0,1)/k^2 amplitudes

    def u0(x):
        return 0.5 + (a[None, None, :] * np.sin(2 * np.pi * k[None, None, :] * x[..., None] + phi)).sum(-1)
    got = inputs.fourier_ic(nx, seed=seed)
    np.testing.assert_allclose(got, gauss_cell_averages(u0, nx), rtol=0, atol=1e-12)
    assert got.mean() == pytest.approx(0.5, abs=1e-13)
    # the same seed gives the same field, another seed another one
    assert np.array_equal(got, inputs.fourier_ic(nx, seed=seed))
    assert not np.allclose(got, inputs.fourier_ic(nx, seed=seed + 1))


def test_breaking_time_of_a_single_mode():
    # u0 = 0.5 + a sin(2 pi x + phi): min u0' = -2 pi |a|, breaking time 1/(2 pi |a|)
    a, _ = inputs.fourier_coeffs(5, K=1)
    assert inputs.fourier_breaking_time(5, K=1) == pytest.approx(1.0 / (2 * np.pi * abs(a[0])), rel=1e-6)


@pytest.mark.parametrize("nt,m,L", [(256, 4, 3), (16384, 4, 6), (65536, 8, 5), (64, 8, 2), (16, 4, 1),
                                    (17, 4, 1), (96, 2, 4)])
def test_levels_rule(nt, m, L):
    # 1 + min{k : nt / m^k <= 16}, stopping where m no longer divides
    assert inputs.levels_for(nt, m) == L


def test_batch_workload_follows_its_recipe():
    insts, u0s = inputs.batch_workload(seed=0, n=64)
    assert len(insts) == len(u0s) == 64
    for i, (d, u0) in enumerate(zip(insts, u0s)):
        nx, nt, m, L = d["nx"], d["nt"], d["m"], d["levels"]
        assert nx in [2 ** e for e in range(8, 14)] and nt in [2 ** e for e in range(10, 15)]
        assert d["flux"] == (0 if i < 32 else 1) and m == 4
        assert np.array_equal(u0, inputs.fourier_ic(nx, seed=i))
        # at most 16 C-points on the coarsest level, nt divisible down to it
        assert nt % m ** (L - 1) == 0 and nt // m ** (L - 1) <= 16 < nt // m ** max(L - 2, 0) or L == 1
        # dt = 0.375 dx / max|u0| (advection: speed 1)
        speed = np.abs(u0).max() if d["flux"] == 0 else 1.0
        assert d["T"] / nt * speed * nx == pytest.approx(0.375, rel=1e-12)
    # the recipe is seeded: the same seed gives the same batch
    again, _ = inputs.batch_workload(seed=0, n=64)
    assert again == insts
