"""Pins for the oracle's semi-discrete operator A(u) (Sec. 2.1, Eq. spaceDisc)
and time steppers (Sec. 2.2, Eqs. SSPRK3, SSPRK1)."""
import numpy as np
import pytest

import oracle as O
from paper_2104_09404_gb300 import inputs

SCHEMES = [O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE]
FLUXES = [O.FLUX_BURGERS, O.FLUX_ADVECTION]
NUMFLUXES = [O.NUMFLUX_LF_SPLIT, O.NUMFLUX_LF_STATE]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("flux", FLUXES)
@pytest.mark.parametrize("numflux", NUMFLUXES)
def test_conservation_telescoping(scheme, flux, numflux):
    # sum_i A_i = -(1/dx) sum_i (F_{i+1/2} - F_{i-1/2}) = 0 on a periodic grid
    rng = np.random.default_rng(1)
    u = rng.standard_normal(37)
    A = O.spatial_op(u, scheme, flux, numflux)
    assert abs(A.sum()) < 1e-11 * np.abs(A).max() * u.size
    assert np.abs(A).max() > 1.0


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("flux", FLUXES)
@pytest.mark.parametrize("numflux", NUMFLUXES)
def test_constant_state_is_steady(scheme, flux, numflux):
    A = O.spatial_op(np.full(16, 0.8125), scheme, flux, numflux)
    assert np.abs(A).max() < 1e-12


def test_first_order_advection_is_upwind():
    rng = np.random.default_rng(2)
    u = rng.standard_normal(20)
    nx = u.size
    dx = 1.0 / nx
    A = O.spatial_op(u, O.SCHEME_FO_FE, O.FLUX_ADVECTION, O.NUMFLUX_LF_SPLIT)
    np.testing.assert_allclose(A, -(u - np.roll(u, 1)) / dx, rtol=1e-14, atol=1e-12)


def test_first_order_burgers_is_global_lf():
    # k = 0: F_{i+1/2} = (f(u_i) + f(u_{i+1}))/2 - alpha (u_{i+1} - u_i)/2, alpha = max|u|
    rng = np.random.default_rng(3)
    u = rng.standard_normal(24)
    nx = u.size
    f = 0.5 * u * u
    a = np.abs(u).max()
    up = np.roll(u, -1)
    F = 0.5 * (f + np.roll(f, -1)) - 0.5 * a * (up - u)
    ref = -(F - np.roll(F, 1)) * nx
    for nf in NUMFLUXES:
        A = O.spatial_op(u, O.SCHEME_FO_FE, O.FLUX_BURGERS, nf)
        np.testing.assert_allclose(A, ref, rtol=1e-12, atol=1e-12)


def test_split_equals_state_form_for_advection():
    # speed 1: f^+ = u, f^- = 0, and Eq. (LFflux) collapses to F = u^-
    u = inputs.fourier_ic(64, seed=4)
    a = O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, O.NUMFLUX_LF_SPLIT)
    b = O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, O.NUMFLUX_LF_STATE)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10)


def test_mirror_symmetry():
    # reflecting x -> -x maps advection with speed 1 to speed -1; for Burgers
    # (odd flux derivative) u(x) -> -u(-x) is a symmetry: A must transform alike
    rng = np.random.default_rng(5)
    u = rng.standard_normal(32)
    # cell i of the reflected grid is cell nx-1-i of the original
    ur = -u[::-1]
    for nf in NUMFLUXES:
        A = O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, nf)
        Ar = O.spatial_op(ur, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, nf)
        np.testing.assert_allclose(Ar, -A[::-1], rtol=1e-11, atol=1e-10)


def _exact_flux_difference(nx, flux):
    # cell averages of u = 0.6 + 0.3 sin(2 pi x); exact A_i = -(f(u(x_{i+1/2})) - f(u(x_{i-1/2})))/dx
    u = inputs.sine_ic(nx, offset=0.6, amp=0.3)
    x = np.arange(nx + 1) / nx
    ux = 0.6 + 0.3 * np.sin(2 * np.pi * x)
    fx = 0.5 * ux * ux if flux == O.FLUX_BURGERS else ux
    return u, -(fx[1:] - fx[:-1]) * nx


def _exact_point_derivative(nx, flux):
    # point values at cell centres of u = 0.6 + 0.3 sin(2 pi x); exact -f(u)_x there
    xc = (np.arange(nx) + 0.5) / nx
    u = 0.6 + 0.3 * np.sin(2 * np.pi * xc)
    ux = 0.3 * 2 * np.pi * np.cos(2 * np.pi * xc)
    return u, -(u * ux if flux == O.FLUX_BURGERS else ux)


def _orders(errs):
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


@pytest.mark.parametrize("flux", FLUXES)
def test_state_form_fifth_order_on_cell_averages(flux):
    # Eq. (LFflux) reconstructs the state from cell averages (finite volumes):
    # A_i approximates the exact flux difference over cell i at 5th order
    errs = []
    for nx in (32, 64, 128):
        u, ref = _exact_flux_difference(nx, flux)
        errs.append(np.abs(O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, flux, O.NUMFLUX_LF_STATE) - ref).max())
    assert _orders(errs).min() > 4.5, errs


@pytest.mark.parametrize("flux", FLUXES)
def test_split_form_fifth_order_on_point_values(flux):
    # the f^+/- splitting applies WENO to f(u_j): the conservative
    # finite-difference form, 5th order when u_j are point values
    errs = []
    for nx in (32, 64, 128):
        u, ref = _exact_point_derivative(nx, flux)
        errs.append(np.abs(O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, flux, O.NUMFLUX_LF_SPLIT) - ref).max())
    assert _orders(errs).min() > 4.5, errs


def test_split_form_second_order_on_cell_averages_for_burgers():
    # f(average of u) differs from the average of f(u) by O(dx^2): on cell
    # averages the split form drops to 2nd order for a nonlinear flux
    errs = []
    for nx in (64, 128, 256):
        u, ref = _exact_flux_difference(nx, O.FLUX_BURGERS)
        errs.append(np.abs(O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS) - ref).max())
    o = _orders(errs)
    assert 1.8 < o.min() and o.max() < 2.3, errs


def test_first_order_scheme_is_first_order():
    errs = []
    for nx in (64, 128, 256):
        u, ref = _exact_flux_difference(nx, O.FLUX_ADVECTION)
        A = O.spatial_op(u, O.SCHEME_FO_FE, O.FLUX_ADVECTION, O.NUMFLUX_LF_SPLIT)
        errs.append(np.abs(A - ref).max())
    orders = _orders(errs)
    assert 0.8 < orders.min() and orders.max() < 1.2


# --------------------------------------------------------------------------
# time steppers
# --------------------------------------------------------------------------

def _upwind_matrix(nx):
    # linear operator of k = 0 advection: A u = -(u_i - u_{i-1})/dx
    I = np.eye(nx)
    S = np.roll(I, 1, axis=0)      # (S u)_i = u_{i-1}
    return -(I - S) * nx


def test_forward_euler_is_identity_plus_h_l():
    # Eq. (SSPRK1) on the linear k = 0 advection operator: (I + hL) u
    nx = 16
    Lm = _upwind_matrix(nx)
    h = 0.7 / nx
    u = np.random.default_rng(6).standard_normal(nx)
    fe = O.step(u, h, O.SCHEME_FO_FE, O.FLUX_ADVECTION)
    np.testing.assert_allclose(fe, u + h * Lm @ u, rtol=1e-13, atol=1e-13)


def test_ssprk3_is_cubic_taylor_polynomial_on_linear_problems():
    # For a linear autonomous operator L, the three stages of Eq. (SSPRK3)
    # compose to I + hL + (hL)^2/2 + (hL)^3/6.  WENO5 advection is linear
    # (weights = linear weights) once every beta << eps; measure L column by
    # column at amplitude 1e-9 (beta ~ 1e-18) and compare one step.
    nx = 12
    amp = 1e-9
    cols = []
    for j in range(nx):
        e = np.zeros(nx); e[j] = amp
        cols.append(O.spatial_op(e, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION) / amp)
    Lm = np.array(cols).T
    h = 0.4 / nx
    u = amp * np.random.default_rng(7).standard_normal(nx)
    got = O.step(u, h, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION)
    hL = h * Lm
    ref = u + hL @ u + hL @ (hL @ u) / 2 + hL @ (hL @ (hL @ u)) / 6
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * scale)
    # the quadratic and cubic terms are far above that tolerance, so a wrong
    # stage weight would be caught
    assert np.abs(hL @ (hL @ (hL @ u))).max() / 6 > 1e-4 * scale


def test_fo_fe_exact_shift_at_unit_cfl():
    # upwind + forward Euler at CFL 1 is the exact shift u_i^{n+1} = u_{i-1}^n
    nx = 32
    u = np.random.default_rng(8).integers(-8, 8, nx).astype(np.float64)
    out = O.step(u, 1.0 / nx, O.SCHEME_FO_FE, O.FLUX_ADVECTION)
    np.testing.assert_array_equal(out, np.roll(u, 1))


def test_weno5_ssprk3_advection_period_convergence():
    # one period of smooth advection returns u0; with dt ~ dx^(5/3) the error
    # decays at 5th order in dx
    errs = []
    for nx in (16, 32, 64):
        u0 = inputs.sine_ic(nx, offset=0.2, amp=1.0)
        nsteps = int(np.ceil(0.5 * nx ** (5.0 / 3.0)))
        out = O.serial(u0, 1.0 / nsteps, nsteps, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION)
        errs.append(np.abs(out - u0).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 4.0, (errs, orders)


def test_ssprk3_third_order_in_time():
    # fixed space grid, shrinking dt: differences converge at 3rd order
    nx = 64
    u0 = inputs.sine_ic(nx, offset=0.5, amp=0.5)
    T = 0.1
    sols = {}
    for n in (40, 80, 160, 1280):
        sols[n] = O.serial(u0, T / n, n)
    e1 = np.abs(sols[40] - sols[1280]).max()
    e2 = np.abs(sols[80] - sols[1280]).max()
    e3 = np.abs(sols[160] - sols[1280]).max()
    assert np.log2(e1 / e2) > 2.7 and np.log2(e2 / e3) > 2.7, (e1, e2, e3)


def test_serial_matches_repeated_steps():
    u0 = inputs.fourier_ic(40, seed=9)
    a = O.serial(u0, 1e-3, 5)
    b = u0.copy()
    for _ in range(5):
        b = O.step(b, 1e-3)
    np.testing.assert_array_equal(a, b)


# ---- classical Lax-Friedrichs + forward Euler and the matched coarse
# ---- integrators (Sec. 3.3, Eqs. fineLF, coarseLFord0/1, fineLFxM) -------

def _E(v):
    return 0.5 * (np.roll(v, -1) + np.roll(v, 1))


def _D(v, dx):
    return (np.roll(v, -1) - np.roll(v, 1)) / (2 * dx)


def test_lf_fe_advection_at_cfl_one_is_the_exact_shift():
    # (u_{i+1} + u_{i-1})/2 - (u_{i+1} - u_{i-1})/2 = u_{i-1}; integer data and
    # a power-of-two nx make every operation exact
    nx = 64
    u = np.random.default_rng(0).integers(-1000, 1000, nx).astype(np.float64)
    got = O.step(u, 1.0 / nx, scheme=O.SCHEME_LF_FE, flux=O.FLUX_ADVECTION)
    np.testing.assert_array_equal(got, np.roll(u, 1))


def test_lf_fe_conserves_and_keeps_constants():
    nx = 64
    u = inputs.fourier_ic(nx, seed=3)
    v = O.step(u, 0.3 / nx, scheme=O.SCHEME_LF_FE)
    assert abs(v.sum() - u.sum()) < 1e-13 * nx
    c = np.full(nx, 0.7)
    np.testing.assert_array_equal(O.step(c, 0.01, scheme=O.SCHEME_LF_FE), c)


def test_matched_integrators_of_one_step_are_the_fine_step():
    nx = 40
    u = inputs.fourier_ic(nx, seed=4)
    fine = O.step(u, 0.2 / nx, scheme=O.SCHEME_LF_FE)
    np.testing.assert_array_equal(O.psi_step(u, 0.2 / nx, 1, 0), fine)
    np.testing.assert_array_equal(O.psi_step(u, 0.2 / nx, 1, 1), fine)


def test_two_step_matching_identities_for_advection():
    # f = u: Phi = E - dt D with E, D commuting, so
    #   Phi^2 - Psi1 = dt^2 D^2 u  and  Phi^2 - Psi0 = -2 dt (E - I) D u + dt^2 D^2 u
    nx, dx = 48, 1.0 / 48
    u = inputs.fourier_ic(nx, seed=5)
    dt = 0.3 * dx
    two = O.step(O.step(u, dt, scheme=O.SCHEME_LF_FE, flux=O.FLUX_ADVECTION), dt,
                 scheme=O.SCHEME_LF_FE, flux=O.FLUX_ADVECTION)
    p1 = O.psi_step(u, dt, 2, 1, flux=O.FLUX_ADVECTION)
    p0 = O.psi_step(u, dt, 2, 0, flux=O.FLUX_ADVECTION)
    Du = _D(u, dx)
    np.testing.assert_allclose(two - p1, dt ** 2 * _D(Du, dx), rtol=0, atol=1e-13)
    np.testing.assert_allclose(two - p0, -2 * dt * (_E(Du) - Du) + dt ** 2 * _D(Du, dx),
                               rtol=0, atol=1e-13)


def test_two_step_first_order_matching_identity_for_burgers():
    # Phi^2(u) = E^2 u - dt (E D f + D f(E u)) + dt^2 D(E u . D f) - dt^3/2 D((D f)^2)
    # exactly for f = u^2/2 (Taylor expansion of f around E u terminates), so
    # Phi^2 - Psi1 is the last two terms
    nx, dx = 64, 1.0 / 64
    u = inputs.fourier_ic(nx, seed=6)
    dt = 0.25 * dx
    two = O.step(O.step(u, dt, scheme=O.SCHEME_LF_FE), dt, scheme=O.SCHEME_LF_FE)
    p1 = O.psi_step(u, dt, 2, 1)
    Df = _D(0.5 * u * u, dx)
    rest = dt ** 2 * _D(_E(u) * Df, dx) - 0.5 * dt ** 3 * _D(Df * Df, dx)
    np.testing.assert_allclose(two - p1, rest, rtol=0, atol=1e-13)


@pytest.mark.parametrize("M", [4, 8])
def test_first_order_matching_error_is_second_order_in_dt(M):
    # Psi1 matches M fine steps up to O(dt^2) (Eq. fineLFxM): halving dt
    # divides the mismatch by ~4; Psi0 only matches to O(dt)
    nx = 64
    u = inputs.fourier_ic(nx, seed=7)

    def fine(dt):
        v = u
        for _ in range(M):
            v = O.step(v, dt, scheme=O.SCHEME_LF_FE)
        return v
    e1 = [np.abs(fine(dt) - O.psi_step(u, dt, M, 1)).max() for dt in (0.02 / nx, 0.01 / nx)]
    e0 = [np.abs(fine(dt) - O.psi_step(u, dt, M, 0)).max() for dt in (0.02 / nx, 0.01 / nx)]
    assert 3.5 < e1[0] / e1[1] < 4.5
    assert 1.7 < e0[0] / e0[1] < 2.3


# ---- Roe flux with the Harten-Hyman entropy fix (Sec. 2.1.2, Eq. roeflux) ---

def test_roe_is_upwind_for_advection():
    # f = u: Roe speed 1, no fix, F = u^-: the same flux as the LF splitting
    nx = 64
    u = inputs.fourier_ic(nx, seed=2)
    for scheme in (O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE):
        a = O.spatial_op(u, scheme, O.FLUX_ADVECTION, O.NUMFLUX_ROE)
        b = O.spatial_op(u, scheme, O.FLUX_ADVECTION, O.NUMFLUX_LF_SPLIT)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_first_order_roe_burgers_is_the_upwind_godunov_flux_away_from_sonic_points():
    # same-sign neighbours: F_{i+1/2} = f(upwind value) exactly, so on positive
    # data A_i = -(f(u_i) - f(u_{i-1}))/dx
    nx = 50
    u = 1.0 + 0.5 * np.random.default_rng(3).random(nx)
    A = O.spatial_op(u, O.SCHEME_FO_FE, O.FLUX_BURGERS, O.NUMFLUX_ROE)
    f = 0.5 * u * u
    np.testing.assert_allclose(A, -(f - np.roll(f, 1)) * nx, rtol=1e-13, atol=0)


def test_entropy_fix_gives_the_godunov_flux_in_a_transonic_rarefaction():
    # u = -a | +a (periodic, so +a | -a at the wrap): the rarefaction
    # interface carries Godunov's f(0) = 0 (without the fix Roe would give
    # a^2/2, an expansion shock); the stationary shock at the wrap carries
    # f(a) = a^2/2, as do all interfaces inside the constant states
    nx, a = 16, 0.8
    u = np.where(np.arange(nx) < nx // 2, -a, a)
    A = O.spatial_op(u, O.SCHEME_FO_FE, O.FLUX_BURGERS, O.NUMFLUX_ROE)
    F = np.full(nx, a * a / 2)        # F[i] = F_{i+1/2}
    F[nx // 2 - 1] = 0.0              # the -a | +a interface
    np.testing.assert_allclose(A, -(F - np.roll(F, 1)) * nx, rtol=0, atol=1e-13)


def test_roe_conserves_and_keeps_constants():
    nx = 64
    u = inputs.fourier_ic(nx, seed=9)
    A = O.spatial_op(u, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, O.NUMFLUX_ROE)
    assert abs(A.sum()) < 1e-12 * nx * nx
    c = np.full(nx, -0.3)
    np.testing.assert_array_equal(O.spatial_op(c, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS,
                                               O.NUMFLUX_ROE), np.zeros(nx))
