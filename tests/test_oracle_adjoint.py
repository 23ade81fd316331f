"""Pins for the oracle's discrete adjoint (vector-Jacobian products of the
stepper through Eqs. SSPRK3, spaceDisc, the LF splitting and the WENO
weights).  Checked against central finite differences of the forward oracle
(independent of the derivative code) and, for linear cases, against the
transpose of the explicitly assembled Jacobian."""
import numpy as np
import pytest

import oracle as O
from paper_2104_09404_gb300 import inputs

H = 1e-6


@pytest.mark.parametrize("seed", range(6))
def test_weno_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(5)
    if seed >= 3:
        q[4] += 3.0               # a jump inside one stencil: strongly nonlinear weights
    g = O.weno5_left_grad(q)
    fd = np.array([(O.weno5_left(q + H * e)[0] - O.weno5_left(q - H * e)[0]) / (2 * H)
                   for e in np.eye(5)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("scheme", [O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE])
@pytest.mark.parametrize("flux", [O.FLUX_BURGERS, O.FLUX_ADVECTION])
def test_step_vjp_dot_product_with_finite_differences(scheme, flux):
    # <(Phi(u+hv) - Phi(u-hv))/2h, w> = <v, Phi'(u)^T w> + O(h^2)
    rng = np.random.default_rng(1)
    nx = 48
    u = inputs.fourier_ic(nx, seed=2)
    dt = 0.3 / nx
    for _ in range(3):
        v, w = rng.standard_normal(nx), rng.standard_normal(nx)
        jv = (O.step(u + H * v, dt, scheme, flux) - O.step(u - H * v, dt, scheme, flux)) / (2 * H)
        vj = O.step_vjp(u, w, dt, scheme, flux)
        assert abs(jv @ w - v @ vj) <= 1e-7 * abs(v @ vj)


def test_linear_upwind_adjoint_is_exact_transpose():
    # k = 0 advection with forward Euler is linear: Phi(u) = M u, Phi'^T = M^T
    nx = 20
    dt = 0.6 / nx
    M = np.array([O.step(e, dt, O.SCHEME_FO_FE, O.FLUX_ADVECTION) for e in np.eye(nx)]).T
    w = np.random.default_rng(3).standard_normal(nx)
    got = O.step_vjp(np.zeros(nx), w, dt, O.SCHEME_FO_FE, O.FLUX_ADVECTION)
    np.testing.assert_allclose(got, M.T @ w, rtol=0, atol=1e-13)


def test_weno5_advection_linear_regime_transpose():
    # at amplitude 1e-9 every beta << eps and WENO5 advection is linear; the
    # adjoint there must be the transpose of the Jacobian assembled column by
    # column from forward steps
    nx, amp = 16, 1e-9
    dt = 0.4 / nx
    J = np.array([O.step(amp * e, dt, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION) / amp
                  for e in np.eye(nx)]).T
    w = np.random.default_rng(4).standard_normal(nx)
    got = O.step_vjp(np.zeros(nx), w, dt, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION)
    np.testing.assert_allclose(got, J.T @ w, rtol=1e-8, atol=1e-10)


def test_alpha_derivative_through_the_argmax():
    # only the alpha term connects a cell's value to fluxes far away: with
    # the maximum in cell k*, perturbing u_{k*} must change A far from k*
    # exactly as the adjoint's alpha term predicts
    nx = 40
    u = 0.3 + 0.1 * np.random.default_rng(9).standard_normal(nx)
    u[7] = 1.5                      # unique maximiser of |u|
    dt = 0.2 / nx
    e = np.zeros(nx); e[7] = 1.0
    w = np.zeros(nx); w[30] = 1.0   # observe a cell far from k*
    jv = (O.step(u + H * e, dt) - O.step(u - H * e, dt)) / (2 * H)
    vj = O.step_vjp(u, w, dt)
    assert abs(jv[30]) > 1e-8       # the far cell does feel u_{k*}, through alpha
    assert vj[7] == pytest.approx(jv[30], rel=1e-6)


def test_serial_adjoint_equals_chained_vjps():
    nx, n, dt = 32, 6, 0.3 / 32
    u0 = inputs.fourier_ic(nx, seed=5)
    lam = np.random.default_rng(6).standard_normal(nx)
    traj = O.serial(u0, dt, n, store_all=True)
    ref = lam.copy()
    for k in range(n - 1, -1, -1):
        ref = O.step_vjp(traj[k], ref, dt)
    np.testing.assert_allclose(O.adjoint_serial(u0, lam, dt, n), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("T", [0.05, 0.3])
def test_gradient_of_objective_matches_central_differences(T):
    # J(u0) = 1/2 ||u(T) - u_target||^2 through serial stepping; 32 random
    # directions, central differences with h = 1e-6, relative 1e-6
    nx, n = 64, 40
    u0 = inputs.fourier_ic(nx, seed=7)
    target = O.serial(inputs.fourier_ic(nx, seed=1007), T / n, n)
    def J(x):
        uT = O.serial(x, T / n, n)
        return 0.5 * np.sum((uT - target) ** 2)
    uT = O.serial(u0, T / n, n)
    grad = O.adjoint_serial(u0, uT - target, T / n, n)
    rng = np.random.default_rng(8)
    for _ in range(32):
        v = rng.standard_normal(nx)
        fd = (J(u0 + H * v) - J(u0 - H * v)) / (2 * H)
        assert abs(grad @ v - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(grad) * np.linalg.norm(v))


# ---- adjoint MGRIT (Algorithm 1 run backward in time on the adjoint system) ----

def _forward(nx, nt, m, L, T, seed, scheme=O.SCHEME_WENO5_SSPRK3, flux=O.FLUX_BURGERS):
    u0 = inputs.fourier_ic(nx, seed=seed)
    f = O.mgrit(u0, nt, m, L, T, scheme=scheme, flux=flux, tol=1e-13, max_iter=80)
    assert f["status"] == O.OK
    return u0, f["uC"]


@pytest.mark.parametrize("scheme,flux", [(O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS),
                                         (O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION),
                                         (O.SCHEME_FO_FE, O.FLUX_BURGERS)])
@pytest.mark.parametrize("L,relax,guess", [(2, O.RELAX_FCF, O.GUESS_EQ17),
                                           (3, O.RELAX_F, O.GUESS_EQ17),
                                           (3, O.RELAX_FCF, O.GUESS_INJECT)])
def test_adjoint_mgrit_fixed_point_is_the_serial_adjoint(scheme, flux, L, relax, guess):
    # the fixed point of the backward V-cycle is the serial adjoint (itself
    # pinned by finite differences above), whatever the hierarchy
    nx, nt, m, T = 32, 64, 4, 0.08
    u0, uC = _forward(nx, nt, m, L, T, seed=3, scheme=scheme, flux=flux)
    lamT = np.random.default_rng(2).standard_normal(nx)
    a = O.adjoint_mgrit(uC, lamT, nt, m, L, T, scheme=scheme, flux=flux, relax=relax,
                        guess=guess, tol=1e-12, max_iter=60)
    assert a["status"] == O.OK
    ref = O.adjoint_serial(u0, lamT, T / nt, nt, scheme=scheme, flux=flux)
    np.testing.assert_allclose(a["lam0"], ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    # every C-point is the serial adjoint at that time: the chained VJPs of
    # the m steps before the next C-point, at the serial forward states
    traj = O.serial(u0, T / nt, nt, scheme=scheme, flux=flux, store_all=True)
    for i in range(nt // m):
        lam = a["lamC"][i + 1]
        for n in range(m * (i + 1) - 1, m * i - 1, -1):
            lam = O.step_vjp(traj[n], lam, T / nt, scheme=scheme, flux=flux)
        np.testing.assert_allclose(a["lamC"][i], lam, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_adjoint_mgrit_two_level_F_relaxation_exact_after_nt_over_m_cycles():
    # forward substitution structure: after k two-level F-cycles the first k
    # backward C-intervals are exact, so by nt/m cycles the residual is roundoff
    nx, nt, m, T = 24, 32, 4, 0.06
    _, uC = _forward(nx, nt, m, 2, T, seed=11)
    lamT = np.random.default_rng(5).standard_normal(nx)
    a = O.adjoint_mgrit(uC, lamT, nt, m, 2, T, relax=O.RELAX_F, tol=0.0, max_iter=nt // m)
    assert a["status"] == O.ENOTCONV
    assert a["res_hist"][-1] < 1e-13 * a["res_hist"][0]


def test_adjoint_mgrit_upwind_advection_mirrors_forward_mgrit():
    # first-order upwind advection with forward Euler is linear and
    # shift-invariant: Phi = (1-c) I + c S with S the periodic right shift, so
    # Phi^T = P Phi P with P the reflection i -> nx-1-i (on every level).  The
    # adjoint V-cycle on lamT must then be the reflected forward V-cycle on
    # P lamT, iterate by iterate: same residual history, reflected C-points.
    nx, nt, m, L, T = 40, 128, 4, 3, 0.4
    rng = np.random.default_rng(7)
    lamT = rng.standard_normal(nx)
    uC = np.zeros((nt // m + 1, nx))       # the states do not enter a linear scheme
    kw = dict(scheme=O.SCHEME_FO_FE, flux=O.FLUX_ADVECTION, relax=O.RELAX_FCF, tol=1e-13,
              max_iter=40)
    a = O.adjoint_mgrit(uC, lamT, nt, m, L, T, **kw)
    f = O.mgrit(lamT[::-1].copy(), nt, m, L, T, **kw)
    assert a["status"] == f["status"] == O.OK
    assert a["iters"] == f["iters"]
    np.testing.assert_allclose(a["res_hist"], f["res_hist"], rtol=1e-10,
                               atol=1e-13 * f["res_hist"][0])
    nc = nt // m
    for i in range(nc + 1):
        np.testing.assert_allclose(a["lamC"][nc - i], f["uC"][i][::-1], rtol=0, atol=1e-13)
