"""Pins for the oracle's MGRIT (Sec. 3, Algorithm 1) against what the
structure of the method fixes: the fixed point is serial time-stepping
(Eqs. monolithicSystem, schurComplement), two-level exactness (forward
substitution through S), the FAS fixed-point property of Eq. (restriction::u),
conservation, and the brute-force monolithic residual on tiny grids."""
import numpy as np
import pytest

import oracle as O
from paper_2104_09404_gb300 import inputs


def serial_traj(u0, nt, T, **kw):
    return O.serial(u0, T / nt, nt, store_all=True, **kw)


@pytest.mark.parametrize("relax", [O.RELAX_F, O.RELAX_FCF])
@pytest.mark.parametrize("guess", [O.GUESS_EQ17, O.GUESS_INJECT])
def test_fixed_point_is_serial_stepping(relax, guess):
    nx, nt, m, T = 32, 64, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=1)
    traj = serial_traj(u0, nt, T)
    r = O.mgrit(u0, nt, m, 3, T, relax=relax, guess=guess, uC_init=traj[::m], tol=1e-12)
    assert r["status"] == O.OK and r["iters"] == 0
    assert r["res_hist"][0] < 1e-13
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-14)


@pytest.mark.parametrize("levels", [2, 3, 4])
@pytest.mark.parametrize("relax", [O.RELAX_F, O.RELAX_FCF])
def test_converged_mgrit_equals_serial(levels, relax):
    nx, nt, m, T = 64, 256, 2, 0.2
    u0 = inputs.sine_ic(nx)
    r = O.mgrit(u0, nt, m, levels, T, relax=relax, tol=1e-10, max_iter=60)
    assert r["status"] == O.OK
    traj = serial_traj(u0, nt, T)
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["uT"], traj[-1], rtol=0, atol=1e-9)
    # residual history ends below tol and the previous one was not
    assert r["res_hist"][-1] < 1e-10
    assert np.all(r["res_hist"][:-1] >= 1e-10)


@pytest.mark.parametrize("k", [1, 2, 5])
def test_two_level_f_relaxation_exact_after_k_cycles(k):
    # forward substitution with S (Eq. schurComplement): after k two-level
    # cycles with F-relaxation the C-points 0..k equal serial stepping
    nx, nt, m, T = 32, 96, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=2)
    traj = serial_traj(u0, nt, T)
    r = O.mgrit(u0, nt, m, 2, T, relax=O.RELAX_F, tol=0.0, max_iter=k)
    assert r["status"] == O.ENOTCONV and r["iters"] == k
    err = np.abs(r["uC"] - traj[::m]).max(axis=1)
    assert err[: k + 1].max() < 1e-13, err
    if k == 1:
        assert err[k + 2:].max() > 1e-9     # not yet exact beyond the front


def test_two_level_converges_within_nt_over_m_cycles():
    nx, nt, m, T = 32, 64, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=3)
    for relax in (O.RELAX_F, O.RELAX_FCF):
        r = O.mgrit(u0, nt, m, 2, T, relax=relax, tol=1e-10, max_iter=nt // m + 1)
        assert r["status"] == O.OK and r["iters"] <= nt // m


@pytest.mark.parametrize("nx", [8, 16])
@pytest.mark.parametrize("nt,m,levels", [(8, 2, 2), (16, 2, 3), (16, 4, 2), (16, 2, 2)])
@pytest.mark.parametrize("scheme", [O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE])
def test_brute_force_monolithic_residual_tiny(nx, nt, m, levels, scheme):
    # every row of A u = g (Eq. monolithicSystem) holds at convergence:
    # u^0 = u0 and u^n = Phi(u^{n-1})
    T = 0.05
    u0 = inputs.fourier_ic(nx, seed=4)
    r = O.mgrit(u0, nt, m, levels, T, scheme=scheme, tol=1e-12, max_iter=40, want_full=True)
    assert r["status"] == O.OK
    u = r["u"]
    np.testing.assert_array_equal(u[0], u0)
    dt = T / nt
    worst = max(np.abs(u[n] - O.step(u[n - 1], dt, scheme)).max() for n in range(1, nt + 1))
    assert worst < 1e-11
    np.testing.assert_allclose(u, serial_traj(u0, nt, T, scheme=scheme), rtol=0, atol=1e-11)


@pytest.mark.parametrize("relax", [O.RELAX_F, O.RELAX_FCF])
def test_every_iterate_conserves_mass(relax):
    # g rows other than g^0 carry zero total mass (flux differences telescope),
    # so any number of unconverged cycles keeps sum_i u_i of every C-point
    nx, nt, m, T = 48, 128, 4, 0.15
    u0 = inputs.fourier_ic(nx, seed=5)
    for k in (1, 3):
        r = O.mgrit(u0, nt, m, 3, T, relax=relax, tol=0.0, max_iter=k)
        sums = r["uC"].sum(axis=1)
        assert np.abs(sums - u0.sum()).max() < 1e-11 * nx


def test_injection_and_eq17_reach_the_same_solution():
    nx, nt, m, T = 32, 128, 2, 0.15
    u0 = inputs.sine_ic(nx)
    a = O.mgrit(u0, nt, m, 3, T, guess=O.GUESS_EQ17, tol=1e-11)
    b = O.mgrit(u0, nt, m, 3, T, guess=O.GUESS_INJECT, tol=1e-11)
    assert a["status"] == O.OK and b["status"] == O.OK
    np.testing.assert_allclose(a["uC"], b["uC"], rtol=0, atol=1e-9)


def test_residual_definition():
    nx, nt, m, T = 24, 48, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=6)
    traj = serial_traj(u0, nt, T)
    uC = traj[::m].copy()
    assert O.residual(uC, nt, m, T) < 1e-14
    # perturbing only the last C-point changes only the last residual row
    d = np.random.default_rng(0).standard_normal(nx) * 1e-3
    uC[-1] += d
    assert O.residual(uC, nt, m, T) == pytest.approx(np.linalg.norm(d), rel=1e-9)


def test_mgrit_first_residual_matches_residual_routine():
    # the first recorded residual is that of the relaxed initial iterate;
    # with F-relaxation the C-points are untouched (all u0), so it equals
    # the residual of the constant-in-time C-point array
    nx, nt, m, T = 24, 48, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=7)
    r = O.mgrit(u0, nt, m, 2, T, relax=O.RELAX_F, tol=0.0, max_iter=0)
    uC = np.tile(u0, (nt // m + 1, 1))
    assert r["res_hist"][0] == pytest.approx(O.residual(uC, nt, m, T), rel=1e-12)


def test_divergence_is_reported():
    # coarse-level CFL far above the explicit limit (Sec. 4): rediscretised
    # coarse steps blow up and the solver reports divergence, not a hang
    u0 = inputs.sine_ic(64)
    r = O.mgrit(u0, 64, 8, 2, 0.5, tol=1e-10, max_iter=20)
    assert r["status"] == O.EDIVERGED
    nan = np.full(16, np.nan)
    r = O.mgrit(nan, 16, 2, 2, 0.1, tol=1e-10, max_iter=5)
    assert r["status"] == O.EDIVERGED and r["iters"] == 0


def test_invalid_arguments():
    u0 = np.zeros(16)
    assert O.mgrit(u0, 10, 4, 2, 0.1)["status"] == O.EINVAL     # nt % m != 0
    assert O.mgrit(u0, 16, 1, 2, 0.1)["status"] == O.EINVAL     # m < 2
    assert O.mgrit(u0, 16, 2, 1, 0.1)["status"] == O.EINVAL     # one level
    assert O.mgrit(u0, 16, 4, 4, 0.1)["status"] == O.EINVAL     # 16 % 4^3 != 0
    assert O.mgrit(np.zeros(4), 16, 4, 2, 0.1)["status"] == O.EINVAL   # WENO5 needs nx >= 5


# ---- F-cycle (Sec. 3.2, Fig. MGcycles) ----------------------------------

@pytest.mark.parametrize("levels", [3, 4])
@pytest.mark.parametrize("relax", [O.RELAX_F, O.RELAX_FCF])
def test_f_cycle_keeps_the_serial_fixed_point(levels, relax):
    # started on the serial trajectory, every FAS coarse correction of the
    # F-cycle's extra coarse visits is zero: cycles leave the C-points in place
    nx, nt, m, T = 32, 256, 2, 0.1
    u0 = inputs.fourier_ic(nx, seed=1)
    traj = serial_traj(u0, nt, T)
    r = O.mgrit(u0, nt, m, levels, T, relax=relax, uC_init=traj[::m], tol=0.0, max_iter=2,
                cycle=O.CYCLE_F)
    assert r["status"] == O.ENOTCONV
    assert np.all(r["res_hist"] < 1e-13)
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-14)


@pytest.mark.parametrize("levels", [3, 4])
@pytest.mark.parametrize("relax", [O.RELAX_F, O.RELAX_FCF])
def test_converged_f_cycle_equals_serial(levels, relax):
    nx, nt, m, T = 64, 256, 2, 0.2
    u0 = inputs.sine_ic(nx)
    r = O.mgrit(u0, nt, m, levels, T, relax=relax, tol=1e-10, max_iter=60, cycle=O.CYCLE_F)
    assert r["status"] == O.OK
    traj = serial_traj(u0, nt, T)
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-9)


def test_two_level_f_cycle_is_the_v_cycle():
    # with one coarse level both cycles visit it once per cycle
    nx, nt, m, T = 40, 128, 4, 0.1
    u0 = inputs.fourier_ic(nx, seed=8)
    v = O.mgrit(u0, nt, m, 2, T, tol=1e-12, cycle=O.CYCLE_V)
    f = O.mgrit(u0, nt, m, 2, T, tol=1e-12, cycle=O.CYCLE_F)
    assert v["iters"] == f["iters"]
    np.testing.assert_array_equal(v["res_hist"], f["res_hist"])
    np.testing.assert_array_equal(v["uC"], f["uC"])


@pytest.mark.parametrize("scheme", [O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE])
def test_f_cycle_brute_force_monolithic_residual_tiny(scheme):
    nx, nt, m, levels, T = 16, 16, 2, 3, 0.05
    u0 = inputs.fourier_ic(nx, seed=4)
    r = O.mgrit(u0, nt, m, levels, T, scheme=scheme, tol=1e-12, max_iter=40, want_full=True,
                cycle=O.CYCLE_F)
    assert r["status"] == O.OK
    u = r["u"]
    worst = max(np.abs(u[n] - O.step(u[n - 1], T / nt, scheme)).max() for n in range(1, nt + 1))
    assert worst < 1e-11


def test_f_cycle_iterates_conserve_mass():
    nx, nt, m, T = 48, 256, 4, 0.15
    u0 = inputs.fourier_ic(nx, seed=5)
    r = O.mgrit(u0, nt, m, 4, T, tol=0.0, max_iter=2, cycle=O.CYCLE_F)
    assert np.abs(r["uC"].sum(axis=1) - u0.sum()).max() < 1e-11 * nx


def test_f_cycle_needs_fewer_cycles_on_a_smooth_case():
    # the extra coarse visits give the F-cycle a better coarse correction
    # (3 vs 5 cycles at 3 levels, 4 vs 7 at 4 levels on this case)
    u0 = inputs.fourier_ic(64, seed=3)
    for levels in (3, 4):
        v = O.mgrit(u0, 1024, 4, levels, 0.1, tol=1e-11, cycle=O.CYCLE_V)
        f = O.mgrit(u0, 1024, 4, levels, 0.1, tol=1e-11, cycle=O.CYCLE_F)
        assert v["status"] == f["status"] == O.OK
        assert f["iters"] < v["iters"]


# ---- matched coarse integrators (Sec. 3.3) -------------------------------

@pytest.mark.parametrize("coarse", [O.COARSE_PSI0, O.COARSE_PSI1])
def test_matched_coarse_integrators_keep_the_fine_fixed_point(coarse):
    # the coarse integrator changes convergence, never the answer: converged
    # MGRIT equals serial stepping of the fine scheme, Eq. (fineLF)
    nx, nt, m, L, T = 64, 512, 2, 5, 0.475
    u0 = inputs.sine_ic(nx, offset=0.0)
    r = O.mgrit(u0, nt, m, L, T, scheme=O.SCHEME_LF_FE, relax=O.RELAX_F, coarse=coarse,
                tol=1e-11, max_iter=40)
    assert r["status"] == O.OK
    traj = serial_traj(u0, nt, T, scheme=O.SCHEME_LF_FE)
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-10)


def _errors(coarse, ncycles, nx=64, nt=512, ic="stationary"):
    # relative space-time L2 error of the level-0 C-points after k cycles
    # (Sec. 4 setting: 5 levels, m = 2, T = 0.475, F-relaxation, V-cycle)
    u0 = inputs.sine_ic(nx, offset=0.0) if ic == "stationary" else inputs.sine_ic(nx, 0.5, 0.5)
    ser = serial_traj(u0, nt, 0.475, scheme=O.SCHEME_LF_FE)[::2]
    out = []
    for k in range(1, ncycles + 1):
        r = O.mgrit(u0, nt, 2, 5, 0.475, scheme=O.SCHEME_LF_FE, relax=O.RELAX_F,
                    coarse=coarse, tol=0.0, max_iter=k)
        e = np.linalg.norm(r["uC"] - ser) / np.linalg.norm(ser)
        out.append(e if np.isfinite(e) else np.inf)
    return np.array(out)


@pytest.mark.parametrize("ic", ["stationary", "moving"])
def test_paper_claim_matching_restores_convergence(ic):
    # Sec. 4 (fine-integrator matching): rediscretisation blows up within a few
    # cycles, zeroth-order matching converges, first-order matching faster
    red = _errors(O.COARSE_REDISC, 4, ic=ic)
    p0 = _errors(O.COARSE_PSI0, 4, ic=ic)
    p1 = _errors(O.COARSE_PSI1, 4, ic=ic)
    assert red.max() > 1.0
    assert np.all(np.diff(p0) < 0) and np.all(np.diff(p1) < 0)
    assert np.all(p1 < p0)
    assert p1[3] < 1e-6


def test_matched_integrators_need_the_lf_fine_scheme():
    u0 = inputs.sine_ic(32)
    r = O.mgrit(u0, 64, 2, 3, 0.1, coarse=O.COARSE_PSI1)
    assert r["status"] == O.EINVAL


@pytest.mark.parametrize("scheme", [O.SCHEME_WENO5_SSPRK3, O.SCHEME_FO_FE])
def test_roe_flux_mgrit_converges_to_serial(scheme):
    nx, nt, m, T = 64, 256, 4, 0.2
    u0 = inputs.sine_ic(nx, offset=0.0)        # transonic: the entropy fix is exercised
    r = O.mgrit(u0, nt, m, 3, T, scheme=scheme, numflux=O.NUMFLUX_ROE, tol=1e-11, max_iter=40)
    assert r["status"] == O.OK
    traj = serial_traj(u0, nt, T, scheme=scheme, numflux=O.NUMFLUX_ROE)
    np.testing.assert_allclose(r["uC"], traj[::m], rtol=0, atol=1e-10)
