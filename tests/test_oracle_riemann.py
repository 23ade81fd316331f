"""Pins of the oracle's shocked Burgers solutions against the exact entropy
solution of a periodic Riemann problem (Sec. 2, Eq. burgers; the schemes of
Secs. 2.1.1-2.2).

u0 = a on (x1, x2), b elsewhere on the unit circle, a > b.  Until the fan
head meets the shock the entropy solution is
  u = b                  for x < x1 + b t,
  u = (x - x1) / t       on the rarefaction fan x1 + b t <= x <= x1 + a t,
  u = a                  up to the shock at x2 + s t, s = (a + b) / 2
                         (Rankine-Hugoniot for f = u^2 / 2),
  u = b                  beyond it.
The exact cell averages of that function are compared with the oracle's
serial stepping at three resolutions.  A conservative, entropy-satisfying
scheme converges to it in L1 at first order (the discontinuity and the fan's
corners limit the rate), puts the shock where the Rankine-Hugoniot speed
does, and the WENO5 schemes stay within O(1e-4) of the data's bounds.  A
wrong flux, sign, speed or upwind direction fails at least one of these.
With b < 0 < a the fan is transonic, where a scheme that ignores the
entropy condition keeps an expansion shock.
"""
import numpy as np
import pytest

import oracle as O

X1, X2, T = 0.2, 0.5, 0.3
CFL = 0.4

SCHEMES = {
    "weno5-lf-split": (O.SCHEME_WENO5_SSPRK3, O.NUMFLUX_LF_SPLIT),
    "weno5-lf-state": (O.SCHEME_WENO5_SSPRK3, O.NUMFLUX_LF_STATE),
    "weno5-roe": (O.SCHEME_WENO5_SSPRK3, O.NUMFLUX_ROE),
    "first-order-lf": (O.SCHEME_FO_FE, O.NUMFLUX_LF_SPLIT),
}


def initial_averages(nx, a, b):
    # x1 and x2 are cell edges at the resolutions used, so these are exact
    c = (np.arange(nx) + 0.5) / nx
    return np.where((c > X1) & (c < X2), a, b)


def exact_averages(nx, a, b, t=T):
    s = 0.5 * (a + b)
    f0, f1, xs = X1 + b * t, X1 + a * t, X2 + s * t
    assert 0.0 <= f0 < f1 < xs < 1.0   # before the fan meets the shock

    def antiderivative(x):
        fan = np.clip(x, f0, f1)
        return (b * np.minimum(x, f0) + ((fan - X1) ** 2 - (f0 - X1) ** 2) / (2 * t)
                + a * np.clip(x - f1, 0.0, xs - f1) + b * np.clip(x - xs, 0.0, None))

    edges = np.linspace(0.0, 1.0, nx + 1)
    return np.diff(antiderivative(edges)) * nx


def solve(nx, a, b, scheme):
    sch, nf = SCHEMES[scheme]
    nt = int(np.ceil(T * nx * max(abs(a), abs(b)) / CFL))
    return O.serial(initial_averages(nx, a, b), T / nt, nt, scheme=sch, numflux=nf)


def shock_position(u, nx, a, b):
    """Right edge of the last cell above the shock's mid value."""
    mid = 0.5 * (a + b)
    j = np.where((u[:-1] >= mid) & (u[1:] < mid))[0]
    assert len(j) == 1
    return (j[0] + 1) / nx


STATES = [pytest.param(1.0, 0.0, id="sonic-fan-edge"), pytest.param(1.0, -0.5, id="transonic-fan")]


@pytest.mark.parametrize("a,b", STATES)
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_riemann_problem_converges_to_the_entropy_solution(scheme, a, b):
    weno = scheme.startswith("weno5")
    errs = []
    for nx in (200, 400, 800):
        u = solve(nx, a, b, scheme)
        errs.append(np.abs(u - exact_averages(nx, a, b)).mean())
        # conservation: the mean of u never changes
        assert abs(u.mean() - initial_averages(nx, a, b).mean()) < 1e-13
        # the shock sits where the Rankine-Hugoniot speed puts it
        assert abs(shock_position(u, nx, a, b) - (X2 + 0.5 * (a + b) * T)) <= 2.0 / nx
        # no oscillations beyond O(1e-4) (first order: none at all)
        slack = 1e-3 if weno else 1e-12
        assert u.min() >= b - slack and u.max() <= a + slack
    errs = np.array(errs)
    # L1 error of order dx, halving with dx (first order at the discontinuity;
    # the first-order scheme's fan corners converge a little slower)
    assert np.all(errs * np.array([200, 400, 800]) < (1.5 if weno else 8.0)), errs
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > (1.9 if weno else 1.6)), ratios


def test_exact_averages_conserve_mass_and_follow_the_rankine_hugoniot_speed():
    # the reference solution itself: its mean is the initial one (the shock
    # speed is exactly the one that conserves mass), and at t -> 0 it is the
    # initial data
    for a, b in ((1.0, 0.0), (1.0, -0.5)):
        for nx in (200, 800):
            ex = exact_averages(nx, a, b)
            assert abs(ex.mean() - initial_averages(nx, a, b).mean()) < 1e-14
            np.testing.assert_allclose(exact_averages(nx, a, b, t=1e-12), initial_averages(nx, a, b),
                                       atol=1e-9)
            # a wrong shock speed breaks conservation
            s_wrong = 0.6 * (a + b)
            xs = X2 + s_wrong * T
            edges = np.linspace(0.0, 1.0, nx + 1)
            moved = ex.copy()
            moved[(edges[:-1] >= X2 + 0.5 * (a + b) * T) & (edges[1:] <= xs)] = a
            assert abs(moved.mean() - ex.mean()) > 1e-3
