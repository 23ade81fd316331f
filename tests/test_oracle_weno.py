"""Pins for the oracle's WENO reconstruction (Sec. 2.1.1, Eqs. C, B, omega, D).

Each check is derived from the definitions, not from the printed tables:
candidate values from exact cell averages of polynomials, smoothness
indicators from the integral in Eq. (B), the linear weights from 5th-order
exactness (Eq. D).
"""
import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle as O


def cell_avgs(coef, edges):
    """Exact averages of the polynomial with coefficients coef over the cells
    delimited by edges."""
    anti = P.polyint(coef)
    v = P.polyval(edges, anti)
    return (v[1:] - v[:-1]) / np.diff(edges)


# cells i-2..i+2 are [j, j+1] for j = -2..2 (dx = 1); interface x_{i+1/2} = 1
EDGES = np.arange(-2.0, 4.0)
XI = 1.0


@pytest.mark.parametrize("seed", range(8))
def test_candidates_exact_for_quadratics(seed):
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(3)
    q = cell_avgs(coef, EDGES)
    _, p, _, _ = O.weno5_left(q)
    exact = P.polyval(XI, coef)
    np.testing.assert_allclose(p, exact, rtol=0, atol=1e-13 * (1 + abs(exact)))


@pytest.mark.parametrize("seed", range(6))
def test_candidates_not_exact_for_cubics(seed):
    # a cubic breaks 3rd-order candidates (guards against a degenerate test)
    rng = np.random.default_rng(100 + seed)
    coef = np.r_[rng.standard_normal(3), 1.0]
    q = cell_avgs(coef, EDGES)
    _, p, _, _ = O.weno5_left(q)
    assert np.all(np.abs(p - P.polyval(XI, coef)) > 1e-3)


def quad_on_stencil(vals, cells):
    """Quadratic whose averages over the three given unit cells are vals."""
    M = np.zeros((3, 3))
    for row, j in enumerate(cells):
        for d in range(3):
            M[row, d] = ((j + 1.0) ** (d + 1) - j ** (d + 1.0)) / (d + 1)
    return np.linalg.solve(M, vals)


def beta_from_integral(coef, h=1.0):
    """Eq. (B): sum_{l=1}^{2} int_{cell i} h^{2l-1} (d^l q/dx^l)^2 dx, cell i = [0, 1]."""
    tot = 0.0
    for l in (1, 2):
        d = P.polyder(coef, l)
        sq = P.polymul(d, d)
        anti = P.polyint(sq)
        tot += h ** (2 * l - 1) * (P.polyval(1.0, anti) - P.polyval(0.0, anti))
    return tot


@pytest.mark.parametrize("seed", range(10))
def test_smoothness_indicators_match_integral_definition(seed):
    rng = np.random.default_rng(200 + seed)
    q = rng.standard_normal(5)
    _, p, beta, _ = O.weno5_left(q)
    # the three 3-cell windows of the 5 cells, as offsets from cell i
    windows = [(0, 1, 2), (-1, 0, 1), (-2, -1, 0)]
    got = {}
    for r_cells in windows:
        vals = np.array([q[c + 2] for c in r_cells])
        coef = quad_on_stencil(vals, r_cells)
        got[r_cells] = (beta_from_integral(coef), P.polyval(XI, coef))
    # each (indicator, candidate) pair of the oracle corresponds to exactly one
    # window, and the three pairs use the three windows
    used = []
    for r in range(3):
        matches = [w for w, (b, v) in got.items()
                   if abs(b - beta[r]) <= 1e-11 * (1 + abs(b)) and abs(v - p[r]) <= 1e-12 * (1 + abs(v))]
        assert len(matches) == 1, (r, beta[r], p[r], got)
        used.append(matches[0])
    assert len(set(used)) == 3


@pytest.mark.parametrize("seed", range(6))
def test_fifth_order_exact_for_quartics_in_linear_weight_limit(seed):
    # with beta << eps the nonlinear weights equal the linear ones, and the
    # linear combination must be exact for quartics (Eq. D, s = 2k+1 = 5)
    rng = np.random.default_rng(300 + seed)
    amp = 1e-7
    coef = amp * rng.standard_normal(5)
    q = cell_avgs(coef, EDGES)
    w, p, beta, om = O.weno5_left(q)
    exact = P.polyval(XI, coef)
    assert np.all(beta < 1e-11)
    spread = np.max(np.abs(p - exact))
    assert spread > 1e-9          # candidates alone are not exact ...
    assert abs(w - exact) < 1e-4 * spread   # ... their weighted combination is


def test_constant_state_gives_linear_weights_and_exact_value():
    w, p, beta, om = O.weno5_left(np.full(5, 0.37))
    assert np.all(np.abs(beta) < 1e-15)     # zero up to rounding of the quadratic form
    assert w == pytest.approx(0.37, rel=0, abs=1e-15)
    # linear weights are the unique ones exact for quartics: recover them
    # from that property with three quartic probes and compare
    A = np.zeros((3, 3))
    b = np.zeros(3)
    for t, deg in enumerate((3, 4, 2)):
        coef = np.zeros(deg + 1); coef[deg] = 1.0
        q = cell_avgs(coef, EDGES)
        _, pc, _, _ = O.weno5_left(q)
        A[t] = pc
        b[t] = P.polyval(XI, coef)
    A[2] = 1.0; b[2] = 1.0   # weights sum to one
    d = np.linalg.solve(A, b)
    np.testing.assert_allclose(om, d, rtol=1e-8)   # beta/eps ~ 1e-10 perturbs omega


def test_eno_property_discontinuity():
    # a jump between cells i+1 and i+2 lies only in the stencil {i..i+2}
    q = np.array([1.0, 1.0, 1.0, 1.0, 5.0])
    _, p, beta, om = O.weno5_left(q)
    smooth = [r for r in range(3) if beta[r] == 0.0]
    rough = [r for r in range(3) if beta[r] > 1.0]
    assert len(smooth) == 2 and len(rough) == 1
    assert om[rough[0]] < 1e-10
    w, _, _, _ = O.weno5_left(q)
    assert abs(w - 1.0) < 1e-10


@pytest.mark.parametrize("ratio", [1.0, 0.25, 7.0])
def test_eps_is_one_millionth(ratio):
    # reading A6: eps = 1e-6.  Only the stencil {i, i+1, i+2} sees the
    # bump, so beta_1 = beta_2 = 0 and alpha_1 / alpha_0 = (d_1/d_0)
    # ((eps + beta_0) / eps)^2.  Scale the bump so that beta_0 = ratio * eps
    # (the indicator is quadratic in the data), then the weight ratio is
    # (d_1/d_0) (1 + ratio)^2 for eps = 1e-6, and far from it for 1e-5.
    unit = np.array([0.0, 0.0, 0.0, 0.0, 1.0])
    _, _, b1, _ = O.weno5_left(unit)
    r0 = int(np.argmax(b1))
    assert b1[r0] > 0 and np.count_nonzero(b1) == 1
    q = unit * np.sqrt(ratio * 1e-6 / b1[r0])
    _, _, beta, om = O.weno5_left(q)
    assert beta[r0] == pytest.approx(ratio * 1e-6, rel=1e-12)
    others = [r for r in range(3) if r != r0]
    for r in others:
        d_ratio = om[r] / om[r0]
        # the linear weights from a constant state (beta = 0)
        _, _, _, lin = O.weno5_left(np.zeros(5))
        assert d_ratio == pytest.approx(lin[r] / lin[r0] * (1.0 + ratio) ** 2, rel=1e-10)
        assert abs(d_ratio - lin[r] / lin[r0] * (1.0 + ratio / 10.0) ** 2) > 1e-3 * d_ratio
