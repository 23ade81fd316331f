"""The WENO tables the paper prints for k = 2 (Sec. 2.1.1, after Eq. D),
stored in tests/golden/weno5_k2_tables.txt, against (a) their definitions,
derived here in exact rational arithmetic, and (b) the oracle's
reconstruction, probed on unit vectors.

(a) pins the printed values themselves (and the reading of their row order:
row r acts on the stencil {i-r, i-r+1, i-r+2}): the candidate coefficients
are the interface values of the quadratics with given cell averages
(Eq. C), the linear weights make the combination the 5-cell quartic
reconstruction (Eq. D), and B_r is the integral of Eq. (B) written as a
quadratic form.  (b) pins the oracle to the printed values through its
outputs only (candidates, indicators, weights).
"""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "weno5_k2_tables.txt")


def load_tables(path=GOLDEN):
    """{name: list of rows of Fractions}, each entry times its table's scale."""
    tables, name, scale = {}, None, None
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                head, rest = line.split("]", 1)
                name = head[1:]
                word, frac = rest.split()
                assert word == "scale"
                scale = Fr(frac)
                tables[name] = []
                continue
            tables[name].append([int(v) * scale for v in line.split()])
    return tables


T = load_tables()


# ---- exact derivations (cell i = [0, 1], cell i+m = [m, m+1], x_{i+1/2} = 1) ----

def cell_moment(j, d):
    """Average of x^d over the cell [j, j+1]."""
    return Fr((j + 1) ** (d + 1) - j ** (d + 1), d + 1)


def inverse(M):
    """Inverse of a square matrix of Fractions (Gauss-Jordan)."""
    n = len(M)
    A = [list(row) + [Fr(int(i == k)) for k in range(n)] for i, row in enumerate(M)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [v / p for v in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [row[n:] for row in A]


def poly_from_averages(cells):
    """Matrix taking the averages over `cells` to the monomial coefficients
    of the polynomial of degree len(cells) - 1 with those averages."""
    n = len(cells)
    return inverse([[cell_moment(j, d) for d in range(n)] for j in cells])


def interface_row(cells):
    """Coefficients of the cell averages in the polynomial's value at x = 1."""
    Minv = poly_from_averages(cells)
    n = len(cells)
    return [sum(Minv[d][col] for d in range(n)) for col in range(n)]


def stencil(r):
    return [-r, -r + 1, -r + 2]


def derived_c():
    return [interface_row(stencil(r)) for r in range(3)]


def derived_d():
    """d_r with sum_r d_r (candidate r on the 5 cells) = the quartic's value."""
    c5 = interface_row([-2, -1, 0, 1, 2])
    cand = []
    for r, row in enumerate(derived_c()):
        full = [Fr(0)] * 5
        for col, v in enumerate(row):
            full[2 - r + col] = v
        cand.append(full)
    # cell i-2 is on stencil 2 only, cell i+2 on stencil 0 only
    d2 = c5[0] / cand[2][0]
    d0 = c5[4] / cand[0][4]
    d1 = (c5[1] - d2 * cand[2][1]) / cand[1][1]
    d = [d0, d1, d2]
    for m in range(5):   # the two remaining equations hold as well
        assert sum(d[r] * cand[r][m] for r in range(3)) == c5[m]
    return d


def derived_B(r):
    """Eq. (B) with dx = 1: int_0^1 (p')^2 + (p'')^2 dx for p = a0 + a1 x + a2 x^2,
    i.e. a^T Q a, Q = [[0,0,0],[0,1,1],[0,1,4/3+4]]; a = Minv s."""
    Minv = poly_from_averages(stencil(r))
    Q = [[Fr(0), Fr(0), Fr(0)], [Fr(0), Fr(1), Fr(1)], [Fr(0), Fr(1), Fr(4, 3) + 4]]
    return [[sum(Minv[a][x] * Q[a][b] * Minv[b][y] for a in range(3) for b in range(3)) for y in range(3)]
            for x in range(3)]


def test_golden_file_shapes():
    assert [len(T["c"]), len(T["c"][0])] == [3, 3]
    assert [len(T["d"]), len(T["d"][0])] == [1, 3]
    for r in range(3):
        assert [len(T["B%d" % r]), len(T["B%d" % r][0])] == [3, 3]


def test_printed_candidate_rows_are_the_cell_average_reconstructions():
    assert derived_c() == T["c"]


def test_printed_candidate_rows_need_the_right_to_left_stencil_order():
    # on the stencils {i+r-2, .., i+r} the rows come out reversed: the
    # printed order is the stencil {i-r, .., i-r+2}
    flipped = [interface_row([r - 2, r - 1, r]) for r in range(3)]
    assert flipped != T["c"] and flipped == T["c"][::-1]


def test_printed_linear_weights_give_the_quartic_reconstruction():
    assert derived_d() == T["d"][0]
    assert sum(T["d"][0]) == 1


@pytest.mark.parametrize("r", range(3))
def test_printed_smoothness_matrices_are_the_integral_of_eq_B(r):
    assert derived_B(r) == T["B%d" % r]


# ---- the oracle against the printed values ------------------------------------

def unit(m):
    q = np.zeros(5)
    q[m] = 1.0
    return q


def test_oracle_candidates_are_the_printed_rows():
    c = np.array(T["c"], dtype=float)
    for m in range(5):
        _, p, _, _ = O.weno5_left(unit(m))
        for r in range(3):
            col = m - (2 - r)   # oracle input q[0..4] = q_{i-2..i+2}
            want = c[r][col] if 0 <= col <= 2 else 0.0
            assert abs(p[r] - want) <= 1e-15, (m, r, p[r], want)


def test_oracle_indicators_are_the_printed_forms():
    # recover each B_r from the oracle's beta_r by polarisation
    got = np.zeros((3, 3, 3))
    for r in range(3):
        cells = [2 - r + k for k in range(3)]
        for a in range(3):
            for b in range(3):
                qa, qb = unit(cells[a]), unit(cells[b])
                bab = O.weno5_left(qa + qb)[2][r]
                ba = O.weno5_left(qa)[2][r]
                bb = O.weno5_left(qb)[2][r]
                got[r, a, b] = ba if a == b else 0.5 * (bab - ba - bb)
    for r in range(3):
        want = np.array(T["B%d" % r], dtype=float)
        np.testing.assert_allclose(got[r], want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("level", [0.0, 1.0, -3.5, 1e3])
def test_oracle_weights_of_a_constant_state_are_the_printed_d(level):
    v, p, beta, om = O.weno5_left(np.full(5, level))
    assert np.all(beta == 0.0)
    np.testing.assert_allclose(om, np.array(T["d"][0], dtype=float), rtol=0, atol=1e-15)
    assert v == pytest.approx(level, rel=1e-15, abs=0)
