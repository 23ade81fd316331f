"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of oracle/mgrit_oracle.c (a wrong table entry, sign, index,
coefficient or step of Algorithm 1), compiles it with the oracle's own flags,
and runs the pin suite against it (MGRIT_ORACLE_LIB points the oracle's
loader at the copy).  Every mutant must fail at least one pin; the unchanged
source, built the same way, must pass them all.

Mistakes that cannot change any result are not listed: the centre row and
column of each B_r are never read (the quadratic form is evaluated on the
stencil minus its middle value), and the coarsest solve's first row is the
restricted u^0, which already equals g^0 (A8).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle.api import compile_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mgrit_oracle.c")
PINS = ["tests/test_oracle_weno.py", "tests/test_oracle_spatial.py", "tests/test_oracle_mgrit.py",
        "tests/test_golden_tables.py", "tests/test_oracle_riemann.py", "tests/test_oracle_adjoint.py"]

# name: (what it breaks, text, replacement, occurrence of the text)
MUTANTS = {
    # Sec. 2.1.1: the printed tables and the weights
    "c-table-sign": ("Eq. (C) row 0", "{  2.0,  5.0, -1.0 },", "{  2.0,  5.0,  1.0 },", 0),
    "d-reversed": ("Eq. (D) weights in stencil order", "TAB_D[3] = { 3.0, 6.0, 1.0 };",
                   "TAB_D[3] = { 1.0, 6.0, 3.0 };", 0),
    "b-corner": ("Eq. (B) matrix B_1", "{ {   8.0, -13.0,   5.0 }", "{ {   9.0, -13.0,   5.0 }", 0),
    "weight-exponent": ("Eq. (omega) exponent 2", "alpha[r] = (TAB_D[r] / 10.0) / (den * den);",
                        "alpha[r] = (TAB_D[r] / 10.0) / den;", 0),
    "stencil-order": ("reading A5 (row r on cells i-r..i-r+2)", "const double *s = &q[2 - r];",
                      "const double *s = &q[r];", 0),
    "weno-eps": ("reading A6 (eps = 1e-6)", "#define WENO_EPS 1e-6", "#define WENO_EPS 1e-5", 0),
    "periodic-wrap": ("periodic indices", "return i < 0 ? i + nx : i;", "return i < 0 ? i + nx - 1 : i;", 0),
    # Secs. 2, 2.1, 2.1.2: flux, splitting, divergence form
    "burgers-flux": ("Eq. (burgers) f = u^2/2", "return flux == ORC_FLUX_BURGERS ? 0.5 * u * u : u;",
                     "return flux == ORC_FLUX_BURGERS ? u * u : u;", 0),
    "lf-split-sign": ("Eq. (LFflux) splitting f+", "t1[j] = 0.5 * (phys_flux(flux, u[j]) + alpha * u[j]);",
                      "t1[j] = 0.5 * (phys_flux(flux, u[j]) - alpha * u[j]);", 0),
    "alpha-min": ("reading A4 (alpha is the maximum)", "if (s > alpha) alpha = s;", "if (s < alpha) alpha = s;", 0),
    "lf-state-sign": ("reading A2 (dissipative sign)", "- 0.5 * alpha * (t2[i] - t1[i]);",
                      "+ 0.5 * alpha * (t2[i] - t1[i]);", 0),
    "divergence-sign": ("Eq. (spaceDisc) sign", "A[i] = -(F[i] - F[wrap(i - 1, nx)]) / dx;",
                        "A[i] = (F[i] - F[wrap(i - 1, nx)]) / dx;", 0),
    "divergence-index": ("Eq. (spaceDisc) interfaces", "A[i] = -(F[i] - F[wrap(i - 1, nx)]) / dx;",
                         "A[i] = -(F[i] - F[wrap(i + 1, nx)]) / dx;", 0),
    "roe-half": ("Eq. (roeflux) dissipation 1/2", "- 0.5 * q * (up - um);", "- q * (up - um);", 0),
    "roe-no-entropy-fix": ("Eq. (roeflux) Harten-Hyman fix",
                           "double q = fabs(lam) < delta ? 0.5 * (lam * lam / delta + delta) : fabs(lam);",
                           "double q = fabs(lam);", 0),
    # Sec. 2.2 and Sec. 3.3: the integrators
    "ssprk3-stage2": ("Eq. (SSPRK3) stage 2",
                      "u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 4.0 * dt * A[i];",
                      "u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 2.0 * dt * A[i];", 0),
    "ssprk3-stage3": ("Eq. (SSPRK3) stage 3",
                      "out[i] = 1.0 / 3.0 * u[i] + 2.0 / 3.0 * u2[i] + 2.0 / 3.0 * dt * A[i];",
                      "out[i] = 1.0 / 3.0 * u[i] + 2.0 / 3.0 * u2[i] + 1.0 / 3.0 * dt * A[i];", 0),
    "lf-fine-sign": ("Eq. (fineLF) sign", "for (int i = 0; i < nx; ++i) out[i] = u1[i] - dt * A[i];",
                     "for (int i = 0; i < nx; ++i) out[i] = u1[i] + dt * A[i];", 0),
    "psi0-factor": ("Eq. (coarseLFord0) M dt", "for (int i = 0; i < nx; ++i) out[i] -= M * dt * b[i];",
                    "for (int i = 0; i < nx; ++i) out[i] -= dt * b[i];", 0),
    "psi1-powers": ("Eq. (coarseLFord1) powers of E", "op_E_pow(nx, M - i, a, t);          /* E^{M-i} u */",
                    "op_E_pow(nx, i - 1, a, t);          /* E^{M-i} u */", 0),
    # Sec. 3.2 and Algorithm 1
    "frelax-g-index": ("Eq. (relaxation) right-hand side",
                       "step_plus_g(M, l, row(M->u[l], nx, m * j + r - 1), m * j + r,",
                       "step_plus_g(M, l, row(M->u[l], nx, m * j + r - 1), m * j + r - 1,", 0),
    "frelax-range": ("reading A14 (m - 1 F-points per chunk)", "for (int r = 1; r < m; ++r)",
                     "for (int r = 1; r < m - 1; ++r)", 0),
    "fcf-without-c": ("FCF-relaxation", "        c_relax(M, l);\n        f_relax(M, l);\n",
                      "        f_relax(M, l);\n", 0),
    "residual-index": ("Eq. (restriction::rhs) residual",
                       "propagate(M, l, m * i, row(M->u[l], nx, m * i - 1), phi, work);",
                       "propagate(M, l, m * i, row(M->u[l], nx, m * i - 2 + (i == 0)), phi, work);", 0),
    "fas-tau-sign": ("Eq. (restriction::rhs) FAS term", "gc[c] = gl[c] + phi[c] - psi[c];",
                     "gc[c] = gl[c] - phi[c] + psi[c];", 0),
    "guess-drops-g": ("Eq. (restriction::u)", "uc[c] = (M->guess == ORC_GUESS_EQ17) ? phi[c] + gl[c] : ul[c];",
                      "uc[c] = (M->guess == ORC_GUESS_EQ17) ? phi[c] : ul[c];", 0),
    "coarse-g-index": ("Eq. (coarseCorr)",
                       "step_plus_g(M, l, row(M->u[l], nx, i - 1), i, row(M->u[l], nx, i), work);",
                       "step_plus_g(M, l, row(M->u[l], nx, i - 1), i - 1, row(M->u[l], nx, i), work);", 0),
    "restrict-without-g0": ("reading A8 (g^0 = u0 on every level)",
                            "memcpy(row(M->g[l + 1], nx, 0), row(M->g[l], nx, 0), sizeof(double) * (size_t)nx);",
                            "", 0),
    "inject-without-last": ("Eq. (interpolation) injection", "for (int i = 0; i <= nc; ++i)",
                            "for (int i = 0; i < nc; ++i)", 0),
    "stop-rule": ("reading A11 (stop when ||r|| < tol)", "if (rk < tol) { st = ORC_OK; break; }",
                  "if (rk < 10 * tol) { st = ORC_OK; break; }", 0),
    "interp-without-frelax": ("Eq. (interpolation) F-relaxation", "    if (do_frelax) f_relax(M, l);\n",
                              "    (void)do_frelax;\n", 0),
    "vcycle-without-recursion": ("Algorithm 1 below level 0",
                                 "        relax(M, l);\n        residual_restrict(M, l, 1);\n"
                                 "        vcycle_from(M, l + 1);\n        interpolate(M, l, 1);\n", "", 0),
    # the same four lines end the F-cycle: its V-cycle after the inner F-cycle
    "fcycle-without-vcycle": ("the F-cycle (reading A17)",
                              "        relax(M, l);\n        residual_restrict(M, l, 1);\n"
                              "        vcycle_from(M, l + 1);\n        interpolate(M, l, 1);\n", "", 1),
    # the discrete adjoint (transposed step)
    "adj-weight-exponent": ("adjoint: forward weights", "alpha[r] = (TAB_D[r] / 10.0) / (den * den);",
                            "alpha[r] = (TAB_D[r] / 10.0) / den;", 1),
    "adj-stencil-order": ("adjoint: stencil rows", "const double *s = &q[2 - r];", "const double *s = &q[r];", 1),
    "adj-weight-derivative": ("adjoint: d alpha / d beta",
                              "dadb[r] = -2.0 * (TAB_D[r] / 10.0) / (den * den * den);",
                              "dadb[r] = 2.0 * (TAB_D[r] / 10.0) / (den * den * den);", 0),
    "adj-mirror-gather": ("adjoint: mirrored stencil of f-", "mufm[wrap(i + 3 - j, nx)] += muF[i] * g[j];",
                          "mufm[wrap(i - 2 + j, nx)] += muF[i] * g[j];", 0),
    "adj-flux-difference": ("adjoint: transposed divergence", "muF[i] = (mu[wrap(i + 1, nx)] - mu[i]) / dx;",
                            "muF[i] = (mu[i] - mu[wrap(i + 1, nx)]) / dx;", 0),
    "adj-alpha-term": ("adjoint: alpha derivative", "mualpha += 0.5 * w[j] * (mufp[j] - mufm[j]);",
                       "mualpha += 0.5 * w[j] * (mufp[j] + mufm[j]);", 0),
    "adj-forward-stage2": ("adjoint: recomputed forward stage",
                           "u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 4.0 * dt * A[i];",
                           "u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 2.0 * dt * A[i];", 1),
    "adj-stage2-weight": ("adjoint: transposed stage 2", "lam_out[i] += 3.0 / 4.0 * l2[i];",
                          "lam_out[i] += 1.0 / 4.0 * l2[i];", 0),
}


def plant(src, text, new, occurrence):
    parts = src.split(text)
    assert len(parts) - 1 > occurrence, "mutation site not found"
    return text.join(parts[:occurrence + 1]) + new + text.join(parts[occurrence + 1:])


def run_pins(lib):
    env = dict(os.environ, MGRIT_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes():
    d = os.path.join(ROOT, "tests", "_build", "mutants.%d" % os.getpid())   # git-ignored
    os.makedirs(d, exist_ok=True)
    src = open(SRC).read()
    jobs = {"unchanged": src}
    for name, (_, text, new, occ) in MUTANTS.items():
        jobs[name] = plant(src, text, new, occ)

    def one(item):
        name, code = item
        c, so = os.path.join(d, name + ".c"), os.path.join(d, name + ".so")
        with open(c, "w") as fh:
            fh.write(code)
        compile_oracle(c, so)
        return name, run_pins(so)

    try:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            return dict(ex.map(one, jobs.items()))
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_unchanged_oracle_passes_the_pins(outcomes):
    rc, out = outcomes["unchanged"]
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    # 1 = a test failed (not a collection or usage error)
    assert rc == 1 and "failed" in out, (MUTANTS[name][0], rc, out)
