"""The sequential chains (serial stepping, the coarsest solve of Eq. coarseCorr)
run on one CTA, on a thread-block cluster or on the grid stepper (one CTA per
SM, boundary cells and partial maxima through global memory, one bounded
wait per RK stage).  All three perform the same floating-point operations per
cell, so they must give the same bits; each must match the oracle's serial
stepping (Sec. 3.1: forward substitution); and a wait that can never complete
must end the launch with MGRIT_ETIMEOUT and leave the context usable."""
import time

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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(got, ref):
    return float(np.abs(np.asarray(got) - ref).max() / np.abs(ref).max())


CASES = [
    # nx, scheme, flux, precision, steps
    (4096, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, 64, 48),
    (2048, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, 64, 48),
    (1000, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, 64, 40),
    (777, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, 64, 40),
    (3000, O.SCHEME_FO_FE, O.FLUX_BURGERS, 64, 64),
    (4096, O.SCHEME_WENO5_SSPRK3, O.FLUX_BURGERS, 32, 48),
    (1500, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION, 32, 40),
]


@pytest.mark.parametrize("nx,scheme,flux,prec,steps", CASES)
def test_one_cta_cluster_and_grid_steppers_agree_bitwise_and_with_the_oracle(M, nx, scheme, flux,
                                                                             prec, steps):
    u0 = inputs.fourier_ic(nx, seed=nx + 1)
    speed = np.abs(u0).max() if flux == O.FLUX_BURGERS else 1.0
    T = 0.5 * steps / (nx * speed)          # CFL 0.5
    outs, used = {}, {}
    for k, name in ((M.SEQ_ONE_CTA, "cta"), (M.SEQ_CLUSTER, "cluster"), (M.SEQ_GRID, "grid")):
        s = M.Solver(nx, steps, 2, 2, scheme, flux, T=T, precision=prec, seq_stepper=k)
        outs[name] = s.serial_step(dev(u0), steps)
        torch.cuda.synchronize()
        used[name] = (s.query(2), s.query(3))
        s.sync_status()
        s.close()
    # the forced shapes were taken (every case here fits all three)
    assert used["cta"] == (1, 0)
    assert used["cluster"][0] >= 2 and used["cluster"][1] == 0
    assert used["grid"][0] == 0 and used["grid"][1] >= 8
    assert torch.equal(outs["cta"], outs["cluster"])
    assert torch.equal(outs["cta"], outs["grid"])
    ref = O.serial(u0, T / steps, steps, scheme, flux)
    assert relerr(outs["grid"].cpu().numpy(), ref) <= (1e-11 if prec == 64 else 1e-4)


def test_mgrit_with_grid_coarsest_solve_matches_oracle(M):
    # two levels at the bench width: the coarsest solve (1024 steps of
    # nx = 4096) runs on the grid stepper
    nx, nt, m, L, T = 4096, 4096, 4, 2, 0.25
    u0 = inputs.fourier_ic(nx, seed=0)
    s = M.Solver(nx, nt, m, L, T=T, max_iter=40, seq_stepper=M.SEQ_GRID)
    st, uT, uC, stats = s.solve(dev(u0))
    assert s.query(3) >= 8
    ref = O.mgrit(u0, nt, m, L, T, max_iter=40)
    assert st == ref["status"] == M.OK and stats.iters == ref["iters"]
    assert relerr(uC.cpu().numpy(), ref["uC"]) <= 1e-11


def test_grid_wait_is_bounded(M):
    # one CTA never publishes its first stage: the waits of the CTAs that read
    # it run out (0.5 s), the launch ends, and the status says so
    nx, n = 4096, 16
    u0 = inputs.fourier_ic(nx, seed=5)
    T = 0.25 * n / nx
    s = M.Solver(nx, n, 2, 2, T=T, seq_stepper=M.SEQ_GRID)
    s.serial_step(dev(u0), 1)
    s.sync_status()
    t0 = time.time()
    st = s.test_grid_timeout()
    assert st == M.ETIMEOUT
    assert time.time() - t0 < 20.0
    # the flag was cleared and the context (and device) still compute
    out = s.serial_step(dev(u0), n)
    s.sync_status()
    assert relerr(out.cpu().numpy(), O.serial(u0, T / n, n)) <= 1e-11
