"""Batched instances (uneven nx, nt, levels and flux in one launch per phase):
every instance must reproduce the single-instance solver, in FP64 and FP32
sweeps, before and after the autotuner changes its CTA shape, and converged
instances must be masked out while the others continue.  Batched and single
launches run the same slab code; where a coarsest solve runs on a different
kernel (single CTA vs cluster) the compiler may contract multiply-adds
differently, so agreement is to 1e-12 relative (in practice bitwise)."""
import numpy as np
import pytest

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


MIXED = [
    dict(nx=64, nt=256, m=2, levels=3, flux=0, T=0.2),
    dict(nx=100, nt=128, m=4, levels=3, flux=1, T=0.1),
    dict(nx=512, nt=256, m=4, levels=2, flux=0, T=0.02),
    dict(nx=777, nt=64, m=4, levels=3, flux=1, T=0.02),
    dict(nx=128, nt=256, m=4, levels=2, flux=0, T=0.25),
    dict(nx=2048, nt=128, m=2, levels=4, flux=0, T=0.004),
]


def single_cpoints(M, d, u0, ncycles, precision, **params):
    # batches run one CTA per chunk; so does the reference context here
    s = M.Solver(d["nx"], d["nt"], d["m"], d["levels"], 0, d["flux"], T=d["T"], precision=precision,
                 chunk_clusters=0, **params)
    s.run_cycles(dev(u0), ncycles)
    torch.cuda.synchronize()
    return s.cpoints()


def close(a, b):
    return float((a - b).abs().max()) <= 1e-12 * float(b.abs().max())


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_cycles_match_single_instances(M, precision):
    u0s = [inputs.fourier_ic(d["nx"], seed=k) for k, d in enumerate(MIXED)]
    b = M.Batch(MIXED, precision=precision)
    b.run_cycles([dev(u) for u in u0s], 2)
    torch.cuda.synchronize()
    for k, d in enumerate(MIXED):
        ref = single_cpoints(M, d, u0s[k], 2, precision)
        assert close(b.cpoints(k), ref), k


# deeper hierarchies, so that the instances' F-cycle launch orders differ
F_MIXED = MIXED + [
    dict(nx=256, nt=512, m=2, levels=5, flux=0, T=0.025),
    dict(nx=160, nt=1024, m=4, levels=4, flux=1, T=0.05),
]


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_f_cycles_match_single_instances(M, precision):
    # batched F-cycle phases interleave the instances' own launch orders
    u0s = [inputs.fourier_ic(d["nx"], seed=40 + k) for k, d in enumerate(F_MIXED)]
    b = M.Batch(F_MIXED, precision=precision, cycle=M.CYCLE_F)
    b.run_cycles([dev(u) for u in u0s], 2)
    torch.cuda.synchronize()
    for k, d in enumerate(F_MIXED):
        ref = single_cpoints(M, d, u0s[k], 2, precision, cycle=M.CYCLE_F)
        assert close(b.cpoints(k), ref), k


def test_batch_f_cycle_solve_matches_single_solves(M):
    insts = [F_MIXED[0], F_MIXED[6], F_MIXED[7], MIXED[4]]
    u0s = [inputs.fourier_ic(d["nx"], seed=50 + k) for k, d in enumerate(insts)]
    b = M.Batch(insts, max_iter=40, cycle=M.CYCLE_F)
    uTs, status, iters, res = b.solve([dev(u) for u in u0s])
    for k, d in enumerate(insts):
        s = M.Solver(d["nx"], d["nt"], d["m"], d["levels"], 0, d["flux"], T=d["T"], max_iter=40,
                     cycle=M.CYCLE_F, chunk_clusters=0)
        st, uT, _, stats = s.solve(dev(u0s[k]))
        assert status[k] == st and iters[k] == stats.iters, (k, status, iters)
        if st == M.OK:
            assert close(uTs[k], uT), k
    # an F-cycle does more work per cycle than a V-cycle of the same hierarchy
    v = M.Batch(insts, max_iter=40)
    assert b.cycle_cell_updates() > v.cycle_cell_updates()


def test_autotuned_shapes_give_identical_results(M):
    u0s = [dev(inputs.fourier_ic(d["nx"], seed=10 + k)) for k, d in enumerate(MIXED)]
    b = M.Batch(MIXED, precision=32)
    b.run_cycles(u0s, 2)
    torch.cuda.synchronize()
    before = [b.cpoints(k) for k in range(len(MIXED))]
    ks_before = [b.query(k, 4) for k in range(len(MIXED))]
    b.autotune(u0s, reps=2)
    shapes = [(b.query(k, 0), b.query(k, 1)) for k in range(len(MIXED))]
    assert all(c in (1, 2, 4, 8, 16) and 32 <= t <= 512 for c, t in shapes)
    # one slab per CTA, and the coarsest solve's cluster size (one CTA below
    # 512 cells)
    assert all(b.query(k, 3) == 1 for k in range(len(MIXED)))
    ks = [b.query(k, 4) for k in range(len(MIXED))]
    assert all(K in (1, 2, 4, 8, 16) for K in ks)
    assert all(K == 1 for K, d in zip(ks, MIXED) if d["nx"] < 512)
    b.run_cycles(u0s, 2)
    torch.cuda.synchronize()
    for k in range(len(MIXED)):
        # every FP32 sweep shape gives the same bits; a coarsest solve moved
        # between one CTA and a cluster (FP64) differs in rounding, which the
        # FP32 copy of the coarse rows can turn into one-ulp FP32 differences
        got, ref = b.cpoints(k), before[k]
        rel = float((got - ref).abs().max() / ref.abs().max())
        assert rel <= (1e-12 if ks[k] == ks_before[k] else 1e-5), (k, rel, ks_before[k], ks[k])


def test_batch_solve_masks_converged_instances(M):
    # instances converge after different numbers of cycles (two-level
    # exactness bounds some by nt/m); each must match its own single solve
    insts = [MIXED[0], MIXED[4], dict(nx=96, nt=64, m=4, levels=2, flux=1, T=0.05), MIXED[1]]
    u0s = [inputs.fourier_ic(d["nx"], seed=20 + k) for k, d in enumerate(insts)]
    b = M.Batch(insts, max_iter=40)
    uTs, status, iters, res = b.solve([dev(u) for u in u0s])
    assert len(set(iters)) > 1          # genuinely different stopping cycles
    for k, d in enumerate(insts):
        s = M.Solver(d["nx"], d["nt"], d["m"], d["levels"], 0, d["flux"], T=d["T"], max_iter=40,
                     chunk_clusters=0)
        st, uT, _, stats = s.solve(dev(u0s[k]))
        assert status[k] == st and iters[k] == stats.iters, (k, status, iters)
        assert close(uTs[k], uT), k
        assert res[k] == pytest.approx(stats.res_hist[stats.iters], rel=1e-9, abs=1e-13)


def test_batch_relaxation_hook_leaves_cycles_unchanged(M):
    # the profiling hook reruns the batched level-0 relaxation; cycles started
    # afterwards from the initial iterate are the cycles of a fresh batch
    u0s = [dev(inputs.fourier_ic(d["nx"], seed=40 + k)) for k, d in enumerate(MIXED)]
    b = M.Batch(MIXED, precision=32)
    b.run_cycles(u0s, 1)
    b.launch_relax(2)
    b.run_cycles(u0s, 2)
    f = M.Batch(MIXED, precision=32)
    f.run_cycles(u0s, 2)
    torch.cuda.synchronize()
    for k in range(len(MIXED)):
        assert torch.equal(b.cpoints(k), f.cpoints(k))
    with pytest.raises(M.MGRITError):
        b.launch_relax(0)


def test_batch_rejects_unsupported_instances(M):
    with pytest.raises(M.MGRITError):
        M.Batch([dict(nx=64, nt=64, m=2, levels=2, flux=0, T=0.1, scheme=1)])
    with pytest.raises(M.MGRITError):
        M.Batch([dict(nx=16384, nt=64, m=2, levels=2, flux=0, T=0.01)], precision=32)
    with pytest.raises(M.MGRITError):
        M.Batch([dict(nx=64, nt=60, m=4, levels=3, flux=0, T=0.1)])


def test_uneven_batch_workload_runs(M):
    # a reduced instance of the 64-instance uneven workload (8 instances)
    insts, u0s = inputs.batch_workload(seed=3, n=8)
    b = M.Batch(insts, precision=32)
    b.run_cycles([dev(u) for u in u0s], 1)
    torch.cuda.synchronize()
    for k, d in enumerate(insts):
        uC = b.cpoints(k)
        assert uC.shape == (d["nt"] // d["m"] + 1, d["nx"])
        # FP32 sweeps: the C-point rows hold u0 rounded to FP32
        assert torch.equal(uC[0], dev(u0s[k]).float().double())


# ----------------------------------------------- batched solves vs the oracle ---
# Every instance of an uneven batch must solve its own problem: the batched
# C-points and u(T) are compared with the oracle's Algorithm 1 on that
# instance alone (Sec. 3.2), with the same outcome and cycle count, so that
# an instance mapped to the wrong arguments, masked at the wrong cycle or
# relaxed with another instance's step would fail here even if the
# single-instance path shared the mistake.
ORACLE_MIX = [
    dict(nx=64, nt=256, m=2, levels=3, flux=0, T=0.2),
    dict(nx=100, nt=128, m=4, levels=2, flux=1, T=0.1),
    dict(nx=512, nt=256, m=4, levels=2, flux=0, T=0.02),
    dict(nx=777, nt=64, m=4, levels=3, flux=1, T=0.004),
    dict(nx=128, nt=256, m=4, levels=2, flux=0, T=0.25),
    dict(nx=2048, nt=128, m=2, levels=3, flux=0, T=0.004),
    dict(nx=256, nt=512, m=2, levels=5, flux=0, T=0.025),
    dict(nx=160, nt=1024, m=4, levels=4, flux=1, T=0.05),
    dict(nx=1000, nt=256, m=4, levels=3, flux=1, T=0.01),
    dict(nx=4096, nt=64, m=4, levels=2, flux=0, T=0.001),
]
ORACLE_SEED = 100


def oracle_solve(d, u0, cycle):
    import oracle as O
    return O.mgrit(u0, d["nt"], d["m"], d["levels"], d["T"], flux=d["flux"], max_iter=40,
                   cycle=cycle)


def rel_max(got, ref):
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(got) - ref).max() / np.abs(ref).max())


def near_tol(hist, tol=1e-10):
    return bool(np.any(np.abs(np.asarray(hist) - tol) <= 1e-3 * tol))


@pytest.mark.parametrize("tuned", [False, True], ids=["rule", "autotuned"])
@pytest.mark.parametrize("cycle", [0, 1], ids=["V", "F"])
def test_batch_solve_matches_oracle_fp64(M, cycle, tuned):
    import oracle as O
    u0s = [inputs.fourier_ic(d["nx"], seed=ORACLE_SEED + k) for k, d in enumerate(ORACLE_MIX)]
    du0 = [dev(u) for u in u0s]
    b = M.Batch(ORACLE_MIX, max_iter=40, cycle=cycle)
    if tuned:
        b.autotune(du0, reps=2)
    uTs, status, iters, res = b.solve(du0)
    assert len(set(iters)) > 1   # instances stop (and are masked) at different cycles
    for k, d in enumerate(ORACLE_MIX):
        ref = oracle_solve(d, u0s[k], cycle)
        assert status[k] == ref["status"] == O.OK, (k, status[k], ref["status"])
        if not near_tol(ref["res_hist"]):
            assert iters[k] == ref["iters"], (k, iters[k], ref["iters"])
        # the masked instance keeps the C-points of its own final cycle
        assert rel_max(b.cpoints(k).cpu().numpy(), ref["uC"]) <= 1e-11, k
        assert rel_max(uTs[k].cpu().numpy(), ref["uT"]) <= 1e-11, k
        floor = 1e-14 * np.abs(ref["uC"]).max() * np.sqrt(ref["uC"].size)
        assert res[k] == pytest.approx(ref["res_hist"][ref["iters"]], rel=1e-8, abs=floor), k


@pytest.mark.parametrize("tuned", [False, True], ids=["rule", "autotuned"])
def test_batch_fp32_solve_within_bound_of_oracle(M, tuned):
    # FP32 sweeps stop at the FP32 fixed point (or on stagnation); their
    # result is compared with the FP64 oracle's converged solution within the
    # stated FP32 bound: relative max-norm 1e-4, relative L1 5e-5
    import oracle as O
    u0s = [inputs.fourier_ic(d["nx"], seed=ORACLE_SEED + k) for k, d in enumerate(ORACLE_MIX)]
    du0 = [dev(u) for u in u0s]
    b = M.Batch(ORACLE_MIX, max_iter=40, precision=32)
    if tuned:
        b.autotune(du0, reps=2)
    uTs, status, iters, res = b.solve(du0)
    for k, d in enumerate(ORACLE_MIX):
        ref = oracle_solve(d, u0s[k], 0)
        assert status[k] == O.OK, (k, status[k])
        got = uTs[k].cpu().numpy()
        assert rel_max(got, ref["uT"]) <= 1e-4, k
        assert np.abs(got - ref["uT"]).sum() / np.abs(ref["uT"]).sum() <= 5e-5, k
        uC = b.cpoints(k).cpu().numpy()
        assert rel_max(uC, ref["uC"]) <= 1e-4, k
