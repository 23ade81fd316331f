"""The bench's multi-rank logic on CPU with the gloo backend (world size 2):
replicas only, so the one exchange is the max of the per-rank times; the
whole-job rate counts the units of all ranks; non-zero ranks of the oracle
arm exit without work or output, and rank 0 prints the contract's line."""
import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    b = _bench()
    ms = [120.0, 80.0][rank]              # this rank's own timed region
    got = b.max_over_ranks(ms, ws)
    rate = b.whole_job_rate(ws, 1000.0, 5, got)
    out.put((rank, got, rate))
    tdist.barrier()
    tdist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the rate counts both replicas
    assert [r[1] for r in res] == [120.0, 120.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 1000.0 * 5 / 0.120)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(42.0, 1) == 42.0
    assert b.whole_job_rate(1, 10.0, 3, 1000.0) == pytest.approx(30.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])

    def no_work(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")
    monkeypatch.setattr(b, "oracle_cycle_rate", no_work)
    assert b.main() == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    # the oracle arm's JSON line on a tiny sample: the contract's keys, its
    # own rate as cpu_baseline and e2e, and no host<->device bytes
    import json
    b = _bench()
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(b, "SAMPLE", dict(nx=64, nt=64, m=4, levels=2, T=0.05, seed=0))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert b.main() == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "cell-updates/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "nx=64" in d["config"]["workload"] and "nt=16384" in d["config"]["sample_of"]
    steps_updates = b.cycle_updates(b.SAMPLE) * 2
    assert d["value"] == pytest.approx(steps_updates / (d["ms_per_step"] * 2 / 1e3), rel=1e-9)
