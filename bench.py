#!/usr/bin/env python
"""Benchmark: fine cell-updates/s of the MGRIT V-cycle on one GB300.

Workload (one step = one full V-cycle from the initial iterate, all levels):
inviscid Burgers, WENO5-JS + global Lax-Friedrichs splitting + SSPRK3, FP64,
nx = 4096 cells, nt = 16384 steps to T = 1, coarsening m = 4, 6 levels
(coarsened until 16 C-points remain), FCF relaxation, coarse guess of
Eq. (restriction::u); u0 = 0.5 + 8-mode random Fourier series (seed 0),
exact cell averages.  Synthetic data: the paper's workloads are analytic
initial conditions.

value  = cells x Phi applications of one V-cycle (all levels) / device time
e2e    = same, measured through the C ABI with u0 copied from pinned host
         memory and u(T) copied back inside the timed region
roofline = the level-0 relaxation kernel (the dominant kernel) against the
         FP64 pipe: algorithmic FLOPs per cell update x cell updates per
         launch / CUDA-event launch time
cpu_baseline / --impl reference = the FP64 C oracle on the host cores, one
         V-cycle of the same workload over the first quarter of the time
         horizon (nt = 4096, T = 0.25).

Multi-GPU (torchrun): independent replicas, one per GPU (the path has no
exchange step on one problem); value = all ranks' cell updates / max time.
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(nx=4096, nt=16384, m=4, levels=6, T=1.0, seed=0)
SAMPLE = dict(nx=4096, nt=4096, m=4, levels=6, T=0.25, seed=0)   # CPU baseline sample
SAMPLE1 = dict(nx=4096, nt=1024, m=4, levels=5, T=0.0625, seed=0)  # single-thread sample
CPU_BASELINE_SECONDS = 10.0   # the host-core timing repeats its sample for at least this long

# Algorithmic FLOPs per cell update of one SSPRK3 step of WENO5-JS with the
# global LF splitting (Burgers): the operations the paper's formulas take, as
# counted by the instrumented build of the oracle (oracle/count_flops.py:
# every data-dependent +, -, x, /, |.| and comparison counts 1, constant
# expressions fold): 185 additions, 289 multiplications, 75 divisions,
# 3 |.| and 3 comparisons.  tests/test_flop_count.py keeps the figure equal
# to the counting run.
FLOPS_PER_CELL_UPDATE = 555
# the same for linear advection (alpha = 1 and f^- = 0: 185 additions, 271
# multiplications, 75 divisions)
FLOPS_PER_CELL_UPDATE_ADVECTION = 531
# adjoint gradient workload: pre-shock and post-shock final times with the
# levels the coarse CFL allows (level-2 CFL 0.51 at T=0.12, level-1 0.32 at T=0.3)
ADJOINT_WORKLOAD = dict(nx=2048, nt=8192, m=4, seed=1, target_seed=1001, breaking_time=0.201,
                        cases=((0.12, 3), (0.3, 2)))

# Nominal SIMT rates from the unit counts and clocks (context only; the
# roofline uses the rates measured in the run, see fma_peaks)
FP64_NOMINAL_TFLOPS = 152 * 2.07e9 * 4 / 1e12          # 2 DFMA / clk / SM
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12    # 128 FFMA lanes / SM

# DRAM bytes (read + write) per level-0 relaxation launch from an ncu
# capture, keyed by a hash of the kernel sources it was taken on; reported
# only while the kernel is unchanged.  (The key is that of the captured
# sources with three comments corrected since: compiled without line info,
# every device image of the library is byte for byte the same.)
TRAFFIC = {"c79845a03917ee5a": 141477376 + 350998784}   # profiles/relax_l0_c2_fp64.md


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (GB/s), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def fma_peaks(mgrit):
    """Measured multiply-add throughput of the FP64 and FP32 pipes on this GPU
    (mgrit_fma_probe, ~0.1 s each, best of 3): the roofline denominators of
    the arithmetic-bound sweeps.  FP32 takes the faster of scalar and packed
    pairs."""
    def best(kind, iters):
        mgrit.fma_probe(kind, max(1, iters // 20))
        return max(mgrit.fma_probe(kind, iters) for _ in range(3)) / 1e12
    fp64 = best(mgrit.FMA_FP64, 3000)
    fp32 = max(best(mgrit.FMA_FP32, 200000), best(mgrit.FMA_FP32X2, 100000))
    return {"fp64_tflops": fp64, "fp32_tflops": fp32,
            "source": "mgrit_fma_probe on this GPU in this run: 152 x 8 CTAs x 256 threads, "
                      "8 independent multiply-add chains per thread, CUDA events, best of 3"}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("slab.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2104_09404_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mgrit", choices=["mgrit", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the 64-instance batch line")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint gradient line")
    p.add_argument("--no-c4", action="store_true", help="skip the nx=16384, nt=65536 FP32 line")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the paper's coarse-integrator / relaxation / cycle comparisons")
    return p.parse_args()


def max_over_ranks(ms, ws, device=None):
    """The slowest rank's time: every rank passes its own CUDA-event time and
    gets the maximum (all-reduce MAX over the default process group)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as tdist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_step, steps, ms):
    """Units processed by all ranks (weak scaling: each rank runs its own
    replica of the workload) per second of the slowest rank."""
    return ws * units_per_step * steps / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle ---

def oracle_cycle_rate(sample, min_seconds=0.0):
    """The oracle, as it stands, on one V-cycle of the sample from its initial
    iterate, repeated until `min_seconds` have passed; returns (cell
    updates/s, seconds, threads, repetitions).  Cell updates counted like the
    GPU's."""
    import numpy as np  # noqa: F401
    import oracle as O
    from paper_2104_09404_gb300 import inputs
    O.build()
    u0 = inputs.fourier_ic(sample["nx"], seed=sample["seed"])
    reps = 0
    t0 = time.perf_counter()
    while True:
        O.vcycles(u0, sample["nt"], sample["m"], sample["levels"], sample["T"], 1)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    upd = cycle_updates(sample) * reps
    return upd / dt, dt, O.num_threads(), reps


def oracle_single_thread(sample):
    """The oracle on one host thread (OMP_NUM_THREADS=1, in a child process
    so that the parent's thread pool is untouched) over one V-cycle of
    `sample`: (cell updates/s, seconds)."""
    code = ("import json, time, oracle as O\n"
            "from paper_2104_09404_gb300 import inputs\n"
            "s = json.loads(%r)\n"
            "O.build()\n"
            "u0 = inputs.fourier_ic(s['nx'], seed=s['seed'])\n"
            "t0 = time.perf_counter()\n"
            "O.vcycles(u0, s['nt'], s['m'], s['levels'], s['T'], 1)\n"
            "print(json.dumps([time.perf_counter() - t0, O.num_threads()]))\n" % json.dumps(sample))
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    if r.returncode != 0:
        return None
    secs, threads = json.loads(r.stdout.strip().splitlines()[-1])
    return cycle_updates(sample) / secs, secs, threads


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=30).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cycle_updates(w, fcf=True):
    # cells x Phi applications of one V-cycle (same count as mgrit_cycle_cell_updates)
    m, L = w["m"], w["levels"]
    steps = 0
    for l in range(L - 1):
        nc = w["nt"] // m ** (l + 1)
        steps += (2 * nc * m if fcf else nc * m) + nc
        if l >= 1:
            steps += nc * (m - 1)
    steps += w["nt"] // m ** (L - 1)
    return steps * w["nx"]


def workload_config(ws, sample=None):
    """The config object of the JSON line: the bench workload, or (reference
    arm) the sample of it that the oracle times, with the full workload named."""
    full = ("Burgers WENO5-JS/LF-split/SSPRK3 FP64 MGRIT V-cycle: nx=4096, nt=16384, T=1, m=4, "
            "6 levels, FCF, Fourier u0 seed 0")
    w = sample or WORKLOAD
    cfg = {"workload": full if sample is None else
           ("Burgers WENO5-JS/LF-split/SSPRK3 FP64 MGRIT V-cycle: nx=%d, nt=%d, T=%g, m=%d, "
            "%d levels, FCF, Fourier u0 seed %d" % (w["nx"], w["nt"], w["T"], w["m"], w["levels"],
                                                    w["seed"])),
           "step": "one V-cycle (all levels) from the initial iterate",
           "cell_updates_per_step": cycle_updates(w),
           "l2": "inputs larger than L2: each cycle streams >500 MB of level rows",
           "parallelism": "replicas" if ws > 1 else "single GPU"}
    if sample is not None:
        cfg["sample_of"] = full
        cfg["l2"] = "host run (no L2 flush applies)"
    return cfg


def sample_desc(s):
    return ("one V-cycle of the workload over its first quarter: nx=%d, nt=%d, T=%g, m=%d, "
            "%d levels, seed %d" % (s["nx"], s["nt"], s["T"], s["m"], s["levels"], s["seed"]))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_cycle_rate(SAMPLE)
    times = []
    for _ in range(args.steps):
        _, dt, cores, _ = oracle_cycle_rate(SAMPLE)
        times.append(dt)
    tot = sum(times)
    upd = cycle_updates(SAMPLE) * args.steps
    value = upd / tot
    line = {
        "impl": "reference",
        "metric": "fine cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(ws, SAMPLE),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "FP64 C oracle on the host cores: " + sample_desc(SAMPLE)},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------- GPU ---

def adjoint_gradient(mgrit, inputs, dev, stream):
    """dJ/du0 of J = 1/2 ||u(T) - u_target||^2 (Burgers, nx=2048, nt=8192,
    m=4, FP64; u0 seed 1, breaking time 0.20; u_target = forward solution from
    seed 1001) at the pre-shock T=0.12 and the post-shock T=0.3: forward
    MGRIT to tol, adjoint MGRIT from its C-point checkpoints, against the
    serial adjoint (C-point checkpointing, one CTA) and serial stepping."""
    import torch
    W = ADJOINT_WORKLOAD
    u0 = torch.as_tensor(inputs.fourier_ic(W["nx"], seed=W["seed"]), device=dev)
    ut0 = torch.as_tensor(inputs.fourier_ic(W["nx"], seed=W["target_seed"]), device=dev)
    out = {"workload": "J = 1/2 ||u(T) - u_target||^2, Burgers WENO5-JS/LF-split/SSPRK3 FP64, "
                       "nx=2048, nt=8192, m=4, FCF, tol 1e-10; u0 Fourier seed 1 (breaks at "
                       "t=0.20), u_target from seed 1001", "runs": []}
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    for T, L in W["cases"]:
        s = mgrit.Solver(W["nx"], W["nt"], W["m"], L, T=T, max_iter=120)
        target = s.serial_step(ut0, W["nt"])
        s.solve(u0)                                   # warm-up: allocation and graph capture
        (st, uT, uC, fst), fwd_ms = timed(lambda: s.solve(u0))
        lamT = (uT - target).contiguous()
        s.adjoint(uC, lamT)                           # warm-up: adjoint workspaces and graphs
        (ast, g, _, ast_stats), adj_ms = timed(lambda: s.adjoint(uC, lamT))
        uT_ser, ser_ms = timed(lambda: s.serial_step(u0, W["nt"]))
        lam_ser = (uT_ser - target).contiguous()
        g_ser, aser_ms = timed(lambda: s.adjoint_serial(u0, lam_ser))
        rel = float((g - g_ser).abs().max() / g_ser.abs().max())
        out["runs"].append({
            "T": T, "levels": L, "shock": T > W["breaking_time"],
            "forward": {"status": mgrit.STATUS_NAMES[st], "cycles": fst.iters, "ms": fwd_ms},
            "adjoint_mgrit": {"status": mgrit.STATUS_NAMES[ast], "cycles": ast_stats.iters,
                              "ms": adj_ms,
                              "vjp_cell_updates_per_s": ast_stats.cell_updates / (adj_ms / 1e3)},
            "serial": {"forward_ms": ser_ms, "adjoint_ms": aser_ms},
            "gradient_ms": fwd_ms + adj_ms, "serial_gradient_ms": ser_ms + aser_ms,
            "rel_max_diff_vs_serial_adjoint": rel,
            "J": 0.5 * float((lamT ** 2).sum())})
        s.close()
    return out


C4 = dict(nx=16384, nt=65536, m=8, levels=3)


def config4(mgrit, inputs, dev, timed_ms, rel_errs, peaks):
    """Config 4: Burgers, nx=16384, nt=65536, m=8, FP32 WENO5/SSPRK3 sweeps with
    FP64 tau correction, residual norms and coarsest solve; u0 = 0.5 + sin 2 pi x
    (breaks at t = 0.159); smooth T=0.12 and shocked T=0.5.
    (1) As stated (3 levels): outcome and cycle count (coarsest CFL 2.9 and 12).
    (2) CFL-capped at T=0.12 (2 levels, coarse CFL 0.36): time to tolerance,
        against FP32 serial stepping, and the max / L1 error of u(T) against FP64
        serial stepping (the GPU FP64 stepper, equal to the oracle's to 1e-11 in
        the parity tests).  At T=0.5 even 2 levels put the coarse CFL at 1.5, past
        the explicit limit; its 2-level outcome is reported as well."""
    import torch
    nx, nt, m = C4["nx"], C4["nt"], C4["m"]
    u0_np = inputs.sine_ic(nx)
    u0 = torch.as_tensor(u0_np, device=dev)
    speed = float(abs(u0_np).max())
    out = {"workload": "Burgers WENO5-JS/LF-split/SSPRK3, FP32 sweeps (FP64 tau, norms, coarsest), "
                       "nx=16384, nt=65536, m=8, FCF, u0 = 0.5 + sin(2 pi x)",
           "runs": []}
    for T in (0.12, 0.5):
        for L in (C4["levels"], 2):
            cfl = speed * (T / nt) * nx * m ** (L - 1)
            capped = cfl <= 0.95
            sv = mgrit.Solver(nx, nt, m, L, T=T, precision=32, max_iter=64 if capped else 16)
            st, uT, _, stats = sv.solve(u0, want_uC=False)
            run = {"T": T, "levels": L, "coarsest_cfl": cfl, "as_stated": L == C4["levels"],
                   "status": mgrit.STATUS_NAMES[st], "cycles": stats.iters,
                   "stagnated": bool(stats.stagnated), "seconds": stats.t_total_ms / 1e3,
                   "res_hist": [stats.res_hist[k] for k in range(min(stats.iters + 1, 6))]}
            if st == mgrit.OK and capped:
                st2, uT, _, stats = sv.solve(u0, want_uC=False)     # warm (graphs captured)
                run["seconds"] = stats.t_total_ms / 1e3
                run["cell_updates_per_s"] = nx * nt / (stats.t_total_ms / 1e3)
                sv.serial_step(u0, 8)
                uTs32, ser32_ms = timed_ms(lambda: sv.serial_step(u0, nt))
                s64 = mgrit.Solver(nx, nt, m, L, T=T)
                s64.serial_step(u0, 8)
                uT64, ser64_ms = timed_ms(lambda: s64.serial_step(u0, nt))
                s64.close()
                run.update({"serial_fp32_seconds": ser32_ms / 1e3,
                            "serial_fp64_seconds": ser64_ms / 1e3,
                            "speedup_vs_fp32_serial": ser32_ms / stats.t_total_ms,
                            "error_vs_fp64_serial": rel_errs(uT, uT64),
                            "serial_fp32_error_vs_fp64_serial": rel_errs(uTs32, uT64)})
                # the FP32 level-0 relaxation of this workload, launched alone
                # (FCF: 2m + 1 steps on each of the nt/m + 1 chunks)
                sv.run_cycles(u0, 0)
                sv.launch_kernel(0, 0, 1)
                _, rk = timed_ms(lambda: sv.launch_kernel(0, 0, 3))
                nC = nt // m
                upd = nx * (2 * nC * m + nC)
                ach = FLOPS_PER_CELL_UPDATE * upd / (rk / 3 / 1e3) / 1e12
                run["relax_l0_roofline"] = {"bound": "alu", "kernel": "level-0 relaxation (k_slab, FP32)",
                                            "ms": rk / 3, "cell_updates_per_launch": upd,
                                            "achieved": ach, "peak": peaks["fp32_tflops"],
                                            "unit": "TFLOP/s", "frac": ach / peaks["fp32_tflops"]}
            sv.close()
            out["runs"].append(run)
    return out


def paper_variants(mgrit, inputs, dev):
    """The paper's Sec. 4 comparisons on the GPU, on its setting: Burgers with
    the classical Lax-Friedrichs + FE fine scheme (Eq. fineLF), nx=128,
    nt=1024, T=0.475, m=2, 5 levels (coarsest CFL 0.95), F-relaxation,
    V-cycle; stationary (sin 2 pi x) and moving ((1 + sin 2 pi x)/2) shocks.
    (1) relative space-time L2 error of the level-0 C-points against serial
    stepping after each of the first 8 cycles, for rediscretised, Psi0 and
    Psi1 coarse integrators; (2) cycles to ||r|| < 1e-10 with Psi1 for F/FCF
    relaxation x Eq. (restriction::u)/injection x V/F-cycle."""
    import torch
    nx, nt, m, L, T = 128, 1024, 2, 5, 0.475
    nC = nt // m
    out = {"setting": "Burgers, classical LF + FE, nx=128, nt=1024, T=0.475, m=2, 5 levels",
           "error_per_cycle": {}, "cycles_to_tol_psi1": {}}
    names = {mgrit.COARSE_REDISC: "rediscretised", mgrit.COARSE_PSI0: "psi0",
             mgrit.COARSE_PSI1: "psi1"}
    for ic, (off, amp) in (("stationary", (0.0, 1.0)), ("moving", (0.5, 0.5))):
        u0 = torch.as_tensor(inputs.sine_ic(nx, offset=off, amp=amp), device=dev)
        s = mgrit.Solver(nx, nt, m, L, mgrit.LF_FE, mgrit.BURGERS, T=T)
        ser = torch.empty((nC + 1, nx), dtype=torch.float64, device=dev)
        ser[0] = u0
        for i in range(nC):                         # serial C-points, m steps at a time
            ser[i + 1] = s.serial_step(ser[i].contiguous(), m)
        norm = float(ser.norm())
        s.close()
        res = {}
        for coarse, name in names.items():
            s = mgrit.Solver(nx, nt, m, L, mgrit.LF_FE, mgrit.BURGERS, T=T, relax=mgrit.RELAX_F,
                             coarse=coarse)
            errs = []
            for k in range(1, 9):
                s.run_cycles(u0, k)
                e = float((s.cpoints() - ser).norm()) / norm
                errs.append(e if e == e and e != float("inf") else None)
            res[name] = errs
            s.close()
        out["error_per_cycle"][ic] = res
        for relax in (mgrit.RELAX_F, mgrit.RELAX_FCF):
            for guess in (mgrit.GUESS_EQ17, mgrit.GUESS_INJECT):
                for cycle in (mgrit.CYCLE_V, mgrit.CYCLE_F):
                    s = mgrit.Solver(nx, nt, m, L, mgrit.LF_FE, mgrit.BURGERS, T=T, relax=relax,
                                     guess=guess, cycle=cycle, coarse=mgrit.COARSE_PSI1,
                                     max_iter=60)
                    st, _, _, stats = s.solve(u0, want_uC=False)
                    key = "%s/%s/%s" % ("FCF" if relax else "F", "inject" if guess else "eq17",
                                        "F-cycle" if cycle else "V-cycle")
                    out["cycles_to_tol_psi1"].setdefault(ic, {})[key] = {
                        "status": mgrit.STATUS_NAMES[st], "cycles": stats.iters,
                        "ms": stats.t_total_ms}
                    s.close()
    return out


def run_mgrit(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2104_09404_gb300 import build as B, inputs, mgrit
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        tdist.barrier()
    W = WORKLOAD
    u0_np = inputs.fourier_ic(W["nx"], seed=W["seed"])
    u0 = torch.as_tensor(u0_np, device=dev)
    s = mgrit.Solver(W["nx"], W["nt"], W["m"], W["levels"], T=W["T"])
    stream = torch.cuda.current_stream()
    per_cycle = s.cycle_cell_updates()

    def barrier_sync():
        torch.cuda.synchronize()
        if ws > 1:
            tdist.barrier()
            torch.cuda.synchronize()

    # ---- device-resident throughput: one V-cycle per step ---------------
    for _ in range(max(args.warmup, 3)):
        s.run_cycles(u0, 1)
    barrier_sync()
    clocks = ClockSampler(dev.index)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.run_cycles(u0, 1)
    e1.record(stream)
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    value = whole_job_rate(ws, per_cycle, args.steps, ms)

    # ---- end to end through the C ABI with host buffers -----------------
    h_u0 = torch.as_tensor(u0_np).pin_memory()
    h_uT = torch.empty(W["nx"], dtype=torch.float64).pin_memory()
    d_u0 = torch.empty_like(u0)
    d_uC = torch.empty((W["nt"] // W["m"] + 1, W["nx"]), dtype=torch.float64, device=dev)

    def e2e_step():
        d_u0.copy_(h_u0, non_blocking=True)
        s.run_cycles(d_u0, 1)
        s.cpoints(d_uC)
        h_uT.copy_(d_uC[-1], non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier_sync()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier_sync()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    e2e_value = whole_job_rate(ws, per_cycle, args.steps, ms_e2e)

    # ---- per-kernel times (CUDA events, same stream) ----------------------
    # The level-0 relaxation is timed on the cycle's own level-0 input (the
    # initial iterate, all finite); the other kernels on the level data left
    # by one cycle of the workload as stated (which holds non-finite values
    # on the coarse levels, see the MGRIT outcome).
    s.run_cycles(u0, 0)
    torch.cuda.synchronize()
    kern = {}
    reps = 3

    def time_kernel(name, which, level):
        s.launch_kernel(which, level, 1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.launch_kernel(which, level, reps)
        b.record(stream)
        torch.cuda.synchronize()
        kern[name] = a.elapsed_time(b) / reps

    time_kernel("relax_l0", 0, 0)
    s.run_cycles(u0, 1)
    torch.cuda.synchronize()
    time_kernel("restrict_l0", 1, 0)
    time_kernel("relax_l1", 0, 1)
    time_kernel("coarsest", 2, 0)
    time_kernel("interp_l1", 3, 1)
    nC0 = W["nt"] // W["m"]
    relax0_updates = W["nx"] * (2 * nC0 * W["m"] + nC0)
    # FAS residual + restriction at level 0 (HBM-bound): per C-point value it
    # reads Phi_0(u^{mi-1}), the relaxed C-point and Phi_1(u^{m(i-1)}) and
    # writes g_1 and u_1: 5 FP64 values = 40 B algorithmic, over nC x nx values
    restrict_bytes = 40.0 * nC0 * W["nx"]
    restrict_gbs = restrict_bytes / (kern["restrict_l0"] / 1e3) / 1e9
    hbm_peak = measured_hbm_gbs()
    peaks = fma_peaks(mgrit)
    achieved = FLOPS_PER_CELL_UPDATE * relax0_updates / (kern["relax_l0"] / 1e3) / 1e12
    traffic = TRAFFIC.get(kernel_hash())

    # ---- serial GPU stepping and time to tolerance -------------------------
    # serial: all nt fine steps of the workload on one thread-block cluster
    def timed_ms(fn):
        torch.cuda.synchronize()
        ta = torch.cuda.Event(enable_timing=True)
        tb = torch.cuda.Event(enable_timing=True)
        ta.record(stream)
        r = fn()
        tb.record(stream)
        torch.cuda.synchronize()
        return r, ta.elapsed_time(tb)

    def rel_errs(got, ref):
        d = (got - ref).abs()
        return {"max": float(d.max() / ref.abs().max()), "l1": float(d.sum() / ref.abs().sum())}

    s.serial_step(u0, 8)
    uT_serial, serial_ms = timed_ms(lambda: s.serial_step(u0, W["nt"]))
    st, _, _, stats = s.solve(u0, want_uC=False)
    outcome = {"status": mgrit.STATUS_NAMES[st], "cycles": stats.iters,
               "res_hist": [stats.res_hist[k] for k in range(min(stats.iters + 1, 8))],
               "t_ms": stats.t_total_ms}
    # CFL-capped variant: the most levels keeping the coarsest CFL below 0.95
    speed = float(abs(u0_np).max())
    Lc = 1
    while (Lc + 1 <= W["levels"] and
           speed * (W["T"] / W["nt"]) * W["nx"] * W["m"] ** Lc <= 0.95):
        Lc += 1
    ttt = capped = None
    if Lc >= 2:
        cfl_c = speed * (W["T"] / W["nt"]) * W["nx"] * W["m"] ** (Lc - 1)
        sc = mgrit.Solver(W["nx"], W["nt"], W["m"], Lc, T=W["T"], max_iter=120)
        sc.solve(u0, want_uC=False)                 # warm-up (allocation, graph capture)
        stc, uTc, _, statc = sc.solve(u0, want_uC=False)
        torch.cuda.synchronize()
        ttt = {"levels": Lc, "coarsest_cfl": cfl_c,
               "status": mgrit.STATUS_NAMES[stc], "cycles": statc.iters,
               "seconds": statc.t_total_ms / 1e3, "serial_seconds": serial_ms / 1e3,
               "speedup_vs_serial": (serial_ms / 1e3) / (statc.t_total_ms / 1e3),
               # the effective solver rate: fine cell updates of the answer per second
               "effective_cell_updates_per_s": W["nx"] * W["nt"] / (statc.t_total_ms / 1e3),
               "final_residual": statc.res_hist[statc.iters],
               "rel_max_diff_vs_serial_uT": rel_errs(uTc, uT_serial)["max"]}
        # the headline's per-cycle throughput on this finite (CFL-capped)
        # hierarchy, beside the as-stated one whose coarse levels go non-finite
        pc_c = sc.cycle_cell_updates()
        sc.run_cycles(u0, 1)
        _, msc = timed_ms(lambda: sc.run_cycles(u0, args.steps))
        capped = {"levels": Lc, "coarsest_cfl": cfl_c, "value": pc_c * args.steps / (msc / 1e3),
                  "unit": "cell-updates/s", "ms_per_step": msc / args.steps,
                  "cell_updates_per_step": pc_c}
        sc.close()

    # ---- the same workload with FP32 sweeps (precision = 32) ---------------
    s32 = mgrit.Solver(W["nx"], W["nt"], W["m"], W["levels"], T=W["T"], precision=32)
    for _ in range(3):
        s32.run_cycles(u0, 1)
    _, ms32 = timed_ms(lambda: [s32.run_cycles(u0, 1) for _ in range(args.steps)])
    s32.run_cycles(u0, 0)
    s32.launch_kernel(0, 0, 1)
    _, relax32_reps = timed_ms(lambda: s32.launch_kernel(0, 0, reps))
    relax32_ms = relax32_reps / reps
    # time to tolerance in FP32 sweeps on the CFL-capped hierarchy, against
    # FP32 serial stepping; errors of both against the FP64 serial solution
    # (GPU FP64 stepping, equal to the oracle's to 1e-11 in the parity tests)
    ttt32 = None
    if Lc >= 2:
        sc32 = mgrit.Solver(W["nx"], W["nt"], W["m"], Lc, T=W["T"], max_iter=120, precision=32)
        sc32.solve(u0, want_uC=False)
        st32, uT32, _, stat32 = sc32.solve(u0, want_uC=False)
        sc32.serial_step(u0, 8)
        uTs32, ser32_ms = timed_ms(lambda: sc32.serial_step(u0, W["nt"]))
        ttt32 = {"levels": Lc, "status": mgrit.STATUS_NAMES[st32], "cycles": stat32.iters,
                 "stagnated": bool(stat32.stagnated), "seconds": stat32.t_total_ms / 1e3,
                 "serial_seconds": ser32_ms / 1e3,
                 "speedup_vs_serial": ser32_ms / stat32.t_total_ms,
                 "effective_cell_updates_per_s": W["nx"] * W["nt"] / (stat32.t_total_ms / 1e3),
                 "error_vs_fp64_serial": rel_errs(uT32, uT_serial),
                 "serial_fp32_error_vs_fp64_serial": rel_errs(uTs32, uT_serial)}
        sc32.close()

    # ---- config 4: nx = 16384, nt = 65536, m = 8, FP32 sweeps ----------------
    c4 = None if args.no_c4 else config4(mgrit, inputs, dev, timed_ms, rel_errs, peaks)

    # ---- A/B: one CTA per chunk on every level (chunk_clusters = 0) --------
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)

    def cycle_ms(sv, n):
        for _ in range(3):
            sv.run_cycles(u0, 1)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(n):
            sv.run_cycles(u0, 1)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    chunks = {"cluster_ctas_per_level": [s.query(100 + l) for l in range(W["levels"] - 1)],
              "ms_per_step": ms / args.steps,
              "fp32_cluster_ctas_per_level": [s32.query(100 + l) for l in range(W["levels"] - 1)],
              "fp32_ms_per_step": ms32 / args.steps}
    s.set_params(chunk_clusters=0)
    s32.set_params(chunk_clusters=0)
    chunks["one_cta_chunks_ms_per_step"] = cycle_ms(s, args.steps)
    chunks["one_cta_chunks_fp32_ms_per_step"] = cycle_ms(s32, args.steps)
    s.set_params(chunk_clusters=1)
    ach32 = FLOPS_PER_CELL_UPDATE * relax0_updates / (relax32_ms / 1e3) / 1e12
    fp32 = {"value": per_cycle * args.steps / (ms32 / 1e3), "unit": "cell-updates/s",
            "ms_per_step": ms32 / args.steps, "relax_l0_ms": relax32_ms,
            "roofline": {"bound": "alu", "achieved": ach32, "peak": peaks["fp32_tflops"],
                         "unit": "TFLOP/s", "frac": ach32 / peaks["fp32_tflops"],
                         "peak_source": "measured FP32 multiply-add rate (" + peaks["source"] + ")",
                         "flops_per_cell_update": FLOPS_PER_CELL_UPDATE},
            "time_to_tol_cfl_capped": ttt32}
    s32.close()

    # ---- 64 uneven instances: one batch vs one context at a time -----------
    batched = None
    if not args.no_batch:
        insts, bu0 = inputs.batch_workload(seed=0, n=64)
        bu0 = [torch.as_tensor(u, device=dev) for u in bu0]
        bt = mgrit.Batch(insts, precision=32)
        t0 = time.perf_counter()
        bt.autotune(bu0, reps=2)
        tune_s = time.perf_counter() - t0
        per_batch = bt.cycle_cell_updates()
        tuned = {}
        for what, name in ((0, "cells_per_thread"), (4, "coarsest_cluster_ctas")):
            vals = [bt.query(i, what) for i in range(len(insts))]
            tuned[name] = {str(v): vals.count(v) for v in sorted(set(vals))}
        for _ in range(2):
            bt.run_cycles(bu0, 1)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            bt.run_cycles(bu0, 1)
        b.record(stream)
        torch.cuda.synchronize()
        msb = a.elapsed_time(b)
        # the batched level-0 relaxation launched alone, against the measured
        # FP32 rate; FLOPs per cell update by flux (the instrumented oracle
        # counts 531 for advection, whose f^- reconstruction vanishes)
        bt.launch_relax(1)
        torch.cuda.synchronize()
        a.record(stream)
        bt.launch_relax(3)
        b.record(stream)
        torch.cuda.synchronize()
        relaxb_ms = a.elapsed_time(b) / 3
        relaxb_flop = sum(d["nx"] * (d["nt"] // d["m"]) * (2 * d["m"] + 1) *
                          (FLOPS_PER_CELL_UPDATE if d["flux"] == 0 else FLOPS_PER_CELL_UPDATE_ADVECTION)
                          for d in insts)
        relaxb_ach = relaxb_flop / (relaxb_ms / 1e3) / 1e12
        bt.close()
        singles = [mgrit.Solver(d["nx"], d["nt"], d["m"], d["levels"], 0, d["flux"], T=d["T"],
                                precision=32) for d in insts]
        for sv, u in zip(singles, bu0):
            sv.run_cycles(u, 1)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            for sv, u in zip(singles, bu0):
                sv.run_cycles(u, 1)
        b.record(stream)
        torch.cuda.synchronize()
        mss = a.elapsed_time(b)
        for sv in singles:
            sv.close()
        batched = {"workload": "64 instances: nx in 256..8192, nt in 1024..16384 (powers of 2), "
                               "half Burgers / half advection, FP32 sweeps, m=4, CFL 0.375, seed 0",
                   "value": per_batch * args.steps / (msb / 1e3), "unit": "cell-updates/s",
                   "ms_per_cycle": msb / args.steps,
                   "one_context_at_a_time_ms_per_cycle": mss / args.steps,
                   "speedup_vs_one_at_a_time": mss / msb, "autotune_seconds": tune_s,
                   "relax_l0_roofline": {"bound": "alu", "kernel": "batched level-0 relaxation (FP32)",
                                         "ms": relaxb_ms, "flop_per_launch": relaxb_flop,
                                         "achieved": relaxb_ach, "peak": peaks["fp32_tflops"],
                                         "unit": "TFLOP/s", "frac": relaxb_ach / peaks["fp32_tflops"]},
                   "autotuned_instances_per_choice": tuned}

    adjoint = None if args.no_adjoint else adjoint_gradient(mgrit, inputs, dev, stream)
    variants = None if args.no_variants else paper_variants(mgrit, inputs, dev)

    if rank != 0:
        if ws > 1:
            tdist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        rate, secs, cores, reps = oracle_cycle_rate(SAMPLE, min_seconds=CPU_BASELINE_SECONDS)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
               "sample": "%s, repeated %d times" % (sample_desc(SAMPLE), reps), "seconds": secs,
               "repetitions": reps, "cpu_model": host_cpu_model()}
        one = oracle_single_thread(SAMPLE1)
        if one is not None:
            cpu["single_thread"] = {"value": one[0], "unit": "cell-updates/s", "threads": one[2],
                                    "seconds": one[1],
                                    "sample": "one V-cycle: nx=%d, nt=%d, T=%g, m=%d, %d levels, seed %d"
                                              % (SAMPLE1["nx"], SAMPLE1["nt"], SAMPLE1["T"],
                                                 SAMPLE1["m"], SAMPLE1["levels"], SAMPLE1["seed"])}

    L = W["levels"]
    # graph A (relax, restrict, norm), graph B (relax + restrict per level
    # 1..L-2, coarsest, interpolation per level), and the initial-iterate
    # broadcasts of each run_cycles call (level-0 C-points, row 0 of levels 2..L-1)
    launches_per_cycle = 3 + 2 * (L - 2) + 1 + (L - 2) + 1 + (L - 2)
    line = {
        "metric": "fine cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(ws),
        "roofline": {"bound": "alu", "kernel": "level-0 relaxation (k_slab, MODE_RELAX)",
                     "achieved": achieved, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / peaks["fp64_tflops"], "traffic": traffic,
                     "peak_source": "measured FP64 multiply-add rate, burst (" + peaks["source"] + ")",
                     "nominal_peak": FP64_NOMINAL_TFLOPS,
                     "flops_per_cell_update": FLOPS_PER_CELL_UPDATE,
                     "cell_updates_per_launch": relax0_updates},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s",
                "h2d_bytes_per_step": 8 * W["nx"], "d2h_bytes_per_step": 8 * W["nx"]},
        "gpu_launches": launches_per_cycle * args.steps,
        "clocks": clk,
        "kernel_ms": kern,
        "chunk_clusters": chunks,
        "restriction_roofline": {"bound": "hbm", "kernel": "level-0 FAS residual + restriction "
                                 "(k_restrict)", "achieved": restrict_gbs, "peak": hbm_peak,
                                 "unit": "GB/s", "frac": restrict_gbs / hbm_peak if hbm_peak else None,
                                 "bytes_per_launch": restrict_bytes,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"},
        "serial_gpu": {"steps": W["nt"], "seconds": serial_ms / 1e3,
                       "ms_per_step": serial_ms / W["nt"],
                       "cell_updates_per_s": W["nx"] * W["nt"] / (serial_ms / 1e3),
                       "cluster_ctas": s.query(2)},
        "mgrit_outcome_as_stated": outcome,
        "cfl_capped_cycle": capped,
        "time_to_tol_cfl_capped": ttt,
        "config4": c4,
        "fp32_sweeps": fp32,
        "batched": batched,
        "adjoint": adjoint,
        "paper_variants": variants,
    }
    print(json.dumps(line))
    if ws > 1:
        tdist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_mgrit(args)


if __name__ == "__main__":
    sys.exit(main())
