"""Launch one kernel of the V-cycle for profiling (e.g. under ncu).

    python -m paper_2104_09404_gb300.profile --case c2 --kernel relax --level 0 --reps 1

(--kernel serial: 64 steps of mgrit_serial_step instead, on the sequential
stepper the context chose at allocation.)  The profiled launches run inside
the NVTX range "profiled"; profile them with
    ncu --nvtx --nvtx-include "profiled/" ...

Cases: c2 = nx 4096, nt 16384, m 4, 6 levels, T 1 (the benchmark workload);
small = nx 4096, nt 2048, m 4, 4 levels, T 0.125 (same kernel shape, 513
CTAs); c4 = nx 16384, nt 65536, m 8, 2 levels, T 0.12, u0 = 0.5 + sin 2 pi x
(config 4, CFL-capped); c4small = the same with nt 8192, T 0.015.  The context is prepared with zero cycles (workspaces allocated,
level-0 C-points = u0), then the chosen kernel is launched `reps` times; it
is the first launch of that kernel in the process.

    python -m paper_2104_09404_gb300.profile --adjoint

runs the adjoint gradient workload instead (nx 2048, nt 8192, m 4, 3 levels,
T 0.12, u0 Fourier seed 1, target seed 1001): a forward solve, then one
adjoint cycle (k_adjoint launches: the forward-trajectory regeneration, then
the level-0 adjoint relaxation).

    python -m paper_2104_09404_gb300.profile --batch

builds the 64-instance uneven batch (inputs.batch_workload, seed 0; FP32
sweeps), autotunes it as the benchmark does, runs one cycle, and then
launches its level-0 relaxation (one k_slab_batch launch per (flux, cells
per thread, threads) class) `reps` times inside the range "profiled".

    python -m paper_2104_09404_gb300.profile --peaks

measures the multiply-add throughput of the FP64 and FP32 pipes
(mgrit_fma_probe: 152 x 8 CTAs of 256 threads, 8 independent chains per
thread, ~0.1 s per launch, best of 3), the roofline denominators of the
arithmetic-bound sweeps, and prints them in TFLOP/s.

    python -m paper_2104_09404_gb300.profile --steppers

times serial stepping (Burgers WENO5/SSPRK3, CFL 0.25, Fourier u0 seed 0) on
each sequential stepper (one CTA, cluster, grid, and the one the context
picks at allocation), FP64 and FP32, at nx = 1024, 2048, 4096 and 16384,
with CUDA events around one mgrit_serial_step call, and prints microseconds
per step with the cluster size and grid size used.
"""
import argparse
import sys

CASES = {
    "c2": dict(nx=4096, nt=16384, m=4, levels=6, T=1.0),
    "small": dict(nx=4096, nt=2048, m=4, levels=4, T=0.125),
    "c1": dict(nx=128, nt=256, m=4, levels=2, T=0.5),
    # config 4 (u0 = 0.5 + sin 2 pi x), CFL-capped to 2 levels, and a short
    # case of the same kernel shape
    "c4": dict(nx=16384, nt=65536, m=8, levels=2, T=0.12, ic="sine"),
    "c4small": dict(nx=16384, nt=8192, m=8, levels=2, T=0.015, ic="sine"),
}
KERNELS = {"relax": 0, "restrict": 1, "coarsest": 2, "interp": 3, "serial": -1}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--case", default="c2", choices=sorted(CASES))
    p.add_argument("--kernel", default="relax", choices=sorted(KERNELS))
    p.add_argument("--level", type=int, default=0)
    p.add_argument("--reps", type=int, default=1)
    p.add_argument("--adjoint", action="store_true")
    p.add_argument("--batch", action="store_true",
                   help="the batched level-0 relaxation of the 64-instance workload")
    p.add_argument("--peaks", action="store_true", help="FP64 / FP32 multiply-add throughput")
    p.add_argument("--steppers", action="store_true",
                   help="microseconds per serial step on each sequential stepper")
    p.add_argument("--precision", type=int, default=64, choices=(64, 32),
                   help="32: the FP32-sweep instances of the kernels")
    a = p.parse_args(argv)
    import torch
    from . import inputs, mgrit
    if a.peaks:
        mgrit.load()
        for kind, name, iters in ((mgrit.FMA_FP64, "FP64 DFMA", 3000),
                                  (mgrit.FMA_FP32, "FP32 FFMA", 200000),
                                  (mgrit.FMA_FP32X2, "FP32 FFMA2 (packed pairs)", 100000)):
            mgrit.fma_probe(kind, iters // 20)
            r = [mgrit.fma_probe(kind, iters) for _ in range(3)]
            print("%-26s %8.3f TFLOP/s (best of 3; %s)" % (name, max(r) / 1e12,
                                                         ", ".join("%.3f" % (x / 1e12) for x in r)))
        return 0
    if a.steppers:
        return time_steppers(torch, inputs, mgrit)
    if a.adjoint:
        nx, nt = 2048, 8192
        s = mgrit.Solver(nx, nt, 4, 3, T=0.12)
        u0 = torch.as_tensor(inputs.fourier_ic(nx, seed=1), device="cuda")
        target = s.serial_step(torch.as_tensor(inputs.fourier_ic(nx, seed=1001), device="cuda"), nt)
        st, uT, uC, _ = s.solve(u0)
        s.set_params(max_iter=0)
        s.adjoint(uC, (uT - target).contiguous())
        torch.cuda.synchronize()
        print("adjoint workload: trajectory + one adjoint cycle")
        return 0
    if a.batch:
        insts, bu0 = inputs.batch_workload(seed=0, n=64)
        bu0 = [torch.as_tensor(u, device="cuda") for u in bu0]
        bt = mgrit.Batch(insts, precision=32)
        bt.autotune(bu0, reps=2)
        bt.run_cycles(bu0, 1)
        bt.launch_relax(1)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("profiled")
        t0.record()
        bt.launch_relax(a.reps)
        t1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        cells = sum(d["nx"] * (d["nt"] // d["m"]) * (2 * d["m"] + 1) for d in insts)
        print("batched level-0 relaxation x%d: %d instances, %d cell updates per launch, "
              "%.3f ms per launch (CUDA events)" % (a.reps, len(insts), cells, t0.elapsed_time(t1) / a.reps))
        bt.close()
        return 0
    c = CASES[a.case]
    s = mgrit.Solver(c["nx"], c["nt"], c["m"], c["levels"], T=c["T"], precision=a.precision)
    u0_np = inputs.sine_ic(c["nx"]) if c.get("ic") == "sine" else inputs.fourier_ic(c["nx"], seed=0)
    u0 = torch.as_tensor(u0_np, device="cuda")
    if a.kernel == "serial":
        # 64 serial steps on the sequential stepper the context chose, in the
        # NVTX range "profiled" (allocation, which times the candidates,
        # comes before it)
        s.serial_step(u0, 1)
        s.sync_status()
        torch.cuda.nvtx.range_push("profiled")
        s.serial_step(u0, 64)
        s.sync_status()
        torch.cuda.nvtx.range_pop()
        print("serial stepping x64 on case %s (grid CTAs %d, cluster CTAs %d)"
              % (a.case, s.query(3), s.query(2)))
        return 0
    s.run_cycles(u0, 0)
    torch.cuda.synchronize()
    # the launches to profile sit in the NVTX range "profiled" (the context's
    # allocation times candidate kernel shapes first: ncu --nvtx
    # --nvtx-include "profiled/" skips those)
    torch.cuda.nvtx.range_push("profiled")
    s.launch_kernel(KERNELS[a.kernel], a.level, a.reps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print("launched %s level %d x%d on case %s" % (a.kernel, a.level, a.reps, a.case))
    return 0


def time_steppers(torch, inputs, mgrit):
    mgrit.load()
    names = ((mgrit.SEQ_AUTO, "auto"), (mgrit.SEQ_ONE_CTA, "one CTA"),
             (mgrit.SEQ_CLUSTER, "cluster"), (mgrit.SEQ_GRID, "grid"))
    print("precision  nx      " + "".join("%-22s" % n for _, n in names))
    for prec in (64, 32):
        for nx, steps in ((1024, 2048), (2048, 2048), (4096, 2048), (16384, 1024)):
            row = []
            for k, _ in names:
                if k == mgrit.SEQ_ONE_CTA and prec == 64 and nx > 8192:
                    row.append("-")         # beyond the one-CTA FP64 slab
                    continue
                s = mgrit.Solver(nx, steps, 2, 2, T=0.25 * steps / nx, precision=prec,
                                 seq_stepper=k)
                u0 = torch.as_tensor(inputs.fourier_ic(nx, seed=0), device="cuda")
                s.serial_step(u0, 4)
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record()
                s.serial_step(u0, steps)
                t1.record()
                torch.cuda.synchronize()
                s.sync_status()
                us = 1e3 * t0.elapsed_time(t1) / steps
                k2, g = s.query(2), s.query(3)
                row.append("%.2f (%s)" % (us, "G=%d" % g if g else "K=%d" % k2))
                s.close()
            print("FP%-8d %-7d " % (prec, nx) + "".join("%-22s" % x for x in row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
