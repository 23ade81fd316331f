"""Algorithmic FLOPs per cell update, counted by instrumenting the oracle.

Builds oracle/flopcount.cpp (the oracle's source compiled as C++ with a
counting number type; test and measurement infrastructure, never part of the
product path), runs one oracle time step of the benchmark state and prints
the operations per cell update, by kind, for each scheme and numerical flux.

    python oracle/count_flops.py            # table
    python oracle/count_flops.py --json     # one JSON object

The first row (WENO5-JS + global Lax-Friedrichs splitting + SSPRK3, Burgers)
is the per-unit figure of the relaxation kernel's roofline.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "flopcount.cpp")
LIB = os.path.join(HERE, "libflopcount.so")
KINDS = ("add", "mul", "div", "abs", "cmp", "sqrt")


def build(force=False):
    deps = [SRC, os.path.join(HERE, "mgrit_oracle.c")]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, deps)):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fpermissive", "-w",
                               "-fPIC", "-shared", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def _lib():
    lib = ctypes.CDLL(build())
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.fc_count_step.restype = None
    lib.fc_count_step.argtypes = [I, D, D, I, I, I, P, P, P]
    lib.fc_count_step_vjp.restype = None
    lib.fc_count_step_vjp.argtypes = [I, D, D, I, I, P, P, P]
    return lib


def count_step(u, dt, scheme=0, flux=0, numflux=0, Lx=1.0, want_result=False):
    """Operations of one oracle step on u, per cell, as a dict by kind (+ total);
    with want_result, also the step's result computed by the counting build."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = (ctypes.c_longlong * len(KINDS))()
    res = np.zeros_like(u)
    _lib().fc_count_step(u.size, Lx, dt, scheme, flux, numflux, u.ctypes.data_as(ctypes.c_void_p),
                         ctypes.cast(out, ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p))
    d = {k: out[i] / u.size for i, k in enumerate(KINDS)}
    d["total"] = sum(out) / u.size
    return (d, res) if want_result else d


def count_step_vjp(u, lam, dt, scheme=0, flux=0, Lx=1.0):
    """Operations of one oracle transposed step, per cell (split flux)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = (ctypes.c_longlong * len(KINDS))()
    _lib().fc_count_step_vjp(u.size, Lx, dt, scheme, flux, u.ctypes.data_as(ctypes.c_void_p),
                             lam.ctypes.data_as(ctypes.c_void_p), ctypes.cast(out, ctypes.c_void_p))
    d = {k: out[i] / u.size for i, k in enumerate(KINDS)}
    d["total"] = sum(out) / u.size
    return d


def table():
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2104_09404_gb300 import inputs
    nx, nt, T = 4096, 16384, 1.0
    u0 = inputs.fourier_ic(nx, seed=0)
    dt = T / nt
    rows = {}
    for name, (scheme, flux, numflux) in (
            ("weno5_ssprk3_burgers_lf_split", (0, 0, 0)),
            ("weno5_ssprk3_advection_lf_split", (0, 1, 0)),
            ("weno5_ssprk3_burgers_lf_state", (0, 0, 1)),
            ("weno5_ssprk3_burgers_roe", (0, 0, 2)),
            ("fo_fe_burgers_lf_split", (1, 0, 0))):
        rows[name] = count_step(u0, dt, scheme, flux, numflux)
    lam = np.random.default_rng(0).standard_normal(nx)
    rows["adjoint_weno5_ssprk3_burgers"] = count_step_vjp(u0, lam, dt)
    return {"state": "nx=4096 Fourier u0 seed 0, dt=1/16384", "per_cell_update": rows}


if __name__ == "__main__":
    t = table()
    if "--json" in sys.argv:
        print(json.dumps(t))
    else:
        print(t["state"])
        for name, d in t["per_cell_update"].items():
            print("%-34s total %7.1f  " % (name, d["total"]) +
                  "  ".join("%s %.1f" % (k, d[k]) for k in KINDS))
