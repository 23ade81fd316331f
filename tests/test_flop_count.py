"""The algorithmic FLOP count of the relaxation kernel's roofline comes from
the instrumented build of the oracle (oracle/flopcount.cpp, run by
oracle/count_flops.py).  Checks that the counting build performs exactly the
oracle's arithmetic, that its counts are per-cell constants, that known small
cases give their closed-form counts, and that the bench uses the counted figure."""
import numpy as np
import pytest

import oracle as O
from oracle import count_flops as C
from paper_2104_09404_gb300 import inputs


def test_counting_build_computes_the_oracle_step_bit_for_bit():
    u = inputs.fourier_ic(256, seed=3)
    for scheme, flux, numflux in ((0, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 2), (1, 0, 0)):
        _, res = C.count_step(u, 1e-3, scheme, flux, numflux, want_result=True)
        np.testing.assert_array_equal(res, O.step(u, 1e-3, scheme, flux, numflux))


def test_counts_are_per_cell_constants():
    a = C.count_step(inputs.fourier_ic(128, seed=1), 1e-3)
    b = C.count_step(inputs.fourier_ic(1000, seed=7), 2e-4)
    assert a == b


def test_first_order_upwind_count_is_its_closed_form():
    # k = 0, forward Euler, advection (alpha = 1, f = u):
    #   alpha: |f'| = 1 is a constant -> nothing;
    #   f^+ = (u + 1 u)/2: 1 add, 1 mul; f^- = (u - 1 u)/2: 1 add, 1 mul;
    #   F_{i+1/2} = f^+_i + f^-_{i+1}: 1 add; A_i = -(F_i - F_{i-1}) / dx: 1 add, 1 div;
    #   u + dt A: 1 mul, 1 add   -> 5 add, 3 mul, 1 div per cell
    d = C.count_step(inputs.fourier_ic(64, seed=2), 1e-3, O.SCHEME_FO_FE, O.FLUX_ADVECTION)
    assert (d["add"], d["mul"], d["div"], d["abs"], d["cmp"]) == (5, 3, 1, 0, 0)


def test_bench_uses_the_counted_figure():
    import bench
    d = C.count_step(inputs.fourier_ic(4096, seed=0), 1.0 / 16384)
    assert bench.FLOPS_PER_CELL_UPDATE == d["total"] == 555
    da = C.count_step(inputs.fourier_ic(4096, seed=0), 1.0 / 16384, O.SCHEME_WENO5_SSPRK3, O.FLUX_ADVECTION)
    assert bench.FLOPS_PER_CELL_UPDATE_ADVECTION == da["total"] == 531
