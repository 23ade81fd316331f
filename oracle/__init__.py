"""FP64 CPU oracle for MGRIT on 1D periodic conservation laws (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is compiled from ``mgrit_oracle.c``
with gcc and shares nothing with the CUDA library.
"""
from .api import (  # noqa: F401
    SCHEME_WENO5_SSPRK3, SCHEME_FO_FE, SCHEME_LF_FE, FLUX_BURGERS, FLUX_ADVECTION,
    NUMFLUX_LF_SPLIT, NUMFLUX_LF_STATE, NUMFLUX_ROE, RELAX_F, RELAX_FCF, GUESS_EQ17, GUESS_INJECT, CYCLE_V, CYCLE_F, COARSE_REDISC, COARSE_PSI0, COARSE_PSI1,
    OK, EINVAL, EDIVERGED, ENOTCONV,
    build, weno5_left, spatial_op, step, serial, mgrit, residual, num_threads, vcycles,
    weno5_left_grad, step_vjp, adjoint_serial, adjoint_mgrit, psi_step,
)
