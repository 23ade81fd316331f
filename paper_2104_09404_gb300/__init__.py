"""GB300-native MGRIT (arXiv:2104.09404) for 1D periodic conservation laws.

The compute path is ``libmgrit.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/mgrit.h``); :mod:`.mgrit` is its thin ctypes binding and
:mod:`.inputs` builds seeded synthetic initial conditions.
"""
from . import inputs  # noqa: F401
