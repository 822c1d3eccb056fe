"""GB300-native FCIQMC time step (Rimu.jl paper, arXiv 2601.19505).

The step runs as hand-written sm_103a CUDA kernels in ``libfciqmc.so`` behind
the C ABI of ``include/fciqmc.h``; this package only marshals arguments into
it (``_lib``) and offers the same calls as Python objects (``fciqmc``), plus
host-side analysis of the recorded time series (``stats``).  There is no CPU
fallback: importing the objects works anywhere, creating a run needs a GPU.
"""
from .fciqmc import (  # noqa: F401
    BH_MOM_1D, BH_REAL_1D, BH_REAL_2D, KEY_DTYPE, MODE_DETERMINISTIC, MODE_INT, MODE_REAL32,
    MODE_REAL64, STATS_DTYPE, Batch, FqError, Hamiltonian, Run, RunError, default_params, keys_from_ints,
    keys_to_ints, version)
