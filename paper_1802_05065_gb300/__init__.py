"""GB300 first-passage-time engine (sm_103a CUDA kernels behind the C ABI of include/fpt.h).

Python front end: ``_lib`` marshals arguments into the CUDA library; ``api`` offers torch-
friendly helpers (device buffers and streams from PyTorch).  No computation of the method runs
in Python.
"""
from ._lib import (  # noqa: F401
    Engine, FptError, Params, Result, Sums, engine_occupancy, load, normals_fill, params_from, philox_fill,
    plain_launch, reduce_steps, run_noalloc, sums_finish, version,
    UNDERDAMPED, OVERDAMPED, FP32, FP64, EULER_MARUYAMA, HEUN, OUT_TIME, OUT_BIAS, TH_ABSOLUTE, TH_FROM_START,
)
