"""GB300 discrete-ordinates transport sweep (the Sweep method, Peter et al. 2022).

The compute path is the CUDA library libsweep.so (C ABI in include/sweep.h); this
package only loads it and marshals arguments. Build it with ``build.build()``.
"""
from ._lib import (EXPORTS, SCHEDULES, SWEEP_FACE_BOUNDARY, SWEEP_FACE_PERIODIC, Context, SweepError, default_opts,
                   load, sweep_opts, sweep_stats)

__all__ = ["Context", "SweepError", "default_opts", "load", "sweep_opts", "sweep_stats", "EXPORTS", "SCHEDULES",
           "SWEEP_FACE_BOUNDARY", "SWEEP_FACE_PERIODIC"]
