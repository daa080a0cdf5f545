"""GB300 discrete-ordinates transport sweep (the Sweep method, Peter et al. 2022).

The compute path is the CUDA library libsweep.so (C ABI in include/sweep.h); this
package only loads it and marshals arguments. Build it with ``build.build()``.
"""
from ._lib import (EXPORTS, SCHEDULES, SWEEP_FACE_BOUNDARY, SWEEP_FACE_PERIODIC, Context, SweepError, default_opts,
                   load, sweep_opts, sweep_stats)



def transport_solve(*args, **kw):
    """Differentiable solve (see autograd.transport_solve); imports torch on first use."""
    from .autograd import transport_solve as f
    return f(*args, **kw)


__all__ = ["transport_solve", "Context", "SweepError", "default_opts", "load", "sweep_opts", "sweep_stats", "EXPORTS", "SCHEDULES",
           "SWEEP_FACE_BOUNDARY", "SWEEP_FACE_PERIODIC"]
