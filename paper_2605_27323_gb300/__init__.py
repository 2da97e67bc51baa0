"""GB300-native Monte Carlo path tracer ("Megakernel vs Wavefront GPU Path Tracing").

The estimator (Eq. 1-3, Sec. 2.2) runs as a megakernel or as a wavefront pipeline (Sec. 2.3, 3,
3.1), with a path-replay adjoint and batched rendering, all in CUDA kernels behind the C ABI of
include/pt.h.  This package holds the ctypes binding (capi), the Python front (tracer), the build
step (build) and the seeded scene generators (scenes).
"""
from .tracer import (Progressive, Scene, autotune_batch, debug_rng, make_camera, make_opts,  # noqa: F401
                     render_batch, render_differentiable)
