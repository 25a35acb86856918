"""B300-native differentiable 3D Gaussian-splat rasterizer.

The hot path of the joint Gaussian optimisation (Sec. 5.2): EWA projection with
SH colour, tile binning with a (tile, depth) sort, front-to-back blending, the
analytic backward to every Gaussian parameter and the camera pose, and a fused
Adam step.  Every step runs in hand-written CUDA kernels behind the C ABI in
include/gs.h; this package is the Python binding (argument marshalling only).

The compiled library is loaded on first use; a missing or unloadable library
raises, there is no fallback path.
"""

__all__ = ["synth"]
