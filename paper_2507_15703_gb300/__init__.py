"""GB300-native simulation of partial-sky CMB maps with 3-D FFTs.

The hot path (Gaussian draw, inverse real 3-D FFT, interpolation at the sky
pixels) runs in hand-written sm_103a CUDA kernels behind the C ABI of
include/cmb3d.h; `cmb3d` is its ctypes binding.
"""
from . import cmb3d  # noqa: F401
from .cmb3d import Plan  # noqa: F401
