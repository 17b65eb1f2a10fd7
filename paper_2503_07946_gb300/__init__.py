"""GB300-native (sm_103a) renderer for 7D Gaussian Splatting (arXiv 2503.07946).

The render path -- conditional slicing, EWA projection + SH, tile binning, compositing and
their adjoint -- runs in the CUDA kernels of libsdgs.so behind the C ABI in include/sdgs.h.
`sdgs` is the ctypes binding, `render` the pipeline and autograd wrappers.
"""
__version__ = "0.1.0"
