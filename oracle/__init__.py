"""FP64 CPU oracle for the 7DGS render path -- TEST INFRASTRUCTURE ONLY.

This package is the slow, plainly written reference that the CUDA kernels are
checked against.  Only the test suite, the package-level `smoke()` check and the
benchmark's CPU-baseline leg may import it; the product path never calls it and
there is no CPU fallback built on it.  It shares no code with the CUDA path:
inputs come from the seeded generator in `synth/`, and every step below is
written from the paper's equations (Sec. 4.2, Eqs. cond_mean / cond_cov /
temp_mod / dir_mod, Algorithm 1 steps 3-6) and the 3DGS projection and
compositing rules the paper adopts (Sec. 4.4), in float64 with plain PyTorch
CPU operations.  Gradients are PyTorch autograd through this same forward.

Modules:
    slicing     Sigma = L L^T, block partition, conditional mean / covariance, modulation
    sh          real spherical-harmonic basis of degree 3 built from its definition
    projection  pinhole camera, EWA 2D covariance, conic, 3-sigma radius, tile rectangle
    binning     per-tile instance lists as a stable sort by (tile, depth, id)
    composite   front-to-back alpha compositing (vectorised per tile; literal loop for tiny cases)
    render      whole pipeline, sampled pixels, projected-input rendering, autograd gradients
"""
