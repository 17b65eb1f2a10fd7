"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This package only draws random scene parameters and builds pinhole cameras; it
contains none of the 7DGS arithmetic (no slicing, projection, binning or
compositing), so both sides can take their inputs from it without sharing
method code.
"""
from .scenes import (  # noqa: F401
    Scene,
    Camera,
    make_scene,
    make_camera,
    look_at,
    config_scene,
    config_cameras,
    perturb_scene,
    random_projected,
    serving_scenes,
    make_agr_weights,
    WHITE,
    BLACK,
)
