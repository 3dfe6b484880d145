"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle and the
benchmark.

This package only draws random numbers and lays them out; it holds none of the
splatting arithmetic (no projection, blending, loss or optimiser code), so the
oracle and the CUDA path can both consume it without sharing method code.
"""
from .scenes import (  # noqa: F401
    Camera,
    Scene,
    camera_c1,
    camera_pose_error,
    with_pose_error,
    ring_cameras,
    mixed_ring_cameras,
    orbit_cameras,
    recon_init,
    ng_anchors,
    scene_c1,
    scene_clustered,
    scene_tiny,
    camera_tiny,
    target_uniform,
    upstream_grads,
)
