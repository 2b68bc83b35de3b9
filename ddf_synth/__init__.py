"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This package only *makes inputs*: procedural meshes, ray batches, network weights and
camera descriptions. It holds none of the method's arithmetic (no labelling, no MLP,
no path tracing, no random numbers drawn by the method itself), so that the oracle
and the GPU path can both consume the same arrays without sharing any of the code
that is being checked.

Everything is deterministic in its seed. Meshes are generated in float64 and rounded
to float32 exactly once; consumers read the float32 arrays.
"""

from .meshes import icosphere, torus, torus_knot, mesh_euler_characteristic
from .rays import (
    uniform_sphere_rays,
    surface_aimed_rays,
    labelled_ray_set,
    sample_surface_points,
    fibonacci_directions,
)
from .weights import ddf_arch_sizes, init_weights, split_weights
from .scenes import default_camera, CameraSpec

__all__ = [
    "icosphere",
    "torus",
    "torus_knot",
    "mesh_euler_characteristic",
    "uniform_sphere_rays",
    "surface_aimed_rays",
    "labelled_ray_set",
    "sample_surface_points",
    "ddf_arch_sizes",
    "init_weights",
    "split_weights",
    "default_camera",
    "CameraSpec",
]
