"""Camera descriptions for the synthetic render workloads (inputs only: the ray
generation from a camera belongs to the renderer on each side)."""

from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class CameraSpec:
    eye: tuple
    look_at: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int
    seed: int = 1
    albedo: float = 0.7
    env: float = 1.0


def default_camera(width: int, height: int, seed: int = 1, azimuth_deg: float = 30.0,
                   elevation_deg: float = 20.0, distance: float = 2.5, vfov_deg: float = 30.0,
                   albedo: float = 0.7, env: float = 1.0) -> CameraSpec:
    """Pinhole camera on a sphere of `distance` around the object, Z-up (the paper's
    renders are Z-up and taken from several azimuth / polar angles), looking at the origin.
    With the defaults every pixel ray meets the unit ball."""
    az = math.radians(azimuth_deg)
    el = math.radians(elevation_deg)
    eye = (distance * math.cos(el) * math.cos(az), distance * math.cos(el) * math.sin(az),
           distance * math.sin(el))
    return CameraSpec(eye=eye, look_at=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), vfov_deg=vfov_deg,
                      width=width, height=height, seed=seed, albedo=albedo, env=env)
