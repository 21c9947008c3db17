"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This package holds geometry and parameter generators only: it contains none of
the method's arithmetic (no ray tracing, enforcement, aggregation or REF solve).
Both the CPU oracle's callers and the CUDA library's callers take their inputs
from here.
"""
from .meshes import (Mesh, cube, plates, discs, perpendicular_squares, small_sat,
                     spacecraft, patch_mesh, two_sided_plates)
from .params import (optical_sets, heat_loads, rays_by_area, uniform_rays, workload)

__all__ = ["Mesh", "cube", "plates", "discs", "perpendicular_squares", "small_sat", "spacecraft",
           "patch_mesh", "two_sided_plates", "optical_sets", "heat_loads", "rays_by_area", "uniform_rays", "workload"]
