"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package generates inputs only: triangle meshes (vertex coordinates and connectivity),
the seeded complex Gaussian starting basis, and the workload descriptions. It holds none
of the method's arithmetic (no Green's function, quadrature, contour or projection), so
the CUDA path and the oracle can both consume it without sharing any method code.
"""
from .meshes import (icosphere, cube_grid, cube_sphere, tetrakis_sphere, Mesh)
from .basis import splitmix64, uniform01, complex_gaussian
from .workloads import WORKLOADS, workload, ContourSpec

__all__ = ["icosphere", "cube_grid", "cube_sphere", "tetrakis_sphere", "Mesh",
           "splitmix64", "uniform01", "complex_gaussian", "WORKLOADS", "workload",
           "ContourSpec"]
