"""The synthetic workloads (mesh, contour, number of nodes, basis width, seed).

Five workloads mirror the paper's experiments (unit sphere and unit cube with Dirichlet
conditions, Section 4) at the sizes this project measures:

1. ``sphere320``: icosphere level 2 (320 triangles); circle centre 4.0 radius 1.0, N = 16,
   nu = 16.
2. ``cube3072``: unit cube, 16 x 16 squares per face (3072 triangles); ellipse centre 6.5,
   semi-axes 1.5 (real) and 0.4 (imaginary), N = 32, nu = 64.
3. ``batch48``: 48 ellipsoids, semi-axes uniform in [0.5, 2], triangle count log-uniform in
   [500, 12000] (cube-sphere, 12 m^2 triangles with m = round(sqrt(T / 12))), circle centre
   uniform in [2, 8] radius 0.8, N drawn from {16, 24, 32}, nu = 32.
4. ``sphere20480``: icosphere level 5; circle centre 7.0 radius 1.0, N = 32, nu = 128.
5. ``ellipsoid98304``: tetrakis sphere level 6 scaled to semi-axes (1.0, 0.7, 0.5); circle
   centre 9.0 radius 1.5, N = 64, nu = 256.

``ellipsoid24576`` (level 5 of the same ellipsoid, same contour, N = 16, nu = 256) is the
small case of workload 5's kernel shape (one node per work unit, 256 basis columns), sized
for profiler captures.

A contour is described by data only (kind, centre, semi-axes); its nodes and weights are
computed by each side on its own. Seeds: problem p of a workload uses 20190609 + p.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .meshes import icosphere, cube_grid, cube_sphere, tetrakis_sphere
from .basis import uniform01

BASE_SEED = 20190609


@dataclass(frozen=True)
class ContourSpec:
    kind: str          # "circle" or "ellipse"
    centre: complex    # centre c
    a: float           # semi-axis along Re (radius for a circle)
    b: float           # semi-axis along Im (equal to a for a circle)


@dataclass
class Problem:
    mesh_fn: object
    contour: ContourSpec
    N: int
    nu: int
    seed: int
    label: str = ""

    def mesh(self):
        return self.mesh_fn()


@dataclass
class Workload:
    name: str
    problems: list = field(default_factory=list)


def _circle(c, r):
    return ContourSpec("circle", complex(c), float(r), float(r))


def _batch48():
    u = uniform01(BASE_SEED, 48 * 8)
    probs = []
    for p in range(48):
        s = u[8 * p: 8 * p + 8]
        axes = tuple(float(0.5 + 1.5 * s[k]) for k in range(3))
        t = math.exp(math.log(500.0) + (math.log(12000.0) - math.log(500.0)) * s[3])
        m = max(2, int(round(math.sqrt(t / 12.0))))
        centre = 2.0 + 6.0 * s[4]
        N = (16, 24, 32)[min(2, int(3.0 * s[5]))]
        probs.append(Problem(lambda m=m, axes=axes: cube_sphere(m, axes),
                             _circle(centre, 0.8), N, 32, BASE_SEED + p,
                             f"ellipsoid{p}_m{m}"))
    return probs


def _make():
    return {
        "sphere320": Workload("sphere320", [Problem(lambda: icosphere(2), _circle(4.0, 1.0),
                                                    16, 16, BASE_SEED, "icosphere_L2")]),
        "cube3072": Workload("cube3072", [Problem(lambda: cube_grid(16),
                                                  ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4),
                                                  32, 64, BASE_SEED, "cube_16x16")]),
        "batch48": Workload("batch48", _batch48()),
        "sphere20480": Workload("sphere20480", [Problem(lambda: icosphere(5), _circle(7.0, 1.0),
                                                        32, 128, BASE_SEED, "icosphere_L5")]),
        "ellipsoid98304": Workload("ellipsoid98304",
                                   [Problem(lambda: tetrakis_sphere(6, (1.0, 0.7, 0.5)),
                                            _circle(9.0, 1.5), 64, 256, BASE_SEED,
                                            "tetrakis_L6")]),
        "ellipsoid24576": Workload("ellipsoid24576",
                                   [Problem(lambda: tetrakis_sphere(5, (1.0, 0.7, 0.5)),
                                            _circle(9.0, 1.5), 16, 256, BASE_SEED,
                                            "tetrakis_L5")]),
    }


WORKLOADS = _make()


def workload(name: str) -> Workload:
    return WORKLOADS[name]
