"""Closed triangle surface meshes used as synthetic BEM workloads.

The paper's experiments run on a uniformly meshed unit cube and unit sphere (Section 4,
Examples 1 and 2) and on a third-party pump casing that is not reproduced here. These
generators build the same kinds of surfaces deterministically:

* ``icosphere(level)``: regular icosahedron on the unit sphere, each level splitting every
  triangle into four through edge midpoints pushed back onto the sphere (20 * 4**level
  flat triangles: level 2 -> 320, level 5 -> 20480).
* ``cube_grid(m)``: surface of [0,1]^3 with m x m squares per face, each square split into
  two along its (i,j)->(i+1,j+1) diagonal (12 m^2 triangles: m = 16 -> 3072).
* ``cube_sphere(m, axes)``: surface of [-1,1]^3 gridded as above, projected radially onto
  the unit sphere and scaled by the semi-axes (an ellipsoid with 12 m^2 triangles).
* ``tetrakis_sphere(level, axes)``: each face of [-1,1]^3 split into four triangles about
  its centre (24), midpoint-subdivided ``level`` times on the flat faces, projected
  radially and scaled (24 * 4**level triangles: level 6 -> 98304).

Every triangle is oriented so that (v1 - v0) x (v2 - v0) points out of the body.
Coordinates are float64, connectivity int32. Nothing here evaluates the method.
"""
from dataclasses import dataclass
import itertools
import numpy as np


@dataclass
class Mesh:
    name: str
    xyz: np.ndarray   # (nv, 3) float64, C-contiguous
    tri: np.ndarray   # (nt, 3) int32, C-contiguous

    @property
    def n(self) -> int:
        return int(self.tri.shape[0])


def _finish(name, pts, tris):
    xyz = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    tri = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
    return Mesh(name, xyz, tri)


def _orient_outward(xyz, tris, centre=(0.0, 0.0, 0.0)):
    """Flip triangles whose normal points towards ``centre`` (star-shaped bodies only)."""
    c = np.asarray(centre)
    out = []
    for a, b, d in tris:
        nrm = np.cross(xyz[b] - xyz[a], xyz[d] - xyz[a])
        mid = (xyz[a] + xyz[b] + xyz[d]) / 3.0 - c
        out.append((a, b, d) if np.dot(nrm, mid) > 0 else (a, d, b))
    return out


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    pts = np.array(pts)
    # faces = vertex triples that are pairwise at the edge length (2 before normalising)
    faces = []
    for a, b, c in itertools.combinations(range(12), 3):
        if all(abs(np.linalg.norm(pts[p] - pts[q]) - 2.0) < 1e-9
               for p, q in ((a, b), (b, c), (a, c))):
            faces.append((a, b, c))
    assert len(faces) == 20
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    return pts, _orient_outward(pts, faces)


def _subdivide(pts, faces, project):
    """Split each triangle into 4 through edge midpoints; ``project`` maps a new point."""
    pts = [np.asarray(p, dtype=np.float64) for p in pts]
    cache = {}

    def mid(a, b):
        key = (a, b) if a < b else (b, a)
        if key not in cache:
            cache[key] = len(pts)
            pts.append(project(0.5 * (pts[a] + pts[b])))
        return cache[key]

    out = []
    for a, b, c in faces:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.array(pts), out


def icosphere(level: int) -> Mesh:
    pts, faces = _icosahedron()
    unit = lambda p: p / np.linalg.norm(p)
    for _ in range(level):
        pts, faces = _subdivide(pts, faces, unit)
    return _finish(f"icosphere_L{level}", pts, faces)


# (origin, u, v) of each face of the cube [lo, hi]^3 with u x v the outward normal;
# origin and axes are given in "corner units" (0 -> lo, 1 -> hi).
_CUBE_FACES = (
    ((0, 0, 0), (0, 0, 1), (0, 1, 0)),   # x = lo, normal -x
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),   # x = hi, normal +x
    ((0, 0, 0), (1, 0, 0), (0, 0, 1)),   # y = lo, normal -y
    ((0, 1, 0), (0, 0, 1), (1, 0, 0)),   # y = hi, normal +y
    ((0, 0, 0), (0, 1, 0), (1, 0, 0)),   # z = lo, normal -z
    ((0, 0, 1), (1, 0, 0), (0, 1, 0)),   # z = hi, normal +z
)


def _cube_lattice(m):
    """Integer lattice vertices (units of 1/m) and triangles of the gridded cube surface."""
    index = {}
    verts = []
    tris = []

    def vid(p):
        if p not in index:
            index[p] = len(verts)
            verts.append(p)
        return index[p]

    for o, u, v in _CUBE_FACES:
        o = np.array(o) * m
        u = np.array(u)
        v = np.array(v)
        for i in range(m):
            for j in range(m):
                p00 = tuple(int(t) for t in o + i * u + j * v)
                p10 = tuple(int(t) for t in o + (i + 1) * u + j * v)
                p11 = tuple(int(t) for t in o + (i + 1) * u + (j + 1) * v)
                p01 = tuple(int(t) for t in o + i * u + (j + 1) * v)
                a, b, c, d = vid(p00), vid(p10), vid(p11), vid(p01)
                tris += [(a, b, c), (a, c, d)]
    return np.array(verts, dtype=np.float64), tris


def cube_grid(m: int) -> Mesh:
    lat, tris = _cube_lattice(m)
    return _finish(f"cube_{m}x{m}", lat / m, tris)


def cube_sphere(m: int, axes=(1.0, 1.0, 1.0)) -> Mesh:
    lat, tris = _cube_lattice(m)
    p = 2.0 * lat / m - 1.0
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    p *= np.asarray(axes, dtype=np.float64)
    return _finish(f"cubesphere_{m}_{axes[0]:.3f}_{axes[1]:.3f}_{axes[2]:.3f}", p, tris)


def tetrakis_sphere(level: int, axes=(1.0, 1.0, 1.0)) -> Mesh:
    corners, quads = [], []
    index = {}

    def vid(p):
        if p not in index:
            index[p] = len(corners)
            corners.append(p)
        return index[p]

    faces = []
    for o, u, v in _CUBE_FACES:
        o = np.array(o, dtype=np.float64) * 2 - 1
        u = np.array(u, dtype=np.float64) * 2
        v = np.array(v, dtype=np.float64) * 2
        c00 = vid(tuple(o)); c10 = vid(tuple(o + u))
        c11 = vid(tuple(o + u + v)); c01 = vid(tuple(o + v))
        ctr = vid(tuple(o + 0.5 * u + 0.5 * v))
        faces += [(c00, c10, ctr), (c10, c11, ctr), (c11, c01, ctr), (c01, c00, ctr)]
    pts = np.array(corners, dtype=np.float64)
    for _ in range(level):
        pts, faces = _subdivide(pts, faces, lambda q: q)
    pts = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    pts = pts * np.asarray(axes, dtype=np.float64)
    return _finish(f"tetrakis_L{level}", pts, faces)
