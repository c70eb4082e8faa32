"""The synthetic inputs: mesh counts, closedness, orientation, areas; basis statistics."""
import collections

import numpy as np
import pytest

import synth


def _edges_closed_and_consistent(mesh):
    """Every directed edge appears once and its reverse exactly once (closed, oriented)."""
    directed = collections.Counter()
    for a, b, c in mesh.tri:
        for p, q in ((a, b), (b, c), (c, a)):
            directed[(int(p), int(q))] += 1
    return all(v == 1 for v in directed.values()) and \
        all(directed.get((q, p), 0) == 1 for (p, q) in directed)


@pytest.mark.parametrize("fn,n", [
    (lambda: synth.icosphere(0), 20), (lambda: synth.icosphere(2), 320),
    (lambda: synth.cube_grid(4), 192), (lambda: synth.cube_grid(16), 3072),
    (lambda: synth.cube_sphere(5, (1.0, 0.7, 0.5)), 300),
    (lambda: synth.tetrakis_sphere(2, (1.0, 0.7, 0.5)), 384),
])
def test_counts_closed_oriented(fn, n):
    m = fn()
    assert m.n == n
    assert m.tri.dtype == np.int32 and m.xyz.dtype == np.float64
    assert _edges_closed_and_consistent(m)
    # Euler characteristic of a sphere-like surface
    nv = m.xyz.shape[0]
    assert nv - (3 * m.n // 2) + m.n == 2
    a, b, c = (m.xyz[m.tri[:, k]] for k in range(3))
    nrm = np.cross(b - a, c - a)
    ctr = (a + b + c) / 3.0 - m.xyz.mean(axis=0)
    assert np.all(np.einsum("ij,ij->i", nrm, ctr) > 0)


def test_areas():
    m = synth.cube_grid(16)
    a, b, c = (m.xyz[m.tri[:, k]] for k in range(3))
    assert abs(0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum() - 6.0) < 1e-12
    # inscribed icospheres approach 4 pi from below
    areas = []
    for L in (1, 2, 3):
        m = synth.icosphere(L)
        a, b, c = (m.xyz[m.tri[:, k]] for k in range(3))
        areas.append(0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum())
    assert areas[0] < areas[1] < areas[2] < 4 * np.pi
    assert np.allclose(np.linalg.norm(synth.icosphere(3).xyz, axis=1), 1.0)


def test_basis_deterministic_and_gaussian():
    V1 = synth.complex_gaussian(1000, 8, 7)
    V2 = synth.complex_gaussian(1000, 8, 7)
    assert V1.flags.f_contiguous and V1.dtype == np.complex128
    assert np.array_equal(V1, V2)
    assert not np.array_equal(V1, synth.complex_gaussian(1000, 8, 8))
    assert abs(np.mean(np.abs(V1) ** 2) - 1.0) < 0.05
    assert abs(np.mean(V1.real)) < 0.05 and abs(np.var(V1.real) - 0.5) < 0.05


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: published first outputs of the generator
    out = synth.splitmix64(0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                     0x06C45D188009454F]


def test_workloads():
    assert synth.workload("sphere320").problems[0].mesh().n == 320
    assert synth.workload("cube3072").problems[0].mesh().n == 3072
    b = synth.workload("batch48").problems
    assert len(b) == 48
    assert all(p.N in (16, 24, 32) and p.nu == 32 for p in b)
    assert all(2.0 <= p.contour.centre.real <= 8.0 for p in b)
