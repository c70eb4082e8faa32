"""Pins of the oracle's low-rank far field (oracle/hmatrix.py), against what the definitions
fix independently of its code:

* the block partition covers every (i, l) exactly once, and every far block satisfies the
  admissibility condition it was chosen by;
* two unit squares a distance D apart form one far block exactly when sqrt(2) <= D - 1
  (the vertex boxes' diagonal against their gap, eta = 1);
* adaptive cross approximation recovers an exactly rank-3 matrix to rounding in 3 steps
  (plus at most the one that finds the zero residual);
* the squared Frobenius norm that the stopping test uses, updated step by step (cross
  terms included), equals ||U_k W_k^T||_F^2 formed explicitly after every step;
* the assembled H-matrix differs from the dense A(k) by less than the requested tolerance
  (relative Frobenius norm), for the single layer and the double layer, and the error falls
  with the tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import assembly as oasm, hmatrix as hm


def test_partition_covers_every_entry_once():
    mesh = synth.icosphere(2)
    cl = hm.cluster_tree(mesh, leaf=16)
    bl = hm.blocks(cl, eta=1.0)
    count = np.zeros((mesh.n, mesh.n), int)
    for t, s, far in bl:
        count[np.ix_(cl[t][0], cl[s][0])] += 1
        if far:
            assert max(hm._diam(cl[t]), hm._diam(cl[s])) <= hm._dist(cl[t], cl[s])
    assert np.all(count == 1)
    assert any(f for _, _, f in bl) and any(not f for _, _, f in bl)


class _Mesh:
    def __init__(self, xyz, tri):
        self.xyz, self.tri, self.n = np.asarray(xyz, float), np.asarray(tri), len(tri)


def _two_squares(D):
    """Two unit squares in the plane z = 0, the second shifted by D along x, each split into
    two triangles."""
    xyz, tri = [], []
    for x0 in (0.0, D):
        b = len(xyz)
        xyz += [(x0, 0, 0), (x0 + 1, 0, 0), (x0 + 1, 1, 0), (x0, 1, 0)]
        tri += [(b, b + 1, b + 2), (b, b + 2, b + 3)]
    return _Mesh(xyz, tri)


@pytest.mark.parametrize("D,far", [(1.0 + np.sqrt(2.0) + 1e-3, True),
                                   (1.0 + np.sqrt(2.0) - 1e-3, False)])
def test_admissibility_of_two_squares(D, far):
    """Each square's box (of its vertices) has diagonal sqrt(2); the gap between the boxes is
    D - 1, so the squares form one far block exactly when sqrt(2) <= D - 1 (eta = 1); the
    boxes of the triangles' centroids would give a diagonal of sqrt(2) / 3."""
    mesh = _two_squares(D)
    cl = hm.cluster_tree(mesh, leaf=2)
    assert sorted(map(sorted, (cl[c][0].tolist() for c in cl[0][1]))) == [[0, 1], [2, 3]]
    bl = hm.blocks(cl, eta=1.0)
    a, b = cl[0][1]
    assert ((a, b, True) in bl) == far and ((b, a, True) in bl) == far
    assert not any(f for t, s, f in bl if t == s)


def test_aca_recovers_a_rank3_matrix():
    rng = np.random.default_rng(2)
    m, n = 40, 33
    P = rng.normal(size=(m, 3)) + 1j * rng.normal(size=(m, 3))
    Q = rng.normal(size=(n, 3)) + 1j * rng.normal(size=(n, 3))
    M = P @ Q.T
    U, W = hm.aca(lambda i: M[i].copy(), lambda j: M[:, j].copy(), m, n, 1e-12, 20)
    assert U.shape[1] <= 4
    assert np.max(np.abs(U @ W.T - M)) < 1e-12 * np.max(np.abs(M))


def test_aca_norm_update_is_exact():
    rng = np.random.default_rng(5)
    m, n = 50, 37
    M = sum(np.outer(rng.normal(size=m) + 1j * rng.normal(size=m),
                     rng.normal(size=n) + 1j * rng.normal(size=n)) * 0.5 ** p for p in range(12))
    U, W, hist = hm.aca(lambda i: M[i].copy(), lambda j: M[:, j].copy(), m, n, 1e-14, 30,
                        history=True)
    assert len(hist) == U.shape[1] >= 8
    for k, h in enumerate(hist, start=1):
        ref = np.linalg.norm(U[:, :k] @ W[:, :k].T, "fro") ** 2
        assert abs(h - ref) <= 1e-12 * ref, (k, h, ref)


@pytest.mark.parametrize("op", [None, (0.0, 1.0)], ids=["single", "double"])
def test_hmatrix_within_tolerance(op):
    mesh = synth.icosphere(3)
    k = 3.0 + 0.1j
    cl = hm.cluster_tree(mesh, leaf=32)
    bl = hm.blocks(cl, eta=1.0)
    A = oasm.matrix(mesh, k, op=op)
    errs = []
    for eps in (1e-4, 1e-7):
        AH = hm.dense(cl, bl, hm.compress(mesh, k, cl, bl, eps=eps, op=op), mesh.n)
        errs.append(np.linalg.norm(A - AH) / np.linalg.norm(A))
        assert errs[-1] < eps
    assert errs[1] < errs[0] / 100
