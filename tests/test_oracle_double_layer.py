"""Pins of the oracle's operator variant T = c_G G + c_H (1/2 I + K) (the double layer K
with its jump; the paper's general T = A H - B G of Eq. HelmBIM) against what the
mathematics fixes, independent of the oracle's own formulas:

* Row sums on the unit sphere. The double-layer potential of the constant density, taken
  to the sphere from inside, is i k^2 j_0(k) h_0'(k) (addition theorem of the Green's
  function; at k -> 0 Gauss's solid-angle integral, -1), so with the jump the row sums of
  H = 1/2 I + K tend to 1 + (sin k / k) e^{ik} (i k - 1), at the rate O(h^2) of the
  inscribed mesh (ratio ~4 per refinement). A wrong sign of the kernel, of the normal, of
  (y - x), or a missing jump moves the limit.
* With the near-field rule the static identity (k -> 0: row sums 0) holds to 1e-5 on
  icosphere L2 (the 7-point rule alone leaves the O(h) error of the 1/r^2 kernel).
* The self entry is the jump 1/2 exactly (x_i lies in the plane of its own panel), its
  k-derivative is 0; away from the diagonal the k-derivative matches central differences.
* The 7-point rule and the 32 x 32 conical rule agree on a well-separated pair.
* The discrete Neumann eigenvalues of the sphere (T = H) sit near the zeros of j_1' and
  j_2' (2.0816, 3.3421; multiplicities 3 and 5, kept by the icosahedral symmetry).
"""
import os

import numpy as np
import pytest

import synth
from oracle import assembly as oasm

HERE = os.path.dirname(os.path.abspath(__file__))
H_OP = (0.0, 1.0)


def _closed_form(k):
    return 1.0 + (np.sin(k) / k) * np.exp(1j * k) * (1j * k - 1.0)


@pytest.mark.parametrize("k", [1.0, 2.5, 3.0 + 0.3j])
def test_row_sums_converge_to_closed_form(k):
    errs = []
    for level in (2, 3):
        H = oasm.matrix(synth.icosphere(level), k, op=H_OP)
        errs.append(np.max(np.abs(H.sum(1) - _closed_form(k))))
    assert errs[1] < 1.3e-2
    assert errs[0] / errs[1] > 3.3, errs


def test_static_identity_with_near_field():
    H = oasm.matrix(synth.icosphere(2), 1e-4, op=H_OP, near=True)
    assert np.max(np.abs(H.sum(1))) < 1e-5


def test_jump_and_derivatives():
    mesh = synth.icosphere(1)
    k = 2.0 + 0.2j
    H = oasm.matrix(mesh, k, op=H_OP)
    assert np.all(np.diag(H) == 0.5)
    Hd = oasm.matrix(mesh, k, deriv=1, op=H_OP)
    assert np.all(np.diag(Hd) == 0.0)
    h = 1e-5
    fd = (oasm.matrix(mesh, k + h, op=H_OP) - oasm.matrix(mesh, k - h, op=H_OP)) / (2 * h)
    off = ~np.eye(mesh.n, dtype=bool)
    assert np.max(np.abs(Hd - fd)[off]) < 1e-8 * np.max(np.abs(Hd))
    Hdn = oasm.matrix(mesh, k, deriv=1, op=H_OP, near=True)
    fdn = (oasm.matrix(mesh, k + h, op=H_OP, near=True) -
           oasm.matrix(mesh, k - h, op=H_OP, near=True)) / (2 * h)
    assert np.max(np.abs(Hdn - fdn)[off]) < 1e-8 * np.max(np.abs(Hdn))


def test_seven_point_rule_against_conical_rule_far_pair():
    mesh = synth.icosphere(3)
    c, _, _, _ = oasm.geometry(mesh)
    i = 0
    d = np.linalg.norm(c - c[i], axis=1)
    l = int(np.argsort(d)[len(d) // 3])          # a panel far from x_i
    k = 2.5 + 0.1j
    H = oasm.matrix(mesh, k, op=H_OP, rows=(i, i + 1))
    v = mesh.xyz[mesh.tri[l]]
    ref = oasm.near_rule(v[0], v[1], v[2], c[i], k, order=32, kind=1)
    assert abs(H[0, l] - ref) < 1e-7 * abs(ref)


def test_combination_is_linear():
    mesh = synth.icosphere(0)
    k = 1.7 + 0.1j
    G = oasm.matrix(mesh, k)
    H = oasm.matrix(mesh, k, op=H_OP)
    T = oasm.matrix(mesh, k, op=(0.3 - 0.2j, 1.1 + 0.5j))
    assert np.max(np.abs(T - ((0.3 - 0.2j) * G + (1.1 + 0.5j) * H))) < 1e-14 * np.max(np.abs(T))


def test_neumann_eigenvalues_near_bessel_zeros():
    rows = np.loadtxt(os.path.join(HERE, "golden", "eigs_sphere320_neumann.txt"), ndmin=2)
    lam = rows[:, 0] + 1j * rows[:, 1]
    mult = rows[:, 2].astype(int)
    for target, m in ((2.081576, 3), (3.342094, 5)):
        j = int(np.argmin(np.abs(lam - target)))
        assert mult[j] == m
        assert abs(lam[j] - target) / target < 0.03
