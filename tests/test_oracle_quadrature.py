"""Pins of the oracle's quadrature and matrix entries against facts fixed independently of
it: exact monomial integrals, Gauss-Legendre moments, a Duffy-transformed tensor rule for
the singular self term, the closed-form static potential of a triangle, finite
differences for dA/dk, and the single-layer closed form on the unit sphere."""
import math

import numpy as np
import pytest

import synth


def test_rule7_integrates_degree5_exactly(oracle_mod):
    b, w = oracle_mod.assembly.rule7()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(b.sum(axis=1), 1.0)
    for a in range(6):
        for c in range(6 - a):
            # reference triangle (0,0), (1,0), (0,1): x = b1, y = b2, area 1/2
            val = 0.5 * np.sum(w * b[:, 1] ** a * b[:, 2] ** c)
            exact = math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
            assert abs(val - exact) < 1e-16, (a, c)
    # and not degree 6 (it is a degree-5 rule)
    val = 0.5 * np.sum(w * b[:, 1] ** 6)
    assert abs(val - math.factorial(6) / math.factorial(8)) > 1e-6


def test_gauss_legendre16_moments(oracle_mod):
    x, w = oracle_mod.assembly.gauss_legendre(16)
    for k in range(32):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    assert abs(np.sum(w * x ** 32) - 2.0 / 33) > 1e-10


def _duffy_self(v, x, k, n=200):
    """Independent rule: split at x into three triangles, Duffy map (s, t) -> x + s (p - x
    + t (q - p)) removes the 1/r singularity; tensor Gauss-Legendre in (s, t)."""
    g, gw = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (g + 1.0); sw = 0.5 * gw
    total = 0.0 + 0.0j
    for e in range(3):
        p, q = v[e], v[(e + 1) % 3]
        jac = np.linalg.norm(np.cross(p - x, q - p))
        for t, tw in zip(s, sw):
            rho = np.linalg.norm(p - x + t * (q - p))
            total += tw * np.sum(sw * np.exp(1j * k * s * rho)) / (4 * np.pi * rho) * jac
    return total


@pytest.mark.parametrize("tri", [
    [(0, 0, 0), (1, 0, 0), (0, 1, 0)],
    [(0.1, 0.2, 0.3), (0.4, 0.25, 0.1), (0.2, 0.5, 0.45)],
    [(0, 0, 0), (1, 0, 0), (0.5, 0.25, 0.0)],
])
@pytest.mark.parametrize("k", [0.0, 3.3, 7.2 + 0.4j, 10.0 - 1.0j])
def test_self_term_against_duffy(oracle_mod, tri, k):
    v = [np.array(p, dtype=float) for p in tri]
    x = (v[0] + v[1] + v[2]) / 3.0
    got = oracle_mod.assembly.self_integral(v[0], v[1], v[2], x, k)
    ref = _duffy_self(v, x, k)
    assert abs(got - ref) <= 1e-11 * abs(ref), (got, ref)


def test_self_term_static_closed_form(oracle_mod):
    """k = 0: sum over edges of d [asinh(s/d)] / (4 pi), the potential of a uniform
    triangle at an interior point (edge-log formula)."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        v = [rng.normal(size=3) for _ in range(3)]
        bary = rng.dirichlet([3, 3, 3])
        x = bary[0] * v[0] + bary[1] * v[1] + bary[2] * v[2]
        ref = 0.0
        for e in range(3):
            p, q = v[e], v[(e + 1) % 3]
            t = (q - p) / np.linalg.norm(q - p)
            sp, sq = np.dot(p - x, t), np.dot(q - x, t)
            d = np.linalg.norm((p - x) - sp * t)
            ref += d * (np.arcsinh(sq / d) - np.arcsinh(sp / d))
        ref /= 4 * np.pi
        got = oracle_mod.assembly.self_integral(v[0], v[1], v[2], x, 0.0)
        assert abs(got.real - ref) < 1e-13 * abs(ref) and abs(got.imag) == 0.0


def test_derivative_matches_finite_difference(oracle_mod):
    m = synth.icosphere(1)
    k = 4.1 + 0.3j
    h = 1e-5
    Ad = oracle_mod.assembly.matrix(m, k, deriv=1)
    fd = (oracle_mod.assembly.matrix(m, k + h) - oracle_mod.assembly.matrix(m, k - h)) / (2 * h)
    assert np.max(np.abs(Ad - fd)) < 1e-8 * np.max(np.abs(Ad))


def test_entries_far_pair_against_fine_rule(oracle_mod):
    """A well-separated pair: the 7-point value agrees with a fine Duffy-free tensor rule
    on the source triangle to the 7-point rule's own accuracy."""
    m = synth.icosphere(3)
    A = oracle_mod.assembly.matrix(m, 5.0 + 0.2j, rows=(0, 1))
    c, area, _, _ = oracle_mod.assembly.geometry(m)
    far = int(np.argmax(np.linalg.norm(c - c[0], axis=1)))
    v = m.xyz[m.tri[far]]
    g, gw = np.polynomial.legendre.leggauss(30)
    s = 0.5 * (g + 1); sw = 0.5 * gw
    ref = 0.0
    for si, swi in zip(s, sw):
        for ti, twi in zip(s, sw):
            y = v[0] + si * (v[1] - v[0]) + si * ti * (v[2] - v[1])
            r = np.linalg.norm(c[0] - y)
            ref += swi * twi * si * np.exp(1j * (5.0 + 0.2j) * r) / (4 * np.pi * r)
    ref *= 2 * area[far]
    assert abs(A[0, far] - ref) < 1e-7 * abs(ref)


def test_row_sum_single_layer_sphere(oracle_mod):
    """sum_l A_il(k) -> (single layer of a unit density on the unit sphere at the surface)
    = i k j0(k) h0(k) = exp(i k) sin(k) / k, at rate O(h^2) on icospheres."""
    k = 2.5
    exact = np.exp(1j * k) * np.sin(k) / k
    errs = []
    for L in (1, 2, 3):
        m = synth.icosphere(L)
        A = oracle_mod.assembly.matrix(m, k, rows=(0, 8))
        errs.append(np.max(np.abs(A.sum(axis=1) - exact)))
    assert errs[2] < errs[1] < errs[0]
    assert 2.5 < errs[1] / errs[2] < 6.0
    assert errs[2] < 2e-2 * abs(exact)
