"""Pins of the oracle's near-field variant: the 64-point conical-product rule on near panel
pairs (centroid distance below twice the larger panel diameter).

- the rule against the closed-form static potential of a triangle at points of its plane
  outside it (edge-log formula with signed edge distances), which fixes its points,
  weights and Jacobian independently of the code;
- the rule against the 7-point rule on a far pair (both exact to the 7-point rule's error);
- the near list against a brute-force numpy evaluation of the criterion;
- the near-variant matrix: near pairs carry the 8 x 8 rule, the rest the 7-point rule;
- what the near rule gains: on adjacent pairs its error against an order-48 reference is
  far below the 7-point rule's."""
import numpy as np
import pytest

import synth


def _static_inplane(v, x):
    """(1 / 4 pi) * integral over the triangle of 1 / |x - y| for x in its plane: the sum
    over edges of the signed distance times the asinh difference."""
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    total = 0.0
    for e in range(3):
        p, q = v[e], v[(e + 1) % 3]
        t = (q - p) / np.linalg.norm(q - p)
        sp, sq = np.dot(p - x, t), np.dot(q - x, t)
        d = np.linalg.norm((p - x) - sp * t)
        sign = np.sign(np.dot(np.cross(p - x, q - x), n))
        total += sign * d * (np.arcsinh(sq / d) - np.arcsinh(sp / d))
    return total / (4 * np.pi)


def test_near_rule_static_closed_form_outside(oracle_mod):
    """Points of the plane beyond an edge (barycentric coordinates with one negative): the
    rule converges to the closed form, to rounding at order 64."""
    rng = np.random.default_rng(5)
    for _ in range(6):
        v = [rng.normal(size=3) for _ in range(3)]
        for b in ([0.8, 0.8, -0.6], [1.2, 0.6, -0.8]):
            b = np.array(b)
            x = b[0] * v[0] + b[1] * v[1] + b[2] * v[2]
            ref = _static_inplane(v, x)
            got = oracle_mod.assembly.near_rule(v[0], v[1], v[2], x, 0.0, order=64)
            assert abs(got.real - ref) < 1e-12 * abs(ref) and abs(got.imag) == 0.0, (got, ref)
            low = oracle_mod.assembly.near_rule(v[0], v[1], v[2], x, 0.0, order=8)
            assert abs(low.real - ref) < 5e-3 * abs(ref)


def test_near_rule_far_pair_matches_rule7(oracle_mod):
    m = synth.icosphere(3)
    c, _, qp, qw = oracle_mod.assembly.geometry(m)
    far = int(np.argmax(np.linalg.norm(c - c[0], axis=1)))
    k = 5.0 + 0.2j
    r = np.linalg.norm(qp[far] - c[0], axis=1)
    ref7 = np.sum(qw[far] * np.exp(1j * k * r) / (4 * np.pi * r))
    v = m.xyz[m.tri[far]]
    got = oracle_mod.assembly.near_rule(v[0], v[1], v[2], c[0], k, order=8)
    assert abs(got - ref7) < 1e-9 * abs(ref7)
    gd = oracle_mod.assembly.near_rule(v[0], v[1], v[2], c[0], k, deriv=1, order=8)
    refd = np.sum(qw[far] * 1j * np.exp(1j * k * r) / (4 * np.pi))
    assert abs(gd - refd) < 1e-9 * abs(refd)


@pytest.mark.parametrize("mesh_fn", [lambda: synth.icosphere(2), lambda: synth.cube_grid(4),
                                     lambda: synth.cube_sphere(5, (1.6, 0.9, 0.6))])
def test_near_pairs_brute_force(oracle_mod, mesh_fn):
    m = mesh_fn()
    v = m.xyz[m.tri]                                  # (n, 3, 3)
    cen = v.mean(axis=1)
    edges = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 1], v[:, 0] - v[:, 2]], axis=1)
    diam = np.linalg.norm(edges, axis=2).max(axis=1)
    dist = np.linalg.norm(cen[:, None, :] - cen[None, :, :], axis=2)
    near = dist < 2.0 * np.maximum(diam[:, None], diam[None, :])
    np.fill_diagonal(near, False)
    row_ptr, cols = oracle_mod.assembly.near_pairs(m)
    assert row_ptr[-1] == near.sum()
    for i in range(m.n):
        assert np.array_equal(cols[row_ptr[i]:row_ptr[i + 1]], np.nonzero(near[i])[0])


def test_near_matrix_composition(oracle_mod):
    m = synth.icosphere(1)
    k = 3.7 - 0.4j
    A7 = oracle_mod.assembly.matrix(m, k)
    An = oracle_mod.assembly.matrix(m, k, near=True)
    row_ptr, cols = oracle_mod.assembly.near_pairs(m)
    mask = np.zeros_like(A7, dtype=bool)
    c, *_ = oracle_mod.assembly.geometry(m)
    for i in range(m.n):
        for l in cols[row_ptr[i]:row_ptr[i + 1]]:
            mask[i, l] = True
            v = m.xyz[m.tri[l]]
            ref = oracle_mod.assembly.near_rule(v[0], v[1], v[2], c[i], k, order=8)
            assert An[i, l] == ref
    assert np.array_equal(An[~mask], A7[~mask])
    assert np.max(np.abs(An[mask] - A7[mask])) > 0.0


def test_near_rule_gain_on_adjacent_pairs(oracle_mod):
    """Adjacent panels of a fine sphere: the 8 x 8 rule is far closer to an order-48
    reference than the 7-point rule is (the reason near pairs get it)."""
    m = synth.icosphere(3)
    c, _, qp, qw = oracle_mod.assembly.geometry(m)
    row_ptr, cols = oracle_mod.assembly.near_pairs(m, rows=(0, 40))
    k = 6.0 + 0.3j
    e7, e8 = [], []
    for i in range(40):
        for l in cols[row_ptr[i]:row_ptr[i + 1]]:
            v = m.xyz[m.tri[l]]
            ref = oracle_mod.assembly.near_rule(v[0], v[1], v[2], c[i], k, order=48)
            r = np.linalg.norm(qp[l] - c[i], axis=1)
            a7 = np.sum(qw[l] * np.exp(1j * k * r) / (4 * np.pi * r))
            a8 = oracle_mod.assembly.near_rule(v[0], v[1], v[2], c[i], k, order=8)
            e7.append(abs(a7 - ref) / abs(ref))
            e8.append(abs(a8 - ref) / abs(ref))
    e7, e8 = np.array(e7), np.array(e8)
    assert e8.max() < 1e-4 and np.median(e8) < 1e-6
    assert e7.max() > 1e-3 and np.median(e7) > 30 * np.median(e8)
