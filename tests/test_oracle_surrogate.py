"""Pins of the surrogate network's oracle (oracle/surrogate.py): the backward pass against
central finite differences of the forward pass in FP64, the forward pass in a case with a
closed form (including the (d/h)^7 decay factor), and the invariances of the canonical features and of the normalised target
(rigid motions, cyclic vertex order, joint scaling of geometry and wavelength)."""
import numpy as np

import synth
from oracle import surrogate as osur, assembly as oasm


def _random_params(rng, scale=0.4):
    p = osur.unpack(np.zeros(osur.SIZE))
    out = {}
    for name, arr in p.items():
        out[name] = rng.normal(scale=scale, size=arr.shape)
    out["in_shift"] = rng.normal(scale=0.1, size=osur.IN)
    out["in_scale"] = 1.0 + 0.2 * rng.random(osur.IN)
    out["out_scale"] = 0.5 + rng.random(osur.OUT)
    return osur.pack(out)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    params = _random_params(rng)
    feat = rng.normal(size=(7, osur.IN))
    target = rng.normal(size=(7, osur.OUT))
    loss, grad = osur.loss_and_grad(params, feat, target)
    u = osur.unpack(np.arange(osur.SIZE))
    trained = np.concatenate([u[n].ravel() for n in osur.TRAINED]).astype(int)
    fixed = np.setdiff1d(np.arange(osur.SIZE), trained)
    assert np.all(grad[fixed] == 0.0)
    h = 1e-6
    for idx in rng.choice(trained, size=60, replace=False):
        e = np.zeros(osur.SIZE)
        e[idx] = h
        lp, _ = osur.loss_and_grad(params + e, feat, target)
        lm, _ = osur.loss_and_grad(params - e, feat, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[idx]) <= 1e-6 * max(abs(grad[idx]), 1e-3 * abs(loss)), (idx, fd, grad[idx])


def test_forward_constant_when_hidden_weights_vanish():
    rng = np.random.default_rng(4)
    p = osur.unpack(_random_params(rng))
    p = {k: v.copy() for k, v in p.items()}
    p["W4"][:] = 0.0
    feat = rng.normal(size=(5, osur.IN))
    out, _ = osur.forward(osur.pack(p), feat)
    # the prediction is out_scale * b4 / (d/h)^7, d/h the norm of the vertices' mean
    c = (feat[:, 0:3] + feat[:, 3:6] + feat[:, 6:9]) / 3.0
    dh = np.sqrt(np.sum(c * c, axis=1))
    assert np.allclose(out * dh[:, None] ** 7, p["b4"] * p["out_scale"], rtol=1e-13, atol=0)


def _rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_features_invariant_under_rigid_motion_and_vertex_order():
    rng = np.random.default_rng(6)
    m = synth.icosphere(3)
    c, *_ = oasm.geometry(m)
    row_ptr, cols = oasm.near_pairs(m, rows=(0, 5))
    k = 7.0 - 0.4j
    for i in range(5):
        for l in cols[row_ptr[i]:row_ptr[i + 1]][:6]:
            v = m.xyz[m.tri[l]]
            h = max(np.linalg.norm(v[1] - v[0]), np.linalg.norm(v[2] - v[0]),
                    np.linalg.norm(v[2] - v[1]))
            f0 = osur.features(v, c[i], k, h)
            Q, t = _rotation(rng), rng.normal(size=3)
            f1 = osur.features(v @ Q.T + t, Q @ c[i] + t, k, h)
            f2 = osur.features(np.roll(v, 1, axis=0), c[i], k, h)
            assert np.max(np.abs(f1 - f0)) < 1e-12 and np.max(np.abs(f2 - f0)) < 1e-12


def test_normalised_target_scale_free():
    """(A_near - A_7) / h depends on the pair's shape and on k h only."""
    m = synth.icosphere(3)
    c, _, qp, qw = oasm.geometry(m)
    row_ptr, cols = oasm.near_pairs(m, rows=(0, 1))
    l = cols[0]
    v = m.xyz[m.tri[l]]
    h = max(np.linalg.norm(v[1] - v[0]), np.linalg.norm(v[2] - v[0]), np.linalg.norm(v[2] - v[1]))

    def corr(scale, k):
        vv, x = v * scale, c[0] * scale
        r = np.linalg.norm(qp[l] * scale - x, axis=1)
        a7 = np.sum(qw[l] * scale ** 2 * np.exp(1j * k * r) / (4 * np.pi * r))
        return (oasm.near_rule(vv[0], vv[1], vv[2], x, k, order=8) - a7) / (h * scale)

    base = corr(1.0, 6.0 + 0.5j)
    for s in (0.3, 2.5):
        # the correction is a small difference of two entries: rounding of the entries sets the bar
        assert abs(corr(s, (6.0 + 0.5j) / s) - base) < 1e-10 * abs(base)
