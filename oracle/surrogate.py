"""Oracle of the near-field surrogate network: plain numpy FP64 forward pass, loss and
backward pass (test infrastructure only: only the tests load it).

The network maps the canonical features of a near panel pair to the pair's near-field
correction (A_near - A_7) / h (h the panel diameter). Features: the triangle's vertices in a
frame with its origin at the collocation point x, e1 along (b - a), e3 along the normal
(b - a) x (c - b) flipped so that a lies on its non-negative side, e2 = e3 x e1 (a the vertex
nearest x, b and c following it in the triangle's order), each divided by h; then Re(k h),
Im(k h). Network: standardisation (f - shift) * scale, then 11 -> 64 -> 64 -> 64 -> 2 with
tanh on the hidden layers; the prediction is out_scale * z / (d/h)^7, z the last layer's
output and d/h the distance from x to the triangle's centroid read off the features.
Loss: mean over samples of sum_o (z_o - target_o (d/h)^7 / out_scale_o)^2.

Parameter layout (one flat array, the same order as the library's):
in_shift[11], in_scale[11], W1[64][11], b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
W4[2][64], b4[2], out_scale[2].
"""
import numpy as np

IN, HID, OUT = 11, 64, 2
_SHAPES = [("in_shift", (IN,)), ("in_scale", (IN,)), ("W1", (HID, IN)), ("b1", (HID,)),
           ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)), ("b3", (HID,)),
           ("W4", (OUT, HID)), ("b4", (OUT,)), ("out_scale", (OUT,)),
           ("feat_lo", (IN,)), ("feat_hi", (IN,))]
SIZE = sum(int(np.prod(s)) for _, s in _SHAPES)
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def unpack(params):
    """Views of the flat parameter array by name."""
    out, o = {}, 0
    params = np.asarray(params)
    for name, shape in _SHAPES:
        size = int(np.prod(shape))
        out[name] = params[o:o + size].reshape(shape)
        o += size
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel()
                           for name, _ in _SHAPES])


def decay(feat):
    """(d/h)^7 per sample, d/h the norm of the mean of the three vertex features."""
    f = np.asarray(feat, dtype=np.float64)
    c = (f[:, 0:3] + f[:, 3:6] + f[:, 6:9]) / 3.0
    return np.sum(c * c, axis=1) ** 3.5


def forward(params, feat):
    """Prediction (n, 2) and the activations needed by the backward pass."""
    p = unpack(np.asarray(params, dtype=np.float64))
    x = (np.asarray(feat, dtype=np.float64) - p["in_shift"]) * p["in_scale"]
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    z = h3 @ p["W4"].T + p["b4"]
    return z * p["out_scale"] / decay(feat)[:, None], (x, h1, h2, h3, z)


def loss_and_grad(params, feat, target):
    """Mean over samples of sum_o (z_o - target_o (d/h)^7 / out_scale_o)^2 and its gradient
    with respect to the flat parameter array (zero for the standardisation and output
    scaling)."""
    p = unpack(np.asarray(params, dtype=np.float64))
    pred, (x, h1, h2, h3, z) = forward(params, feat)
    n = pred.shape[0]
    diff = z - np.asarray(target, dtype=np.float64) * decay(feat)[:, None] / p["out_scale"]
    loss = np.sum(diff * diff) / n
    dz = 2.0 * diff / n                                   # dL/dz, z the pre-scaling output
    g = {name: np.zeros(shape) for name, shape in _SHAPES}
    g["W4"] = dz.T @ h3
    g["b4"] = dz.sum(axis=0)
    d3 = (dz @ p["W4"]) * (1.0 - h3 * h3)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def features(tri_vertices, x, k, h):
    """Canonical features of one pair: triangle vertices (3, 3), collocation point x (3,),
    wavenumber k, panel diameter h. Written from the frame's definition above."""
    v = np.asarray(tri_vertices, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    d = np.linalg.norm(v - x, axis=1)
    a = 0
    for q in (1, 2):
        if d[q] < d[a]:
            a = q
    A, B, C = v[a], v[(a + 1) % 3], v[(a + 2) % 3]
    e1 = (B - A) / np.linalg.norm(B - A)
    e3 = np.cross(B - A, C - B)
    e3 /= np.linalg.norm(e3)
    if np.dot(A - x, e3) < 0.0:
        e3 = -e3
    e2 = np.cross(e3, e1)
    f = []
    for P in (A, B, C):
        r = P - x
        f += [np.dot(r, e1) / h, np.dot(r, e2) / h, np.dot(r, e3) / h]
    k = complex(k)
    return np.array(f + [k.real * h, k.imag * h])
