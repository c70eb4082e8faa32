"""Fits the polynomials of trig_poly.cuh and writes that header.

The fused kernel can evaluate part of its sines and cosines on the FP32 FMA pipe instead
of the MUFU unit. The phase phi is reduced in half revolutions, t = phi / pi, n = rint(t),
f = t - n in [-1/2, 1/2], so that e^{i phi} = (-1)^n e^{i pi f}, and then
    cos(pi f) ~ C(u),  sin(pi f) ~ f S(u),  u = f^2,
with C and S of degree 4 in u. Both are minimax fits (Remez exchange, here in float64 on a
fine grid) of the absolute error over f in [0, 1/2]: for the sine the error weight is f
(the error of f S(u)), for the cosine 1. The coefficients are rounded to FP32. Evaluated
by Horner's rule in FP32 the error is below 2e-7 (the fits' own error is below 5e-8).

Usage: python paper_1906_03938_gb300/csrc/trig_poly_fit.py  (rewrites trig_poly.cuh)
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "trig_poly.cuh")
SIN_DEG, COS_DEG = 4, 4
PI = np.pi


def _sin_over_f(u):
    f = np.sqrt(u)
    return np.where(f > 0, np.sin(PI * f) / np.where(f > 0, f, 1.0), PI)


def _cos(u):
    return np.cos(PI * np.sqrt(u))


def remez(g, w, a, b, deg, iters=40, grid=400001):
    """Coefficients c (ascending powers) of the degree-deg polynomial p minimising
    max |w(u) (p(u) - g(u))| over [a, b], and that maximum (on the grid)."""
    n = deg + 2
    x = (a + b) / 2 - (b - a) / 2 * np.cos(np.pi * np.arange(n) / (n - 1))
    xs = np.linspace(a, b, grid)
    ws, gs = w(xs), g(xs)
    c = None
    for _ in range(iters):
        A = np.zeros((n, n))
        A[:, :deg + 1] = x[:, None] ** np.arange(deg + 1)[None, :]
        A[:, deg + 1] = (-1.0) ** np.arange(n) / w(x)
        sol = np.linalg.solve(A, g(x))
        c = sol[:deg + 1]
        err = ws * (np.polyval(c[::-1], xs) - gs)
        # one extremum per run of equal sign, then the window of n alternating extrema
        # whose smallest magnitude is largest
        runs = np.split(np.arange(grid), np.where(np.diff(np.sign(err)) != 0)[0] + 1)
        ext = [r[np.argmax(np.abs(err[r]))] for r in runs if len(r)]
        if len(ext) < n:
            break
        best = max(range(len(ext) - n + 1), key=lambda s: np.min(np.abs(err[ext[s:s + n]])))
        x = xs[ext[best:best + n]]
    err = ws * (np.polyval(c[::-1], xs) - gs)
    return c, float(np.max(np.abs(err)))


def fit():
    """(sin coefficients, cos coefficients) as float32 arrays, ascending powers of u."""
    cs, _ = remez(_sin_over_f, lambda u: np.sqrt(u) + 1e-300, 0.0, 0.25, SIN_DEG)
    cc, _ = remez(_cos, lambda u: np.ones_like(u), 0.0, 0.25, COS_DEG)
    return cs.astype(np.float32), cc.astype(np.float32)


def eval_f32(f, cs, cc):
    """The header's evaluation order in FP32 (Horner in u), for a float32 array f."""
    f = f.astype(np.float32)
    u = f * f
    s = cs[-1]
    for k in range(len(cs) - 2, -1, -1):
        s = s * u + cs[k]
    c = cc[-1]
    for k in range(len(cc) - 2, -1, -1):
        c = c * u + cc[k]
    return c.astype(np.float32), (f * s).astype(np.float32)


def header_text(cs, cc):
    def lit(v):
        return f"{float(v):.9e}f"
    lines = [
        "// Polynomial sine and cosine on the FP32 FMA pipe (generated by trig_poly_fit.py:",
        "// minimax fits of cos(pi f) and sin(pi f) / f in u = f^2 over |f| <= 1/2, FP32",
        "// coefficients). The phase is reduced in half revolutions: t = phi / pi, n = rint(t)",
        "// (by the 1.5 * 2^23 shift, which leaves n in the low bits of t + shift), f = t - n,",
        "// e^{i phi} = (-1)^n e^{i pi f}; phi may be any FP32 value below ~1e6.",
        "#pragma once",
        "",
        "namespace bem {",
        "namespace trig {",
        "",
        "constexpr float kInvPi = 0.318309886f;",
        "constexpr float kRoundShift = 12582912.0f;   // 1.5 * 2^23: x + s - s = rint(x)",
    ]
    for k, v in enumerate(cs):
        lines.append(f"constexpr float kS{k} = {lit(v)};")
    for k, v in enumerate(cc):
        lines.append(f"constexpr float kC{k} = {lit(v)};")
    lines += ["", "}  // namespace trig", "}  // namespace bem", ""]
    return "\n".join(lines)


def read_header(path=HEADER):
    """The coefficients stored in the header (sin, cos), as float32 arrays."""
    vals = {}
    for line in open(path):
        line = line.strip()
        if line.startswith("constexpr float k") and ("kS" in line or "kC" in line):
            name = line.split()[2]
            if name[1] in "SC" and name[2:].isdigit():
                vals[name] = np.float32(float(line.split("=")[1].strip().rstrip(";").rstrip("f")))
    cs = np.array([vals[f"kS{k}"] for k in range(SIN_DEG + 1)], dtype=np.float32)
    cc = np.array([vals[f"kC{k}"] for k in range(COS_DEG + 1)], dtype=np.float32)
    return cs, cc


if __name__ == "__main__":
    cs, cc = fit()
    with open(HEADER, "w") as fh:
        fh.write(header_text(cs, cc))
    f = np.linspace(-0.5, 0.5, 200001).astype(np.float32)
    c, s = eval_f32(f, cs, cc)
    print("max |cos err|", np.max(np.abs(c - np.cos(PI * f.astype(np.float64)))),
          "max |sin err|", np.max(np.abs(s - np.sin(PI * f.astype(np.float64)))))
