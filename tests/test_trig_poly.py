"""The FMA-pipe sine and cosine of the fused kernel (csrc/trig_poly.cuh, csrc/f32x2.cuh).

* The header's coefficients are exactly what the committed fit script produces (minimax
  fits by the Remez exchange, rounded to FP32), so they can be regenerated and checked.
* Evaluated in FP32 in the kernel's order (Horner in u = f^2), cos(pi f) and sin(pi f)
  stay within 2e-7 of the exact values over |f| <= 1/2.
* The half-revolution reduction of the kernel, emulated here step by step in FP32
  (t = phi / pi, the 1.5 * 2^23 shift, n from the low bit of the shifted value, sign
  flip), gives e^{i phi} within 2e-7 + (the FP32 rounding of phi / pi) over the phases
  the kernel meets (0 to 40 rad), with the sign logic right in every half revolution."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_1906_03938_gb300", "csrc")


def _fitmod():
    spec = importlib.util.spec_from_file_location("trig_poly_fit",
                                                  os.path.join(SRC, "trig_poly_fit.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_matches_the_fit():
    m = _fitmod()
    cs, cc = m.fit()
    hs, hc = m.read_header(os.path.join(SRC, "trig_poly.cuh"))
    assert np.array_equal(cs, hs) and np.array_equal(cc, hc)
    assert open(os.path.join(SRC, "trig_poly.cuh")).read() == m.header_text(cs, cc)


def test_fp32_evaluation_error():
    m = _fitmod()
    cs, cc = m.read_header(os.path.join(SRC, "trig_poly.cuh"))
    f = np.linspace(-0.5, 0.5, 400001).astype(np.float32)
    c, s = m.eval_f32(f, cs, cc)
    x = np.pi * f.astype(np.float64)
    assert np.max(np.abs(c - np.cos(x))) < 2e-7
    assert np.max(np.abs(s - np.sin(x))) < 2e-7
    # odd / even symmetry is exact (the sine is f times an even polynomial)
    assert np.array_equal(s[::-1], -s) and np.array_equal(c[::-1], c)


def test_half_revolution_reduction_and_sign():
    m = _fitmod()
    cs, cc = m.read_header(os.path.join(SRC, "trig_poly.cuh"))
    f32 = np.float32
    inv_pi, shift = f32(0.318309886), f32(12582912.0)
    ph = np.concatenate([np.linspace(0.0, 40.0, 300001),
                         np.pi * np.arange(0, 13) + 1e-3]).astype(np.float32)
    t = (ph * inv_pi).astype(np.float32)
    tb = (t + shift).astype(np.float32)
    n = (tb - shift).astype(np.float32)
    f = (t - n).astype(np.float32)
    assert np.all(np.abs(f) <= 0.5)
    c, s = m.eval_f32(f, cs, cc)
    odd = (tb.view(np.uint32) & 1).astype(bool)
    assert np.array_equal(odd, (n.astype(np.int64) % 2) == 1)
    sign = np.where(odd, -1.0, 1.0)
    z = sign * (c.astype(np.float64) + 1j * s.astype(np.float64))
    exact = np.exp(1j * ph.astype(np.float64))
    # FP32 rounding of t = phi / pi (and of the constant) moves the phase by ~ |t| 2^-24 pi
    bound = 2.5e-7 + np.pi * np.abs(t.astype(np.float64)) * 2.0 ** -23
    assert np.all(np.abs(z - exact) <= bound)
