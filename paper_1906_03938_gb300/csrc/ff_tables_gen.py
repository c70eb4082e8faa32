"""Writes ff_tables.cuh: the constants of the double-FP32 ("float-float") evaluation of
e^{i k r} used by the fast residual kernel, computed here in 60-digit arithmetic (mpmath)
and split into FP32 pairs (hi, lo) with hi = fl32(v), lo = fl32(v - hi):

* cos(j pi / 32), sin(j pi / 32), j = 0..63 (the table of the phase reduction by pi / 32);
* 2^(j / 32), j = 0..31 (the table of the exponential's reduction by 1 / 32 in base 2);
* pi / 32 in three FP32 parts P1 + P2 + P3 with P1 of 12 significant bits, so that j P1
  is exact in FP32 for j < 2^11 (Cody and Waite's additive reduction);
* log2(e) and ln(2) as FP32 pairs, 32 / pi as one FP32.

Usage: python paper_1906_03938_gb300/csrc/ff_tables_gen.py  (rewrites ff_tables.cuh)
"""
import os

import mpmath
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "ff_tables.cuh")
mpmath.mp.dps = 60


def split(v):
    """(hi, lo) FP32 pair of the high-precision value v."""
    hi = np.float32(float(v))
    lo = np.float32(float(v - mpmath.mpf(float(hi))))
    return hi, lo


def round_bits(v, bits):
    """v rounded to `bits` significant bits (a float exactly representable in FP32)."""
    m, e = mpmath.frexp(v)
    return mpmath.ldexp(mpmath.nint(m * 2 ** bits), e - bits)


def tables():
    cs = [split(mpmath.cos(j * mpmath.pi / 32)) for j in range(64)]
    sn = [split(mpmath.sin(j * mpmath.pi / 32)) for j in range(64)]
    e2 = [split(mpmath.power(2, mpmath.mpf(j) / 32)) for j in range(32)]
    q = mpmath.pi / 32
    p1 = round_bits(q, 12)
    p2 = mpmath.mpf(float(np.float32(float(q - p1))))
    p3 = mpmath.mpf(float(np.float32(float(q - p1 - p2))))
    consts = {
        "kP1": np.float32(float(p1)), "kP2": np.float32(float(p2)), "kP3": np.float32(float(p3)),
        "kInvPi32": np.float32(float(32 / mpmath.pi)),
    }
    pairs = {"kLog2e": split(1 / mpmath.log(2)), "kLn2": split(mpmath.log(2))}
    return cs, sn, e2, consts, pairs


def lit(v):
    return f"{float(v):.9e}f"


def header_text():
    cs, sn, e2, consts, pairs = tables()
    out = ["// Constants of the double-FP32 evaluation of e^{i k r} (generated by",
           "// ff_tables_gen.py from 60-digit values; each pair is hi = fl32(v),",
           "// lo = fl32(v - hi)).", "#pragma once", "", "namespace bem {", "namespace ff {", ""]
    for name, v in consts.items():
        out.append(f"constexpr float {name} = {lit(v)};")
    for name, (h, l) in pairs.items():
        out.append(f"constexpr float {name}Hi = {lit(h)};")
        out.append(f"constexpr float {name}Lo = {lit(l)};")
    out.append("")
    out.append("// cos(j pi / 32), sin(j pi / 32): {cos hi, cos lo, sin hi, sin lo}, j = 0..63")
    out.append("__device__ __constant__ float kTrigTable[64][4] = {")
    for j in range(64):
        out.append(f"    {{{lit(cs[j][0])}, {lit(cs[j][1])}, {lit(sn[j][0])}, {lit(sn[j][1])}}},")
    out.append("};")
    out.append("// 2^(j / 32): {hi, lo}, j = 0..31")
    out.append("__device__ __constant__ float kExp2Table[32][2] = {")
    for j in range(32):
        out.append(f"    {{{lit(e2[j][0])}, {lit(e2[j][1])}}},")
    out.append("};")
    out += ["", "}  // namespace ff", "}  // namespace bem", ""]
    return "\n".join(out)


if __name__ == "__main__":
    with open(HEADER, "w") as f:
        f.write(header_text())
    print("wrote", HEADER)
