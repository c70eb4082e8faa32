"""Writes the stored expected eigenvalues under tests/golden/ by calling only the oracle.

For each workload, the discrete eigenvalues of A(k) strictly inside its contour (the plain
definition of the method's output, Section 1: all k inside the contour with T(k)u = 0),
found by the oracle's successive-linear-problems refinement started from the closed-form
continuum eigenvalues inside the contour (unit sphere: zeros of spherical Bessel functions,
Table 3; unit cube: pi sqrt(n1^2 + n2^2 + n3^2), Table 1) and from every neighbour that the
refinement reveals. "sphere320_near" is the same sphere with the near-field variant of A
(8 x 8 conical rule on near panel pairs). "sphere320_neumann" is the sphere with the
operator T = 1/2 I + K (the double layer with its jump: the interior Neumann problem, the
paper's T = A H - B G with B = 0), started from the zeros of j_1' and j_2' (2.0816,
3.3421) inside the circle of centre 2.75 and radius 0.9. "sphere20480_near" is the icosphere
of level 5 with the near-field variant inside the circle of centre 7 and radius 1, started
from the zeros of j_0, j_3 and j_1 there (6.2832, 6.9879, 7.7253; about two hours on eight
cores: every step factorises the dense n = 20480 matrix). "batch48_p<i>" is problem i of
the 48-ellipsoid sweep (no closed form: started from a grid of points inside its circle).
Usage:
python tests/golden/make_golden.py [sphere320] [cube3072] [sphere320_near] [sphere320_neumann]
                                   [sphere20480_near] [batch48_p9] [batch48_p14]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth                      # noqa: E402
from oracle import refine, contour  # noqa: E402

STARTS = {
    "sphere320": [3.141593, 4.493409],
    "cube3072": [5.441398, 7.695299],
    "sphere320_near": [3.141593, 4.493409],
    "sphere320_neumann": [2.081576, 3.342094],
    "sphere20480_near": [6.283185, 6.987932, 7.725252],
}
OPERATOR = {"sphere320_neumann": (0.0, 1.0)}
CONTOUR = {"sphere320_neumann": synth.ContourSpec("circle", 2.75 + 0j, 0.9, 0.9)}


def _batch_starts(spec):
    """Starts for an ellipsoid of the 48-problem sweep (no closed form): the circle's
    centre, six points at half its radius and two on the real axis at 0.85 of it."""
    c, r = spec.centre, spec.a
    pts = [c] + [c + 0.5 * r * np.exp(2j * np.pi * k / 6) for k in range(6)]
    return pts + [c - 0.85 * r, c + 0.85 * r]


def main(names):
    for name in names:
        near = name.endswith("_near")
        base = name.split("_")[0]
        if base == "batch48":   # batch48_p<i>: problem i of the sweep
            prob = synth.workload(base).problems[int(name.split("_p")[1])]
            starts, radius = _batch_starts(prob.contour), prob.contour.a
        else:
            prob = synth.workload(base).problems[0]
            starts, radius = STARTS[name], 0.2
        mesh = prob.mesh()
        spec = CONTOUR.get(name, prob.contour)
        op = OPERATOR.get(name)
        found = refine.discrete_eigs(mesh, starts, radius=radius,
                                     keep=lambda l: bool(contour.inside(l, spec, -0.05)),
                                     near=near, op=op)
        path = os.path.join(HERE, f"eigs_{name}.txt")
        with open(path, "w") as f:
            f.write(f"# discrete eigenvalues of A(k) inside the contour of {name}"
                    f"{' (near-field variant of A)' if near else ''}"
                    f"{f' (operator c_G G + c_H (I/2 + K), (c_G, c_H) = {op})' if op else ''}\n")
            f.write(f"# mesh {mesh.name} (n = {mesh.n}), contour {spec}\n")
            f.write("# written by tests/golden/make_golden.py (oracle only)\n")
            f.write("# re im multiplicity inside\n")
            for lam, mult in found:
                if not contour.inside(lam, spec, -0.05):   # a start that wandered off
                    continue
                ins = int(bool(contour.inside(lam, spec)))
                f.write(f"{lam.real:.17g} {lam.imag:.17g} {mult} {ins}\n")
        print(name, found)


if __name__ == "__main__":
    main(sys.argv[1:] or list(STARTS))
