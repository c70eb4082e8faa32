"""The double-FP32 residual (bem_residual_arith, arith 1) against the FP64 residual
(arith 0) through the C ABI, and the FP64 one against the oracle.

Bar, from the arithmetic: every off-diagonal entry is evaluated in pairs of FP32 numbers
(~48 significant bits) to a relative error of about 1e-13; A(lambda) x and A'(lambda) x
sum n such terms, so the two arithmetics agree to 1e-11 of the largest component (and the
relative residuals to 1e-10 of themselves). The cases cover a ragged last block of rows,
the near-field corrections (which stay FP64) and wavenumbers with Im k of both signs."""
import numpy as np
import pytest
import torch

import synth
from oracle import assembly as oasm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _relerr(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("case", ["sphere320", "cube_ragged", "sphere1280_near"])
def test_double_fp32_residual_matches_fp64(bem, case):
    if case == "sphere320":
        mesh, near = synth.icosphere(2), 0
        lam = np.array([3.2 + 0.05j, 4.4 - 0.3j, 4.0 + 0.9j])
    elif case == "cube_ragged":
        mesh, near = synth.cube_grid(5), 0            # 150 panels: a ragged 128-row block
        lam = np.array([5.5 - 0.2j, 7.0 + 0.4j])
    else:
        mesh, near = synth.icosphere(3), 1
        lam = np.array([6.3 + 0.0j, 7.7 - 1.0j])
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    if near:
        ctx.set_near_field(1)
    X = synth.complex_gaussian(mesh.n, len(lam), 17)
    Xd = bem.fortran(torch.from_numpy(X).to("cuda:0"))
    rel64, R64, D64 = ctx.residual_arith(lam, Xd, arith=0, deriv=True)
    relff, Rff, Dff = ctx.residual_arith(lam, Xd, arith=1, deriv=True)
    R64, D64, Rff, Dff = (t.cpu().numpy() for t in (R64, D64, Rff, Dff))
    for c in range(len(lam)):
        assert _relerr(Rff[:, c], R64[:, c]) < 1e-11, (case, c)
        assert _relerr(Dff[:, c], D64[:, c]) < 1e-11, (case, c)
        assert abs(relff[c] - rel64[c]) <= 1e-10 * rel64[c]
    # the FP64 arithmetic itself against the oracle's dense FP64 matrix (and its k-derivative)
    for c in range(len(lam)):
        A = oasm.matrix(mesh, lam[c], near=bool(near))
        Ad = oasm.matrix(mesh, lam[c], deriv=1, near=bool(near))
        assert _relerr(R64[:, c], A @ X[:, c]) < 1e-11
        assert _relerr(D64[:, c], Ad @ X[:, c]) < 1e-11
    ctx.close()
