"""The order test of Section 4, Example 3 (bem_select_order) against the oracle's
(oracle/contour.py select_order on dense FP64 matrices), through the C ABI.

The GPU applies T(z) in double-FP32 arithmetic (entries to ~1e-13), the oracle in FP64, so
the relative errors of the Cauchy approximation on the inner circle agree to 1e-6 of
themselves down to ~1e-11, and both choose the same order. The errors fall geometrically
with N (the nearest singularity of T sits outside the contour)."""
import numpy as np
import pytest
import torch

import synth
from oracle import assembly as oasm, contour as ocon

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


@pytest.mark.parametrize("near", [0, 1])
def test_select_order_matches_oracle(bem, near):
    mesh = synth.icosphere(2)
    spec = synth.ContourSpec("circle", 4.0 + 0.2j, 1.0, 1.0)
    N_list = [4, 8, 12, 16, 24, 32]
    X = synth.complex_gaussian(mesh.n, 3, 12)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    if near:
        ctx.set_near_field(1)
    Xd = bem.fortran(torch.from_numpy(X).to("cuda:0"))
    chosen, errs = ctx.select_order("circle", spec.centre, spec.a, spec.b, N_list, Xd, 1e-6,
                                    nsamples=6)
    ref_chosen, ref = ocon.select_order(lambda z: oasm.matrix(mesh, z, near=bool(near)), spec,
                                        N_list, X, 1e-6, nsamples=6)
    print("errors", errs, ref)
    for e, r in zip(errs, ref):
        assert abs(e - r) <= 1e-6 * r + 1e-11, (e, r)
    assert chosen == ref_chosen
    assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1) if errs[k] > 1e-10)
    ctx.close()
