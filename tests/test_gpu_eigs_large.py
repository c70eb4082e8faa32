"""Per-eigenvalue accuracy of the whole method at the large workloads (bem_solve: Algorithm 1
basis, CholeskyQR2, mixed projection, reduced solve, refinement), through the C ABI.

* sphere20480 with the near-field rule (icosphere level 5, circle 7 / 1, N = 32, nu = 128):
  against the oracle's eigenvalues of the same discrete operator
  (tests/golden/eigs_sphere20480_near.txt: 6.28451 x 1, the level-5 split of the zero
  6.9879 of j_3 into 6.989352 x 3 and 6.989424 x 4, and 7.72688 x 3), every one found with
  its multiplicity, no
  converged extra inside the circle, relative error <= 1e-8 and FP64 residual <= 1e-8
  (the metric's accuracy qualifier).
* ellipsoid98304 (98304 panels, circle 9 / 1.5, N = 64, nu = 256): the oracle cannot
  factorise A at this size, so every converged eigenpair inside the circle is certified by
  its FP64 residual <= 1e-8, and the FP64 residual vector A(lambda) x itself is checked
  against the oracle's rows of A(lambda) on sampled rows, to 1e-12 of sum_l |A_il| |x_l|
  (the residual is a cancellation of terms that size)."""
import os

import numpy as np
import pytest
import torch

import bench
import synth
from oracle import assembly as oasm

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _solve(bem, name, near, seed_offset=0):
    prob = synth.workload(name).problems[0]
    mesh, c = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    ctx.set_near_field(near)
    V0 = bem.fortran(torch.from_numpy(
        synth.complex_gaussian(mesh.n, prob.nu, prob.seed + seed_offset)).to("cuda:0"))
    lam, X, rel = ctx.solve(V0, q=10, precision=bem.PREC_MIXED, tol=1e-14)
    return ctx, prob, mesh, lam, X, rel


@pytest.mark.skipif(not os.path.exists(os.path.join(HERE, "golden", "eigs_sphere20480_near.txt")),
                    reason="stored oracle eigenvalues of sphere20480 absent")
def test_sphere20480_near_eigenvalues_against_oracle(bem):
    ctx, prob, mesh, lam, X, rel = _solve(bem, "sphere20480", 1)
    gold = bench.read_golden("sphere20480_near")
    res = bench.eig_compare(lam, X.cpu().numpy(), rel, gold, prob.contour, 1e-8, conv=1e-8)
    print("sphere20480", lam, rel)
    assert not res["missing"] and not res["extras"], res
    assert res["eig_rel_err_max"] <= 1e-8
    ctx.close()


def test_ellipsoid98304_eigenpairs_certified_by_fp64_residual(bem):
    ctx, prob, mesh, lam, X, rel = _solve(bem, "ellipsoid98304", 1)
    c = prob.contour
    inside = bench.inside_contour(lam, c, 0.02)
    conv = np.where(inside & (rel <= 1e-8))[0]
    print("ellipsoid98304", lam, rel)
    assert len(conv) >= 1, (lam, rel)
    # the FP64 residual vectors of two converged pairs against the oracle on sampled rows
    for k in conv[:2]:
        x = X[:, k:k + 1].contiguous()
        xr = bem.fortran(x)
        rr, R, _ = ctx.residual_arith(np.array([lam[k]]), xr, arith=0)
        assert abs(rr[0] - rel[k]) <= 1e-6 * rel[k]
        xh = x.cpu().numpy()
        Rh = R.cpu().numpy()[:, 0]
        for r0 in (0, mesh.n // 2, mesh.n - 64):
            # the residual is a cancellation: compare at the rounding level of its terms,
            # 1e-12 of sum_l |A_il| |x_l| (FP64 rounding with a wide margin)
            Arows = oasm.matrix(mesh, lam[k], rows=(r0, r0 + 64), near=True)
            ref = Arows @ xh[:, 0]
            mass = np.abs(Arows) @ np.abs(xh[:, 0])
            got = Rh[r0:r0 + 64]
            assert np.all(np.abs(got - ref) <= 1e-12 * mass), np.max(np.abs(got - ref) / mass)
    ctx.close()
