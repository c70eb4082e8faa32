"""GPU parity of the near-field variant of A (8 x 8 conical rule on near panel pairs)
against the oracle's near variant, through the C ABI.

Bars: the pair list bit-exact (index work); FP64 projection and residuals 1e-11 relative;
mixed projection 1e-4 (the mixed path's bar); eigenvalues from bem_solve with the near
field on against the oracle's near-variant eigenvalues (tests/golden/eigs_sphere320_near.txt)
to 1e-10, which exercises the FP64 refinement's near-field derivatives too."""
import os

import numpy as np
import pytest
import torch

import bench
import synth
from oracle import assembly as oasm, rr as orr

pytestmark = pytest.mark.gpu
TOL64 = 1e-11
TOLMIX = 1e-4
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _dev(V):
    import paper_1906_03938_gb300 as b
    return b.fortran(torch.from_numpy(np.asarray(V)).to("cuda:0"))


def _relerr(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("mesh_fn", [lambda: synth.icosphere(2), lambda: synth.cube_grid(4),
                                     lambda: synth.cube_sphere(5, (1.6, 0.9, 0.6)),
                                     lambda: synth.tetrakis_sphere(2, (1.0, 0.7, 0.5))])
def test_near_pairs_bit_exact(bem, mesh_fn):
    m = mesh_fn()
    ctx = bem.Context(0)
    ctx.set_mesh(m.xyz, m.tri)
    ctx.set_near_field(1)
    row_ptr, cols = ctx.near_pairs()
    ref_ptr, ref_cols = oasm.near_pairs(m)
    assert np.array_equal(row_ptr.astype(np.int64), ref_ptr)
    assert np.array_equal(cols.astype(np.int64), ref_cols)
    ctx.close()


@pytest.mark.parametrize("case", ["sphere320", "ragged108"])
def test_near_projection_fp64_and_mixed(bem, case):
    if case == "sphere320":
        prob = synth.workload("sphere320").problems[0]
        mesh, spec, N, nu, seed = prob.mesh(), prob.contour, prob.N, prob.nu, prob.seed
    else:
        mesh = synth.cube_grid(3)
        spec, N, nu, seed = synth.ContourSpec("ellipse", 6.5 + 0.1j, 1.5, 0.4), 7, 5, 3
    V = synth.complex_gaussian(mesh.n, nu, seed)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    ctx.set_near_field(1)
    B64, Y64 = ctx.project(_dev(V), bem.PREC_FP64, AV=True)
    Bm, Ym = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
    ctx.check()
    P, Yo = orr.project(mesh, z, V, near=True)
    P7, _ = orr.project(mesh, z, V)
    for j in range(N):
        ref = w[j] * P[j]
        assert _relerr(Y64[j].cpu().numpy(), Yo[j]) < TOL64, j
        assert _relerr(B64[j].cpu().numpy(), ref) < TOL64, j
        assert _relerr(Ym[j].cpu().numpy(), Yo[j]) < TOLMIX, j
        assert _relerr(Bm[j].cpu().numpy(), ref) < TOLMIX, j
        # the near field changes the operator well above the FP64 bar
        assert _relerr(w[j] * P7[j], ref) > 1e3 * TOL64
    # switching it off restores the 7-point operator
    ctx.set_near_field(0)
    B0 = ctx.project(_dev(V), bem.PREC_FP64).cpu().numpy()
    for j in range(N):
        assert _relerr(B0[j], w[j] * P7[j]) < TOL64
    ctx.close()


def test_near_residual_fp64(bem):
    mesh = synth.icosphere(2)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_near_field(1)
    X = synth.complex_gaussian(mesh.n, 3, 9)
    lam = np.array([3.18, 4.2 + 0.3j, 5.0 - 0.5j])
    rel, R = ctx.residual(lam, _dev(X), want_R=True)
    for c in range(3):
        A = oasm.matrix(mesh, lam[c], near=True)
        r = A @ X[:, c]
        assert _relerr(R[:, c].cpu().numpy(), r) < TOL64
        assert abs(rel[c] - np.linalg.norm(r) / np.linalg.norm(X[:, c])) < 1e-12 * rel[c]
    ctx.close()


def _golden(name):
    rows = np.loadtxt(os.path.join(HERE, "golden", f"eigs_{name}.txt"), ndmin=2)
    return [(complex(r[0], r[1]), int(r[2])) for r in rows if int(r[3]) == 1]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_near_solve_sphere320_against_golden(bem, precision):
    prob = synth.workload("sphere320").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, prob.N)
    ctx.set_near_field(1)
    V0 = _dev(synth.complex_gaussian(mesh.n, prob.nu, prob.seed))
    prec = bem.PREC_FP64 if precision == "fp64" else bem.PREC_MIXED
    lam, X, rel = ctx.solve(V0, q=10, precision=prec, tol=1e-14)
    res = bench.eig_compare(lam, X.cpu().numpy(), rel, _golden("sphere320_near"), spec, 1e-10)
    assert not res["missing"] and not res["extras"], res
    ctx.close()
