"""GPU parity of the reduced linearised eigensolve (Section 3.1) against the oracle.

The GPU solves the shifted-and-inverted linearisation by subspace iteration + Rayleigh-Ritz;
the oracle solves the full (N+1) nu pencil with LAPACK. Both start from the same weighted
projected matrices, so their eigenvalues inside the contour must agree to rounding of the
converged iteration (bar: 1e-9 relative)."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import bench
import synth
from oracle import contour as ocon, rr as orr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _ctx_with_contour(bem, spec, N):
    mesh = synth.icosphere(0)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return ctx, z, w


def _to_dev(Bhat):
    return torch.from_numpy(np.ascontiguousarray(Bhat)).to("cuda:0")


def test_reduced_solve_reproduces_matrix_polynomial(bem):
    """B^_j = w_j T(z_j) for a quadratic T: the eigenvalues inside the circle are those of
    the textbook companion form (exact reproduction by the Cauchy formula)."""
    rng = np.random.default_rng(5)
    nu = 6
    A0, A1, A2 = (rng.normal(size=(nu, nu)) + 1j * rng.normal(size=(nu, nu)) for _ in range(3))
    A2 *= 0.05
    I, Z = np.eye(nu), np.zeros((nu, nu))
    ref = sla.eigvals(np.block([[Z, I], [-A0, -A1]]), np.block([[I, Z], [Z, A2]]))
    ref = ref[np.isfinite(ref)]
    c = ref[np.argsort(np.abs(ref))[2]]
    rho = 0.6 * np.sort(np.abs(ref - c))[4]
    spec = synth.ContourSpec("circle", complex(c), float(rho), float(rho))
    ctx, z, w = _ctx_with_contour(bem, spec, 16)
    Bhat = np.stack([w[j] * (A0 + z[j] * A1 + z[j] ** 2 * A2) for j in range(16)])
    # shift off the eigenvalue the circle is centred on (S must be regular)
    lam, Y, res, it = ctx.solve_reduced(_to_dev(Bhat), c + 0.1 * rho * np.exp(0.3j), p=32,
                                        tol=1e-13)
    want = ref[np.abs(ref - c) < 0.999 * rho]
    got = lam[(np.abs(lam - c) < 0.999 * rho) & (res < 1e-10)]
    assert len(want) >= 2 and len(got) == len(want), (want, lam, res)
    for l in want:
        assert np.min(np.abs(got - l)) <= 1e-10 * abs(l)
    Yh = Y.cpu().numpy()
    for k in np.where((np.abs(lam - c) < 0.999 * rho) & (res < 1e-10))[0]:
        T = A0 + lam[k] * A1 + lam[k] ** 2 * A2
        assert np.linalg.norm(T @ Yh[:, k]) < 1e-9 * np.linalg.norm(T) * np.linalg.norm(Yh[:, k])
    ctx.close()


def test_reduced_solve_sphere320_matches_oracle_pencil(bem):
    prob = synth.workload("sphere320").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    Q, _ = orr.orthonormalize(V)
    z, w = ocon.from_spec(spec, prob.N)
    P, _ = orr.project(mesh, z, Q)
    Bhat = w[:, None, None] * P
    lam_o, Y_o = orr.reduced_eigs(Bhat, z)
    inside_o = lam_o[np.abs(lam_o - spec.centre) < 0.98 * spec.a]
    ctx, zg, wg = _ctx_with_contour(bem, spec, prob.N)
    lam, Y, res, it = ctx.solve_reduced(_to_dev(Bhat), spec.centre, p=64, tol=1e-12)
    print("iterations", it, "inside (oracle)", len(inside_o))
    conv = lam[res < 1e-9]
    for l in inside_o:
        assert np.min(np.abs(conv - l)) <= 1e-9 * abs(l), (l, np.min(np.abs(lam - l)))
    ctx.close()


def _check_against_golden(name, lam, X, rel, tol, spec):
    """Every golden eigenvalue found (with its multiplicity of independent vectors and a
    converged residual) and no converged extra strictly inside the contour."""
    res = bench.eig_compare(lam, X.cpu().numpy(), rel, bench.read_golden(name), spec, tol)
    print(name, "found", lam, "relres", rel)
    assert not res["missing"], res
    assert not res["extras"], res
    assert res["ok"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_sphere320_against_golden(bem, precision):
    prob = synth.workload("sphere320").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, prob.N)
    V0 = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, prob.seed)).to("cuda:0"))
    prec = bem.PREC_FP64 if precision == "fp64" else bem.PREC_MIXED
    lam, X, rel = ctx.solve(V0, q=10, precision=prec, tol=1e-14)
    _check_against_golden("sphere320", lam, X, rel, 1e-10, spec)
    ctx.close()


def test_solve_cube3072_mixed_against_golden(bem):
    """Full bench workload, mixed projection + FP64 refinement: the three discrete
    eigenvalues inside the ellipse (5.44004, and the split pair 7.69320 / 7.69325 x2)."""
    import time
    prob = synth.workload("cube3072").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, prob.N)
    V0 = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, prob.seed)).to("cuda:0"))
    t0 = time.perf_counter()
    lam, X, rel = ctx.solve(V0, q=10, precision=bem.PREC_MIXED, tol=1e-14)
    print("cube3072 solve seconds", time.perf_counter() - t0)
    _check_against_golden("cube3072", lam, X, rel, 1e-10, spec)
    ctx.close()
