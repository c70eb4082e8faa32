"""GPU parity of the Chebyshev variant (Eq. Chebyshev, Eq. sc1_chebyshev_red, Algorithm 2's
setting) against oracle/chebyshev.py, and the variant end to end on the unit sphere.

Bars: nodes to rounding; coefficients to 1e-13 relative; eigenvalues of an interpolated
matrix polynomial near the interval to 1e-10; sphere320's eigenvalues inside the interval,
found through the Chebyshev interpolant and refined in FP64, against the oracle's discrete
eigenvalues (tests/golden/eigs_sphere320.txt) to 1e-10."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import synth
from oracle import assembly as oasm, chebyshev as och

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _ctx(bem, c, a, N, mesh=None):
    mesh = mesh or synth.icosphere(0)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour("chebyshev", c, a, a, N)
    return ctx, z, w


def test_nodes_and_coefficients(bem):
    ctx, z, w = _ctx(bem, 3.8, 1.2, 11)
    assert np.max(np.abs(z - och.nodes(3.8, 1.2, 11))) < 1e-15 * 8 and np.all(w == 1.0)
    rng = np.random.default_rng(1)
    P = rng.normal(size=(11, 5, 5)) + 1j * rng.normal(size=(11, 5, 5))
    B = ctx.chebyshev_coeffs(torch.from_numpy(P).to("cuda:0")).cpu().numpy()
    ref = och.coefficients(P)
    assert np.max(np.abs(B - ref)) < 1e-13 * np.max(np.abs(ref))
    ctx.close()


@pytest.mark.parametrize("N", [4, 5, 8, 14])
def test_shift_invert_operator_matches_dense_solve(bem, N):
    """The GPU's recurrence solve of (A - sigma M) w' = M w against the oracle's dense
    solve of the colleague pencil, for coefficients that are all significant."""
    rng = np.random.default_rng(N)
    nu, p = 5, 7
    c, a = 0.0, 1.0
    ctx, _, _ = _ctx(bem, c, a, N)
    B = np.stack([(rng.normal(size=(nu, nu)) + 1j * rng.normal(size=(nu, nu))) * 0.5 ** i
                  for i in range(N)])
    W = rng.normal(size=((N - 1) * nu, p)) + 1j * rng.normal(size=((N - 1) * nu, p))
    for sigma in (0.0, 0.05, 0.3 - 0.2j):
        HW = ctx.chebyshev_apply(torch.from_numpy(B).to("cuda:0"), c + a * sigma,
                                 torch.from_numpy(W).to("cuda:0")).cpu().numpy()
        ref = och.shift_invert_apply(B, sigma, W)
        assert np.max(np.abs(HW - ref)) < 1e-12 * np.max(np.abs(ref)), (N, sigma)
    ctx.close()


def test_solve_matrix_polynomial(bem):
    rng = np.random.default_rng(5)
    nu = 6
    A0, A1, A2 = (rng.normal(size=(nu, nu)) + 1j * rng.normal(size=(nu, nu)) for _ in range(3))
    A2 *= 0.05
    I, Z = np.eye(nu), np.zeros((nu, nu))
    ref = sla.eigvals(np.block([[Z, I], [-A0, -A1]]), np.block([[I, Z], [Z, A2]]))
    ref = ref[np.isfinite(ref)]
    # an interval around the real parts of three eigenvalues
    order = np.argsort(np.abs(ref))
    pick = ref[order[:3]]
    c = float(np.mean(pick.real))
    a = float(np.max(np.abs(pick.real - c))) + 0.5
    ctx, z, _ = _ctx(bem, c, a, 10)
    P = np.stack([A0 + zk * A1 + zk ** 2 * A2 for zk in z])
    B = ctx.chebyshev_coeffs(torch.from_numpy(P).to("cuda:0"))
    lam, Y, res, it = ctx.solve_chebyshev(B, c + 0.05 * a, p=24, tol=1e-13)
    zeta = (lam - c) / a
    got = lam[(np.abs(zeta.real) < 1) & (np.abs(zeta.imag) < 0.25) & (res < 1e-10)]
    want = ref[(np.abs((ref.real - c) / a) < 1) & (np.abs(ref.imag / a) < 0.25)]
    assert len(want) >= 1 and len(got) >= len(want), (want, lam, res)
    for l in want:
        assert np.min(np.abs(got - l)) <= 1e-10 * max(1.0, abs(l))
    # the oracle's linearisation gives the same eigenvalues from the GPU's coefficients
    lo, _ = och.eigs(B.cpu().numpy(), c, a)
    for l in got:
        assert np.min(np.abs(lo - l)) <= 1e-10 * max(1.0, abs(l))
    ctx.close()


def _golden(name):
    rows = np.loadtxt(os.path.join(HERE, "golden", f"eigs_{name}.txt"), ndmin=2)
    return [(complex(r[0], r[1]), int(r[2])) for r in rows if int(r[3]) == 1]


def test_sphere320_through_chebyshev_interpolant(bem):
    prob = synth.workload("sphere320").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    # basis: Algorithm 1 on the closed contour, orthonormalised
    ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, prob.N)
    V = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, prob.seed)).to("cuda:0"))
    ctx.inverse_power(V, 10, spec.centre)
    ctx.cholqr2(V, want_R=False)
    # Chebyshev interpolant on [2.8, 4.8]
    c, a = 3.8, 1.0
    ctx.set_contour("chebyshev", c, a, a, 14)
    P = ctx.project(V, bem.PREC_FP64)
    B = ctx.chebyshev_coeffs(P)
    lam, Y, res, _ = ctx.solve_chebyshev(B, c, p=32, tol=1e-10)
    keep = np.where((np.abs(lam.real - c) < a) & (np.abs(lam.imag) < 0.1) & (res < 1e-6))[0]
    X = ctx.ritz_vectors(V, Y[:, keep].contiguous())
    lam_r, rel, _ = ctx.refine(lam[keep], X, tol=1e-14)
    Xh = X.cpu().numpy()
    for lg, mult in _golden("sphere320"):
        near = np.where(np.abs(lam_r - lg) <= 1e-10 * abs(lg))[0]
        assert len(near) >= 1, (lg, lam_r)
        sv = np.linalg.svd(Xh[:, near] / np.linalg.norm(Xh[:, near], axis=0), compute_uv=False)
        assert np.sum(sv > 1e-6) >= mult, (lg, sv)
        assert np.all(rel[near] < 1e-10)
    ctx.close()


def test_algorithm2_matches_oracle(bem):
    """Algorithm 2 (bem_inverse_power_chebyshev: FP32 iterate, G factorised in FP32, the
    right-hand side by the node-summed BF16x3 kernel) against the oracle's FP64 Algorithm 2
    on the dense Chebyshev coefficients of A, q = 3 steps from the same basis: the same
    directions to 1e-3 (column by column, up to a scalar), as Algorithm 1's test."""
    mesh = synth.icosphere(1)
    c, a, N, nu, q = 3.6, 1.0, 8, 6, 3
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, _ = ctx.set_contour("chebyshev", c, a, a, N)
    V0 = synth.complex_gaussian(mesh.n, nu, 9)
    Vd = bem.fortran(torch.from_numpy(V0).to("cuda:0"))
    ctx.inverse_power_chebyshev(Vd, q)
    ctx.check()
    got = Vd.cpu().numpy()
    B = och.coefficients([oasm.matrix(mesh, zk) for zk in och.nodes(c, a, N)])
    ref = och.inverse_power(B, V0, q)
    for col in range(nu):
        g, r = got[:, col], ref[:, col]
        al = np.vdot(r, g) / np.vdot(r, r)
        assert np.linalg.norm(g - al * r) <= 1e-3 * np.linalg.norm(g), col
    ctx.close()


def test_sphere320_through_algorithm2_basis(bem):
    """The whole Chebyshev route with Algorithm 2's basis: q = 10 steps on the interval
    [2.8, 4.8], CholeskyQR2, FP64 projection at the Chebyshev points, colleague solve,
    refinement; the golden eigenvalues of the unit sphere inside the interval (pi and
    4.4934 x 3 on the level-2 mesh) with their multiplicities to 1e-10."""
    prob = synth.workload("sphere320").problems[0]
    mesh = prob.mesh()
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    c, a = 3.8, 1.0
    ctx.set_contour("chebyshev", c, a, a, 14)
    V = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, prob.seed)).to("cuda:0"))
    ctx.inverse_power_chebyshev(V, 10)
    ctx.cholqr2(V, want_R=False)
    P = ctx.project(V, bem.PREC_FP64)
    B = ctx.chebyshev_coeffs(P)
    lam, Y, res, _ = ctx.solve_chebyshev(B, c, p=32, tol=1e-10)
    keep = np.where((np.abs(lam.real - c) < a) & (np.abs(lam.imag) < 0.1) & (res < 1e-6))[0]
    X = ctx.ritz_vectors(V, Y[:, keep].contiguous())
    lam_r, rel, _ = ctx.refine(lam[keep], X, tol=1e-14)
    Xh = X.cpu().numpy()
    for lg, mult in _golden("sphere320"):
        near = np.where(np.abs(lam_r - lg) <= 1e-10 * abs(lg))[0]
        assert len(near) >= 1, (lg, lam_r)
        sv = np.linalg.svd(Xh[:, near] / np.linalg.norm(Xh[:, near], axis=0), compute_uv=False)
        assert np.sum(sv > 1e-6) >= mult, (lg, sv)
        assert np.all(rel[near] < 1e-10)
    ctx.close()
