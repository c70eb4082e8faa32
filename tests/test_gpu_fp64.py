"""GPU parity of the plain FP64 path against the CPU oracle, through the C ABI.

Bar: the projected matrices and A(z_j) V agree with the oracle to 1e-11 relative (per
node, max-norm of the difference over max-norm of the oracle's matrix); entries, self
terms, CholeskyQR2 and residuals likewise."""
import numpy as np
import pytest
import torch

import synth
from oracle import assembly as oasm, contour as ocon, rr as orr, refine as oref

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _ctx(bem, mesh, spec, N):
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return ctx, z, w


def _dev(V):
    import paper_1906_03938_gb300 as b
    return b.fortran(torch.from_numpy(np.asarray(V)).to("cuda:0"))


def _relerr(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def test_contour_matches_oracle(bem):
    mesh = synth.icosphere(1)
    for spec, N in ((synth.ContourSpec("circle", 4.0 + 0.5j, 1.2, 1.2), 16),
                    (synth.ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4), 7)):
        ctx, z, w = _ctx(bem, mesh, spec, N)
        zo, wo = ocon.from_spec(spec, N)
        assert np.max(np.abs(z - zo)) < 1e-15 * 8 and np.max(np.abs(w - wo)) < 1e-16 * 8
        ctx.close()


@pytest.mark.parametrize("case", ["sphere320", "ragged108"])
def test_project_fp64_matches_oracle(bem, case):
    if case == "sphere320":
        prob = synth.workload("sphere320").problems[0]
        mesh, spec, N, nu, seed = prob.mesh(), prob.contour, prob.N, prob.nu, prob.seed
    else:   # 108 rows (not a multiple of the 32-row tile), nu = 5, odd N, ellipse
        mesh = synth.cube_grid(3)
        spec, N, nu, seed = synth.ContourSpec("ellipse", 6.5 + 0.1j, 1.5, 0.4), 7, 5, 3
    V = synth.complex_gaussian(mesh.n, nu, seed)
    ctx, z, w = _ctx(bem, mesh, spec, N)
    B, Y = ctx.project(_dev(V), bem.PREC_FP64, AV=True)
    torch.cuda.synchronize()
    P, Yo = orr.project(mesh, z, V)
    for j in range(N):
        assert _relerr(Y[j].cpu().numpy(), Yo[j]) < TOL, j
        assert _relerr(B[j].cpu().numpy(), w[j] * P[j]) < TOL, j
    ctx.close()


def test_entries_and_self_terms_via_unit_columns(bem):
    """V = columns of the identity returns columns of A(z_j), diagonal (self term) included."""
    mesh = synth.icosphere(1)
    spec = synth.ContourSpec("circle", 3.5 - 0.2j, 1.0, 1.0)
    ctx, z, w = _ctx(bem, mesh, spec, 3)
    cols = [0, 1, 17, 63, 79]
    E = np.zeros((mesh.n, len(cols)), dtype=complex)
    E[cols, range(len(cols))] = 1.0
    _, Y = ctx.project(_dev(E), bem.PREC_FP64, AV=True)
    torch.cuda.synchronize()
    for j in range(3):
        A = oasm.matrix(mesh, z[j])
        assert _relerr(Y[j].cpu().numpy(), A[:, cols]) < TOL
        d = Y[j].cpu().numpy()[cols, range(len(cols))]
        assert np.max(np.abs(d - np.diag(A)[cols]) / np.abs(np.diag(A)[cols])) < TOL
    ctx.close()


def test_project_edge_cases(bem):
    mesh = synth.icosphere(0)             # 20 triangles: smaller than one tile
    spec = synth.ContourSpec("circle", 4.0, 1.0, 1.0)
    for N, nu in ((1, 1), (2, 20), (5, 3)):
        V = synth.complex_gaussian(mesh.n, nu, 7)
        ctx, z, w = _ctx(bem, mesh, spec, N)
        B = ctx.project(_dev(V), bem.PREC_FP64)
        torch.cuda.synchronize()
        P, _ = orr.project(mesh, z, V)
        for j in range(N):
            assert _relerr(B[j].cpu().numpy(), w[j] * P[j]) < TOL
        ctx.close()


def test_project_full_size_cube3072_sampled(bem):
    """Full bench workload: sampled rows of A(z_j) V against the oracle, and the projection
    against V^H Y_j formed from the returned Y (consistency of the contraction)."""
    prob = synth.workload("cube3072").problems[0]
    mesh = prob.mesh()
    V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    ctx, z, w = _ctx(bem, mesh, prob.contour, prob.N)
    B, Y = ctx.project(_dev(V), bem.PREC_FP64, AV=True)
    torch.cuda.synchronize()
    Yh = Y.cpu().numpy()
    Bh = B.cpu().numpy()
    for r0 in (0, 1531, 3040):
        rows = (r0, r0 + 32)
        _, Yo = orr.project(mesh, z[::8], V, rows=rows)
        for jj, j in enumerate(range(0, prob.N, 8)):
            assert _relerr(Yh[j, rows[0]:rows[1]], Yo[jj]) < TOL
    for j in (0, 13, 31):
        ref = w[j] * (V.conj().T @ Yh[j])
        assert _relerr(Bh[j], ref) < 1e-12
    ctx.close()


def test_cholqr2_matches_definition(bem):
    V = synth.complex_gaussian(1000, 24, 5)
    V[:, 3] = V[:, 3] + 100.0 * V[:, 2]                 # ill-conditioned but full rank
    ctx = bem.Context(0)
    Vd = _dev(V)
    R = ctx.cholqr2(Vd).cpu().numpy()
    Q = Vd.cpu().numpy()
    Qo, Ro = orr.orthonormalize(V)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(24))) < 1e-13
    assert _relerr(Q, Qo) < 1e-10 and _relerr(R, Ro) < 1e-11
    assert np.max(np.abs(Q @ R - V)) < 1e-12 * np.max(np.abs(V))
    ctx.close()


def test_cholqr2_rejects_rank_deficient(bem):
    V = synth.complex_gaussian(100, 4, 5)
    V[:, 3] = V[:, 1]
    ctx = bem.Context(0)
    with pytest.raises(bem.BemError) as e:
        ctx.cholqr2(_dev(V))
    assert e.value.status in (-4,)
    ctx.close()


def test_residual_matches_oracle(bem):
    mesh = synth.icosphere(2)
    spec = synth.workload("sphere320").problems[0].contour
    ctx, z, w = _ctx(bem, mesh, spec, 4)
    X = synth.complex_gaussian(mesh.n, 3, 9)
    lam = np.array([3.18, 4.2 + 0.3j, 5.0 - 0.5j])
    rel, R = ctx.residual(lam, _dev(X), want_R=True)
    for c in range(3):
        A = oasm.matrix(mesh, lam[c])
        r = A @ X[:, c]
        assert _relerr(R[:, c].cpu().numpy(), r) < TOL
        assert abs(rel[c] - np.linalg.norm(r) / np.linalg.norm(X[:, c])) < 1e-12 * rel[c]
    ctx.close()


def test_invalid_arguments_are_rejected(bem):
    mesh = synth.icosphere(0)
    ctx = bem.Context(0)
    with pytest.raises(bem.BemError):           # project before a mesh is set
        ctx.project(_dev(np.ones((20, 2), complex)))
    bad = mesh.tri.copy()
    bad[3, 1] = 10_000                          # vertex index out of range (device check)
    with pytest.raises(bem.BemError) as e:
        ctx.set_mesh(mesh.xyz, bad)
    assert e.value.status == -1
    flat = mesh.tri.copy()
    flat[0, 2] = flat[0, 1]                     # zero-area triangle
    with pytest.raises(bem.BemError):
        ctx.set_mesh(mesh.xyz, flat)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    with pytest.raises(bem.BemError):
        ctx.set_contour("circle", 4.0, -1.0, 1.0, 8)
    ctx.set_contour("circle", 4.0, 1.0, 1.0, 8)
    with pytest.raises(bem.BemError):
        ctx.project(_dev(np.ones((20, 300), complex)))   # nu > 256
    ctx.close()


def test_cholqr2_fp32_first_pass_orthonormal(bem):
    """Without R the first pass runs in FP32; the FP64 second pass must still give
    orthonormal columns spanning the input."""
    V = synth.complex_gaussian(3072, 64, 8)
    V[:, 5] = V[:, 5] + 30.0 * V[:, 4]
    ctx = bem.Context(0)
    Vd = _dev(V)
    ctx.cholqr2(Vd, want_R=False)
    Q = Vd.cpu().numpy()
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(64))) < 1e-13
    assert np.max(np.abs(Q @ (Q.conj().T @ V) - V)) < 1e-12 * np.max(np.abs(V))
    Qo, _ = orr.orthonormalize(V)
    # same basis up to a unitary diagonal (both are the positive-diagonal QR factor)
    assert _relerr(Q, Qo) < 1e-10
    ctx.close()


@pytest.mark.parametrize("n,nu,boost", [(2000, 24, 1e4), (600, 130, 0.0), (3072, 64, 300.0)])
def test_cholqr2_without_R_routes(bem, n, nu, boost):
    """Without R: an FP32 pass that gives up (boost 1e4: condition ~1e5), the FP64 route for
    nu > 128, and a second pass whose Gram matrix is near the identity must all give the
    positive-diagonal QR factor of the input to FP64 accuracy."""
    V = synth.complex_gaussian(n, nu, 11)
    if boost:
        V[:, 7] = V[:, 7] + boost * V[:, 6]
    ctx = bem.Context(0)
    Vd = _dev(V)
    ctx.cholqr2(Vd, want_R=False)
    Q = Vd.cpu().numpy()
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(nu))) < 1e-13
    assert np.max(np.abs(Q @ (Q.conj().T @ V) - V)) < 1e-12 * np.max(np.abs(V))
    Qo, _ = orr.orthonormalize(V)
    assert _relerr(Q, Qo) < 1e-8 * max(1.0, boost / 100.0)
    ctx.close()


def test_async_mode_same_results_and_deferred_status(bem):
    """bem_set_async: the set-up, orthonormalisation and projection pipeline gives the same
    bits as the synchronous calls, and a rank-deficient basis is reported by bem_check
    instead of by bem_cholqr2."""
    prob = synth.workload("sphere320").problems[0]
    mesh, spec = prob.mesh(), prob.contour
    V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    out = []
    for mode in (False, True):
        ctx = bem.Context(0)
        ctx.set_async(mode)
        ctx.set_mesh(mesh.xyz, mesh.tri)
        ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, prob.N)
        Vd = _dev(V)
        ctx.cholqr2(Vd, want_R=False)
        B = ctx.project(Vd, bem.PREC_MIXED)
        ctx.check()
        out.append((Vd.cpu(), B.cpu()))
        ctx.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    ctx = bem.Context(0)
    ctx.set_async(True)
    Vbad = V.copy()
    Vbad[:, 3] = Vbad[:, 2]
    ctx.cholqr2(_dev(Vbad), want_R=False)          # returns at once
    with pytest.raises(bem.BemError):
        ctx.check()
    ctx.close()
