"""GPU parity of Algorithm 1's node-summed operator and of the inverse power steps built on
it, through the C ABI, against the CPU oracle (oracle/assembly.py, oracle/rr.py).

bem_apply_sum forms Y = sum_j c_j A(z_j) X_j (one block per node: the right-hand side of
Eq. linsyssim) or (sum_j c_j A(z_j)) X (one block: the Schur complement S applied) with the
fused kernel: FP32 entries, scaled by c_j in FP32, split into BF16 hi/lo and contracted on
the tensor core (3 products per K-block and operand half), FP32 accumulation over all nodes
and columns. Each element obeys the split-precision bound of the projection:
|Y_gpu - Y_ref| <= (2^-15 + 4 u32 sqrt(6 N n / 16)) (sum_j |c_j| |A(z_j)| |X_j|).

bem_inverse_power (q steps from v_j = u / (z_j - s); S factorised in FP32) must give the
oracle's dense FP64 iterate to 1e-3 in direction (column by column, up to a scalar)."""
import numpy as np
import pytest
import torch

import synth
from oracle import assembly as oasm, rr as orr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


CASES = {
    # (mesh, contour, N, nu): twins and a G = 4 unit; ragged rows with an odd node count;
    # nu = 72 (two nodes per unit with one basis block per node)
    "sphere320": (lambda: synth.icosphere(2), synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0), 16, 16),
    "ragged108": (lambda: synth.cube_grid(3), synth.ContourSpec("ellipse", 6.5 + 0.1j, 1.5, 0.4), 7, 5),
    "nu72": (lambda: synth.icosphere(1), synth.ContourSpec("ellipse", 5.0 + 0j, 1.2, 0.5), 12, 72),
    # nu = 256: two column chunks of the accumulator (one node per unit)
    "nu256": (lambda: synth.icosphere(2), synth.ContourSpec("circle", 9.0 + 0j, 1.5, 1.5), 4, 256),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("per_node", [True, False])
def test_apply_sum_matches_oracle(bem, case, per_node):
    mk, spec, N, nu = CASES[case]
    mesh = mk()
    n = mesh.n
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    rng = np.random.default_rng(3)
    coef = (rng.normal(size=N) + 1j * rng.normal(size=N)) / N
    if per_node:
        X = np.stack([synth.complex_gaussian(n, nu, 40 + j) for j in range(N)])
        Xd = torch.from_numpy(np.ascontiguousarray(X.transpose(0, 2, 1))).to("cuda:0").transpose(1, 2)
    else:
        X = synth.complex_gaussian(n, nu, 40)
        Xd = bem.fortran(torch.from_numpy(X).to("cuda:0"))
    Y = ctx.apply_sum(coef, Xd, per_node=per_node).cpu().numpy()
    ref = np.zeros((n, nu), complex)
    mass = np.zeros((n, nu))
    for j in range(N):
        A = oasm.matrix(mesh, z[j])
        Xj = X[j] if per_node else X
        ref += coef[j] * (A @ Xj)
        mass += abs(coef[j]) * (np.abs(A) @ np.abs(Xj))
    bound = 2.0 ** -15 + 4 * 2.0 ** -24 * np.sqrt(6 * N * n / 16)
    ratio = np.max(np.abs(Y - ref) / (bound * mass))
    rel = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    print(f"{case} per_node={per_node}: worst error / bound {ratio:.3f}, max rel {rel:.2e}")
    assert ratio <= 1.0
    ctx.close()


@pytest.mark.parametrize("case", ["sphere320", "cube3072"])
def test_inverse_power_matches_oracle(bem, case):
    """sphere320: two LU panels; cube3072 (n = 3072): twelve panels of 256 columns, so every
    level of the blocked factorisation (sub-panel pivoting, in-panel updates, interchanges,
    block rows, tensor-core trailing updates) is exercised."""
    prob = synth.workload(case).problems[0]
    mesh, spec, N = prob.mesh(), prob.contour, prob.N
    nu = prob.nu if case == "sphere320" else 8
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    V0 = synth.complex_gaussian(mesh.n, nu, prob.seed)
    q = 3 if case == "sphere320" else 2
    shift = spec.centre + (0.0 if case == "sphere320" else 0.3j)
    Vd = bem.fortran(torch.from_numpy(V0).to("cuda:0"))
    ctx.inverse_power(Vd, q, shift)
    ug = Vd.cpu().numpy()
    Bfull = np.stack([w[j] * oasm.matrix(mesh, z[j]) for j in range(N)])
    uo = orr.inverse_power(Bfull, z, shift, V0, q)
    worst = 0.0
    for c in range(nu):
        a = np.vdot(uo[:, c], ug[:, c]) / np.vdot(uo[:, c], uo[:, c])
        worst = max(worst, np.linalg.norm(ug[:, c] - a * uo[:, c]) / np.linalg.norm(ug[:, c]))
    print(case, "inverse power: worst column direction error", worst)
    assert worst < 1e-3
    ctx.close()


def _sphere_ctx(bem):
    prob = synth.workload("sphere320").problems[0]
    mesh, spec, N = prob.mesh(), prob.contour, prob.N
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return prob, mesh, spec, ctx, z, w


def test_solve_sum_matches_dense_solve(bem):
    """Matrix-free GMRES on S = sum_j w_j A(z_j) / (z_j - s) against the dense FP64 solve.
    GMRES stops on its own operator's true residual (tol 1e-4: that operator carries the
    split-precision error, ~3e-5 relative, so smaller residuals are not meaningful). Then
    X - X_dense = S^-1 (residual + (S_gpu - S) X), so the bar is cond(S) (tol + 1e-4)."""
    prob, mesh, spec, ctx, z, w = _sphere_ctx(bem)
    c = w / (z - spec.centre)
    S = sum(c[j] * oasm.matrix(mesh, z[j]) for j in range(len(z)))
    B = synth.complex_gaussian(mesh.n, 6, 77)
    tol = 1e-4
    X, iters, rel = ctx.solve_sum(c, bem.fortran(torch.from_numpy(B).to("cuda:0")), tol=tol,
                                  max_iter=600)
    Xo = np.linalg.solve(S, B)
    err = np.linalg.norm(X.cpu().numpy() - Xo) / np.linalg.norm(Xo)
    ores = np.linalg.norm(B - S @ X.cpu().numpy(), axis=0) / np.linalg.norm(B, axis=0)
    cond = np.linalg.cond(S)
    print(f"GMRES: {iters} Arnoldi steps, own residual {rel.max():.1e}, "
          f"oracle residual {ores.max():.1e}, solution error {err:.1e}, cond {cond:.1f}")
    assert np.all(rel <= tol)
    assert err < cond * (tol + 1e-4)
    ctx.close()


def test_inverse_power_matrix_free_matches_oracle(bem):
    """q = 3 steps with GMRES solves to 1e-4: each solve's relative error is at most
    cond(S) (tol + 1e-4), and the direction errors of the steps add up."""
    prob, mesh, spec, ctx, z, w = _sphere_ctx(bem)
    V0 = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    q, tol = 3, 1e-4
    Vd = bem.fortran(torch.from_numpy(V0).to("cuda:0"))
    its = ctx.inverse_power_mf(Vd, q, spec.centre, tol=tol, max_iter=600)
    ug = Vd.cpu().numpy()
    Bfull = np.stack([w[j] * oasm.matrix(mesh, z[j]) for j in range(len(z))])
    uo = orr.inverse_power(Bfull, z, spec.centre, V0, q)
    cond = np.linalg.cond(np.einsum("j,jab->ab", 1.0 / (z - spec.centre), Bfull))
    worst = 0.0
    for col in range(prob.nu):
        a = np.vdot(uo[:, col], ug[:, col]) / np.vdot(uo[:, col], uo[:, col])
        worst = max(worst, np.linalg.norm(ug[:, col] - a * uo[:, col]) / np.linalg.norm(ug[:, col]))
    print(f"matrix-free inverse power: {its} Arnoldi steps, worst column direction error "
          f"{worst:.2e}, cond(S) {cond:.1f}")
    assert worst < q * cond * (tol + 1e-4)
    ctx.close()
