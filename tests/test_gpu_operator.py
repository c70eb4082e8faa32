"""GPU parity of the operator variant T = c_G G + c_H (1/2 I + K) (the general form of
Eq. HelmBIM: Neumann (0, 1) and Robin conditions) against the oracle
(oracle/assembly.py with op=), through the C ABI.

Bars: the FP64 projection to 1e-11 relative (max-norm per node) as for the single layer;
the mixed projection and the node-summed apply to 1e-4 (the BF16x3 split keeps ~2^-17 of
each operand; the operator factor adds a few FP32 operations per point); residuals
||T(lam) x|| to 1e-11 of ||T|| ||x||; the Neumann eigenvalues of the sphere, found by the
whole method (Algorithm 1, CholeskyQR2, projection, reduced solve, FP64 refinement), to
1e-10 of the oracle's (tests/golden/eigs_sphere320_neumann.txt), with their
multiplicities."""
import os

import numpy as np
import pytest
import torch

import bench
import synth
from oracle import assembly as oasm, rr as orr

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
NEUMANN = (0.0, 1.0)
ROBIN = (0.5 + 0.2j, 1.0 - 0.3j)
SPEC = synth.ContourSpec("circle", 2.75 + 0j, 0.9, 0.9)


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


def _ctx(bem, mesh, op, spec=SPEC, N=8, near=0):
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_operator(*op)
    if near:
        ctx.set_near_field(near)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return ctx, z, w


@pytest.mark.parametrize("op", [NEUMANN, ROBIN], ids=["neumann", "robin"])
@pytest.mark.parametrize("case", ["sphere320", "ragged108"])
def test_projection_matches_oracle(bem, op, case):
    if case == "sphere320":
        mesh, spec, N, nu = synth.icosphere(2), SPEC, 8, 16
    else:
        mesh, spec, N, nu = synth.cube_grid(3), synth.ContourSpec("ellipse", 4.5 + 0.1j, 1.2, 0.4), 7, 5
    ctx, z, w = _ctx(bem, mesh, op, spec, N)
    V = synth.complex_gaussian(mesh.n, nu, 12)
    P, Yo = orr.project(mesh, z, V, op=op)
    B64, Y64 = ctx.project(_dev(V), bem.PREC_FP64, AV=True)
    Bm, Ym = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
    ctx.check()
    e64 = max(_relerr(B64[j].cpu().numpy(), w[j] * P[j]) for j in range(N))
    em = max(max(_relerr(Bm[j].cpu().numpy(), w[j] * P[j]), _relerr(Ym[j].cpu().numpy(), Yo[j]))
             for j in range(N))
    print(f"{case} op={op}: FP64 {e64:.1e}, mixed {em:.1e}")
    assert e64 < 1e-11 and em < 1e-4
    ctx.close()


def test_projection_with_near_field(bem):
    mesh = synth.icosphere(3)
    ctx, z, w = _ctx(bem, mesh, NEUMANN, N=4, near=1)
    V = synth.complex_gaussian(mesh.n, 8, 5)
    rows = (0, 64)
    _, Yo = orr.project(mesh, z, V, rows=rows, near=True, op=NEUMANN)
    _, Y64 = ctx.project(_dev(V), bem.PREC_FP64, AV=True)
    _, Ym = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
    ctx.check()
    e64 = max(_relerr(Y64[j, rows[0]:rows[1]].cpu().numpy(), Yo[j]) for j in range(4))
    em = max(_relerr(Ym[j, rows[0]:rows[1]].cpu().numpy(), Yo[j]) for j in range(4))
    print(f"near field, Neumann: FP64 {e64:.1e}, mixed {em:.1e}")
    assert e64 < 1e-11 and em < 1e-4
    ctx.close()


def test_apply_sum_and_residual(bem):
    mesh = synth.icosphere(2)
    ctx, z, w = _ctx(bem, mesh, ROBIN)
    N = len(z)
    rng = np.random.default_rng(4)
    c = (rng.normal(size=N) + 1j * rng.normal(size=N)) / N
    X = synth.complex_gaussian(mesh.n, 6, 8)
    Y = ctx.apply_sum(c, _dev(X), per_node=False).cpu().numpy()
    ref = sum(c[j] * oasm.matrix(mesh, z[j], op=ROBIN) for j in range(N)) @ X
    assert _relerr(Y, ref) < 1e-4
    lam = np.array([2.3 + 0.05j, 3.1 - 0.02j])
    Xr = synth.complex_gaussian(mesh.n, 2, 9)
    rel = ctx.residual(lam, _dev(Xr))
    for col in range(2):
        A = oasm.matrix(mesh, lam[col], op=ROBIN)
        want = np.linalg.norm(A @ Xr[:, col]) / np.linalg.norm(Xr[:, col])
        assert abs(rel[col] - want) <= 1e-11 * np.linalg.norm(A, 2)
    ctx.close()


def test_operator_restrictions(bem):
    mesh = synth.icosphere(1)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    with pytest.raises(bem.BemError):
        ctx.set_operator(0.0, 0.0)
    ctx.set_operator(*NEUMANN)
    ctx.set_contour("circle", 2.75, 0.9, 0.9, 8)
    with pytest.raises(bem.BemError):
        bem.Batch([ctx], [_dev(synth.complex_gaussian(mesh.n, 4, 1))])
    ctx.close()


def _golden(name):
    rows = np.loadtxt(os.path.join(HERE, "golden", f"eigs_{name}.txt"), ndmin=2)
    return [(complex(r[0], r[1]), int(r[2])) for r in rows if int(r[3]) == 1]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_neumann_sphere320_against_golden(bem, precision):
    mesh = synth.icosphere(2)
    ctx, z, w = _ctx(bem, mesh, NEUMANN, N=16)
    V0 = _dev(synth.complex_gaussian(mesh.n, 16, 20190609))
    prec = bem.PREC_FP64 if precision == "fp64" else bem.PREC_MIXED
    lam, X, rel = ctx.solve(V0, q=10, precision=prec, tol=1e-14)
    res = bench.eig_compare(lam, X.cpu().numpy(), rel, _golden("sphere320_neumann"),
                            SPEC, 1e-10)
    assert not res["missing"] and not res["extras"], res
    ctx.close()
