"""GPU parity of the mixed-precision path (FP32 evaluation, BF16x3 tcgen05 contraction)
against the CPU oracle, through the C ABI.

Tolerance, from the arithmetic: FP32 coordinates relative to the tile and MUFU
exponentials carry ~1e-6 relative error per entry; the BF16x3 split keeps ~2^-17 of each
operand, so each product term is good to ~1e-5; sums of n terms of both signs stay in that
range. The bar is 1e-4 relative (max-norm per node) on the projected matrices and on
A(z_j)V; the FP64 refinement of the eigenpairs recovers full accuracy afterwards."""
import numpy as np
import pytest
import torch

import synth
from oracle import contour as ocon, rr as orr

pytestmark = pytest.mark.gpu
TOL = 1e-4


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


def _run(bem, mesh, spec, N, nu, seed, AV=True):
    V = synth.complex_gaussian(mesh.n, nu, seed)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    out = ctx.project(_dev(V), bem.PREC_MIXED, AV=AV)
    ctx.check()
    return ctx, V, z, w, out


@pytest.mark.parametrize("case", ["sphere320", "ragged108", "nu1", "nu130", "g3_twins",
                                  "odd_n_twins"])
def test_mixed_matches_oracle(bem, case):
    if case == "g3_twins":
        # nu = 72 leaves room for 3 nodes per work unit: twin pairs (32 ellipse nodes, all
        # conjugate) straddle the unit boundaries and fall back to single evaluation there
        mesh, spec, N, nu = synth.icosphere(1), synth.ContourSpec("ellipse", 6.0 + 0j, 1.5, 0.4), 32, 72
    elif case == "odd_n_twins":
        # 7 circle nodes: three twin pairs and the real node theta = pi on its own
        mesh, spec, N, nu = synth.icosphere(1), synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0), 7, 40
    elif case == "sphere320":
        mesh, spec, N, nu = synth.icosphere(2), synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0), 16, 16
    elif case == "ragged108":
        mesh, spec, N, nu = synth.cube_grid(3), synth.ContourSpec("ellipse", 6.5 + 0.1j, 1.5, 0.4), 7, 5
    elif case == "nu1":
        mesh, spec, N, nu = synth.icosphere(1), synth.ContourSpec("circle", 3.0 + 0j, 0.5, 0.5), 3, 1
    else:
        mesh, spec, N, nu = synth.icosphere(2), synth.ContourSpec("circle", 5.0 + 0j, 1.0, 1.0), 5, 130
    ctx, V, z, w, (B, Y) = _run(bem, mesh, spec, N, nu, 21)
    P, Yo = orr.project(mesh, z, V)
    Bh, Yh = B.cpu().numpy(), Y.cpu().numpy()
    errs = []
    for j in range(N):
        errs.append((_relerr(Yh[j], Yo[j]), _relerr(Bh[j], w[j] * P[j])))
    worst = np.max(errs, axis=0)
    print(f"{case}: worst rel err Y {worst[0]:.2e}, Bhat {worst[1]:.2e}")
    assert worst[0] < TOL and worst[1] < TOL
    ctx.close()


def test_mixed_deterministic(bem):
    mesh, spec = synth.icosphere(2), synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    ctx, V, z, w, (B1, _) = _run(bem, mesh, spec, 8, 24, 3)
    B2 = ctx.project(_dev(V), bem.PREC_MIXED)
    ctx.check()
    assert torch.equal(B1, B2)
    ctx.close()


def test_mixed_full_size_cube3072(bem):
    """The bench workload: sampled rows of A(z_j)V against the oracle, and all projected
    matrices against the plain FP64 GPU path."""
    prob = synth.workload("cube3072").problems[0]
    mesh = prob.mesh()
    ctx, V, z, w, (B, Y) = _run(bem, mesh, prob.contour, prob.N, prob.nu, prob.seed)
    Bf = ctx.project(_dev(V), bem.PREC_FP64)
    ctx.check()
    Bh, Bfh, Yh = B.cpu().numpy(), Bf.cpu().numpy(), Y.cpu().numpy()
    worst_b = max(_relerr(Bh[j], Bfh[j]) for j in range(prob.N))
    worst_y = 0.0
    for r0 in (0, 1531, 3040):
        rows = (r0, r0 + 32)
        _, Yo = orr.project(mesh, z[::8], V, rows=rows)
        for jj, j in enumerate(range(0, prob.N, 8)):
            worst_y = max(worst_y, _relerr(Yh[j, rows[0]:rows[1]], Yo[jj]))
    print(f"cube3072: worst rel err Bhat vs FP64 GPU {worst_b:.2e}, sampled Y vs oracle {worst_y:.2e}")
    assert worst_b < TOL and worst_y < TOL
    ctx.close()


@pytest.mark.parametrize("scale,centre", [(1.0, 4.0), (2.0, 3.5)])
def test_mixed_self_terms_both_routes(bem, scale, centre):
    """Diagonal entries of the mixed path (unit columns) against the oracle's self integral:
    small panels against the wavelength take the moment series (|k| rho ~ 1), panels of a
    doubled icosahedron at k ~ 3.5 + i the direct angular quadrature (|k| rho > 3.5)."""
    from oracle import assembly as oasm
    mesh = synth.icosphere(1 if scale == 1.0 else 0)
    mesh = synth.Mesh(mesh.name, mesh.xyz * scale, mesh.tri)
    spec = synth.ContourSpec("circle", centre + 0j, 1.0, 1.0)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, _ = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, 4)
    E = np.eye(mesh.n, dtype=complex)
    _, Y = ctx.project(_dev(E), bem.PREC_MIXED, AV=True)
    ctx.check()
    for j in range(4):
        A = oasm.matrix(mesh, z[j])
        d = np.diag(Y[j].cpu().numpy())
        assert np.max(np.abs(d - np.diag(A)) / np.abs(np.diag(A))) < 2e-5, j
        assert _relerr(Y[j].cpu().numpy(), A) < TOL
    ctx.close()


@pytest.mark.parametrize("kind,N,twins", [("ellipse", 32, 16), ("circle", 7, 3),
                                          ("circle", 1, 0), ("chebyshev", 12, 0)])
def test_node_order(bem, kind, N, twins):
    """The schedule is a permutation of the nodes; its twin pairs (at the front) have
    bit-equal real parts, so the shared sine and cosine are exactly each node's own, and
    for a contour symmetric about the real axis they are conjugates."""
    mesh = synth.icosphere(0)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, _ = ctx.set_contour(kind, 5.0 + 0j, 1.25, 0.5, N)
    order, tw = ctx.node_order()
    assert sorted(order.tolist()) == list(range(N))
    assert tw == twins
    for P in range(tw):
        a, b = z[order[2 * P]], z[order[2 * P + 1]]
        assert np.float32(a.real) == np.float32(b.real)
        assert a.real == b.real and a.imag == -b.imag
    ctx.close()


@pytest.mark.parametrize("np_poly", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("case", ["twins_g4", "single_g1"])
def test_mixed_eval_split_matches_oracle(bem, case, np_poly):
    """Every split of the sines and cosines between the MUFU unit and the FMA-pipe
    polynomials (bem_set_eval_split) meets the mixed path's bar against the oracle, for
    units of four nodes with twin pairs (ellipse) and units of one node (nu = 130)."""
    if case == "twins_g4":
        mesh, spec, N, nu = synth.cube_grid(4), synth.ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4), 8, 24
    else:
        mesh, spec, N, nu = synth.icosphere(2), synth.ContourSpec("circle", 9.0 + 0j, 1.5, 1.5), 4, 130
    V = synth.complex_gaussian(mesh.n, nu, 31)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    ctx.set_eval_split(np_poly)
    B, Y = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
    ctx.check()
    P, Yo = orr.project(mesh, z, V)
    Bh, Yh = B.cpu().numpy(), Y.cpu().numpy()
    worst = max(max(_relerr(Yh[j], Yo[j]), _relerr(Bh[j], w[j] * P[j])) for j in range(N))
    print(f"{case} poly points {np_poly}: worst rel err {worst:.2e}")
    assert worst < TOL
    ctx.close()


@pytest.mark.parametrize("case", ["ellipse_nu136", "odd_circle_nu130", "robin_ellipse_nu200"])
def test_twin_clusters_match_single_node_units(bem, case):
    """Units of one node (nu > 128) run each twin pair on a two-CTA cluster, every entry of
    a pair evaluated once for both nodes and half of each block sent to the partner through
    distributed shared memory. The same FP32 operations act on the same values as with one
    node per CTA, so the projected matrices and A(z_j)V agree bit for bit; both meet the
    mixed path's bar against the oracle. A circle with an odd node count leaves its real
    node unpaired (its cluster partner idles); the Robin operator covers the general kernel."""
    op = None
    if case == "ellipse_nu136":
        mesh, spec, N, nu = synth.cube_grid(4), synth.ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4), 8, 136
    elif case == "odd_circle_nu130":
        mesh, spec, N, nu = synth.icosphere(2), synth.ContourSpec("circle", 5.0 + 0j, 1.0, 1.0), 5, 130
    else:
        mesh, spec, N, nu = synth.cube_grid(3), synth.ContourSpec("ellipse", 6.0 + 0j, 1.5, 0.4), 6, 200
        op = (0.5 + 0.0j, 1.0 + 0.0j)
    V = synth.complex_gaussian(mesh.n, nu, 41)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    if op is not None:
        ctx.set_operator(*op)
    twins = ctx.node_order()[1]
    assert twins == N // 2
    out = {}
    for on in (True, False):
        ctx.set_twin_clusters(on)
        B, Y = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
        ctx.check()
        shape = ctx.mixed_shape()
        assert shape["nodes_per_unit"] == 1 and shape["paired"] == on
        out[on] = (B.cpu().numpy(), Y.cpu().numpy())
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    P, Yo = orr.project(mesh, z, V, op=op)
    Bh, Yh = out[True]
    worst = max(max(_relerr(Yh[j], Yo[j]), _relerr(Bh[j], w[j] * P[j])) for j in range(N))
    print(f"{case}: twin clusters bit-identical to single-node units; worst rel err {worst:.2e}")
    assert worst < TOL
    ctx.close()
