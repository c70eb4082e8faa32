"""GPU parity of the grouped (batched) mixed projection: one launch of the fused kernel over
the work units of many problems, recorded as a CUDA graph.

Bar: each problem's projected matrices agree with the oracle to the mixed path's 1e-4
(relative, max-norm per node), and with the same context's single-problem mixed projection
to 2e-5 (the two may split the columns differently, which changes only FP32 rounding)."""
import numpy as np
import pytest
import torch

import synth
from oracle import rr as orr

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _relerr(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def _setup(bem, problems):
    ctxs, Vs, Vh, zs, ws, meshes = [], [], [], [], [], []
    for prob in problems:
        mesh = prob.mesh()
        ctx = bem.Context(0)
        ctx.set_mesh(mesh.xyz, mesh.tri)
        z, w = ctx.set_contour(prob.contour.kind, prob.contour.centre, prob.contour.a,
                               prob.contour.b, prob.N)
        V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
        ctxs.append(ctx)
        Vh.append(V)
        Vs.append(bem.fortran(torch.from_numpy(V).to("cuda:0")))
        zs.append(z)
        ws.append(w)
        meshes.append(mesh)
    return ctxs, Vs, Vh, zs, ws, meshes


def _small_problems():
    # ellipsoids like the 48-problem sweep, small enough for the oracle: ragged sizes
    # (not multiples of the 128-row tile), node counts 16 / 24, several basis widths
    out = []
    for p, (m, axes, c, N, nu) in enumerate([(4, (0.6, 0.9, 1.3), 4.0, 16, 8),
                                              (5, (1.2, 0.7, 0.5), 6.0, 24, 16),
                                              (7, (1.0, 1.0, 1.0), 3.5, 16, 32),
                                              (6, (1.9, 1.1, 0.8), 2.5, 24, 5),
                                              (9, (0.8, 1.4, 1.0), 5.0, 16, 32)]):
        out.append(synth.workloads.Problem(lambda m=m, axes=axes: synth.cube_sphere(m, axes),
                                           synth.ContourSpec("circle", c + 0j, 0.8, 0.8), N, nu,
                                           synth.workloads.BASE_SEED + 100 + p, f"small{p}"))
    return out


def test_batch_matches_oracle_and_single(bem):
    probs = _small_problems()
    ctxs, Vs, Vh, zs, ws, meshes = _setup(bem, probs)
    out = bem.project_batched(ctxs, Vs)
    torch.cuda.synchronize()
    for k, prob in enumerate(probs):
        B = out[k].cpu().numpy()
        P, _ = orr.project(meshes[k], zs[k], Vh[k])
        single = ctxs[k].project(Vs[k], bem.PREC_MIXED).cpu().numpy()
        for j in range(prob.N):
            ref = ws[k][j] * P[j]
            assert _relerr(B[j], ref) < TOL, (k, j)
            assert _relerr(B[j], single[j]) < 2e-5, (k, j)
    for c in ctxs:
        c.close()


def test_batch_graph_replay_autotune_and_state(bem):
    probs = _small_problems()[:3]
    ctxs, Vs, Vh, zs, ws, meshes = _setup(bem, probs)
    batch = bem.Batch(ctxs, Vs, autotune=True)
    info = batch.info()
    assert info["splits"] in (0, 1, 2, 3, 4) and info["nodes_per_unit"] in (0, 2)
    assert info["units"] > 0 and info["tuned_ms"] > 0
    first = [B.clone() for B in batch.run()]
    torch.cuda.synchronize()
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(first[k], batch.Bhat[k])   # replays are deterministic
        P, _ = orr.project(meshes[k], zs[k], Vh[k])
        for j in range(probs[k].N):
            assert _relerr(batch.Bhat[k][j].cpu().numpy(), ws[k][j] * P[j]) < TOL
    before = ctxs[0].launches
    batch.run()
    torch.cuda.synchronize()
    assert ctxs[0].launches > before
    # a context whose contour changed invalidates the recorded graph
    ctxs[1].set_contour("circle", 4.5, 0.8, 0.8, 16)
    with pytest.raises(bem.BemError) as e:
        batch.run()
    assert e.value.status == -7
    batch.close()
    for c in ctxs:
        c.close()


def test_batch_rejects_bad_arguments(bem):
    probs = _small_problems()[:2]
    ctxs, Vs, *_ = _setup(bem, probs)
    with pytest.raises(bem.BemError):                 # the same context twice
        bem.project_batched([ctxs[0], ctxs[0]], [Vs[0], Vs[0]])
    empty = bem.Context(0)
    with pytest.raises(bem.BemError):                 # a context without a mesh
        import paper_1906_03938_gb300 as b
        hs, vp, ld, nus, bp = b._batch_arrays([ctxs[0], empty], [Vs[0], Vs[0]],
                                              [Vs[0], Vs[0]])
        st = b.load().bem_project_batched(hs, 2, vp, ld, nus, bp, b.PREC_MIXED, b._stream(None))
        if st != 0:
            raise b.BemError("bem_project_batched", st, "")
    for c in ctxs + [empty]:
        c.close()


def test_batch48_full_against_single(bem):
    """The 48-ellipsoid sweep at full size: every problem of the grouped launch against the
    same context's single-problem projection, the three smallest also against the oracle."""
    probs = synth.workload("batch48").problems
    ctxs, Vs, Vh, zs, ws, meshes = _setup(bem, probs)
    batch = bem.Batch(ctxs, Vs, autotune=False)
    out = batch.run()
    torch.cuda.synchronize()
    for c in ctxs:
        c.check()
    sizes = [m.n for m in meshes]
    smallest = set(np.argsort(sizes)[:3].tolist())
    for k, prob in enumerate(probs):
        B = out[k].cpu().numpy()
        single = ctxs[k].project(Vs[k], bem.PREC_MIXED).cpu().numpy()
        assert np.all(np.isfinite(B))
        for j in range(prob.N):
            assert _relerr(B[j], single[j]) < 2e-5, (k, j)
        if k in smallest:
            P, _ = orr.project(meshes[k], zs[k], Vh[k])
            for j in range(0, prob.N, 3):
                assert _relerr(B[j], ws[k][j] * P[j]) < TOL, (k, j)
    batch.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("problem", [9, 14])
def test_batch48_problem_eigenvalues_against_oracle(bem, problem):
    """The whole method (Algorithm 1, CholeskyQR2, mixed projection, reduced solve,
    refinement) on a problem of the 48-ellipsoid sweep with stored oracle eigenvalues
    (tests/golden/eigs_batch48_p<i>.txt, pinned complete by the argument principle): every
    one found, no converged extra inside the circle, 1e-10 relative."""
    import os
    import bench
    if bench.read_golden(f"batch48_p{problem}") is None:
        pytest.skip("stored list absent")
    prob = synth.workload("batch48").problems[problem]
    mesh, c = prob.mesh(), prob.contour
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    V0 = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, prob.seed)).to("cuda:0"))
    lam, X, rel = ctx.solve(V0, q=10, precision=bem.PREC_MIXED, tol=1e-14)
    res = bench.eig_compare(lam, X.cpu().numpy(), rel, bench.read_golden(f"batch48_p{problem}"),
                            c, 1e-10)
    print(problem, lam, rel)
    assert not res["missing"] and not res["extras"], res
    ctx.close()
