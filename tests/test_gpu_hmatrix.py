"""GPU parity of the low-rank far field (bem_set_hmatrix, precision BEM_PREC_HMATRIX)
against the FP64 projection and the oracle's H-matrix (oracle/hmatrix.py).

The H-matrix replaces each far block by its adaptive cross approximation to relative
accuracy eps, and evaluates entries and products in FP32: the projected matrices must then
agree with the FP64 dense projection to about eps plus the FP32 level, bar 1e-4 (max-norm per
node) at eps = 1e-6; the block structure must match the oracle's (the same definitions), and
the products A_H V the oracle's H-matrix products to the same bar."""
import numpy as np
import pytest
import torch

import synth
from oracle import hmatrix as ohm

pytestmark = pytest.mark.gpu


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


def _ctx(bem, mesh, spec, N, op=None, near=0):
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    if op:
        ctx.set_operator(*op)
    if near:
        ctx.set_near_field(near)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return ctx, z, w


@pytest.mark.parametrize("level,op,near", [(3, None, 0), (4, None, 0), (3, (0.0, 1.0), 0),
                                           (4, None, 1)],
                         ids=["L3", "L4", "L3-neumann", "L4-near"])
def test_hmatrix_projection_matches_fp64(bem, level, op, near):
    mesh = synth.icosphere(level)
    spec = synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    N, nu = 8, 24
    ctx, z, w = _ctx(bem, mesh, spec, N, op, near)
    ctx.set_hmatrix(leaf=16 if level == 3 else 32, eta=1.0, eps=1e-6, rmax=64)
    V = _dev(synth.complex_gaussian(mesh.n, nu, 3))
    B64, Y64 = ctx.project(V, bem.PREC_FP64, AV=True)
    Bh, Yh = ctx.project(V, bem.PREC_HMATRIX, AV=True)
    ctx.check()
    eb = max(_relerr(Bh[j].cpu().numpy(), B64[j].cpu().numpy()) for j in range(N))
    ey = max(_relerr(Yh[j].cpu().numpy(), Y64[j].cpu().numpy()) for j in range(N))
    st = ctx.hmatrix_stats()
    print(f"L{level} op={op} near={near}: Bhat {eb:.1e}, AV {ey:.1e}, stats {st}")
    assert eb < 1e-4 and ey < 1e-4
    assert 0 < st["mean_rank"] <= 64 and st["far_blocks"] > 0
    ctx.close()


@pytest.mark.parametrize("nu", [100, 200], ids=["nu100-two-chunks", "nu200-four-chunks"])
def test_hmatrix_wide_bases(bem, nu):
    """Basis widths of two and four 64-column chunks (ragged: zero-padded columns)."""
    mesh = synth.icosphere(4)
    spec = synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    N = 4
    ctx, z, w = _ctx(bem, mesh, spec, N)
    ctx.set_hmatrix(leaf=32, eta=1.0, eps=1e-6, rmax=64)
    V = _dev(synth.complex_gaussian(mesh.n, nu, 7))
    B64, Y64 = ctx.project(V, bem.PREC_FP64, AV=True)
    Bh, Yh = ctx.project(V, bem.PREC_HMATRIX, AV=True)
    ctx.check()
    eb = max(_relerr(Bh[j].cpu().numpy(), B64[j].cpu().numpy()) for j in range(N))
    ey = max(_relerr(Yh[j].cpu().numpy(), Y64[j].cpu().numpy()) for j in range(N))
    st, work = ctx.hmatrix_stats(), ctx.hmatrix_work()
    print(f"nu={nu}: Bhat {eb:.1e}, AV {ey:.1e}, {work}")
    assert eb < 1e-4 and ey < 1e-4
    # the dense work is every entry outside the far blocks, evaluated once
    n2 = float(mesh.n) ** 2
    assert abs(work["dense_entries"] - (1.0 - st["far_fraction"]) * n2) <= 1e-9 * n2
    assert work["far_row_terms"] > 0 and work["far_col_terms"] > 0
    ctx.close()


@pytest.mark.parametrize("level", [0, 1], ids=["root-leaf", "no-far-blocks"])
def test_hmatrix_without_far_blocks(bem, level):
    """A mesh of one leaf (20 panels) and one whose admissible blocks are all too small to be
    far (80 panels): every entry dense, the leaf kernel alone (no cross approximation)."""
    mesh = synth.icosphere(level)
    spec = synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    N, nu = 5, 3
    ctx, z, w = _ctx(bem, mesh, spec, N)
    ctx.set_hmatrix(leaf=32, eta=1.0, eps=1e-6, rmax=64)
    V = _dev(synth.complex_gaussian(mesh.n, nu, 9))
    B64, Y64 = ctx.project(V, bem.PREC_FP64, AV=True)
    Bh, Yh = ctx.project(V, bem.PREC_HMATRIX, AV=True)
    ctx.check()
    st, work = ctx.hmatrix_stats(), ctx.hmatrix_work()
    assert st["far_blocks"] == 0 and st["far_fraction"] == 0.0
    assert work["dense_entries"] == float(mesh.n) ** 2 and work["far_row_terms"] == 0.0
    eb = max(_relerr(Bh[j].cpu().numpy(), B64[j].cpu().numpy()) for j in range(N))
    ey = max(_relerr(Yh[j].cpu().numpy(), Y64[j].cpu().numpy()) for j in range(N))
    assert eb < 1e-4 and ey < 1e-4
    ctx.close()


def test_structure_and_products_match_oracle(bem):
    mesh = synth.icosphere(3)
    spec = synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    ctx, z, w = _ctx(bem, mesh, spec, 2)
    ctx.set_hmatrix(leaf=16, eta=1.0, eps=1e-6, rmax=64)
    V = synth.complex_gaussian(mesh.n, 8, 4)
    _, Yh = ctx.project(_dev(V), bem.PREC_HMATRIX, AV=True)
    st = ctx.hmatrix_stats()
    cl = ohm.cluster_tree(mesh, leaf=16)
    bl = ohm.blocks(cl, eta=1.0, leaf=16)
    assert st["far_blocks"] > 0
    assert st["far_blocks"] == sum(1 for b in bl if b[2])
    assert st["dense_blocks"] == sum(1 for b in bl if not b[2])
    for j in range(2):
        comp = ohm.compress(mesh, z[j], cl, bl, eps=1e-6)
        Yo = ohm.apply(cl, bl, comp, V)
        assert _relerr(Yh[j].cpu().numpy(), Yo) < 1e-4
    ctx.close()


def test_hmatrix_arguments(bem):
    mesh = synth.icosphere(1)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour("circle", 4.0, 1.0, 1.0, 4)
    V = _dev(synth.complex_gaussian(mesh.n, 4, 1))
    with pytest.raises(bem.BemError):
        ctx.project(V, bem.PREC_HMATRIX)          # no far field configured
    for bad in (dict(leaf=0), dict(leaf=64), dict(eps=0.0), dict(rmax=0), dict(rmax=500)):
        with pytest.raises(bem.BemError):
            ctx.set_hmatrix(**bad)
    ctx.close()
