"""Full-size parity of the mixed path on the two large workloads, on sampled rows.

sphere20480 (icosphere level 5, 20480 panels, circle 7 / 1, N = 32, nu = 128) and
ellipsoid98304 (98304 panels, circle 9 / 1.5, N = 64, nu = 256), both with the near-field
rule on (mode 1), at the launch configuration of the single-problem projection. The oracle
computes (A(z_j) V) on sampled rows (all columns, all nodes, near-field variant). At these
sizes a flat relative bar is not what the arithmetic fixes: each product term carries the
split-precision error (hi + lo of each operand keeps 2^-17 of it, so ~2^-16 per product)
and the FP32 accumulation over the K-blocks adds ~u32 sqrt(6 n / 16) relative to the sum of
the terms' magnitudes. So every element must satisfy
|Y_gpu - Y_oracle| <= (2^-15 + 4 u32 sqrt(6 n / 16)) * (|A(z_j)| |V|)_(i, c), the
magnitudes taken from the oracle's rows of A(z_j) (a factor 2 of margin on each term).
The projected matrices are checked against w_j V^H (A(z_j) V) formed from the GPU's own
full A(z_j) V in FP64 by the same kind of bound: the contraction runs in BF16x3 on the
tensor core when nu <= 128 (3 products per 16-row K-block and half of the output), so
|B_j - ref| <= |w_j| (2^-15 + 4 u32 sqrt(3 n / 16)) (|V|^T |A(z_j) V|) elementwise."""
import numpy as np
import pytest
import torch

import synth
from oracle import assembly as oasm, contour as ocon, rr as orr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def _relerr(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("name", ["sphere20480", "ellipsoid98304"])
def test_large_workload_sampled_rows(bem, name):
    prob = synth.workload(name).problems[0]
    mesh = prob.mesh()
    V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    c = prob.contour
    z, w = ctx.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    zo, wo = ocon.from_spec(c, prob.N)
    assert np.max(np.abs(z - zo)) < 1e-14 * np.max(np.abs(zo))
    ctx.set_near_field(1)
    Vd = bem.fortran(torch.from_numpy(V).to("cuda:0"))
    B, Y = ctx.project(Vd, bem.PREC_MIXED, AV=True)
    ctx.check()
    # the contraction: Bhat_j against w_j V^H Y_j in FP64 from the returned Y
    u32 = 2.0 ** -24
    cbound = 2.0 ** -15 + 4 * u32 * np.sqrt(3 * mesh.n / 16)
    for j in (0, prob.N // 2, prob.N - 1):
        ref = w[j] * (Vd.conj().transpose(0, 1) @ Y[j]).cpu().numpy()
        mass = abs(w[j]) * (Vd.abs().transpose(0, 1) @ Y[j].abs()).cpu().numpy()
        r = np.max(np.abs(B[j].cpu().numpy() - ref) / (cbound * mass))
        assert r <= 1.0, (j, r, _relerr(B[j].cpu().numpy(), ref))
    # sampled rows against the oracle (near-field variant), all nodes
    rng = np.random.default_rng(7)
    R = 16   # rows per sample block (one oracle thread per row)
    starts = sorted(rng.choice(mesh.n - R, size=2, replace=False).tolist()) + [mesh.n - R]
    coef = 2.0 ** -15 + 4 * u32 * np.sqrt(6 * mesh.n / 16)
    absV = np.abs(V)
    worst = 0.0
    for r0 in starts:
        _, Yo = orr.project(mesh, z, V, rows=(r0, r0 + R), near=True)
        Yg = Y[:, r0:r0 + R, :].cpu().numpy()
        for j in range(prob.N):
            mass = np.abs(oasm.matrix(mesh, z[j], rows=(r0, r0 + R), near=True)) @ absV
            ratio = np.max(np.abs(Yg[j] - Yo[j]) / (coef * mass))
            worst = max(worst, ratio)
            assert ratio <= 1.0, (r0, j, ratio, _relerr(Yg[j], Yo[j]))
    print(name, "worst error / bound", worst)
    del Y
    ctx.close()
