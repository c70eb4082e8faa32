"""Failure detection on the GPU without a GPU fault: the fused kernel's bounded waits and
the device status word.

* Every pipeline-stage wait of the fused mixed-precision kernel polls an mbarrier a bounded
  number of times. With the bound set to zero (bem_set_wait_limit) every wait gives up at
  once: the kernel records BEM_ETIMEOUT, its blocks drain their copies and tensor-core
  products in flight (those drains keep the full bound), release their tensor memory and
  return. bem_check reports the timeout, and the next projection on the same context, with
  the default bound again, matches the oracle (the context stayed usable).
* A non-finite entry in the basis is recorded in the status word by the projection's
  preparation kernel and by CholeskyQR2; both report it instead of returning NaN silently,
  and a clean call on the same context succeeds afterwards."""
import numpy as np
import pytest
import torch

import synth
from oracle import contour as ocon, rr as orr

pytestmark = pytest.mark.gpu
TOL = 1e-4   # the mixed path's bar (see test_gpu_mixed)


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


def _setup(bem, N=8):
    mesh = synth.icosphere(2)
    spec = synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0)
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    z, w = ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    return ctx, mesh, z, w


def _check_against_oracle(ctx, bem, mesh, z, w, V):
    B, Y = ctx.project(_dev(V), bem.PREC_MIXED, AV=True)
    ctx.check()
    P, Yo = orr.project(mesh, z, V)
    Bh, Yh = B.cpu().numpy(), Y.cpu().numpy()
    for j in range(len(z)):
        assert _relerr(Yh[j], Yo[j]) < TOL
        assert _relerr(Bh[j], w[j] * P[j]) < TOL


@pytest.mark.parametrize("nu", [16, 72, 136])
def test_stage_wait_runs_out_and_context_recovers(bem, nu):
    """nu = 136: units of one node, twin pairs on two-CTA clusters; the partners leave the
    cluster together after any half sent between them has landed."""
    ctx, mesh, z, w = _setup(bem)
    V = synth.complex_gaussian(mesh.n, nu, 9)
    ctx.set_wait_limit(0)
    ctx.project(_dev(V), bem.PREC_MIXED)
    with pytest.raises(bem.BemError) as e:
        ctx.check()
    assert e.value.status == bem.STATUS_CODES["BEM_ETIMEOUT"], str(e.value)
    assert "wait-timeout" in str(e.value)
    # the status word was cleared by the check; the default bound restores normal service
    ctx.set_wait_limit(1 << 24)
    _check_against_oracle(ctx, bem, mesh, z, w, V)
    if nu > 128:
        assert ctx.mixed_shape()["paired"]
    ctx.close()


def test_non_finite_basis_is_reported(bem):
    ctx, mesh, z, w = _setup(bem, N=4)
    V = synth.complex_gaussian(mesh.n, 8, 4)
    Vbad = V.copy()
    Vbad[17, 3] = np.nan
    ctx.project(_dev(Vbad), bem.PREC_MIXED)
    with pytest.raises(bem.BemError) as e:
        ctx.check()
    assert e.value.status == bem.STATUS_CODES["BEM_EKERNEL"]
    assert "non-finite" in str(e.value)
    with pytest.raises(bem.BemError) as e:
        ctx.cholqr2(_dev(Vbad))
    assert e.value.status == bem.STATUS_CODES["BEM_EKERNEL"]
    _check_against_oracle(ctx, bem, mesh, z, w, V)
    ctx.close()
