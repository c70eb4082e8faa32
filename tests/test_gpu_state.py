"""Context statistics and checkpoints: a context restored from a checkpoint reproduces the
saved context's projections bit for bit; damaged checkpoints are rejected on the host."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    return b


def test_checkpoint_roundtrip_and_stats(bem):
    prob = synth.workload("sphere320").problems[0]
    mesh, c = prob.mesh(), prob.contour
    a = bem.Context(0)
    a.set_mesh(mesh.xyz, mesh.tri)
    a.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    a.surrogate_init(seed=9)
    a.set_near_field(2)
    st = a.stats()
    assert st["n"] == mesh.n and st["N"] == prob.N and st["near_mode"] == 2
    assert st["near_pairs"] > 0 and st["surrogate_ready"] == 1
    blob = a.save_state()
    b = bem.Context(0)
    b.load_state(blob)
    sb = b.stats()
    assert (sb["n"], sb["N"], sb["near_mode"], sb["near_pairs"]) == \
        (st["n"], st["N"], st["near_mode"], st["near_pairs"])
    assert np.array_equal(a.surrogate_params(1), b.surrogate_params(1))
    V = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, prob.nu, 3)).to("cuda:0"))
    for prec in (bem.PREC_FP64, bem.PREC_MIXED):
        Ba = a.project(V, prec)
        Bb = b.project(V, prec)
        torch.cuda.synchronize()
        assert torch.equal(Ba, Bb)
    # damaged checkpoints
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(bem.BemError) as e:
        b.load_state(bytes(bad))
    assert e.value.status == -1
    with pytest.raises(bem.BemError) as e:
        b.load_state(blob[:len(blob) // 2])
    assert e.value.status == -1
    a.close()
    b.close()


def test_checkpoint_keeps_the_operator(bem):
    """A Robin operator survives the round trip (same projections bit for bit); a state of
    the earlier layout (tag BEMSTAT1, no operator) loads as the single layer."""
    mesh = synth.icosphere(1)
    a = bem.Context(0)
    a.set_mesh(mesh.xyz, mesh.tri)
    a.set_operator(0.5 + 0.2j, 1.0 - 0.3j)
    a.set_contour("circle", 2.75, 0.9, 0.9, 8)
    blob = a.save_state()
    assert blob[:8] == b"BEMSTAT2"
    b = bem.Context(0)
    b.load_state(blob)
    V = bem.fortran(torch.from_numpy(synth.complex_gaussian(mesh.n, 8, 4)).to("cuda:0"))
    for prec in (bem.PREC_FP64, bem.PREC_MIXED):
        assert torch.equal(a.project(V, prec), b.project(V, prec))
    # the earlier layout: the same header without the operator's four doubles
    hdr = 8 + 6 * 8 + 4 * 8
    old = b"BEMSTAT1" + blob[8:hdr] + blob[hdr + 32:]
    c = bem.Context(0)
    c.load_state(old)
    ref = bem.Context(0)
    ref.set_mesh(mesh.xyz, mesh.tri)
    ref.set_contour("circle", 2.75, 0.9, 0.9, 8)
    assert torch.equal(c.project(V, bem.PREC_FP64), ref.project(V, bem.PREC_FP64))
    for x in (a, b, c, ref):
        x.close()
