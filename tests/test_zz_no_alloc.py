"""The allocation-free projection entry point, for callers that cannot call cudaMalloc
(for example code running under a locked or externally owned memory pool).

It is called through the C ABI and compared with the ordinary FP64 entry point
(bem_project) on the same inputs, twice in a row, at the tolerance of the FP64 parity
tests. This file sorts last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def bem():
    import paper_1906_03938_gb300 as b
    from paper_1906_03938_gb300 import build
    build.build()
    b.load()
    return b


def _noalloc(bem, mesh, xyz, tri, spec, N, Vd, out):
    lib = bem.load()
    kind = bem.CONTOUR_CIRCLE if spec.kind == "circle" else bem.CONTOUR_ELLIPSE
    c = complex(spec.centre)
    st = lib.bem_project_fp64_noalloc(
        0, mesh.xyz.shape[0], ctypes.c_void_p(xyz.data_ptr()), mesh.n,
        ctypes.c_void_p(tri.data_ptr()), kind, c.real, c.imag, spec.a, spec.b, N,
        ctypes.c_void_p(Vd.data_ptr()), Vd.stride(1), Vd.shape[1],
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


CASES = {
    "sphere320": lambda: (synth.icosphere(2), synth.ContourSpec("circle", 4.0 + 0j, 1.0, 1.0), 16, 16),
    "ragged108": lambda: (synth.cube_grid(3), synth.ContourSpec("ellipse", 6.5 + 0.1j, 1.5, 0.4), 7, 5),
    # 32 nodes of 3 MB products each do not fit together: exercises the node groups
    "cube3072": lambda: (synth.cube_grid(16), synth.ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4), 32, 64),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_project_twice(bem, case):
    mesh, spec, N, nu = CASES[case]()
    V = synth.complex_gaussian(mesh.n, nu, 11)
    Vd = bem.fortran(torch.from_numpy(V).to("cuda:0"))
    ctx = bem.Context(0)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(spec.kind, spec.centre, spec.a, spec.b, N)
    ref = ctx.project(Vd, bem.PREC_FP64).cpu().numpy()
    ctx.close()
    xyz = torch.from_numpy(mesh.xyz).to("cuda:0")
    tri = torch.from_numpy(mesh.tri).to("cuda:0")
    for call in range(2):
        out = torch.full((N, nu, nu), complex(np.nan, np.nan), dtype=torch.complex128,
                         device="cuda:0")
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(bem, mesh, xyz, tri, spec, N, Vd, out) == bem.BEM_OK
        if call == 1:   # after the first call nothing more is taken from the device
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.transpose(1, 2).cpu().numpy()
        for j in range(N):
            err = np.max(np.abs(got[j] - ref[j])) / np.max(np.abs(ref[j]))
            assert err < TOL, (case, call, j, err)


def test_noalloc_rejects_sizes_beyond_its_array(bem):
    mesh = synth.tetrakis_sphere(6, (1.0, 0.7, 0.5))      # 98304 triangles, 64 nodes
    V = torch.zeros((256, mesh.n), dtype=torch.complex128, device="cuda:0").transpose(0, 1)
    out = torch.zeros((64, 256, 256), dtype=torch.complex128, device="cuda:0")
    xyz = torch.from_numpy(mesh.xyz).to("cuda:0")
    tri = torch.from_numpy(mesh.tri).to("cuda:0")
    st = _noalloc(bem, mesh, xyz, tri, synth.ContourSpec("circle", 9.0 + 0j, 1.5, 1.5), 64, V,
                  out)
    assert st == -1                                       # BEM_EINVAL, nothing launched
    assert torch.count_nonzero(out).item() == 0
    # the reason is kept for the calling thread
    assert b"too large" in bem.load().bem_noalloc_last_error()
