"""Unit test (CPU) of the library's small dense complex eigensolver (Hessenberg reduction,
shifted QR, back substitution), compiled for the host from the same header the CUDA
kernels use. Checked against the definition A v = lambda v and against LAPACK's
eigenvalues."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("small_eig") / "libsmall_eig.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_1906_03938_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "helpers", "small_eig_host.cpp"),
                           "-o", str(out)])
    L = ctypes.CDLL(str(out))
    L.small_eig_host.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 3
    L.small_eig_host.restype = ctypes.c_int
    return L


def _eig(lib, A):
    m = A.shape[0]
    Af = np.asfortranarray(A.astype(np.complex128)).copy(order="F")
    w = np.zeros(m, complex)
    V = np.zeros((m, m), complex, order="F")
    st = lib.small_eig_host(m, Af.ctypes.data, w.ctypes.data, V.ctypes.data)
    return st, w, V


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (5, 2), (16, 3), (64, 4), (128, 5)])
def test_random_matrices(lib, m, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    st, w, V = _eig(lib, A)
    assert st == 0
    ref = np.linalg.eigvals(A)
    for x in ref:
        assert np.min(np.abs(w - x)) < 1e-10 * max(1, np.abs(ref).max())
    res = np.linalg.norm(A @ V - V * w[None, :], axis=0)
    assert np.all(res < 1e-10 * np.linalg.norm(A))
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)


def test_structured_cases(lib):
    # diagonal, triangular, repeated eigenvalues, a Jordan-free defective-looking case
    D = np.diag([3.0, 1.0 + 2j, -4.0, 1.0 + 2j])
    st, w, _ = _eig(lib, D)
    assert st == 0 and np.allclose(np.sort_complex(w), np.sort_complex(np.diag(D)))
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(20, 20)) + 1j * rng.normal(size=(20, 20)))
    lam = np.array([2.0] * 5 + list(rng.normal(size=15) + 1j * rng.normal(size=15)))
    A = Q @ np.diag(lam) @ Q.conj().T
    st, w, V = _eig(lib, A)
    assert st == 0
    assert np.sum(np.abs(w - 2.0) < 1e-9) == 5
    assert np.linalg.norm(A @ V - V * w[None, :]) < 1e-10 * np.linalg.norm(A)
