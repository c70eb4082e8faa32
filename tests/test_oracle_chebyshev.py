"""Pins of the Chebyshev oracle (oracle/chebyshev.py): the interpolant reproduces the samples
at the nodes and any polynomial of degree < N exactly; the colleague linearisation of a
scalar Chebyshev series has the roots numpy's Chebyshev module finds, and that of a matrix
polynomial the eigenvalues of its textbook companion pencil."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import chebyshev as och


def test_interpolation_at_nodes_and_polynomial_exactness():
    rng = np.random.default_rng(2)
    c, a, N = 4.0, 1.3, 12
    x = och.nodes(c, a, N)
    samples = rng.normal(size=(N, 3, 3)) + 1j * rng.normal(size=(N, 3, 3))
    B = och.coefficients(samples)
    for k in range(N):
        assert np.max(np.abs(och.evaluate(B, (x[k] - c) / a) - samples[k])) < 1e-13
    P = [rng.normal(size=(2, 2)) for _ in range(5)]     # degree 4 matrix polynomial
    T = lambda z: sum(P[i] * z ** i for i in range(5))
    B = och.coefficients(np.stack([T(xk) for xk in x]))
    for z in (3.1, 4.7 + 0.2j, 5.5):
        assert np.max(np.abs(och.evaluate(B, (z - c) / a) - T(z))) < 1e-11 * np.max(np.abs(T(z)))
    assert np.max(np.abs(B[5:])) < 1e-12


def test_scalar_colleague_roots_match_numpy():
    rng = np.random.default_rng(3)
    b = rng.normal(size=7) + 1j * rng.normal(size=7)
    B = b[:, None, None]
    zeta, _ = och.eigs(B, 0.0, 1.0)
    ref = np.polynomial.chebyshev.chebroots(b)
    assert len(zeta) == 6
    for r in ref:
        assert np.min(np.abs(zeta - r)) < 1e-10 * max(1.0, abs(r))


def test_matrix_polynomial_eigenvalues():
    rng = np.random.default_rng(4)
    nu = 3
    A0, A1, A2 = (rng.normal(size=(nu, nu)) + 1j * rng.normal(size=(nu, nu)) for _ in range(3))
    I, Z = np.eye(nu), np.zeros((nu, nu))
    ref = sla.eigvals(np.block([[Z, I], [-A0, -A1]]), np.block([[I, Z], [Z, A2]]))
    c, a, N = 0.0, 2.0, 8
    x = och.nodes(c, a, N)
    B = och.coefficients(np.stack([A0 + xk * A1 + xk ** 2 * A2 for xk in x]))
    lam, _ = och.eigs(B, c, a)
    # the trailing coefficients are rounding noise; eigenvalues near the interval are exact
    near = [r for r in ref if abs(r - c) < 3 * a]
    assert len(near) >= 4
    for r in near:
        assert np.min(np.abs(lam - r)) < 1e-9 * max(1.0, abs(r))


def test_shift_invert_is_inverse_of_pencil():
    rng = np.random.default_rng(5)
    B = rng.normal(size=(6, 2, 2)) + 1j * rng.normal(size=(6, 2, 2))
    A, M = och.pencil(B)
    W = rng.normal(size=(A.shape[0], 3))
    sigma = 0.3 - 0.1j
    X = och.shift_invert_apply(B, sigma, W)
    assert np.max(np.abs((A - sigma * M) @ X - M @ W)) < 1e-12 * np.max(np.abs(M @ W))


@pytest.mark.parametrize("m", [5, 6])
def test_algorithm2_step_is_inverse_iteration_on_the_pencil(m):
    """Algorithm 2's step (recurrence on the block rows, then G u = b) equals one step of
    plain inverse iteration A^{-1} M w on the explicit colleague pencil, for an odd and an
    even number of blocks (the paper prints b separately for each parity)."""
    rng = np.random.default_rng(m)
    n = 7
    B = rng.normal(size=(m + 1, n, n)) + 1j * rng.normal(size=(m + 1, n, n))
    W = rng.normal(size=(m * n, 3)) + 1j * rng.normal(size=(m * n, 3))
    got = och.inverse_power_step(B, W)
    ref = och.shift_invert_apply(B, 0.0, W)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_algorithm2_converges_to_eigenvector_nearest_centre():
    """q steps of Algorithm 2 on a matrix polynomial with known eigenvalues: the u-part
    aligns with the eigenvector of the eigenvalue nearest the interval's centre."""
    rng = np.random.default_rng(4)
    n = 6
    lam = np.array([0.05, 0.6, -0.7, 1.5, -1.8, 2.2])
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    # T(zeta) = Q diag(zeta - lam) Q^H: degree 1, interpolated exactly by m = 4
    x = np.cos(np.pi * (np.arange(5) + 0.5) / 5)
    B = och.coefficients([Q @ np.diag(xx - lam) @ Q.conj().T for xx in x])
    U = och.inverse_power(B, rng.normal(size=(n, 1)) + 0j, 30)
    u = U[:, 0] / np.linalg.norm(U[:, 0])
    assert 1 - abs(np.vdot(Q[:, 0], u)) < 1e-10
