"""Pins of the oracle's Rayleigh-Ritz layer: orthonormalisation, projection, the reduced
linearisation (Eq. EVP_red) and the inverse power / subspace iteration (Algorithms 1, 3),
against problems whose eigenvalues are known by construction or by a textbook
companion linearisation that uses none of the Cauchy machinery. Algorithm 1 in its
Schur-complement form is also pinned against plain inverse iteration on the explicit
(N + 1) n linearisation (a sign error in its v-update or the extra u^(j) term of the
printed listing fail it)."""
import numpy as np
import scipy.linalg as sla
import pytest

import synth
from oracle import contour, rr, assembly


def test_orthonormalize_definition():
    V = synth.complex_gaussian(200, 12, 3)
    Q, R = rr.orthonormalize(V)
    assert np.allclose(Q.conj().T @ Q, np.eye(12), atol=1e-14)
    assert np.allclose(Q @ R, V, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.abs(np.diag(R).imag) < 1e-14)
    assert np.all(np.diag(R).real > 0)


def test_projection_entries_and_covariance(oracle_mod):
    m = synth.icosphere(1)
    n = m.n
    z, _ = contour.nodes_weights("circle", 4.0, 1.0, 1.0, 4)
    # unit vectors pick single entries: (E^H A E)[a, b] = A[i_a, i_b]
    idx = [0, 7, 33]
    E = np.zeros((n, 3), dtype=complex)
    E[idx, range(3)] = 1.0
    P, Y = rr.project(m, z, E)
    for j in range(4):
        A = assembly.matrix(m, z[j])
        assert np.allclose(P[j], A[np.ix_(idx, idx)], rtol=0, atol=1e-15)
        assert np.allclose(Y[j], A[:, idx], rtol=0, atol=1e-15)
    # P(V U) = U^H P(V) U for unitary U (catches V^T in place of V^H)
    V = synth.complex_gaussian(n, 5, 11)
    U, _ = np.linalg.qr(synth.complex_gaussian(5, 5, 12))
    P1, _ = rr.project(m, z, V)
    P2, _ = rr.project(m, z, V @ U)
    for j in range(4):
        assert np.allclose(P2[j], U.conj().T @ P1[j] @ U, rtol=0, atol=1e-12)


def _quadratic(nu, seed):
    rng = np.random.default_rng(seed)
    A0, A1, A2 = (rng.normal(size=(nu, nu)) + 1j * rng.normal(size=(nu, nu)) for _ in range(3))
    A2 = 0.05 * A2
    return A0, A1, A2


def _companion_eigs(A0, A1, A2):
    """Textbook first companion form of A0 + z A1 + z^2 A2."""
    nu = A0.shape[0]
    I = np.eye(nu)
    Z = np.zeros((nu, nu))
    L = np.block([[Z, I], [-A0, -A1]])
    M = np.block([[I, Z], [Z, A2]])
    lam = sla.eigvals(L, M)
    return lam[np.isfinite(lam)]


def test_reduced_linearisation_reproduces_matrix_polynomial():
    """Circle contour: T~ = T / (1 + w^N) inside, so the zeros inside are reproduced to
    rounding for a polynomial T of degree < N."""
    nu = 6
    A0, A1, A2 = _quadratic(nu, 5)
    T = lambda t: A0 + t * A1 + t * t * A2
    ref = _companion_eigs(A0, A1, A2)
    c = ref[np.argsort(np.abs(ref))[2]]          # centre the circle on one eigenvalue
    rho = 0.6 * np.sort(np.abs(ref - c))[4]       # a few eigenvalues inside
    z, w = contour.nodes_weights("circle", c, rho, rho, 16)
    Bhat = np.stack([w[j] * T(z[j]) for j in range(16)])
    lam, Y = rr.reduced_eigs(Bhat, z)
    want = ref[np.abs(ref - c) < rho * 0.999]
    got = lam[np.abs(lam - c) < rho * 0.999]
    assert len(want) >= 2 and len(got) == len(want)
    for l in want:
        assert np.min(np.abs(got - l)) <= 1e-11 * abs(l)
    # the y part is a null vector of T(lambda)
    for k in np.where(np.abs(lam - c) < rho * 0.999)[0]:
        assert np.linalg.norm(T(lam[k]) @ Y[:, k]) < 1e-10 * np.linalg.norm(T(lam[k]))


def test_reduced_linearisation_ellipse_converges():
    nu = 4
    A0, A1, A2 = _quadratic(nu, 9)
    T = lambda t: A0 + t * A1 + t * t * A2
    ref = _companion_eigs(A0, A1, A2)
    c = ref[np.argsort(np.abs(ref))[0]]
    a = 0.5 * np.sort(np.abs(ref - c))[1]
    errs = []
    for N in (16, 32, 64):
        z, w = contour.nodes_weights("ellipse", c, a, 0.6 * a, N)
        lam, _ = rr.reduced_eigs(np.stack([w[j] * T(z[j]) for j in range(N)]), z)
        errs.append(np.min(np.abs(lam - c)))
    assert errs[2] < 1e-10 * abs(c) and errs[1] < errs[0]


def _linear_nlevp(n, lam_in, lam_out, seed):
    """T(z) = X diag(lambda) X^{-1} - z I with known eigenvalues."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    X = X / np.linalg.norm(X, axis=0)
    D = np.concatenate([lam_in, lam_out])
    K = X @ np.diag(D) @ np.linalg.inv(X)
    return lambda t: K - t * np.eye(n)


def test_inverse_power_is_inverse_iteration_on_the_linearisation():
    """Algorithm 1 in Schur-complement form (reading of its right-hand side: no u^(j) term)
    against plain inverse iteration w <- (A - s M)^{-1} M w on the explicit Cauchy
    linearisation of sum_j B_j / (z_j - z): unknowns (v_1 .. v_N, x), rows
    z_j v_j - x = lambda v_j and sum_j B_j v_j = 0, M = diag(I, .., I, 0). After q steps the
    x-part is parallel to the oracle's u (both iterations scale by scalars only)."""
    rng = np.random.default_rng(21)
    n, N, nu, q, s = 9, 6, 3, 4, 0.3 + 0.2j
    z = 2.0 * np.exp(2j * np.pi * (np.arange(N) + 0.5) / N)
    B = rng.normal(size=(N, n, n)) + 1j * rng.normal(size=(N, n, n))
    V0 = synth.complex_gaussian(n, nu, 22)
    u = rr.inverse_power(B, z, s, V0, q)
    dim = (N + 1) * n
    A = np.zeros((dim, dim), complex)
    M = np.zeros((dim, dim), complex)
    for j in range(N):
        blk = slice(j * n, (j + 1) * n)
        A[blk, blk] = z[j] * np.eye(n)
        A[blk, N * n:] = -np.eye(n)
        A[N * n:, blk] = B[j]
        M[blk, blk] = np.eye(n)
    K = np.linalg.solve(A - s * M, M)
    for c in range(nu):
        w = np.zeros(dim, complex)
        for j in range(N):
            w[j * n:(j + 1) * n] = V0[:, c] / (z[j] - s)
        for _ in range(q):
            w = K @ w
            w = w / np.linalg.norm(w)
        x = w[N * n:]
        cos = abs(np.vdot(x, u[:, c])) / (np.linalg.norm(x) * np.linalg.norm(u[:, c]))
        assert abs(cos - 1.0) < 1e-12, (c, cos)


def test_subspace_iteration_finds_known_eigenvalues():
    """Algorithms 1 and 3 on an n = 60 problem with 4 eigenvalues inside a circle."""
    n, nu = 60, 8
    c, rho = 5.0, 1.0
    lam_in = np.array([4.6, 5.2 + 0.1j, 5.3 - 0.2j, 4.9 + 0.3j])
    rng = np.random.default_rng(2)
    ang = rng.uniform(0, 2 * np.pi, n - 4)
    lam_out = c + rho * (1.6 + 3 * rng.uniform(size=n - 4)) * np.exp(1j * ang)
    T = _linear_nlevp(n, lam_in, lam_out, 4)
    N = 32
    z, w = contour.nodes_weights("circle", c, rho, rho, N)
    Bfull = np.stack([w[j] * T(z[j]) for j in range(N)])
    V0 = synth.complex_gaussian(n, nu, 1)
    lam, X, hist = rr.subspace_iteration(Bfull, z, c, V0, q=10, tol=1e-12, maxit=10,
                                         nwant=4)
    inside = np.abs(lam - c) < rho
    # Ritz values of the unconverged directions may fall inside too; their residual
    # ||T(lambda) x|| exposes them
    res = np.array([np.linalg.norm(T(lam[k]) @ X[:, k]) for k in range(len(lam))])
    got = lam[inside & (res < 1e-8)]
    assert len(got) == 4
    assert np.all(res[inside & (res >= 1e-8)] > 1e-3)
    for l in lam_in:
        assert np.min(np.abs(got - l)) < 1e-10
    assert hist[-1] <= 1e-10
