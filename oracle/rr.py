"""Rayleigh-Ritz projection and the reduced Cauchy linearisation (Section 3), oracle side.

Conventions (each a reading of the paper, recorded in the design notes):

* Weighted samples B_j = w_j A(z_j) with the trapezoid weights of ``contour`` so that
  T~(z) = sum_j B_j / (z_j - z) (Eq. TzApp, Eq. TzAppF0 with omega_j = -w_j).
* Projection (Eq. RR_approx): B^_j = V^H B_j V; ``project`` returns the unweighted
  P_j = V^H A(z_j) V and B^_j = w_j P_j.
* Reduced linearisation (Eq. EVP_red, Eq. sc1_cauchy_red) in this sign convention: with
  v_j = y / (lambda - z_j), lambda v_j = z_j v_j + y and sum_j B^_j v_j = 0, i.e. the
  pencil A w = lambda M w with A = [[diag(z_j I), 1 (x) I], [B^_0 .. B^_{N-1}, 0]],
  M = diag(I, .., I, 0), w = [v_0; ..; v_{N-1}; y]. Nodes are indexed j = 0 .. N-1.
* Inverse power step (Algorithm 1; Eq. wjp1, Eq. vjp1, Eq. viupd, Eq. linsyssim) with
  shift s, from (A - s M) w' = M w:
      S u' = sum_j B_j v_j / (z_j - s),  S = sum_j B_j / (z_j - s),
      v_j' = (v_j - u') / (z_j - s).
  The paper's right-hand side also carries u^(j); the algebra (M has a zero last block)
  drops it, and so does this oracle. Iterates are rescaled to unit norm (direction only).
* Starting blocks: v_j = u / (z_j - s) for a given u (the paper's refresh
  v_i = u / (lambda - sigma_i) taken at lambda = s); after an outer step the refresh uses
  the Ritz pairs (lambda, x): v_j = x / (lambda - z_j).
"""
import numpy as np
import scipy.linalg as sla

from . import assembly


def project(mesh, z, V, rows=None, threads=0, near=False, op=None):
    """P_j = V^H A(z_j) V (unweighted, Eq. RR_approx) and Y_j = A(z_j) V (near=True: the
    near-field variant of A)."""
    Y = assembly.apply(mesh, z, V, rows=rows, threads=threads, near=near, op=op)
    Vh = np.asarray(V).conj().T
    if rows is not None:
        Vh = Vh[:, rows[0]:rows[1]]
    P = np.stack([Vh @ Y[j] for j in range(Y.shape[0])])
    return P, Y


def orthonormalize(V):
    """The thin QR factor Q of V whose R has a positive real diagonal (what CholeskyQR2
    returns in exact arithmetic); also returns that R."""
    Q, R = np.linalg.qr(np.asarray(V, dtype=np.complex128))
    d = np.diag(R)
    ph = d / np.abs(d)
    return Q * ph[None, :], ph.conj()[:, None] * R


def linearization(Bhat, z):
    """The (N+1) nu pencil (A, M) of the reduced Cauchy problem."""
    N, nu, _ = Bhat.shape
    D = (N + 1) * nu
    A = np.zeros((D, D), dtype=np.complex128)
    M = np.zeros((D, D), dtype=np.complex128)
    I = np.eye(nu)
    for j in range(N):
        sl = slice(j * nu, (j + 1) * nu)
        A[sl, sl] = z[j] * I
        A[sl, N * nu:] = I
        A[N * nu:, sl] = Bhat[j]
        M[sl, sl] = I
    return A, M


def reduced_eigs(Bhat, z):
    """Finite eigenvalues lambda of the reduced pencil and the y-parts of their vectors."""
    N, nu, _ = Bhat.shape
    A, M = linearization(Bhat, z)
    lam, W = sla.eig(A, M)
    ok = np.isfinite(lam)
    lam = lam[ok]
    Y = W[N * nu:, ok]
    Y = Y / np.linalg.norm(Y, axis=0, keepdims=True)
    return lam, Y


def approx_residual(Bfull_apply, z, lam, X):
    """|| sum_j B_j X f_j(Lambda) ||_F with f_j(l) = 1 / (z_j - l) (the paper's stopping
    test in this sign convention); ``Bfull_apply(j, X)`` returns B_j X."""
    R = 0
    for j in range(len(z)):
        R = R + Bfull_apply(j, X) / (z[j] - lam)[None, :]
    return np.linalg.norm(R)


def inverse_power(Bfull, z, s, V0, q, v_start=None):
    """q steps of Algorithm 1 for every column; Bfull: (N, n, n) weighted samples B_j.
    v_start: optional (N, n, nu) starting v-blocks (default v_j = V0 / (z_j - s))."""
    d = 1.0 / (np.asarray(z) - s)
    S = np.einsum("j,jab->ab", d, Bfull)
    lu = sla.lu_factor(S)
    V = (np.asarray(V0)[None, :, :] * d[:, None, None]) if v_start is None else v_start.copy()
    u = None
    for _ in range(q):
        rhs = np.einsum("j,jab,jbc->ac", d, Bfull, V)
        u = sla.lu_solve(lu, rhs)
        V = (V - u[None, :, :]) * d[:, None, None]
        scale = np.sqrt(np.sum(np.abs(V) ** 2, axis=(0, 1)))
        V = V / scale[None, None, :]
        u = u / scale[None, :]
    return u


def subspace_iteration(Bfull, z, s, V0, q, tol=1e-12, maxit=20, nwant=None):
    """Algorithm 3 with outer refresh: returns (lam, X, history). Dense, small n only."""
    n, nu = V0.shape
    U = inverse_power(Bfull, z, s, V0, q)
    hist = []
    lam = X = None
    for it in range(maxit):
        Q, _ = orthonormalize(U)
        Bhat = np.einsum("ia,jib,bc->jac", Q.conj(), Bfull, Q)
        lam_all, Yv = reduced_eigs(Bhat, z)
        order = np.argsort(np.abs(lam_all - s))[:nu]
        lam = lam_all[order]
        X = Q @ Yv[:, order]
        X = X / np.linalg.norm(X, axis=0, keepdims=True)
        k = nu if nwant is None else nwant
        res = approx_residual(lambda j, Xs: Bfull[j] @ Xs, z, lam[:k], X[:, :k])
        hist.append(res)
        if res <= tol:
            break
        vstart = X[None, :, :] / (lam[None, None, :] - np.asarray(z)[:, None, None])
        U = inverse_power(Bfull, z, s, X, q, v_start=vstart)
    return lam, X, hist
