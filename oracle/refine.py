"""Discrete eigenvalues of A(k) and their residuals, oracle side.

The paper measures an eigenpair by the relative residual ||T(lambda) u||_2 / ||u||_2
(Section 4, Example 1) and targets all eigenvalues inside the contour (Section 1). The
final answer therefore has a plain definition, independent of the Cauchy and
Rayleigh-Ritz machinery: the k inside the contour at which A(k) is singular. This module
computes it directly:

* ``residual``: ||A(lambda) x|| / ||x|| per column (dense FP64 assembly).
* ``slp``: successive linear problems (Ruhe 1973): at the current lambda solve the linear
  pencil A(lambda) x = -theta A'(lambda) x for the theta of least modulus and step
  lambda <- lambda + theta until |theta| <= tol |lambda|. The fixed point is a k with
  A(k) singular whatever the derivative's accuracy; near a simple or semisimple
  eigenvalue the convergence is quadratic. At the converged lambda, the number of theta
  with |theta| <= mult_tol |lambda| is the multiplicity and the other small theta point
  at neighbouring eigenvalues.
* ``discrete_eigs``: SLP from every start, then from every neighbour it reveals, until the
  set inside the search radius is closed.
* ``sigma_min`` and ``winding_count`` (the argument principle on det A) are independent
  checks of the above.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import assembly


def residual(mesh, lam, X, near=False, op=None):
    X = np.atleast_2d(np.asarray(X, dtype=np.complex128).T).T
    lam = np.atleast_1d(lam)
    out = []
    for c in range(X.shape[1]):
        A = assembly.matrix(mesh, lam[c], near=near, op=op)
        out.append(np.linalg.norm(A @ X[:, c]) / np.linalg.norm(X[:, c]))
    return np.array(out)


def sigma_min(mesh, k, near=False, op=None):
    s = np.linalg.svd(assembly.matrix(mesh, k, near=near, op=op), compute_uv=False)
    return s[-1], s[0]


def _small_thetas(A, Ad, count):
    """The ``count`` values theta of least modulus with A x = -theta Ad x."""
    n = A.shape[0]
    if n <= 400:
        th = sla.eigvals(A, -Ad)
        th = th[np.isfinite(th)]
        return th[np.argsort(np.abs(th))[:count]]
    lu = sla.lu_factor(A)
    op = spla.LinearOperator((n, n), matvec=lambda x: -sla.lu_solve(lu, Ad @ x),
                             dtype=np.complex128)
    mu = spla.eigs(op, k=count, which="LM", return_eigenvectors=False, tol=1e-11,
                   maxiter=5000)
    th = 1.0 / mu
    return th[np.argsort(np.abs(th))]


def slp(mesh, lam0, tol=1e-14, maxit=30, count=6, near=False, op=None):
    lam = complex(lam0)
    th = None
    for _ in range(maxit):
        A = assembly.matrix(mesh, lam, near=near, op=op)
        Ad = assembly.matrix(mesh, lam, deriv=1, near=near, op=op)
        th = _small_thetas(A, Ad, count)
        lam = lam + th[0]
        if abs(th[0]) <= tol * abs(lam):
            break
    A = assembly.matrix(mesh, lam, near=near, op=op)
    Ad = assembly.matrix(mesh, lam, deriv=1, near=near, op=op)
    th = _small_thetas(A, Ad, count)
    return lam, th


def discrete_eigs(mesh, starts, radius=0.3, mult_tol=1e-9, dedup=1e-8, count=8,
                  keep=None, near=False, op=None):
    """Eigenvalues (with multiplicity) reached from ``starts`` and their neighbours within
    ``radius``; ``keep(lam)`` restricts which neighbours are followed."""
    found = []      # list of (lam, multiplicity)
    queue = [complex(s) for s in starts]
    seen = 0
    while queue and seen < 60:
        seen += 1
        s = queue.pop(0)
        if any(abs(s - f) <= 1e-6 * abs(f) for f, _ in found):
            continue
        lam, th = slp(mesh, s, count=count, near=near, op=op)
        if any(abs(lam - f) <= dedup * abs(f) for f, _ in found):
            continue
        mult = int(np.sum(np.abs(th) <= mult_tol * abs(lam)))
        found.append((lam, max(mult, 1)))
        for t in th:
            if mult_tol * abs(lam) < abs(t) < radius:
                cand = lam + t
                if keep is None or keep(cand):
                    queue.append(cand)
    found.sort(key=lambda p: (p[0].real, p[0].imag))
    return found


def winding_count(mesh, spec, M=256, near=False, op=None):
    """(1 / 2 pi i) \\oint tr(A(z)^{-1} A'(z)) dz by the trapezoid rule on the contour:
    the number of eigenvalues inside (argument principle)."""
    theta = 2.0 * np.pi * np.arange(M) / M
    a, b = spec.a, spec.b
    total = 0.0 + 0.0j
    for t in theta:
        zz = spec.centre + a * np.cos(t) + 1j * b * np.sin(t)
        dz = -a * np.sin(t) + 1j * b * np.cos(t)
        A = assembly.matrix(mesh, zz, near=near, op=op)
        Ad = assembly.matrix(mesh, zz, deriv=1, near=near, op=op)
        total += np.trace(np.linalg.solve(A, Ad)) * dz
    return total * (2.0 * np.pi / M) / (2.0j * np.pi)
