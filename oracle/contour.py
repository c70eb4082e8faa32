"""Contour quadrature for the Cauchy integral representation (Section 2, Eq. Tz, Eq. TzApp).

T(z) = (1 / 2 pi i) \\oint T(t) / (t - z) dt is discretised by the trapezoid rule in the
angle theta (the paper uses trapezoid nodes in its experiments; its one mention of
Gauss-Legendre is read as a slip, see the design notes). With
theta_j = 2 pi (j + 1/2) / N, j = 0 .. N-1, on the ellipse t(theta) = c + a cos(theta)
+ i b sin(theta) (a circle when a = b = rho):

    z_j = c + a cos(theta_j) + i b sin(theta_j)
    w_j = t'(theta_j) (2 pi / N) / (2 pi i) = (b cos(theta_j) + i a sin(theta_j)) / N

so that T(z) ~ sum_j w_j T(z_j) / (z_j - z). The paper writes the same sum as
sum_i omega_i T(sigma_i) / (z - sigma_i), i.e. omega_i = -w_i; the sign is carried by
the linearisation below instead.
"""
import numpy as np


def nodes_weights(kind: str, centre: complex, a: float, b: float, N: int):
    if kind == "circle":
        b = a
    elif kind != "ellipse":
        raise ValueError(f"unknown contour kind {kind!r}")
    theta = 2.0 * np.pi * (np.arange(N) + 0.5) / N
    z = complex(centre) + a * np.cos(theta) + 1j * b * np.sin(theta)
    w = (b * np.cos(theta) + 1j * a * np.sin(theta)) / N
    return z, w


def from_spec(spec, N: int):
    return nodes_weights(spec.kind, spec.centre, spec.a, spec.b, N)


def inside(lam, spec, margin: float = 0.0):
    """True where lam lies inside the contour shrunk by the relative ``margin``."""
    lam = np.asarray(lam)
    x = (lam.real - spec.centre.real) / spec.a
    y = (lam.imag - spec.centre.imag) / spec.b
    return np.sqrt(x * x + y * y) < 1.0 - margin


def inner_points(spec, nsamples: int):
    """Sample points on the inner contour (same centre, semi-axes halved: the circle of
    radius r/2 of Section 4, Example 3) at angles 2 pi (s + 1/4) / nsamples."""
    b = spec.a if spec.kind == "circle" else spec.b
    t = 2.0 * np.pi * (np.arange(nsamples) + 0.25) / nsamples
    return complex(spec.centre) + 0.5 * spec.a * np.cos(t) + 0.5j * b * np.sin(t)


def approximation_error(Tfun, spec, N: int, X, nsamples: int = 8):
    """The order test of Section 4, Example 3: the largest relative error
    ||T~(zeta) X - T(zeta) X||_F / ||T(zeta) X||_F over the sample points zeta of the inner
    contour, T~ the N-node Cauchy approximation sum_j w_j T(z_j) / (z_j - zeta) and X a
    block of test vectors; Tfun(z) returns the matrix T(z)."""
    z, w = from_spec(spec, N)
    TX = [Tfun(zj) @ X for zj in z]
    err = 0.0
    for zeta in inner_points(spec, nsamples):
        approx = sum(w[j] / (z[j] - zeta) * TX[j] for j in range(N))
        exact = Tfun(zeta) @ X
        err = max(err, np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    return err


def select_order(Tfun, spec, N_list, X, tol, nsamples: int = 8):
    """The smallest N of N_list whose approximation error is <= tol (None if none), and the
    errors of every N."""
    errs = [approximation_error(Tfun, spec, N, X, nsamples) for N in N_list]
    chosen = next((N for N, e in zip(N_list, errs) if e <= tol), None)
    return chosen, errs
