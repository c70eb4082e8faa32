"""Pins of the oracle's contour quadrature (Eq. Tz, Eq. TzApp) against exact identities of
the trapezoid rule."""
import numpy as np
import pytest

from oracle import contour


@pytest.mark.parametrize("N", [8, 16, 32])
@pytest.mark.parametrize("deg", [0, 3, "N-1"])
def test_circle_reproduces_polynomials(N, deg):
    """On a circle with theta_j = 2 pi (j + 1/2) / N, for a polynomial T of degree < N:
    sum_j w_j T(z_j) / (z_j - z) = T(z) / (1 + ((z - c) / rho)^N) exactly."""
    d = N - 1 if deg == "N-1" else deg
    c, rho = 4.0 + 0.5j, 1.3
    z, w = contour.nodes_weights("circle", c, rho, rho, N)
    rng = np.random.default_rng(N + d)
    coef = rng.normal(size=d + 1) + 1j * rng.normal(size=d + 1)
    T = lambda t: np.polyval(coef, t - c)
    scale = np.sum(np.abs(coef) * rho ** np.arange(d, -1, -1))   # size of the largest terms
    for zz in (c, c + 0.3 - 0.2j, c + 0.9 * rho * np.exp(0.7j)):
        approx = np.sum(w * T(z) / (z - zz))
        exact = T(zz) / (1.0 + ((zz - c) / rho) ** N)
        assert abs(approx - exact) <= 1e-14 * N * scale


@pytest.mark.parametrize("N", [8, 32])
def test_ellipse_integrates_polynomials_to_zero(N):
    """(1 / 2 pi i) \\oint p(t) dt = 0; the trapezoid rule is exact for deg p <= N - 2."""
    z, w = contour.nodes_weights("ellipse", 6.5, 1.5, 0.4, N)
    for d in range(N - 1):
        p = (z - 6.5) ** d
        assert abs(np.sum(w * p)) < 1e-13 * max(1.0, np.max(np.abs(p)))
    # degree N - 1 is not exact on a non-circular ellipse
    assert abs(np.sum(w * (z - 6.5) ** (N - 1))) > 1e-8 * (1.5 ** (N - 1))


def test_ellipse_cauchy_kernel_converges():
    """sum_j w_j / (z_j - z0) -> 1 for z0 inside (exponentially in N)."""
    errs = []
    for N in (16, 32, 64):
        z, w = contour.nodes_weights("ellipse", 0.0, 1.5, 1.0, N)
        errs.append(abs(np.sum(w / (z - 0.1j)) - 1.0))
    assert errs[2] < 1e-12 and errs[1] < errs[0]


def test_equal_axes_ellipse_is_circle():
    z1, w1 = contour.nodes_weights("ellipse", 2.0 - 1j, 0.8, 0.8, 24)
    z2, w2 = contour.nodes_weights("circle", 2.0 - 1j, 0.8, 0.8, 24)
    assert np.allclose(z1, z2, atol=0, rtol=0) and np.allclose(w1, w2, atol=0, rtol=0)
    assert np.allclose(w2, (z2 - (2.0 - 1j)) / 24, rtol=1e-15, atol=1e-17)
    # nodes stay off the real axis through the centre for even N (half-step offset)
    assert np.min(np.abs(z2.imag + 1.0)) > 0.0


def test_order_selection_closed_form_for_polynomials():
    """The order test of Section 4, Example 3 on a matrix polynomial of degree 2 < N: the
    trapezoid Cauchy sum reproduces T(zeta) / (1 + u^N), u = (zeta - c) / rho, so the
    relative error at every inner point is exactly |u^N / (1 + u^N)| with |u| = 1/2
    (independent of the test vectors), and the selected order is the first N whose
    closed-form error meets the tolerance."""
    import synth
    from oracle import contour as con
    rng = np.random.default_rng(2)
    A0, A1, A2 = (rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5)) for _ in range(3))

    def T(z):
        return A0 + z * A1 + z * z * A2

    spec = synth.ContourSpec("circle", 2.0 + 1.0j, 1.5, 1.5)
    X = rng.normal(size=(5, 3)) + 1j * rng.normal(size=(5, 3))
    N_list = [4, 8, 12, 16, 24]
    chosen, errs = con.select_order(T, spec, N_list, X, 2e-5, nsamples=8)
    for N, e in zip(N_list, errs):
        u = (con.inner_points(spec, 8) - spec.centre) / spec.a
        closed = np.max(np.abs(u ** N / (1 + u ** N)))
        assert abs(e - closed) <= 1e-12 + 1e-9 * closed, (N, e, closed)
    assert chosen == 16   # 2^-16 / (1 - 2^-16) < 2e-5 < 2^-12 / (1 + 2^-12)
