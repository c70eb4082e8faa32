"""Oracle of the Chebyshev variant (Section 2, Eq. Chebyshev; Section 3, Eq. sc1_chebyshev_red;
Algorithm 2's setting): interpolation of T on a real interval and the linearisation of the
interpolant. Plain numpy / scipy, test infrastructure only.

Interval [c - a, c + a] (shifted by i c_im if given). Nodes: the Chebyshev points of the
first kind x_k = c + a cos(pi (k + 1/2) / N), k = 0..N-1. Interpolant of degree m = N - 1:
T~(z) = sum_i B_i T_i(zeta), zeta = (z - c) / a, with
B_i = (2 - delta_i0) / N sum_k T(x_k) cos(i pi (k + 1/2) / N).
Linearisation (colleague form) of sum_i B_i T_i(zeta) y = 0 with v_i = T_i(zeta) y,
w = [v_0; ...; v_{m-1}]: A w = zeta M w,
A = [[0, I], [I, 0, I], ..., [-B_0, ..., -B_{m-3}, B_m - B_{m-2}, -B_{m-1}]],
M = diag(I, 2I, ..., 2I, 2 B_m) (the paper's Eq. sc1_chebyshev_red; its Eq. sc1_chebyshev
for the full matrices).
"""
import numpy as np
import scipy.linalg as sla


def nodes(c, a, N, c_im=0.0):
    k = np.arange(N)
    return c + a * np.cos(np.pi * (k + 0.5) / N) + 1j * c_im


def coefficients(samples):
    """B_i from the samples T(x_k) (array (N, ...))."""
    samples = np.asarray(samples)
    N = samples.shape[0]
    k = np.arange(N)
    out = []
    for i in range(N):
        cik = np.cos(i * np.pi * (k + 0.5) / N) * (1.0 if i == 0 else 2.0) / N
        out.append(np.tensordot(cik, samples, axes=(0, 0)))
    return np.stack(out)


def evaluate(B, zeta):
    """sum_i B_i T_i(zeta) by the three-term recurrence."""
    t_prev, t = 1.0, zeta
    acc = B[0] * t_prev
    if len(B) > 1:
        acc = acc + B[1] * t
    for i in range(2, len(B)):
        t_prev, t = t, 2 * zeta * t - t_prev
        acc = acc + B[i] * t
    return acc


def pencil(B):
    """(A, M) of the colleague linearisation for coefficients B_0..B_m (m >= 2)."""
    B = np.asarray(B)
    m = B.shape[0] - 1
    nu = B.shape[1]
    I = np.eye(nu)
    A = np.zeros((m * nu, m * nu), dtype=complex)
    M = np.zeros((m * nu, m * nu), dtype=complex)

    def blk(r, c):
        return slice(r * nu, (r + 1) * nu), slice(c * nu, (c + 1) * nu)

    A[blk(0, 1)] = I
    M[blk(0, 0)] = I
    for r in range(1, m - 1):
        A[blk(r, r - 1)] = I
        A[blk(r, r + 1)] = I
        M[blk(r, r)] = 2 * I
    for i in range(m - 2):
        A[blk(m - 1, i)] = -B[i]
    A[blk(m - 1, m - 2)] += B[m] - B[m - 2]
    A[blk(m - 1, m - 1)] = -B[m - 1]
    M[blk(m - 1, m - 1)] = 2 * B[m]
    return A, M


def eigs(B, c, a):
    """Eigenvalues z = c + a zeta of the linearisation and the y-parts of its eigenvectors."""
    A, M = pencil(B)
    zeta, W = sla.eig(A, M)
    ok = np.isfinite(zeta)
    nu = np.asarray(B).shape[1]
    return c + a * zeta[ok], W[:nu, ok]


def shift_invert_apply(B, sigma, Wblk):
    """(A - sigma M)^{-1} M W, the plain definition (dense solve)."""
    A, M = pencil(B)
    return np.linalg.solve(A - sigma * M, M @ Wblk)


def cheb_at_zero(m):
    """T_i(0), i = 0..m-1: 1, 0, -1, 0, 1, ..."""
    return np.array([np.cos(i * np.pi / 2) for i in range(m)]).round()


def inverse_power_step(B, W):
    """One step of Algorithm 2 (inverse power for the Chebyshev interpolant, the shift at the
    interval's centre, zeta = 0): w' = A^{-1} M w for the colleague pencil of ``pencil``,
    w = [v_0; ..; v_{m-1}] (blocks of n rows, any number of columns).

    Steps in the paper's order: y = M w (block diagonal: y_0 = v_0, y_r = 2 v_r,
    y_{m-1} = 2 B_m v_{m-1}); the block rows 0..m-2 of A w' = y give the recurrence
    v'_1 = y_0, v'_{r+1} = y_r - v'_{r-1} (Eq. reccurenceCheb_odd / _even), so that every
    v'_i = E_i + T_i(0) u with u = v'_0 and E from the recurrence started at E_0 = 0; the
    last block row then leaves G u = b with G = sum_i T_i(0) L_i and b = y_{m-1} - sum_i
    L_i E_i, L_i the blocks of that row (Eq. Gmtx, Eq. bodd / beven: here derived from the
    block row, whatever the parity of m). Returns w'."""
    B = np.asarray(B)
    m = B.shape[0] - 1
    n = B.shape[1]
    W = np.asarray(W).reshape(m, n, -1)
    y = [W[0]] + [2 * W[r] for r in range(1, m - 1)] + [2 * B[m] @ W[m - 1]]
    E = [np.zeros_like(W[0]), y[0]]
    for r in range(1, m - 1):
        E.append(y[r] - E[r - 1])
    L = [-B[i] for i in range(m - 2)] + [B[m] - B[m - 2], -B[m - 1]]
    s = cheb_at_zero(m)
    G = sum(s[i] * L[i] for i in range(m))
    b = y[m - 1] - sum(L[i] @ E[i] for i in range(m))
    u = np.linalg.solve(G, b)
    return np.concatenate([E[i] + s[i] * u for i in range(m)], axis=0)


def inverse_power(B, V0, q):
    """q steps of Algorithm 2 from the blocks v_i = T_i(0) V0 (the eigenvector form at the
    shift), each step's columns rescaled to unit norm (direction only); returns the u-parts
    (the y-part of the linearisation, v_0) after q steps."""
    B = np.asarray(B)
    m = B.shape[0] - 1
    s = cheb_at_zero(m)
    V0 = np.asarray(V0, dtype=np.complex128)
    W = np.concatenate([s[i] * V0 for i in range(m)], axis=0)
    for _ in range(q):
        W = inverse_power_step(B, W)
        W = W / np.linalg.norm(W, axis=0)
    return W[:V0.shape[0]]
