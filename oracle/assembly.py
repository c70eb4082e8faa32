"""Oracle wrappers for the BEM matrix A(k) (Section 1, Eq. GreenFun; the single-layer part of
Eq. HelmBIM with constant elements collocated at centroids) and its operator variant
T = c_G G + c_H (1/2 I + K) (the double layer K with its jump; Eq. HelmBIM's general form).
``op`` = (c_G, c_H), default (1, 0). See ``bem_oracle.c``."""
import ctypes
import numpy as np

from ._lib import lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mesh_arrays(mesh):
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
    return xyz, tri


def rule7():
    b = np.zeros((7, 3))
    w = np.zeros(7)
    lib().oracle_rule7(_p(b), _p(w))
    return b, w


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _p(x), _p(w))
    return x, w


def geometry(mesh):
    xyz, tri = _mesh_arrays(mesh)
    n = tri.shape[0]
    c = np.zeros((n, 3)); a = np.zeros(n); qp = np.zeros((n, 7, 3)); qw = np.zeros((n, 7))
    lib().oracle_geometry(_p(xyz), n, _p(tri), _p(c), _p(a), _p(qp), _p(qw))
    return c, a, qp, qw


def self_integral(v0, v1, v2, x, k, deriv=0):
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (v0, v1, v2, x)]
    out = np.zeros(2)
    k = complex(k)
    lib().oracle_self_integral(*[_p(a) for a in arrs], k.real, k.imag, int(deriv), _p(out))
    return complex(out[0], out[1])


def _op4(op):
    cg, ch = (1.0, 0.0) if op is None else op
    cg, ch = complex(cg), complex(ch)
    return np.array([cg.real, cg.imag, ch.real, ch.imag])


def matrix(mesh, k, deriv=0, rows=None, threads=0, near=False, op=None):
    """Dense A(k) (deriv=0) or dA/dk (deriv=1) as an (r1-r0) x n complex128 array; near=True
    uses the 64-point conical rule on near pairs (see ``bem_oracle.c``)."""
    xyz, tri = _mesh_arrays(mesh)
    n = tri.shape[0]
    r0, r1 = (0, n) if rows is None else rows
    A = np.zeros((r1 - r0, n), dtype=np.complex128)
    k = complex(k)
    o = _op4(op)
    lib().oracle_matrix_op(_p(xyz), n, _p(tri), k.real, k.imag, int(deriv), r0, r1, _p(A),
                           int(threads), int(bool(near)), _p(o))
    return A


def apply(mesh, z, V, rows=None, threads=0, near=False, op=None):
    """Y[j] = (A(z_j) V)[rows] for all nodes; returns (N, r1-r0, nu) complex128."""
    xyz, tri = _mesh_arrays(mesh)
    n = tri.shape[0]
    V = np.asfortranarray(V, dtype=np.complex128)
    assert V.shape[0] == n
    nu = V.shape[1]
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    N = z.shape[0]
    r0, r1 = (0, n) if rows is None else rows
    Y = np.zeros(N * (r1 - r0) * nu, dtype=np.complex128)
    o = _op4(op)
    lib().oracle_apply_op(_p(xyz), n, _p(tri), N, _p(z), nu, _p(V), r0, r1, _p(Y), int(threads),
                          int(bool(near)), _p(o))
    # block j is column-major (rows x nu)
    return np.stack([Y[j * (r1 - r0) * nu:(j + 1) * (r1 - r0) * nu].reshape(nu, r1 - r0).T
                     for j in range(N)])


def near_rule(v0, v1, v2, x, k, deriv=0, order=8, kind=0):
    """The conical-product rule of the given order (order x order points) for the integral of
    g(k, |x - y|) (kind 0) or dg/dn_y (kind 1, normal of the triangle in its vertex order)
    over the triangle (v0, v1, v2), collapsed at the vertex nearest x."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (v0, v1, v2, x)]
    out = np.zeros(2)
    k = complex(k)
    lib().oracle_near_rule_kind(*[_p(a) for a in arrs], k.real, k.imag, int(deriv), int(order),
                                int(kind), _p(out))
    return complex(out[0], out[1])


def near_pairs(mesh, rows=None):
    """CSR of the near pairs: (row_ptr, cols), cols increasing within each row."""
    xyz, tri = _mesh_arrays(mesh)
    n = tri.shape[0]
    r0, r1 = (0, n) if rows is None else rows
    counts = np.zeros(r1 - r0, dtype=np.int64)
    lib().oracle_near_pairs(_p(xyz), n, _p(tri), r0, r1, _p(counts), None, None)
    row_ptr = np.zeros(r1 - r0 + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    cols = np.zeros(int(row_ptr[-1]), dtype=np.int64)
    lib().oracle_near_pairs(_p(xyz), n, _p(tri), r0, r1, _p(counts), _p(row_ptr), _p(cols))
    return row_ptr, cols


def entries(mesh, k, rows, cols, near=False, op=None):
    """T_il(k) for the pairs (rows[t], cols[t]) (complex128 array)."""
    xyz, tri = _mesh_arrays(mesh)
    n = tri.shape[0]
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    assert r.shape == c.shape
    out = np.zeros(r.size, dtype=np.complex128)
    k = complex(k)
    o = _op4(op)
    lib().oracle_entries(_p(xyz), n, _p(tri), k.real, k.imag, _p(r), _p(c), r.size, _p(out),
                         int(bool(near)), _p(o))
    return out
