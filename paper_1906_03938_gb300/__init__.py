"""Python binding of the GB300 BEM eigen-solver hot path (C ABI in include/bem_gb300.h).

Argument marshalling only: every step runs in the CUDA library ``_build/libbem_gb300.so``.
The raw entry points keep their C names (``bem_create``, ``bem_set_mesh``, ...); the
``Context`` class wraps them for torch tensors (device memory, streams) and numpy arrays
(host inputs). Importing this package does not touch the GPU; loading the library fails
loudly if it has not been built: there is no CPU fallback.

Layouts: complex arrays are complex128 (interleaved re, im). An n x nu basis is a device
tensor whose memory is column-major, i.e. ``V.stride() == (1, ld)`` with ``ld >= n``
(``fortran(V)`` makes one). Projected matrices come back as a (N, nu, nu) tensor whose
[j] slice is the matrix Bhat_j itself.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbem_gb300.so")

BEM_OK = 0
STATUS = {0: "BEM_OK", -1: "BEM_EINVAL", -2: "BEM_ENOMEM", -3: "BEM_ECUDA", -4: "BEM_EKERNEL",
          -5: "BEM_ETIMEOUT", -6: "BEM_ENOCONV", -7: "BEM_ESTATE"}
STATUS_CODES = {v: k for k, v in STATUS.items()}
PREC_FP64 = 0
PREC_MIXED = 1
PREC_HMATRIX = 2
CONTOUR_CIRCLE = 0
CONTOUR_ELLIPSE = 1
CONTOUR_CHEBYSHEV = 2

# name -> (restype, argtypes) of every symbol declared in include/bem_gb300.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "bem_create": (_I, [ctypes.POINTER(_P), _I]),
    "bem_destroy": (None, [_P]),
    "bem_last_error": (ctypes.c_char_p, [_P]),
    "bem_version": (ctypes.c_char_p, []),
    "bem_set_mesh": (_I, [_P, _I64, _P, _I64, _P, _P]),
    "bem_set_contour": (_I, [_P, _I, _D, _D, _D, _D, _I, _P, _P, _P]),
    "bem_project": (_I, [_P, _P, _I64, _I, _P, _P, _I, _P]),
    "bem_node_order": (_I, [_P, _P, _P]),
    "bem_set_async": (_I, [_P, _I]),
    "bem_set_wait_limit": (_I, [_P, ctypes.c_uint32]),
    "bem_set_eval_split": (_I, [_P, _I]),
    "bem_set_refine_residual": (_I, [_P, _I]),
    "bem_set_twin_clusters": (_I, [_P, _I]),
    "bem_mixed_shape": (_I, [_P, _P, _P, _P, _P]),
    "bem_set_operator": (_I, [_P, _D, _D, _D, _D]),
    "bem_set_hmatrix": (_I, [_P, _I, _D, _D, _I]),
    "bem_hmatrix_stats": (_I, [_P, _P, _P, _P, _P, _P]),
    "bem_hmatrix_work": (_I, [_P, _P, _P, _P]),
    "bem_apply_sum": (_I, [_P, _P, _P, _I64, _I, _I, _P, _P]),
    "bem_solve_sum": (_I, [_P, _P, _P, _I64, _I, _D, _I, _P, _I64, ctypes.POINTER(_I), _P, _P]),
    "bem_inverse_power_mf": (_I, [_P, _P, _I64, _I, _I, _D, _D, _D, _I, ctypes.POINTER(_I), _P]),
    "bem_cholqr2": (_I, [_P, _P, _I64, _I64, _I, _P, _P]),
    "bem_residual": (_I, [_P, _I, _P, _P, _I64, _P, _P, _P]),
    "bem_residual_arith": (_I, [_P, _I, _P, _P, _I64, _P, _P, _P, _I, _P]),
    "bem_kernel_launches": (_I64, [_P]),
    "bem_check": (_I, [_P, _P]),
    "bem_solve_reduced": (_I, [_P, _P, _I, _D, _D, _I, _I, _D, _P, _P, _P,
                               ctypes.POINTER(_I), _P]),
    "bem_ritz_vectors": (_I, [_P, _P, _I64, _I, _P, _I, _P, _I64, _P]),
    "bem_inverse_power": (_I, [_P, _P, _I64, _I, _I, _D, _D, _P]),
    "bem_inverse_power_chebyshev": (_I, [_P, _P, _I64, _I, _I, _P]),
    "bem_select_order": (_I, [_P, _I, _D, _D, _D, _D, _P, _I, _I, _P, _I64, _I, _D, _P, _P, _P]),
    "bem_refine": (_I, [_P, _I, _P, _P, _I64, _D, _I, _P, _P, _P]),
    "bem_solve": (_I, [_P, _P, _I64, _I, _I, _I, _D, _I, _P, _P, _I64, ctypes.POINTER(_I),
                       _P, _P]),
    "bem_set_timing": (_I, [_P, _I]),
    "bem_kernel_times": (_I, [_P, _P, _I, ctypes.POINTER(_I)]),
    "bem_microbench": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "bem_project_fp64_noalloc": (_I, [_I, _I64, _P, _I64, _P, _I, _D, _D, _D, _D, _I, _P,
                                      _I64, _I, _P, _P]),
    "bem_noalloc_last_error": (ctypes.c_char_p, []),
    "bem_chebyshev_coeffs": (_I, [_P, _P, _I, _P, _P]),
    "bem_solve_chebyshev": (_I, [_P, _P, _I, _D, _D, _I, _I, _D, _P, _P, _P, ctypes.POINTER(_I),
                                 _P]),
    "bem_chebyshev_apply": (_I, [_P, _P, _I, _D, _D, _P, _I, _P, _P]),
    "bem_set_near_field": (_I, [_P, _I, _P]),
    "bem_near_pairs": (_I, [_P, ctypes.POINTER(_I64), _P, _P, _P]),
    "bem_surrogate_size": (_I, []),
    "bem_surrogate_init": (_I, [_P, ctypes.c_uint64, _P]),
    "bem_surrogate_set": (_I, [_P, _P, _I64, _P]),
    "bem_surrogate_get": (_I, [_P, _I, _P, _I64, _P]),
    "bem_surrogate_usage": (_I, [_P, _P, _P, _P]),
    "bem_surrogate_samples": (_I, [_P, _D, _D, _D, _D, _I64, ctypes.c_uint64, _P, _P, _P, _P,
                                   _P]),
    "bem_surrogate_forward": (_I, [_P, _P, _I64, _P, _P]),
    "bem_surrogate_grad": (_I, [_P, _P, _P, _I64, _P, ctypes.POINTER(_D), _P]),
    "bem_surrogate_train": (_I, [_P, _P, _P, _I64, _I, _I, _D, _I, ctypes.c_uint64, _P, _P]),
    "bem_batch_create": (_I, [_P, _I, _P, _P, _P, _P, _I, _I, ctypes.POINTER(_P), _P]),
    "bem_batch_run": (_I, [_P, _P]),
    "bem_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64),
                            ctypes.POINTER(_D)]),
    "bem_batch_destroy": (None, [_P]),
    "bem_project_batched": (_I, [_P, _I, _P, _P, _P, _P, _I, _P]),
}

class Stats(ctypes.Structure):
    """bem_stats_t"""
    _fields_ = [("device", ctypes.c_int), ("n", ctypes.c_int64), ("nv", ctypes.c_int64),
                ("N", ctypes.c_int), ("near_mode", ctypes.c_int), ("near_pairs", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("surrogate_ready", ctypes.c_int)]


SIGNATURES.update({
    "bem_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "bem_save_state": (_I, [_P, _P, ctypes.POINTER(ctypes.c_size_t), _P]),
    "bem_load_state": (_I, [_P, _P, ctypes.c_size_t, _P]),
})

_lib = None


class BemError(RuntimeError):
    def __init__(self, name, status, msg):
        super().__init__(f"{name} failed with {STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: build it with ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):
    # raw C entry points under their own names: paper_1906_03938_gb300.bem_project(...)
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(_P)
    return _P(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return _P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def fortran(t):
    """Column-major copy of a 2-D tensor (stride (1, rows))."""
    return t.transpose(0, 1).contiguous().transpose(0, 1)


def _check_fortran(V, name):
    if V.dim() != 2 or V.stride(0) != 1 or V.stride(1) < V.shape[0]:
        raise ValueError(f"{name} must be a column-major 2-D tensor (use fortran())")


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = _P()
        st = self._lib.bem_create(ctypes.byref(h), int(device))
        if st != BEM_OK:
            raise BemError("bem_create", st, "no usable CUDA device")
        self._h = h
        self.device = device
        self.n = 0
        self.N = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, name, st):
        if st != BEM_OK:
            raise BemError(name, st, self._lib.bem_last_error(self._h).decode())

    def check(self, stream=None):
        """Synchronise and raise if a kernel recorded a device-side failure."""
        self._chk("bem_check", self._lib.bem_check(self._h, _stream(stream)))

    @property
    def launches(self) -> int:
        return int(self._lib.bem_kernel_launches(self._h))

    def set_timing(self, enable=True):
        self._chk("bem_set_timing", self._lib.bem_set_timing(self._h, int(bool(enable))))

    def kernel_times(self, max_out=256):
        ms = np.zeros(max_out)
        cnt = _I(0)
        self._chk("bem_kernel_times", self._lib.bem_kernel_times(self._h, _ptr(ms), max_out,
                                                                  ctypes.byref(cnt)))
        return ms[:cnt.value]

    def microbench(self, kind):
        """Measured device throughput in ops/s: 'fp64_fma', 'fp32_fma', 'fp32x2_fma'
        (flops), 'ex2', 'sin', 'cos', 'rsqrt' (MUFU operations), 'sincos_poly' (phases
        whose sine and cosine the FMA-pipe polynomials give)."""
        kinds = {"fp64_fma": 0, "fp32_fma": 1, "ex2": 2, "sin": 3, "cos": 4, "rsqrt": 5,
                 "fp32x2_fma": 6, "sincos_poly": 7}
        r = _D(0.0)
        self._chk("bem_microbench", self._lib.bem_microbench(self._h, kinds[kind], ctypes.byref(r)))
        return r.value

    def set_near_field(self, mode, stream=None):
        """0: 7-point rule everywhere; 1: 8 x 8 conical rule on near pairs; 2: surrogate
        network for the near pairs in the mixed projection."""
        self._chk("bem_set_near_field", self._lib.bem_set_near_field(self._h, int(mode),
                                                                     _stream(stream)))

    def near_pairs(self, stream=None):
        """(row_ptr, cols) of the current mesh's near pairs (numpy int32)."""
        nnz = _I64()
        self._chk("bem_near_pairs", self._lib.bem_near_pairs(self._h, ctypes.byref(nnz), None,
                                                             None, _stream(stream)))
        row_ptr = np.zeros(self.n + 1, dtype=np.int32)
        cols = np.zeros(max(1, nnz.value), dtype=np.int32)
        self._chk("bem_near_pairs", self._lib.bem_near_pairs(self._h, ctypes.byref(nnz),
                                                             _ptr(row_ptr), _ptr(cols),
                                                             _stream(stream)))
        return row_ptr, cols[:nnz.value]

    # ---- surrogate network of the near-field correction ----
    def surrogate_init(self, seed=1, stream=None):
        self._chk("bem_surrogate_init", self._lib.bem_surrogate_init(self._h, int(seed),
                                                                     _stream(stream)))

    def surrogate_params(self, which=0):
        out = np.zeros(self._lib.bem_surrogate_size(), dtype=np.float32)
        self._chk("bem_surrogate_get", self._lib.bem_surrogate_get(self._h, int(which), _ptr(out),
                                                                   out.size, None))
        return out

    def surrogate_set(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._chk("bem_surrogate_set", self._lib.bem_surrogate_set(self._h, _ptr(p), p.size, None))

    def surrogate_usage(self, stream=None):
        """(network, rule): samples of the near-field projections since the last call whose
        correction came from the network, and from the plain 8 x 8 rule (features outside
        the training box); resets the counters."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._chk("bem_surrogate_usage", self._lib.bem_surrogate_usage(
            self._h, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
        return a.value, b.value

    def surrogate_samples(self, count, k_re, k_im, seed=1, with_pairs=False, stream=None):
        """(features (count, 11), targets (count, 2)[, pairs (count, 2), k (count,)])."""
        import torch
        dev = torch.device("cuda", self.device)
        feat = torch.empty((count, 11), dtype=torch.float32, device=dev)
        targ = torch.empty((count, 2), dtype=torch.float32, device=dev)
        pairs = torch.empty((count, 2), dtype=torch.int32, device=dev) if with_pairs else None
        ks = torch.empty((count,), dtype=torch.complex128, device=dev) if with_pairs else None
        self._chk("bem_surrogate_samples", self._lib.bem_surrogate_samples(
            self._h, float(k_re[0]), float(k_re[1]), float(k_im[0]), float(k_im[1]), int(count),
            int(seed), _ptr(feat), _ptr(targ), _ptr(pairs), _ptr(ks), _stream(stream)))
        return (feat, targ, pairs, ks) if with_pairs else (feat, targ)

    def surrogate_forward(self, feat, stream=None):
        import torch
        out = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        self._chk("bem_surrogate_forward", self._lib.bem_surrogate_forward(
            self._h, _ptr(feat), feat.shape[0], _ptr(out), _stream(stream)))
        return out

    def surrogate_grad(self, feat, targ, stream=None):
        import torch
        g = torch.empty(self._lib.bem_surrogate_size(), dtype=torch.float32, device=feat.device)
        loss = _D()
        self._chk("bem_surrogate_grad", self._lib.bem_surrogate_grad(
            self._h, _ptr(feat), _ptr(targ), feat.shape[0], _ptr(g), ctypes.byref(loss),
            _stream(stream)))
        return loss.value, g

    def surrogate_train(self, feat, targ, epochs, batch=4096, lr=1e-3, fit_scaling=True, seed=1,
                        stream=None):
        losses = np.zeros(int(epochs))
        self._chk("bem_surrogate_train", self._lib.bem_surrogate_train(
            self._h, _ptr(feat), _ptr(targ), feat.shape[0], int(epochs), int(batch), float(lr),
            int(bool(fit_scaling)), int(seed), _ptr(losses), _stream(stream)))
        return losses

    def stats(self):
        st = Stats()
        self._chk("bem_stats", self._lib.bem_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in Stats._fields_}

    def save_state(self):
        """Checkpoint (bytes) of the mesh, contour, near-field mode and network."""
        n = ctypes.c_size_t(0)
        self._chk("bem_save_state", self._lib.bem_save_state(self._h, None, ctypes.byref(n), None))
        buf = ctypes.create_string_buffer(n.value)
        self._chk("bem_save_state", self._lib.bem_save_state(self._h, buf, ctypes.byref(n), None))
        return buf.raw[:n.value]

    def load_state(self, data):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._chk("bem_load_state", self._lib.bem_load_state(self._h, buf, len(data), None))
        st = self.stats()
        self.n, self.N = int(st["n"]), int(st["N"])

    def set_mesh(self, xyz, tri, stream=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        self._chk("bem_set_mesh", self._lib.bem_set_mesh(self._h, xyz.shape[0], _ptr(xyz),
                                                          tri.shape[0], _ptr(tri),
                                                          _stream(stream)))
        self.n = int(tri.shape[0])

    def set_contour(self, kind, centre, a, b, N, stream=None):
        kinds = {"circle": CONTOUR_CIRCLE, "ellipse": CONTOUR_ELLIPSE,
                 "chebyshev": CONTOUR_CHEBYSHEV}
        k = kinds[kind] if isinstance(kind, str) else int(kind)
        z = np.zeros(2 * N)
        w = np.zeros(2 * N)
        c = complex(centre)
        self._chk("bem_set_contour", self._lib.bem_set_contour(
            self._h, k, c.real, c.imag, float(a), float(b), int(N), _ptr(z), _ptr(w),
            _stream(stream)))
        self.N = int(N)
        return z.view(np.complex128), w.view(np.complex128)

    def apply_sum(self, coef, X, per_node=True, stream=None):
        """Y = sum_j c_j A(z_j) X_j (per_node: X of shape (N, n, nu), each block column-major)
        or (sum_j c_j A(z_j)) X (X n x nu column-major); Y n x nu complex128 column-major."""
        import torch
        c = np.ascontiguousarray(np.asarray(coef, dtype=np.complex128)).view(np.float64)
        if c.size != 2 * self.N:
            raise ValueError("apply_sum: one coefficient per node")
        if per_node:
            if X.dim() != 3 or X.shape[0] != self.N or X.stride(1) != 1:
                raise ValueError("apply_sum: X must be (N, n, nu) with column-major blocks")
            n, nu = X.shape[1], X.shape[2]
            ldx = X.stride(2)
            if X.stride(0) != ldx * nu:
                raise ValueError("apply_sum: node blocks must be ldx * nu apart")
        else:
            _check_fortran(X, "X")
            n, nu = X.shape
            ldx = X.stride(1)
        Y = torch.empty((nu, n), dtype=torch.complex128, device=X.device).t()
        self._chk("bem_apply_sum", self._lib.bem_apply_sum(
            self._h, c.ctypes.data_as(_P), _P(X.data_ptr()), int(ldx), int(nu),
            1 if per_node else 0, _P(Y.data_ptr()), _stream(stream)))
        return Y

    def set_operator(self, c_g=1.0, c_h=0.0):
        """T = c_G G + c_H (I/2 + K): (1, 0) single layer, (0, 1) Neumann, else Robin."""
        cg, ch = complex(c_g), complex(c_h)
        self._chk("bem_set_operator", self._lib.bem_set_operator(
            self._h, cg.real, cg.imag, ch.real, ch.imag))

    def set_hmatrix(self, leaf=32, eta=1.0, eps=1e-6, rmax=48):
        """Low-rank far field for projections with precision PREC_HMATRIX."""
        self._chk("bem_set_hmatrix", self._lib.bem_set_hmatrix(
            self._h, int(leaf), float(eta), float(eps), int(rmax)))

    def hmatrix_stats(self):
        fb, db = _I64(0), _I64(0)
        ff, mr = ctypes.c_double(0), ctypes.c_double(0)
        xr = _I(0)
        self._chk("bem_hmatrix_stats", self._lib.bem_hmatrix_stats(
            self._h, ctypes.byref(fb), ctypes.byref(db), ctypes.byref(ff), ctypes.byref(mr),
            ctypes.byref(xr)))
        return {"far_blocks": fb.value, "dense_blocks": db.value, "far_fraction": ff.value,
                "mean_rank": mr.value, "max_rank": xr.value}

    def hmatrix_work(self):
        """Algorithmic work of one node of the last far-field projection (node average):
        dense entries, far rank x rows, far rank x columns."""
        d, r, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        self._chk("bem_hmatrix_work", self._lib.bem_hmatrix_work(
            self._h, ctypes.byref(d), ctypes.byref(r), ctypes.byref(c)))
        return {"dense_entries": d.value, "far_row_terms": r.value, "far_col_terms": c.value}

    def set_async(self, on=True):
        """Asynchronous mode: cholqr2 leaves its status check to check()."""
        self._chk("bem_set_async", self._lib.bem_set_async(self._h, 1 if on else 0))

    def set_wait_limit(self, polls):
        """Polls of each pipeline-stage wait of the fused kernel before it gives up with
        BEM_ETIMEOUT (0: at once); the default is 1 << 24."""
        self._chk("bem_set_wait_limit", self._lib.bem_set_wait_limit(self._h, int(polls)))

    def set_eval_split(self, poly_points=-1):
        """Quadrature points (0..4 of 7) per entry whose sine and cosine the fused kernel
        takes from the FMA-pipe polynomials; -1: the measured default."""
        self._chk("bem_set_eval_split", self._lib.bem_set_eval_split(self._h, int(poly_points)))

    def set_refine_residual(self, arith=0):
        """Arithmetic of the residuals refine/solve report: 0 FP64, 1 double-FP32."""
        self._chk("bem_set_refine_residual", self._lib.bem_set_refine_residual(self._h, int(arith)))

    def set_twin_clusters(self, on=True):
        """Twin pairs on two-CTA clusters when a unit of the fused kernel holds one node
        (bases of more than 128 columns); on by default."""
        self._chk("bem_set_twin_clusters", self._lib.bem_set_twin_clusters(self._h, 1 if on else 0))

    def mixed_shape(self):
        """Work decomposition of the last mixed projection: nodes per unit, whether twin
        pairs ran on clusters, column splits, CTAs launched."""
        g, pr, sp = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        u = ctypes.c_int64(0)
        self._chk("bem_mixed_shape", self._lib.bem_mixed_shape(
            self._h, ctypes.byref(g), ctypes.byref(pr), ctypes.byref(sp), ctypes.byref(u)))
        return {"nodes_per_unit": g.value, "paired": bool(pr.value), "splits": sp.value,
                "ctas": u.value}

    def node_order(self):
        """(order, twins): the mixed kernel's node schedule (slot -> node) and the number
        of twin pairs (nodes with equal FP32 real parts) at its front."""
        order = np.zeros(self.N, dtype=np.int32)
        tw = _I(0)
        self._chk("bem_node_order", self._lib.bem_node_order(
            self._h, order.ctypes.data_as(_P), ctypes.byref(tw)))
        return order, int(tw.value)

    def project(self, V, precision=PREC_FP64, AV=False, Bhat=None, stream=None):
        """Bhat_j = w_j V^H A(z_j) V for all nodes; optionally Y_j = A(z_j) V."""
        import torch
        _check_fortran(V, "V")
        n, nu = V.shape
        if Bhat is None:
            Bhat = torch.empty((self.N, nu, nu), dtype=torch.complex128, device=V.device)
        Y = None
        if AV is True:
            Y = torch.empty((self.N, nu, n), dtype=torch.complex128, device=V.device)
        elif AV is not False and AV is not None:
            Y = AV
        self._chk("bem_project", self._lib.bem_project(
            self._h, _ptr(V), V.stride(1), nu, _ptr(Bhat), _ptr(Y), int(precision),
            _stream(stream)))
        Bm = Bhat.transpose(1, 2)
        return (Bm, Y.transpose(1, 2)) if Y is not None else Bm

    def solve_reduced(self, Bhat, shift, p=None, max_iter=200, tol=1e-12, stream=None):
        """Eigenpairs of the reduced linearised problem from Bhat (N x nu x nu matrices,
        as returned by project). Returns (lam, Y, res, iters): Ritz values, y-parts
        (nu x p tensor), reduced residuals."""
        import torch
        N, nu, _ = Bhat.shape
        if p is None:
            p = min(N * nu, 256, max(2 * nu, 32))
        Bm = Bhat.transpose(1, 2).contiguous()        # column-major per node
        lam = np.zeros(2 * p)
        res = np.zeros(p)
        Y = torch.empty((p, nu), dtype=torch.complex128, device=Bhat.device)
        it = _I(0)
        sh = complex(shift)
        self._chk("bem_solve_reduced", self._lib.bem_solve_reduced(
            self._h, _ptr(Bm), nu, sh.real, sh.imag, int(p), int(max_iter), float(tol),
            _ptr(lam), _ptr(Y), _ptr(res), ctypes.byref(it), _stream(stream)))
        return lam.view(np.complex128), Y.transpose(0, 1), res, it.value

    def chebyshev_coeffs(self, P, stream=None):
        """Chebyshev coefficients B_0..B_{N-1} of the reduced interpolant from the projections
        P (N x nu x nu, as returned by project on a Chebyshev contour)."""
        import torch
        N, nu, _ = P.shape
        Pm = P.transpose(1, 2).contiguous()
        Bm = torch.empty_like(Pm)
        self._chk("bem_chebyshev_coeffs", self._lib.bem_chebyshev_coeffs(
            self._h, _ptr(Pm), nu, _ptr(Bm), _stream(stream)))
        return Bm.transpose(1, 2)

    def chebyshev_apply(self, B, shift, W, stream=None):
        """(A - sigma M)^{-1} M W for the colleague pencil of B (W: (N-1) nu x p)."""
        import torch
        N, nu, _ = B.shape
        Bm = B.transpose(1, 2).contiguous()
        Wc = fortran(W)
        HW = fortran(torch.empty_like(Wc))
        sh = complex(shift)
        self._chk("bem_chebyshev_apply", self._lib.bem_chebyshev_apply(
            self._h, _ptr(Bm), nu, sh.real, sh.imag, _ptr(Wc), Wc.shape[1], _ptr(HW),
            _stream(stream)))
        return HW

    def solve_chebyshev(self, B, shift, p=None, max_iter=200, tol=1e-12, stream=None):
        """Eigenpairs of sum_i B_i T_i(zeta) y = 0 nearest shift: (lam, Y, res, iters)."""
        import torch
        N, nu, _ = B.shape
        if p is None:
            p = min((N - 1) * nu, 256, max(2 * nu, 32))
        Bm = B.transpose(1, 2).contiguous()
        lam = np.zeros(2 * p)
        res = np.zeros(p)
        Y = torch.empty((p, nu), dtype=torch.complex128, device=B.device)
        it = _I(0)
        sh = complex(shift)
        self._chk("bem_solve_chebyshev", self._lib.bem_solve_chebyshev(
            self._h, _ptr(Bm), nu, sh.real, sh.imag, int(p), int(max_iter), float(tol),
            _ptr(lam), _ptr(Y), _ptr(res), ctypes.byref(it), _stream(stream)))
        return lam.view(np.complex128), Y.transpose(0, 1), res, it.value

    def ritz_vectors(self, V, Y, stream=None):
        import torch
        _check_fortran(V, "V")
        n, nu = V.shape
        Yc = fortran(Y) if not (Y.stride(0) == 1 and Y.stride(1) == nu) else Y
        k = Yc.shape[1]
        X = torch.empty((k, n), dtype=torch.complex128, device=V.device)
        self._chk("bem_ritz_vectors", self._lib.bem_ritz_vectors(
            self._h, _ptr(V), V.stride(1), nu, _ptr(Yc), k, _ptr(X), n, _stream(stream)))
        return X.transpose(0, 1)

    def inverse_power(self, V, q, shift, stream=None):
        """q steps of Algorithm 1 on every column of V (in place)."""
        _check_fortran(V, "V")
        n, nu = V.shape
        sh = complex(shift)
        self._chk("bem_inverse_power", self._lib.bem_inverse_power(
            self._h, _ptr(V), V.stride(1), nu, int(q), sh.real, sh.imag, _stream(stream)))

    def select_order(self, kind, centre, a, b, N_list, X, tol, nsamples=8, stream=None):
        """(N chosen or None, errors): the first order whose Cauchy approximation meets tol
        on the inner contour (Section 4, Example 3), for test vectors X (n x ncols)."""
        _check_fortran(X, "X")
        kinds = {"circle": CONTOUR_CIRCLE, "ellipse": CONTOUR_ELLIPSE}
        Ns = np.ascontiguousarray(N_list, dtype=np.int32)
        err = np.zeros(len(Ns))
        ch = _I(0)
        c = complex(centre)
        self._chk("bem_select_order", self._lib.bem_select_order(
            self._h, kinds[kind], c.real, c.imag, float(a), float(b), _ptr(Ns), len(Ns),
            int(nsamples), _ptr(X), X.stride(1), X.shape[1], float(tol), ctypes.byref(ch),
            _ptr(err), _stream(stream)))
        return (ch.value if ch.value > 0 else None), err

    def inverse_power_chebyshev(self, V, q, stream=None):
        """q steps of Algorithm 2 (Chebyshev contour) on every column of V (in place)."""
        _check_fortran(V, "V")
        n, nu = V.shape
        self._chk("bem_inverse_power_chebyshev", self._lib.bem_inverse_power_chebyshev(
            self._h, _ptr(V), V.stride(1), nu, int(q), _stream(stream)))

    def inverse_power_mf(self, V, q, shift, tol=1e-4, max_iter=400, stream=None):
        """q steps of Algorithm 1 with matrix-free GMRES solves (in place); returns the total
        number of Arnoldi steps."""
        _check_fortran(V, "V")
        n, nu = V.shape
        sh = complex(shift)
        it = _I(0)
        self._chk("bem_inverse_power_mf", self._lib.bem_inverse_power_mf(
            self._h, _ptr(V), V.stride(1), nu, int(q), sh.real, sh.imag, float(tol),
            int(max_iter), ctypes.byref(it), _stream(stream)))
        return int(it.value)

    def solve_sum(self, coef, B, tol=1e-4, max_iter=400, stream=None):
        """X with (sum_j c_j A(z_j)) X = B by matrix-free GMRES; returns (X, iters, relres)."""
        import torch
        _check_fortran(B, "B")
        n, nu = B.shape
        c = np.ascontiguousarray(np.asarray(coef, dtype=np.complex128)).view(np.float64)
        if c.size != 2 * self.N:
            raise ValueError("solve_sum: one coefficient per node")
        X = torch.empty((nu, n), dtype=torch.complex128, device=B.device).t()
        it = _I(0)
        rel = np.zeros(nu)
        self._chk("bem_solve_sum", self._lib.bem_solve_sum(
            self._h, c.ctypes.data_as(_P), _ptr(B), B.stride(1), nu, float(tol), int(max_iter),
            _ptr(X), X.stride(1), ctypes.byref(it), rel.ctypes.data_as(_P), _stream(stream)))
        return X, int(it.value), rel

    def refine(self, lam, X, tol=1e-13, maxit=40, stream=None):
        """FP64 refinement of eigenpairs (X refined in place); returns (lam, relres, iters)."""
        _check_fortran(X, "X")
        n, m = X.shape
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).reshape(m)).copy()
        rel = np.zeros(m)
        its = np.zeros(m, dtype=np.int32)
        self._chk("bem_refine", self._lib.bem_refine(
            self._h, m, _ptr(lam.view(np.float64)), _ptr(X), X.stride(1), float(tol), int(maxit),
            _ptr(rel), _ptr(its), _stream(stream)))
        return lam, rel, its

    def solve(self, V0, q=10, precision=PREC_FP64, tol=1e-13, kmax=None, stream=None):
        """Eigenpairs inside the contour: (lam, X, relres)."""
        import torch
        _check_fortran(V0, "V0")
        n, nu = V0.shape
        kmax = kmax or min(n, 2 * nu)
        lam = np.zeros(2 * kmax)
        rel = np.zeros(kmax)
        X = torch.zeros((kmax, n), dtype=torch.complex128, device=V0.device)
        k = _I(0)
        self._chk("bem_solve", self._lib.bem_solve(
            self._h, _ptr(V0), V0.stride(1), nu, int(q), int(precision), float(tol), int(kmax),
            _ptr(lam), _ptr(X), n, ctypes.byref(k), _ptr(rel), _stream(stream)))
        kk = k.value
        return lam.view(np.complex128)[:kk], X.transpose(0, 1)[:, :kk], rel[:kk]

    def cholqr2(self, V, want_R=True, stream=None):
        import torch
        _check_fortran(V, "V")
        n, nu = V.shape
        R = torch.empty((nu, nu), dtype=torch.complex128, device=V.device) if want_R else None
        self._chk("bem_cholqr2", self._lib.bem_cholqr2(self._h, _ptr(V), n, V.stride(1), nu,
                                                        _ptr(R), _stream(stream)))
        return R.transpose(0, 1) if R is not None else None

    def residual(self, lam, X, want_R=False, stream=None):
        import torch
        _check_fortran(X, "X")
        n, m = X.shape
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).reshape(m))
        rel = np.zeros(m)
        R = torch.empty((m, n), dtype=torch.complex128, device=X.device) if want_R else None
        self._chk("bem_residual", self._lib.bem_residual(
            self._h, m, _ptr(lam.view(np.float64)), _ptr(X), X.stride(1), _ptr(R), _ptr(rel),
            _stream(stream)))
        return (rel, R.transpose(0, 1)) if want_R else rel

    def residual_arith(self, lam, X, arith=1, deriv=False, stream=None):
        """(relres, R, Rd): residuals of the columns of X at lam in FP64 (arith 0) or
        double-FP32 (arith 1), R = A(lam) x and, with deriv, Rd = A'(lam) x."""
        import torch
        _check_fortran(X, "X")
        n, m = X.shape
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).reshape(m))
        rel = np.zeros(m)
        R = torch.empty((m, n), dtype=torch.complex128, device=X.device)
        Rd = torch.empty((m, n), dtype=torch.complex128, device=X.device) if deriv else None
        self._chk("bem_residual_arith", self._lib.bem_residual_arith(
            self._h, m, _ptr(lam.view(np.float64)), _ptr(X), X.stride(1), _ptr(R), _ptr(Rd), _ptr(rel),
            int(arith), _stream(stream)))
        return rel, R.transpose(0, 1), (Rd.transpose(0, 1) if deriv else None)


def _batch_arrays(ctxs, Vs, Bhats):
    n = len(ctxs)
    hs = (_P * n)(*[c._h for c in ctxs])
    vp = (_P * n)(*[V.data_ptr() for V in Vs])
    ld = (_I64 * n)(*[V.stride(1) for V in Vs])
    nus = (_I * n)(*[V.shape[1] for V in Vs])
    bp = (_P * n)(*[B.data_ptr() for B in Bhats])
    return hs, vp, ld, nus, bp


def _batch_outputs(ctxs, Vs):
    """Raw output buffers (the library writes each Bhat_j column-major) and their views."""
    import torch
    for c, V in zip(ctxs, Vs):
        _check_fortran(V, "V")
        if V.shape[0] != c.n:
            raise ValueError("each V must have as many rows as its context's mesh has panels")
    raw = [torch.empty((c.N, V.shape[1], V.shape[1]), dtype=torch.complex128, device=V.device)
           for c, V in zip(ctxs, Vs)]
    return raw, [r.transpose(1, 2) for r in raw]


class Batch:
    """Grouped mixed-precision projection of several contexts, recorded as a CUDA graph.

    ``Batch(ctxs, Vs, autotune=True)`` plans and records; ``run()`` replays it into
    ``self.Bhat`` (a list of (N_k, nu_k, nu_k) tensors, whose [j] slice is Bhat_j)."""

    def __init__(self, ctxs, Vs, autotune=False, stream=None):
        self._lib = load()
        self.ctxs = list(ctxs)
        self.Vs = list(Vs)
        self._raw, self.Bhat = _batch_outputs(self.ctxs, self.Vs)
        hs, vp, ld, nus, bp = _batch_arrays(self.ctxs, self.Vs, self._raw)
        h = _P()
        st = self._lib.bem_batch_create(hs, len(self.ctxs), vp, ld, nus, bp, PREC_MIXED,
                                        int(bool(autotune)), ctypes.byref(h), _stream(stream))
        if st != BEM_OK:
            raise BemError("bem_batch_create", st,
                           self._lib.bem_last_error(self.ctxs[0]._h).decode())
        self._h = h

    def run(self, stream=None):
        st = self._lib.bem_batch_run(self._h, _stream(stream))
        if st != BEM_OK:
            raise BemError("bem_batch_run", st, self._lib.bem_last_error(self.ctxs[0]._h).decode())
        return self.Bhat

    def info(self):
        s, g, u, t = _I(), _I(), _I64(), _D()
        self._lib.bem_batch_info(self._h, ctypes.byref(s), ctypes.byref(g), ctypes.byref(u),
                                 ctypes.byref(t))
        return {"splits": s.value, "nodes_per_unit": g.value, "units": u.value,
                "tuned_ms": t.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bem_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def project_batched(ctxs, Vs, stream=None):
    """One-shot grouped projection (synchronous); returns the list of Bhat tensors."""
    lib = load()
    ctxs = list(ctxs)
    Vs = list(Vs)
    raw, Bhat = _batch_outputs(ctxs, Vs)
    hs, vp, ld, nus, bp = _batch_arrays(ctxs, Vs, raw)
    st = lib.bem_project_batched(hs, len(ctxs), vp, ld, nus, bp, PREC_MIXED, _stream(stream))
    if st != BEM_OK:
        raise BemError("bem_project_batched", st, lib.bem_last_error(ctxs[0]._h).decode())
    return Bhat
