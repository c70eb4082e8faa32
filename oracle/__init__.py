"""Plain FP64 CPU oracle of the Cauchy rational approximation + Rayleigh-Ritz method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package. It shares no code with the
CUDA path; both only read the inputs made by ``synth``.

Modules
-------
_lib      ctypes loader of the C part (entries of A(k), its k-derivative, A(z_j) V)
contour   trapezoid nodes and weights on a circle or ellipse (Eq. TzApp)
rr        projection, orthonormalisation, reduced linearisation (Eq. EVP_red,
          Eq. sc1_cauchy_red), inverse power step (Algorithm 1), reduced subspace
          iteration (Algorithm 3)
refine    residual ||A(l) x|| / ||x||, successive-linear-problems refinement of eigenvalues,
          sigma_min of A(k), argument-principle count
"""
from ._lib import build, lib
from . import contour, assembly, rr, refine

__all__ = ["build", "lib", "contour", "assembly", "rr", "refine"]
