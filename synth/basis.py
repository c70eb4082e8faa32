"""Seeded complex Gaussian starting bases.

The paper starts its subspace construction from random vectors (Section 3.2; Algorithm 3,
"initially random vectors"). Both the CUDA path and the oracle receive the same basis as
data, generated here once on the host:

* SplitMix64 (Steele, Lea, Flood 2014) in counter form: output k of stream ``seed`` is
  mix(seed + (k + 1) * 0x9E3779B97F4A7C15).
* Uniforms in (0, 1]: the top 53 bits plus one, times 2**-53.
* Box-Muller: z = sqrt(-ln u1) * exp(2 pi i u2), so Re z and Im z are independent
  N(0, 1/2) and E|z|^2 = 1.

The basis is an n x nu complex128 array in column-major (Fortran) order: column c holds
entries c*n .. c*n + n - 1, each an interleaved (re, im) pair.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream started at ``seed``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    bits = splitmix64(seed, count, offset) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (2.0 ** -53)


def complex_gaussian(n: int, nu: int, seed: int) -> np.ndarray:
    """n x nu complex128 Fortran-ordered basis; entry (i, c) uses stream slots 2(c n + i), +1."""
    u = uniform01(seed, 2 * n * nu)
    u1 = u[0::2]
    u2 = u[1::2]
    z = np.sqrt(-np.log(u1)) * np.exp(2j * np.pi * u2)
    return np.asfortranarray(z.reshape(nu, n).T)
