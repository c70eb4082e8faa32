"""Build and load the oracle's C part (``bem_oracle.c``) with gcc; test infrastructure only."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libbem_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain -O2, no fast-math, OpenMP over rows)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        i32 = ctypes.c_int
        L.oracle_rule7.argtypes = [P, P]
        L.oracle_gauss_legendre.argtypes = [i32, P, P]
        L.oracle_geometry.argtypes = [P, i64, P, P, P, P, P]
        L.oracle_self_integral.argtypes = [P, P, P, P, d, d, i32, P]
        L.oracle_matrix.argtypes = [P, i64, P, d, d, i32, i64, i64, P, i32, i32]
        L.oracle_apply.argtypes = [P, i64, P, i32, P, i32, P, i64, i64, P, i32, i32]
        L.oracle_near_rule.argtypes = [P, P, P, P, d, d, i32, i32, P]
        L.oracle_near_pairs.argtypes = [P, i64, P, i64, i64, P, P, P]
        L.oracle_matrix_op.argtypes = [P, i64, P, d, d, i32, i64, i64, P, i32, i32, P]
        L.oracle_apply_op.argtypes = [P, i64, P, i32, P, i32, P, i64, i64, P, i32, i32, P]
        L.oracle_near_rule_kind.argtypes = [P, P, P, P, d, d, i32, i32, i32, P]
        L.oracle_entries.argtypes = [P, i64, P, d, d, P, P, i64, P, i32, P]
        L.oracle_max_threads.restype = i32
        _lib = L
    return _lib
