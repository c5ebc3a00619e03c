"""Build and load the oracle's C tile routines (oracle/orc_tiles.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc_tiles.c")
_LIB = os.path.join(_HERE, "_orc_tiles.so")

# No -ffast-math, no FMA contraction: every operation is one IEEE rounding.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
          "-fno-fast-math", "-fno-unsafe-math-optimizations"]


def build(force=False):
    """Compile orc_tiles.c into _orc_tiles.so next to it (gcc)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_scal_f32": (None, [fp, i64, ctypes.c_float]),
            "orc_potrf": (i, [dp, i, i]),
            "orc_trsm": (None, [dp, i, dp, i, i, i]),
            "orc_syrk": (None, [dp, i, i, i, dp, i]),
            "orc_gemm": (None, [dp, i, dp, i, dp, i, i, i, i]),
            "orc_round_format": (d, [d, i, i, d, i]),
            "orc_scale_exponent": (i, [d, d]),
            "orc_quantise": (None, [dp, i64, i, i, i, d, i, dp]),
            "orc_gemm_lowp": (None, [dp, i, dp, i, d, fp, i, i, i, i, i]),
            "orc_gemm_abs": (None, [dp, i, dp, i, dp, i, i, i, i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
