"""numpy front-end of the oracle's C tile routines.

TEST INFRASTRUCTURE ONLY.  A tile is a numpy array of shape (b, b) in
Fortran (column-major) order, so ``T[r, c]`` is element (r, c) stored at
r + c*b, the layout the task bodies are defined on.  Every routine mutates
its output in place, like a task body acting on a registered buffer
(Section 2).
"""
import ctypes

import numpy as np

from ._clib import lib

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)

# Low-precision formats (significant bits, minimum normal exponent, largest
# finite value, saturating).  bfloat16 keeps binary32's exponent range; E4M3
# (OCP FP8) has 4 significant bits, bias 7, no infinities and saturates to 448.
BF16 = (8, -126, float((2 - 2 ** -7) * 2.0 ** 127), 0)
E4M3 = (4, -6, 448.0, 1)
FORMATS = {"bf16": BF16, "e4m3": E4M3}


def _ptr(a, ty):
    assert a.flags.f_contiguous or a.ndim == 1, "tiles must be column-major"
    return a.ctypes.data_as(ty)


def _ld(a):
    return a.shape[0]


def scal_f32(x, f):
    """x[i] <- fl32(x[i] * f) for every element (the Section 2 example)."""
    assert x.dtype == np.float32 and x.flags.c_contiguous
    lib().orc_scal_f32(x.ctypes.data_as(_fp), x.size, ctypes.c_float(np.float32(f)))


def potrf(A):
    """In-place Cholesky-Crout of the lower triangle; returns info (0 = ok)."""
    assert A.dtype == np.float64
    n = A.shape[0]
    return lib().orc_potrf(_ptr(A, _dp), n, _ld(A))


def trsm(L, A):
    """A <- A L^{-T} (right side, L lower, non-unit)."""
    m, n = A.shape
    lib().orc_trsm(_ptr(L, _dp), _ld(L), _ptr(A, _dp), m, n, _ld(A))


def syrk(A, C):
    """C <- C - A A^T on the lower triangle of C."""
    n, k = A.shape
    lib().orc_syrk(_ptr(A, _dp), n, k, _ld(A), _ptr(C, _dp), _ld(C))


def gemm(A, B, C):
    """C <- C - A B^T."""
    m, k = A.shape
    n = B.shape[0]
    lib().orc_gemm(_ptr(A, _dp), _ld(A), _ptr(B, _dp), _ld(B), _ptr(C, _dp), m, n, k, _ld(C))


def round_format(x, fmt):
    """Round value(s) to the format, one rounding from FP64, ties to even
    (binary32 inputs widen exactly)."""
    p, emin, mx, sat = FORMATS[fmt]
    f = lib().orc_round_format
    xs = np.asarray(x, dtype=np.float64).ravel()
    out = np.array([f(float(v), p, emin, mx, sat) for v in xs])
    return out.reshape(np.shape(x))


def scale_exponent(amax, fmt):
    """Exponent e of the per-tile power-of-two scale 2^e: smallest e with
    amax <= fmt_max * 2^e for E4M3; bfloat16 keeps binary32's range, so its
    scale is 1 (e = 0)."""
    if fmt == "bf16":
        return 0
    return lib().orc_scale_exponent(float(amax), FORMATS[fmt][2])


def quantise(X, fmt):
    """Return (Q, e): Q = round_format(X / 2^e) (one rounding from FP64) as
    float64 values in Fortran order, e the tile's scale exponent from
    max |X|."""
    p, emin, mx, sat = FORMATS[fmt]
    X = np.asfortranarray(X, dtype=np.float64)
    e = scale_exponent(np.max(np.abs(X)) if X.size else 0.0, fmt)
    Q = np.empty_like(X, order="F")
    lib().orc_quantise(X.ctypes.data_as(_dp), X.size, e, p, emin, mx, sat,
                       Q.ctypes.data_as(_dp))
    return Q, e


def gemm_lowp(QA, QB, s, C, lower=False):
    """C(binary32) <- fl32(C - s * QA QB^T); products summed in FP64."""
    assert C.dtype == np.float32 and C.flags.f_contiguous
    m, k = QA.shape
    n = QB.shape[0]
    lib().orc_gemm_lowp(_ptr(QA, _dp), _ld(QA), _ptr(QB, _dp), _ld(QB), float(s),
                        C.ctypes.data_as(_fp), m, n, k, _ld(C), 1 if lower else 0)


def gemm_abs(QA, QB):
    """sum_p |QA(r,p) QB(c,p)| as an m x n Fortran array."""
    m, k = QA.shape
    n = QB.shape[0]
    out = np.zeros((m, n), order="F")
    lib().orc_gemm_abs(_ptr(QA, _dp), _ld(QA), _ptr(QB, _dp), _ld(QB),
                       out.ctypes.data_as(_dp), m, n, k, m)
    return out
