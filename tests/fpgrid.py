"""Test helpers for the low-precision grids (bfloat16, E4M3): an exact
rounding in rational arithmetic, the format's midpoints, binary32 ulps and
the two-step FP64 -> binary32 -> format chain a single rounding must not
equal.  Independent of both the oracle's rounding code and the device's."""
import math
from fractions import Fraction

import numpy as np
import torch

# (significant bits, minimum normal exponent, largest finite value, saturating)
FORMATS = {"bf16": (8, -126, float((2 - 2 ** -7) * 2.0 ** 127), 0),
           "e4m3": (4, -6, 448.0, 1)}


def exact_round(x, fmt):
    """RN_fmt(x) with ties to even, computed on rationals: the nearest point
    of the grid {k * 2^(E - p + 1)}, E = max(floor(log2|x|), emin); above the
    largest finite value the result saturates (E4M3) or overflows (bf16)."""
    p, emin, maxval, sat = FORMATS[fmt]
    if x == 0 or math.isnan(x):
        return x
    X = Fraction(x)
    sgn = -1 if X < 0 else 1
    A = abs(X)
    E = A.numerator.bit_length() - A.denominator.bit_length()
    while Fraction(2) ** E > A:
        E -= 1
    while Fraction(2) ** (E + 1) <= A:
        E += 1
    E = max(E, emin)
    q = Fraction(2) ** (E - p + 1)
    n = A / q
    k = n.numerator // n.denominator
    rem = n - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    y = k * q
    if y > Fraction(maxval):
        return sgn * maxval if sat else sgn * math.inf
    return sgn * float(y)


def grid_midpoints(fmt, rng, n):
    """n random midpoints between neighbouring values of the format's grid
    (positive, normal and subnormal ranges, below the largest value)."""
    p, emin, maxval, _ = FORMATS[fmt]
    top = int(math.floor(math.log2(maxval)))
    out = []
    for _ in range(n):
        E = int(rng.integers(emin - 1, top)) if fmt == "e4m3" else int(rng.integers(-130, 120))
        E = max(E, emin)
        q = 2.0 ** (E - p + 1)
        k = int(rng.integers(2 ** (p - 1) if E > emin else 0, 2 ** p - 1))
        out.append((k + 0.5) * q)
    return np.array(out)


def ulp32(m):
    """Spacing of binary32 values at |m| (2^-149 in binary32's subnormal range)."""
    return 2.0 ** np.maximum(np.floor(np.log2(np.abs(m))) - 23, -149)


def chain_round(x, fmt):
    """The two-step chain FP64 -> binary32 -> format (what the pin must
    reject): numpy's binary32 conversion, then torch's format conversion."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    t = torch.from_numpy(x32)
    dt = torch.bfloat16 if fmt == "bf16" else torch.float8_e4m3fn
    return t.to(dt).to(torch.float64).numpy()
