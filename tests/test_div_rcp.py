"""The FP64 substitution chains of the tile kernels (TRSM, TRTRI, the rows
below a POTRF block) divide by a pivot through its reciprocal: q = RN(a r),
then one correction RN(q + RN(a - q d) r) by fused multiply-adds.  By
Markstein's theorem that is the correctly rounded quotient, so the kernels
keep the results of plain division (Section 2's reading of the tile
routines as textbook loops, and the integer-exact Cholesky pins).  This pins
the method itself on the host against IEEE division, bit for bit: random
operands over 90 binades (significands near 2 weighted), integer quotients
and square-root pivots, and signed zeros."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_quotient_from_reciprocal_is_the_ieee_quotient(tmp_path):
    exe = str(tmp_path / "div_rcp_check")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-o", exe,
                           os.path.join(HERE, "div_rcp_check.c"), "-lm"])
    out = subprocess.run([exe, "20000000"], capture_output=True, text=True, check=True).stdout.split()
    assert out[0] == "pairs" and int(out[1]) > 21_000_000
    assert out[2] == "mismatches" and int(out[3]) == 0, out
