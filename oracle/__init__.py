"""The oracle: a plain, slow, sequential CPU implementation of what the
device executor computes.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in
__graft_entry__.py and the CPU-baseline leg of bench.py may import it.  It
shares no code with the CUDA path (paper_1304_0878_b300/), and neither side
imports the other; the seeded input generators in synth/ feed both.

Parts:
  executor.py  sequential executor: every task runs at submission, in
               submission order (Sections 2-3 of the paper)
  dag.py       dependency rule from access modes and submission order
               (Section 2), partitions (Section 5.1), brute-force legality
  tiles.py     FP64 tile bodies, vector scaling, low-precision rounding
               (C routines in orc_tiles.c)
  cholesky.py  tiled Cholesky task list, tile layout, residual check
  mixed.py     mixed-precision tiled Cholesky
  ir.py        triangular solves, refinement, backward error
"""
from ._clib import build  # noqa: F401
from . import dag, tiles, cholesky, mixed, ir, executor  # noqa: F401
