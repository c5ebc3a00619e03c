"""Writes the stored expected values under tests/golden/ from the oracle
alone (and the seeded input generators).  Run from the repository root:

    python tests/golden/make_golden.py

The paper prints no numeric results, so every stored value here is the
oracle's, on inputs small enough to read by eye:
  * cholesky_dag_t4.txt: the tiled Cholesky task list at T = 4 in
    right-looking submission order and the edges the dependency rule derives
    (Section 2: access modes and invocation order determine the graph;
    Section 5.1: the tiled factorisation over registered tiles);
  * vector_chain.txt: the Section 2 vector-scaling example as a chain of
    three tasks on eight binary32 values, as bit patterns;
  * integer_cholesky_n6.txt: an integer SPD matrix A = L0 L0^T and the
    factor the oracle computes (exact: every step stays on integers).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import cholesky as och, dag, tiles as otl  # noqa: E402


def cholesky_dag(T=4):
    lines = ["# tiled Cholesky, T = %d: task list (right-looking order) and derived edges" % T,
             "# (Section 5.1: the tiled factorisation over registered tiles; Section 2: access modes",
             "# and invocation order determine the dependency graph).  Written by the oracle.",
             "# task <index> <kind> <tile i,j:mode> ...   (mode 1 = R, 3 = RW)"]
    for n, (kind, acc) in enumerate(och.task_list(T)):
        lines.append("task %d %s %s" % (n, kind, " ".join("%d,%d:%d" % (i, j, m) for (i, j), m in acc)))
    edges = dag.derive_edges(och.accesses(T))
    lines.append("# edge <pred> <succ>")
    lines += ["edge %d %d" % e for e in edges]
    lines.append("critical_path %d" % dag.critical_path(len(och.task_list(T)), edges))
    return "\n".join(lines) + "\n"


def vector_chain():
    x = np.array([1.0, -0.5, 3.0e-39, 1.5e38, 0.1, -7.25, 1e-45, 2.0 / 3.0], dtype=np.float32)
    f = np.array([1.1, 0.75, 3.0], dtype=np.float32)
    y = x.copy()
    for fk in f:
        otl.scal_f32(y, fk)
    lines = ["# Section 2 vector scaling as a chain of three RW tasks x *= f_k (k in order),",
             "# one binary32 rounding per multiply; values as IEEE-754 bit patterns (hex).",
             "# Written by the oracle."]
    lines.append("x " + " ".join("%08x" % v for v in x.view(np.uint32)))
    lines.append("f " + " ".join("%08x" % v for v in f.view(np.uint32)))
    lines.append("y " + " ".join("%08x" % v for v in y.view(np.uint32)))
    return "\n".join(lines) + "\n"


def integer_cholesky(N=6, seed=4):
    A, L0 = synth.integer_spd(N, seed)
    L, info = och.dense_potrf(A)
    assert info == 0
    L = np.tril(L)
    lines = ["# integer SPD A = L0 L0^T (synth.integer_spd(%d, seed=%d)) and the oracle's factor" % (N, seed),
             "# (Section 5.1's Cholesky task bodies; every step is exact on these integers)"]
    lines += ["A " + " ".join("%d" % v for v in row) for row in A.astype(np.int64)]
    lines += ["L " + " ".join(repr(float(v)) for v in row) for row in L]
    return "\n".join(lines) + "\n"


FILES = {"cholesky_dag_t4.txt": cholesky_dag, "vector_chain.txt": vector_chain,
         "integer_cholesky_n6.txt": integer_cholesky}

if __name__ == "__main__":
    oracle.build()
    for name, fn in FILES.items():
        with open(os.path.join(HERE, name), "w") as fh:
            fh.write(fn())
        print("wrote", name)
