"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle) against the oracle as it stands, against what fixes them
independently of it, and against the C ABI on the host."""
import importlib.util
import os

import numpy as np
import pytest

import synth
import paper_1304_0878_b300 as b3t

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _read(name):
    with open(os.path.join(GOLD, name)) as f:
        return f.read()


@pytest.mark.parametrize("name", ["cholesky_dag_t4.txt", "vector_chain.txt", "integer_cholesky_n6.txt"])
def test_oracle_reproduces_stored_values(orc, name):
    assert _maker().FILES[name]() == _read(name)


def _rows(text, tag):
    return [l.split()[1:] for l in text.splitlines() if l.startswith(tag + " ")]


def test_cholesky_dag_golden_closed_forms_and_library():
    text = _read("cholesky_dag_t4.txt")
    T = 4
    tasks = _rows(text, "task")
    edges = [(int(a), int(b)) for a, b in _rows(text, "edge")]
    assert len(tasks) == T + T * (T - 1) + T * (T - 1) * (T - 2) // 6
    assert int(_rows(text, "critical_path")[0][0]) == 3 * T - 2
    assert all(p < s for p, s in edges) and len(set(edges)) == len(edges)
    # the C ABI derives the stored edges for the same submission
    c = b3t.Context(host_only=True)
    c.cholesky_submit([0x10000000 + (i << 20) for i in range(T * (T + 1) // 2)], T, 64)   # one task per tile
    assert sorted(c.dag_edges()) == edges
    c.close()


def test_vector_chain_golden_is_in_order_binary32():
    text = _read("vector_chain.txt")
    x, f, y = (np.array([int(v, 16) for v in _rows(text, t)[0]], dtype=np.uint32).view(np.float32)
               for t in ("x", "f", "y"))
    with np.errstate(over="ignore"):
        z = x.copy()
        for fk in f:
            z = (z * fk).astype(np.float32)      # numpy: one binary32 rounding per multiply
        # the product folded into one factor rounds differently somewhere
        folded = (x * np.float32(f[0] * f[1] * f[2])).astype(np.float32)
    assert np.array_equal(z.view(np.uint32), y.view(np.uint32))
    assert np.isinf(y[3]) and y[6] == np.float32(3) * np.float32(1e-45)     # overflow; subnormal kept
    assert not np.array_equal(folded.view(np.uint32), y.view(np.uint32))


def test_integer_cholesky_golden_is_exact():
    text = _read("integer_cholesky_n6.txt")
    A = np.array([[int(v) for v in r] for r in _rows(text, "A")], dtype=np.int64)
    L = np.array([[float(v) for v in r] for r in _rows(text, "L")])
    A0, L0 = synth.integer_spd(6, 4)
    assert np.array_equal(A, A0.astype(np.int64)) and np.array_equal(L, L0)
    assert np.array_equal(L.astype(np.int64) @ L.astype(np.int64).T, A)
