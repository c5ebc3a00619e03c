"""Pins for the dependency oracle (Section 2: access modes plus invocation
order define the task graph).  The rule is checked against its meaning: by
brute force over every order of tiny task sets, a schedule is legal exactly
when it is a topological order of the derived graph."""
import numpy as np
import pytest

import synth
from oracle import dag, cholesky
from oracle.dag import R, W, RW


def test_hand_cases():
    # RAW, WAR, WAW, readers in parallel, handle named twice
    acc = [[(0, W)], [(0, R)], [(0, R)], [(0, RW)], [(0, R), (0, W)], [(1, R)]]
    assert dag.derive_edges(acc) == [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4)]
    # W-only after W-only: WAW edge
    assert dag.derive_edges([[(5, W)], [(5, W)]]) == [(0, 1)]
    # independent handles: no edges
    assert dag.derive_edges([[(0, RW)], [(1, RW)], [(2, R)]]) == []


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_legal_orders_equal_topological_orders(seed):
    n = 4 + seed % 4          # 4..7 tasks
    acc = synth.random_accesses(n, nhandles=3 + seed % 3, maxbuf=3, seed=seed)
    edges = dag.derive_edges(acc)
    assert dag.legal_orders(acc) == dag.topological_orders(n, edges)


@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_with_partitions(seed):
    rng = np.random.default_rng(100 + seed)
    parts = {10: (0, 1, 2)}   # handle 10 is the parent of 0, 1, 2
    n = 6
    acc = []
    for _ in range(n):
        hs = rng.choice([0, 1, 2, 3, 10], size=int(rng.integers(1, 3)), replace=False)
        acc.append([(int(h), int(rng.integers(1, 4))) for h in hs])
    edges = dag.derive_edges(acc, parts)
    assert dag.legal_orders(acc, parts) == dag.topological_orders(n, edges)


@pytest.mark.parametrize("T,ntasks,nedges,cp", [(8, 120, 252, 22)])
def test_cholesky_dag_counts_small(T, ntasks, nedges, cp):
    acc = cholesky.accesses(T)
    e = dag.derive_edges(acc)
    assert len(acc) == ntasks == T + T * (T - 1) + T * (T - 1) * (T - 2) // 6
    assert len(e) == nedges
    assert dag.critical_path(len(acc), e) == cp == 3 * (T - 1) + 1


def test_cholesky_dag_counts_full_size():
    T = 64
    acc = cholesky.accesses(T)
    e = dag.derive_edges(acc)
    assert len(acc) == 45760
    assert len(e) == 131040
    assert dag.critical_path(len(acc), e) == 190


def test_vector_chain_dag():
    nb, nk = 256, 8
    acc = [[(b, RW)] for k in range(nk) for b in range(nb)]   # k-major
    e = dag.derive_edges(acc)
    assert len(e) == nb * (nk - 1) == 1792
    assert dag.critical_path(len(acc), e) == nk


def test_cholesky_bruteforce_t2():
    # T = 2: POTRF, TRSM, SYRK, POTRF -> a chain; only one legal order
    acc = cholesky.accesses(2)
    assert len(acc) == 4
    edges = dag.derive_edges(acc)
    assert dag.legal_orders(acc) == dag.topological_orders(4, edges) == {(0, 1, 2, 3)}


def test_transitive_closure_small():
    e = [(0, 1), (1, 2), (0, 3)]
    assert dag.transitive_closure(4, e) == {(0, 1), (1, 2), (0, 2), (0, 3)}


@pytest.mark.parametrize("seed", range(8))
def test_ranks_by_path_enumeration(seed):
    # upward and downward ranks (Section 5.3) against every path of small
    # random DAGs enumerated one by one: the upward rank of v is the largest
    # cost sum over paths starting at v, the downward rank the largest cost
    # sum over paths ending at v with v's own cost left out
    rng = np.random.default_rng(900 + seed)
    n = 10
    edges = sorted({(int(a), int(b)) for a, b in rng.integers(0, n, size=(18, 2)) if a < b})
    cost = [float(c) for c in rng.integers(1, 9, size=n)]
    adj = {v: [b for a, b in edges if a == v] for v in range(n)}
    paths = []

    def walk(p):
        paths.append(p)
        for s in adj[p[-1]]:
            walk(p + [s])
    for v in range(n):
        walk([v])
    up = [max(sum(cost[x] for x in p) for p in paths if p[0] == v) for v in range(n)]
    down = [max(sum(cost[x] for x in p[:-1]) for p in paths if p[-1] == v) for v in range(n)]
    assert dag.upward_rank(n, edges, cost) == up
    assert dag.downward_rank(n, edges, cost) == down
    # the longest path through v is the same from both ends
    longest = max(sum(cost[x] for x in p) for p in paths)
    assert max(u + d for u, d in zip(up, down)) == longest == max(up)


def test_ranks_of_a_chain():
    # closed form: a chain of n tasks with costs c_i
    cost = [3.0, 1.0, 4.0, 1.0, 5.0]
    edges = [(i, i + 1) for i in range(4)]
    assert dag.upward_rank(5, edges, cost) == [14.0, 11.0, 10.0, 6.0, 5.0]
    assert dag.downward_rank(5, edges, cost) == [0.0, 3.0, 4.0, 8.0, 9.0]
