"""Oracle for dependency inference: which task must run before which.

TEST INFRASTRUCTURE ONLY.

Section 2 of the paper: buffer parameters are accessed read-only, write-only
or read-write, and those access modes together with the order in which tasks
are invoked determine the task dependency graph.  The mode encoding follows
the generated task body of Section 3.2, where a read-write buffer is passed
with mode value 3, i.e. R = 1, W = 2, RW = R|W.

Rule (one reading of Section 2, the classic RAW / WAR / WAW hazards), per
buffer, in submission order:
  * R access  : edge from the last writer (read-after-write).
  * W or RW   : edges from every reader since the last write (write-after-
                read); if there is none, an edge from the last writer
                (write-after-write / read-after-write).  The task becomes the
                last writer and the reader list is cleared.
  * A buffer named twice by one task gets the OR of its modes; no self-edges;
    duplicate edges are merged.
Partitioned buffers (Section 5.1, "filters"): accessing the parent accesses
every part with the same mode; parts are independent of one another.

Also here: brute-force legality over all orders of tiny task sets, which
pins the rule to its meaning rather than to its own statement.
"""
import hashlib
import itertools

R, W, RW = 1, 2, 3


def expand(handle, parts):
    """Leaves a handle stands for: its parts if partitioned, else itself."""
    return parts.get(handle, (handle,))


def derive_edges(accesses, parts=None):
    """accesses[t] = list of (handle, mode) of task t, in submission order.
    parts = {parent: (child, ...)}.  Returns the sorted list of (pred, succ)."""
    parts = parts or {}
    last_writer = {}
    readers = {}
    edges = set()
    for t, acc in enumerate(accesses):
        modes = {}
        for h, m in acc:
            assert m in (R, W, RW)
            for leaf in expand(h, parts):
                modes[leaf] = modes.get(leaf, 0) | m
        for leaf, m in modes.items():
            lw = last_writer.get(leaf)
            rd = readers.setdefault(leaf, [])
            if m & W:
                preds = list(rd) if rd else ([lw] if lw is not None else [])
                for p in preds:
                    if p != t:
                        edges.add((p, t))
                last_writer[leaf] = t
                readers[leaf] = []
            else:
                if lw is not None and lw != t:
                    edges.add((lw, t))
                rd.append(t)
    return sorted(edges)


def successors(n, edges):
    succ = [[] for _ in range(n)]
    for p, s in edges:
        succ[p].append(s)
    return succ


def transitive_closure(n, edges):
    """Set of (a, b) with a path a -> b; tasks are numbered topologically
    (every edge goes from an earlier to a later submission)."""
    succ = successors(n, edges)
    reach = [set() for _ in range(n)]
    for a in range(n - 1, -1, -1):
        for b in succ[a]:
            reach[a].add(b)
            reach[a] |= reach[b]
    return {(a, b) for a in range(n) for b in reach[a]}


def critical_path(n, edges):
    """Number of tasks on the longest path."""
    depth = [1] * n
    pred = [[] for _ in range(n)]
    for p, s in edges:
        pred[s].append(p)
    for t in range(n):
        for p in pred[t]:
            depth[t] = max(depth[t], depth[p] + 1)
    return max(depth) if n else 0


def upward_rank(n, edges, cost):
    """Upward rank of every task (Section 5.3 names upward and downward ranks
    as scheduling hints): the largest total cost over the paths that start at
    the task and follow edges to the end of the graph, the task's own cost
    included.  Written as that definition, by recursion over successors."""
    succ = successors(n, edges)
    memo = {}

    def longest(t):
        if t not in memo:
            memo[t] = cost[t] + max((longest(s) for s in succ[t]), default=0.0)
        return memo[t]

    # every edge goes from an earlier to a later submission: evaluating from
    # the last task backwards keeps the recursion shallow
    for t in range(n - 1, -1, -1):
        longest(t)
    return [memo[t] for t in range(n)]


def downward_rank(n, edges, cost):
    """Downward rank of every task (the other scheduling hint Section 5.3
    names): the largest total cost over the paths from a task without
    predecessors to the task, the task's own cost excluded.  Written as that
    definition, by recursion over predecessors."""
    pred = [[] for _ in range(n)]
    for p, s in edges:
        pred[s].append(p)
    memo = {}

    def longest(t):
        if t not in memo:
            memo[t] = max((longest(p) + cost[p] for p in pred[t]), default=0.0)
        return memo[t]

    for t in range(n):
        longest(t)
    return [memo[t] for t in range(n)]


def depth(n, edges):
    """Edges on the longest path from a source to each task."""
    d = [0] * n
    pred = [[] for _ in range(n)]
    for p, s in edges:
        pred[s].append(p)
    for t in range(n):
        for p in pred[t]:
            d[t] = max(d[t], d[p] + 1)
    return d


def topological_orders(n, edges):
    """All linear extensions (brute force; tiny n only)."""
    pos_pred = [set() for _ in range(n)]
    for p, s in edges:
        pos_pred[s].add(p)
    out = set()
    for perm in itertools.permutations(range(n)):
        seen = set()
        ok = True
        for t in perm:
            if not pos_pred[t] <= seen:
                ok = False
                break
            seen.add(t)
        if ok:
            out.add(perm)
    return out


def _h(*vals):
    return hashlib.blake2b(repr(vals).encode(), digest_size=12).hexdigest()


def run_symbolic(order, accesses, parts=None):
    """Execute tasks symbolically in `order`.  Each task reads the values of
    its R / RW leaves and writes, to every W / RW leaf, a hash of its id, the
    leaf and everything it read (a W-only leaf ignores its old contents).
    Returns (what each task read, the sequence of values written to each
    leaf).  The write sequence, not only the final value, is observable: a
    buffer may be read back between tasks (acquire, Section 3.4)."""
    parts = parts or {}
    mem = {}
    hist = {}
    seen = {}
    for t in order:
        modes = {}
        for h, m in accesses[t]:
            for leaf in expand(h, parts):
                modes[leaf] = modes.get(leaf, 0) | m
        inputs = tuple((leaf, mem.get(leaf, ("init", leaf)))
                       for leaf in sorted(modes) if modes[leaf] & R)
        seen[t] = inputs
        for leaf in sorted(modes):
            if modes[leaf] & W:
                mem[leaf] = _h(t, leaf, inputs)
                hist.setdefault(leaf, []).append(mem[leaf])
    return seen, hist


def legal_orders(accesses, parts=None):
    """Orders in which every task reads exactly what it reads in submission
    order and every buffer receives the same sequence of writes: the
    schedules the sequential program (Section 3) cannot tell apart from
    itself."""
    n = len(accesses)
    ref = run_symbolic(range(n), accesses, parts)
    return {perm for perm in itertools.permutations(range(n))
            if run_symbolic(perm, accesses, parts) == ref}
