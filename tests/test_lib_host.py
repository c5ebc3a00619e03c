"""C-ABI library on the host (no GPU): it loads, exports every function of
include/b3t.h, derives exactly the oracle's dependency edges, and reports
the errors the paper's tooling diagnoses (Section 3.2) as return codes."""
import subprocess

import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from oracle import dag, cholesky as och

R, W, RW = 1, 2, 3


@pytest.fixture
def ctx():
    b3t.lib()
    c = b3t.Context(host_only=True)
    yield c
    c.close()


def fake_ptr(i):
    return 0x10000000 + (i << 20)   # distinct, 16-byte aligned, never dereferenced


def test_exports_every_header_symbol():
    names = b3t.header_symbols()
    assert len(names) >= 20
    out = subprocess.check_output(["nm", "-D", "--defined-only", b3t._lib.LIB_PATH]).decode()
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = b3t.lib()
    for n in names:
        assert hasattr(L, n)


@pytest.mark.skipif(torch.cuda.is_available(), reason="a CUDA device is present")
def test_init_without_device_reports_enodev():
    with pytest.raises(b3t.B3TError) as e:
        b3t.Context()
    assert e.value.code == b3t._lib.ENODEV


def _submit_accesses(c, accesses, nhandles, parts=None):
    hs = [c.data_register(fake_ptr(i), 64, 4) for i in range(nhandles)]
    pmap = {}
    for parent, nkids in (parts or {}).items():
        pmap[parent] = c.data_partition(hs[parent], nkids, 64 // nkids)
    cls = {}
    for acc in accesses:
        modes = tuple(m for _, m in acc)
        if modes not in cls:
            cls[modes] = c.task_decl("t", b3t.NOOP, list(modes))
        c.task_submit(cls[modes], [hs[h] for h, _ in acc])
    return hs, pmap


@pytest.mark.parametrize("seed", range(60))
def test_edges_match_oracle_random(ctx, seed):
    n = 5 + seed % 20
    nh = 2 + seed % 6
    acc = synth.random_accesses(n, nhandles=nh, maxbuf=min(3, nh), seed=1000 + seed)
    _submit_accesses(ctx, acc, nh)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc)


def test_edges_match_oracle_with_partitions(ctx):
    rng = np.random.default_rng(5)
    hs = [ctx.data_register(fake_ptr(i), 64, 4) for i in range(3)]
    kids = ctx.data_partition(hs[0], 4, 16)           # handle 0 -> 4 parts
    # oracle names: parts 10..13 of parent 0; plain handles 1, 2
    parts = {0: (10, 11, 12, 13)}
    lib_of = {0: hs[0], 1: hs[1], 2: hs[2], 10: kids[0], 11: kids[1], 12: kids[2], 13: kids[3]}
    acc = []
    cls = {}
    for _ in range(40):
        k = int(rng.integers(1, 4))
        names = rng.choice([0, 1, 2, 10, 11, 12, 13], size=k, replace=False)
        a = [(int(h), int(rng.integers(1, 4))) for h in names]
        modes = tuple(m for _, m in a)
        if modes not in cls:
            cls[modes] = ctx.task_decl("t", b3t.NOOP, list(modes))
        ctx.task_submit(cls[modes], [lib_of[h] for h, _ in a])
        acc.append(a)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc, parts)


@pytest.mark.parametrize("T", [1, 2, 8, 64])
def test_cholesky_submission_edges(ctx, T):
    b = 64      # one POTRF task per diagonal tile (b >= 128 splits it into panels)
    ptrs = [fake_ptr(i) for i in range(och.ntiles(T))]
    ctx.cholesky_submit(ptrs, T, b)
    nt, ne = ctx.dag_stats()
    acc = och.accesses(T)
    assert nt == len(acc)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc)


def test_mixed_submission_edges(ctx):
    from oracle import mixed
    T, b = 6, 128
    nt = och.ntiles(T)
    Wp = [fake_ptr(i) for i in range(nt)]
    Lp = [fake_ptr(1000 + i) for i in range(nt)]
    Qp = [fake_ptr(2000 + i) for i in range(nt)]
    ctx.cholesky_mx_submit(Wp, Lp, Qp, T, b, b3t.FMT_BF16)
    key = {}
    acc = []
    for kind, a in mixed.task_list(T):
        acc.append([(key.setdefault(buf, len(key)), m) for buf, m in a])
        if kind == mixed.TRSM_MX:
            # the library submits QUANT(L_ik: R, Q_ik: W) right after TRSM_MX
            (_, i, k) = a[2][0]
            acc.append([(key.setdefault(("L", i, k), len(key)), R),
                        (key.setdefault(("Q", i, k), len(key)), W)])
    assert ctx.dag_stats()[0] == len(acc)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc)


def test_chain_edges(ctx):
    nb, nk = 256, 8
    hs = [ctx.data_register(fake_ptr(i), 1 << 20, 4) for i in range(nb)]
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    for k in range(nk):
        for i in range(nb):
            ctx.task_submit(cl, [hs[i]], b3t.pack_f32(1.5))
    assert ctx.dag_stats() == (2048, 1792)
    acc = [[(i, RW)] for k in range(nk) for i in range(nb)]
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc)


def test_error_codes(ctx):
    E = b3t._lib
    h = ctx.data_register(fake_ptr(1), 1024, 4)
    with pytest.raises(b3t.B3TError) as e:
        ctx.data_register(fake_ptr(1), 1024, 4)
    assert e.value.code == E.EEXIST
    with pytest.raises(b3t.B3TError) as e:
        ctx.data_lookup(fake_ptr(2))           # unregistered pointer
    assert e.value.code == E.ENOENT
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    with pytest.raises(b3t.B3TError) as e:     # declaration vs kind signature
        ctx.task_decl("bad", b3t.SCAL_F32, [R], 4)
    assert e.value.code == E.EINVAL
    with pytest.raises(b3t.B3TError) as e:     # wrong scalar blob
        ctx.task_decl("bad", b3t.TRSM, [R, RW], 4)
    assert e.value.code == E.EINVAL
    with pytest.raises(b3t.B3TError) as e:     # mode used differs from declared
        ctx.task_submit(cl, [h], b3t.pack_f32(2.0), modes=[R])
    assert e.value.code == E.EINVAL
    with pytest.raises(b3t.B3TError) as e:
        ctx.task_submit(cl, [12345], b3t.pack_f32(2.0))
    assert e.value.code == E.ENOENT
    with pytest.raises(b3t.B3TError) as e:     # pointer form: lookup failure
        ctx.task_submit_ptrs(cl, [fake_ptr(3)], b3t.pack_f32(2.0))
    assert e.value.code == E.ENOENT
    ctx.task_submit_ptrs(cl, [fake_ptr(1)], b3t.pack_f32(2.0))
    # tile kinds check buffer shapes: f32 buffer where f64 tile is expected
    t = ctx.data_register(fake_ptr(9), 128 * 128, 4, 128)
    cp = ctx.task_decl("potrf", b3t.POTRF, [RW], 4)
    with pytest.raises(b3t.B3TError) as e:
        ctx.task_submit(cp, [t], b3t.pack_i32(0))
    assert e.value.code == E.EINVAL
    assert ctx.dag_stats()[0] == 1
    with pytest.raises(b3t.B3TError) as e:     # no device in host-only mode
        ctx.task_wait()
    assert e.value.code == E.ENODEV
    assert ctx.dag_stats() == (0, 0)
    ctx.data_unregister(h)
    with pytest.raises(b3t.B3TError) as e:
        ctx.task_submit(cl, [h], b3t.pack_f32(2.0))
    assert e.value.code == E.ENOENT


def test_acquire_errors(ctx):
    # Section 3.4 (acquire): an unknown handle and a mode outside R/W/RW are
    # errors; with nothing pending, acquiring a registered buffer returns at once
    E = b3t._lib
    h = ctx.data_register(fake_ptr(5), 64, 4)
    with pytest.raises(b3t.B3TError) as e:
        ctx.data_acquire(h + 100, R)
    assert e.value.code == E.ENOENT
    for bad in (0, 4):
        with pytest.raises(b3t.B3TError) as e:
            ctx.data_acquire(h, bad)
        assert e.value.code == E.EINVAL
    ctx.data_acquire(h, RW)


def test_q_bytes():
    assert b3t.q_bytes(512, b3t.FMT_BF16) == 512 * 512 * 2 + 16
    assert b3t.q_bytes(256, b3t.FMT_E4M3) == 256 * 256 + 16
    assert b3t.q_bytes(100, b3t.FMT_BF16) == 0


def test_strerror():
    assert "unregistered" in b3t.strerror(b3t._lib.ENOENT)
    assert "positive definite" in b3t.strerror(b3t._lib.EDOM)


@pytest.mark.parametrize("T,b", [(1, 256), (3, 512), (4, 256), (3, 128), (2, 192)])
def test_cholesky_panel_dag_edges(ctx, T, b):
    # b >= 256: each diagonal tile is partitioned into b/128 column panels
    # (b = 128 and 192: 64-column panels) and POTRF becomes POTRF_D /
    # PANEL_TRSM / PANEL_UPD tasks on the parts
    ptrs = [fake_ptr(i) for i in range(och.ntiles(T))]
    ctx.cholesky_submit(ptrs, T, b)
    np_ = b // (128 if b >= 256 else 64)
    parts = {och.tile_index(k, k, T): tuple(("P", k, kk) for kk in range(np_)) for k in range(T)}
    acc = []
    for k in range(T):
        P = parts[och.tile_index(k, k, T)]
        for kk in range(np_):
            acc.append([(P[kk], RW)])
            if kk < np_ - 1:
                acc.append([(P[kk], RW)])
            for jj in range(kk + 1, np_):
                acc.append([(P[kk], R), (P[jj], RW)])
        for i in range(k + 1, T):
            acc.append([(och.tile_index(k, k, T), R), (och.tile_index(i, k, T), RW)])
        for i in range(k + 1, T):
            acc.append([(och.tile_index(i, k, T), R), (och.tile_index(i, i, T), RW)])
            for j in range(k + 1, i):
                acc.append([(och.tile_index(i, k, T), R), (och.tile_index(j, k, T), R),
                            (och.tile_index(i, j, T), RW)])
    assert ctx.dag_stats()[0] == len(acc)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc, parts)


def test_tiles_unregister_forgets_panel_parts(ctx):
    # a diagonal tile of b = 256 is split into two 128-column panels whose
    # second part is looked up by its own address; after the tiles are
    # unregistered a new buffer at that address must register afresh
    p = fake_ptr(0)
    ctx.cholesky_submit([p], 1, 256)
    with pytest.raises(b3t.B3TError) as e:      # host-only: the wait drops the batch, reports no device
        ctx.tiles_unregister([p], 1)
    assert e.value.code == b3t._lib.ENODEV
    part1 = p + 256 * 128 * 8
    ctx.cholesky_submit([part1], 1, 64)
    assert ctx.dag_stats()[0] == 1


@pytest.mark.parametrize("T", [1, 3, 6])
def test_inverse_solve_edges(ctx, T):
    # TRTRI per diagonal tile, then the solve with inverted diagonal tiles:
    # forward Z_k = U_k^T Y_k, Y_i -= L_ik Z_k; backward Y_k = U_k Z_k,
    # Z_i -= L_ki^T Y_k (Y and Z partitioned into T parts)
    b, nrhs = 128, 4
    L = [fake_ptr(i) for i in range(och.ntiles(T))]
    U = [fake_ptr(1000 + k) for k in range(T)]
    Y, Z = fake_ptr(2000), fake_ptr(3000)
    ctx.chol_inv_submit(L, U, T, b)
    ctx.chol_solve_inv_submit(L, U, Y, Z, T, b, nrhs, b * nrhs)
    ti = lambda i, j: och.tile_index(i, j, T)    # noqa: E731
    parts = {"Y": tuple(("Y", k) for k in range(T)), "Z": tuple(("Z", k) for k in range(T))}
    acc = [[(ti(k, k), R), (("U", k), W)] for k in range(T)]
    for k in range(T):
        acc.append([(("U", k), R), (("Y", k), R), (("Z", k), RW)])
        for i in range(k + 1, T):
            acc.append([(ti(i, k), R), (("Z", k), R), (("Y", i), RW)])
    for k in reversed(range(T)):
        acc.append([(("U", k), R), (("Z", k), R), (("Y", k), RW)])
        for i in range(k):
            acc.append([(ti(k, i), R), (("Y", k), R), (("Z", i), RW)])
    assert ctx.dag_stats()[0] == len(acc)
    assert sorted(ctx.dag_edges()) == dag.derive_edges(acc, parts)


def test_ir_work_elems_layout():
    # residual parts, a scratch block vector and T inverted tiles, each
    # region a multiple of 32 doubles from the start
    T, b, nrhs = 5, 128, 3
    part = b * nrhs + (b // 16) * (3 * nrhs + 1)      # 16-row residual items
    assert b3t.resid_part_elems(b, nrhs) == part
    r32 = lambda n: (n + 31) // 32 * 32    # noqa: E731
    assert b3t.ir_work_elems(T, b, nrhs) == r32(T * part) + r32(T * b * nrhs) + T * b * b
    assert b3t.ir_work_elems(T, 100, nrhs) == 0


def test_fan_out_fan_in_edges(ctx):
    # one writer of buffer 0, then readers of it that each update a buffer
    # of their own, repeated: each writer waits for every reader of the
    # round before (write after read), each reader for the writer
    nh, rounds = 17, 5
    acc = [a for _ in range(rounds) for a in [[(0, RW)]] + [[(0, R), (i, RW)] for i in range(1, nh)]]
    _submit_accesses(ctx, acc, nh)
    ed = sorted(ctx.dag_edges())
    assert ed == dag.derive_edges(acc)
    assert ctx.dag_stats() == (rounds * nh, (rounds - 1) * (nh - 1) * 3 + (nh - 1))


def test_bench_empty_dags_follow_the_oracle():
    # the scheduler-throughput DAGs: the Cholesky-shaped one submits the
    # oracle's accesses in the oracle's order; the others have the stated
    # task and edge counts under the oracle's rule
    import bench
    for shape, _ in bench.EMPTY_DAGS:
        modes, nh, nt, gen = bench.empty_dag(shape)
        acc = [[(h, modes[c][k]) for k, h in enumerate(bs)] for c, bs in gen()]
        assert len(acc) == nt and max(h for a in acc for h, _ in a) == nh - 1
        if shape == "cholesky":
            T = 64
            ref = [[(i * (i + 1) // 2 + j, m) for (i, j), m in a] for _, a in och.task_list(T)]
            assert acc == ref
            assert len(dag.derive_edges(acc)) == 131040


def test_bench_scipy_serving_sample():
    # the serving workload's library CPU baseline stops after its time
    # budget (here: after the first request) and reports what it sampled
    import bench
    r = bench.scipy_serving_sample(0.0, 4)
    assert r["solves_per_s"] > 0 and r["cores"] >= 1
    assert r["sample"].startswith("first 1 of the 4 served requests")


from hypothesis import given, settings, HealthCheck, strategies as st   # noqa: E402

_acc = st.lists(st.lists(st.tuples(st.sampled_from([0, 1, 2, 10, 11, 12]), st.sampled_from([R, W, RW])),
                         min_size=0, max_size=4), min_size=1, max_size=40)


@settings(max_examples=200, deadline=None, suppress_health_check=[HealthCheck.function_scoped_fixture])
@given(acc=_acc)
def test_edges_match_oracle_property(acc):
    # any task set, including buffers named twice by one task (modes OR-ed),
    # tasks without buffers, and a partitioned buffer named both whole and by
    # part: the library derives exactly the oracle's edges
    c = b3t.Context(host_only=True)
    try:
        hs = [c.data_register(fake_ptr(i), 64, 4) for i in range(3)]
        kids = c.data_partition(hs[0], 3, 16)
        lib_of = {0: hs[0], 1: hs[1], 2: hs[2], 10: kids[0], 11: kids[1], 12: kids[2]}
        cls = {}
        for a in acc:
            modes = tuple(m for _, m in a)
            if modes not in cls:
                cls[modes] = c.task_decl("t", b3t.NOOP, list(modes))
            c.task_submit(cls[modes], [lib_of[h] for h, _ in a])
        assert sorted(c.dag_edges()) == dag.derive_edges(acc, {0: (10, 11, 12)})
        assert c.dag_stats()[0] == len(acc)
    finally:
        c.close()


def test_bench_empty_dags_edge_counts(ctx):
    # the library derives the closed-form edge counts of the 1M-task shapes:
    # chains 1000 x 999; fan-out / fan-in: each writer after the first waits
    # for the 999 readers before it, each reader for its round's writer and
    # for its own buffer's previous reader
    import bench
    want = {"chains": 1000 * 999, "fan": 999 * 999 + 1000 * 999 + 999 * 999}
    for shape, n_edges in want.items():
        c = b3t.Context(host_only=True)
        modes, nh, nt, gen = bench.empty_dag(shape)
        hs = [c.data_register(fake_ptr(i), 16, 4) for i in range(nh)]
        cls = [c.task_decl("empty", b3t.NOOP, m) for m in modes]
        for k, bs in gen():
            c.task_submit(cls[k], [hs[h] for h in bs])
        assert c.dag_stats() == (nt, n_edges)
        c.close()


def test_bench_oracle_empty_dags_rates():
    import bench
    r = bench.oracle_empty_dags(0.0)
    assert set(r) == {"chains", "fan", "cholesky"}
    assert all(v["tasks_per_s"] > 0 and v["cores"] == 1 and v["kind"] == "oracle" for v in r.values())


def test_c_abi_from_plain_c(tmp_path):
    # include/b3t.h compiles as C99 with warnings as errors, and a C program
    # linked against libb3t.so declares, registers, submits by pointer and
    # reads the derived graph and the error codes (tests/c_abi_host.c)
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(b3t._lib.LIB_PATH)
    exe = str(tmp_path / "c_abi_host")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c_abi_host.c"), "-o", exe, "-L", libdir, "-lb3t",
                           "-Wl,-rpath," + libdir])
    out = subprocess.check_output([exe], text=True, timeout=60)
    assert out.strip() == "c abi ok"


# ---- scheduling priorities (Section 5.3: upward rank as a hint)

NOOP_COST = 1000.0   # the library's cost estimate of an empty task (ns)


def _levels_from_rank(rank, L=8):
    m = max(rank)
    return [min(L - 1, int(L * r / (m * 1.000001))) for r in rank]


@pytest.mark.parametrize("seed", range(12))
def test_upward_rank_is_longest_path(seed):
    rng = np.random.default_rng(700 + seed)
    n, nh = int(rng.integers(20, 120)), int(rng.integers(3, 12))
    acc = [[(int(h), int(rng.choice([R, W, RW])))
            for h in rng.choice(nh, size=int(rng.integers(1, 4)), replace=False)] for _ in range(n)]
    with b3t.Context(host_only=True, prio_policy=b3t.PRIO_UPWARD) as c:
        _submit_accesses(c, acc, nh)
        rank, level = c.dag_levels()
    edges = dag.derive_edges(acc)
    ref = dag.upward_rank(n, edges, [NOOP_COST] * n)
    assert rank == ref
    assert level == _levels_from_rank(ref)
    # with one level, the queue is FIFO (every task on level 0)
    with b3t.Context(host_only=True, prio_levels=1) as c:
        _submit_accesses(c, acc, nh)
        assert c.dag_levels()[1] == [0] * n


@pytest.mark.parametrize("seed", range(6))
def test_depth_policy_is_longest_path_from_sources(seed):
    rng = np.random.default_rng(800 + seed)
    n, nh = 60, 6
    acc = [[(int(h), int(rng.choice([R, W, RW])))
            for h in rng.choice(nh, size=int(rng.integers(1, 3)), replace=False)] for _ in range(n)]
    with b3t.Context(host_only=True, prio_policy=1) as c:
        _submit_accesses(c, acc, nh)
        rank, level = c.dag_levels()
    d = dag.depth(n, dag.derive_edges(acc))
    assert rank == [float(x) for x in d]
    assert level == [min(7, x) for x in d]


def _critical_levels(up, down, L=8):
    longest = max(up)
    return [L - 1 if d + u >= longest * (1 - 1e-9) else min(L - 2, int((L - 1) * u / (longest * 1.000001)))
            for u, d in zip(up, down)]


@pytest.mark.parametrize("seed", range(8))
def test_critical_policy_puts_the_longest_paths_on_top(seed):
    # critical path first (Section 5.3's upward and downward ranks): a task
    # whose longest path through it is the graph's longest path takes the
    # top level, the others the levels below by upward rank
    rng = np.random.default_rng(1000 + seed)
    n, nh = int(rng.integers(20, 120)), int(rng.integers(3, 12))
    acc = [[(int(h), int(rng.choice([R, W, RW])))
            for h in rng.choice(nh, size=int(rng.integers(1, 4)), replace=False)] for _ in range(n)]
    with b3t.Context(host_only=True, prio_policy=b3t.PRIO_CRITICAL) as c:
        _submit_accesses(c, acc, nh)
        rank, level = c.dag_levels()
    with b3t.Context(host_only=True) as c:          # the default policy
        _submit_accesses(c, acc, nh)
        assert c.dag_levels() == (rank, level)
    edges = dag.derive_edges(acc)
    cost = [NOOP_COST] * n
    up, down = dag.upward_rank(n, edges, cost), dag.downward_rank(n, edges, cost)
    assert rank == up
    assert level == _critical_levels(up, down)
    top = [t for t in range(n) if level[t] == 7]
    assert any(down[t] == 0 for t in top) and any(up[t] == NOOP_COST for t in top)


def test_critical_policy_on_the_cholesky_dag():
    # T = 8: the per-kind costs are read back from the ranks (rank minus the
    # largest successor rank); the top level is exactly the tasks on a
    # longest cost-weighted path
    T, b = 8, 64
    with b3t.Context(host_only=True, prio_policy=b3t.PRIO_CRITICAL) as c:
        c.cholesky_submit([fake_ptr(i) for i in range(T * (T + 1) // 2)], T, b)
        rank, level = c.dag_levels()
        edges = c.dag_edges()
        n = c.dag_stats()[0]
    succ = [[] for _ in range(n)]
    for p, s_ in edges:
        succ[p].append(s_)
    cost = [rank[t] - max((rank[s_] for s_ in succ[t]), default=0.0) for t in range(n)]
    up, down = dag.upward_rank(n, edges, cost), dag.downward_rank(n, edges, cost)
    assert np.allclose(rank, up, rtol=1e-6)
    assert level == _critical_levels(up, down)
    assert level[0] == 7 and level[n - 1] == 7      # POTRF(0) and the last POTRF


@pytest.mark.parametrize("T,cp", [(8, 22), (64, 190)])
def test_cholesky_upward_rank_follows_the_critical_path(T, cp):
    # tile kinds cost differently; the rank must still be the longest path of
    # per-task costs: rank(t) - max over successors is one constant per kind,
    # the ranks drop along every edge, POTRF(0) holds the largest, and
    # following the largest-ranked successor from it walks a path whose costs
    # add up to that rank.  With equal costs (the same accesses as empty
    # tasks) that walk is the closed-form critical path of 3T - 2 tasks.
    b = 64
    with b3t.Context(host_only=True, prio_policy=b3t.PRIO_UPWARD) as c:
        nt = T * (T + 1) // 2
        tiles = [fake_ptr(i) for i in range(nt)]
        c.cholesky_submit(tiles, T, b)
        rank, level = c.dag_levels()
        edges = c.dag_edges()
        n = c.dag_stats()[0]
    acc_kinds = [k for k, _ in och.task_list(T)]
    assert len(acc_kinds) == n
    succ = dag.successors(n, edges)
    own = {}
    for t in range(n):
        m = max((rank[s] for s in succ[t]), default=0.0)
        assert all(rank[t] > rank[s] for s in succ[t])
        own.setdefault(acc_kinds[t], []).append(rank[t] - m)
    # one cost per kind (the ranks are binary32: differences agree to ~1e-5)
    for k, v in own.items():
        assert max(v) - min(v) <= 2e-5 * max(rank), (k, min(v), max(v))
    kc = {k: float(np.mean(v)) for k, v in own.items()}
    cost = [kc[k] for k in acc_kinds]
    ref = dag.upward_rank(n, edges, cost)
    assert np.allclose(rank, ref, rtol=1e-5)
    assert int(np.argmax(rank)) == 0
    t, total = 0, cost[0]
    while succ[t]:
        t = max(succ[t], key=lambda s: rank[s])
        total += cost[t]
    assert total == pytest.approx(rank[0], rel=1e-5)
    assert level[0] == 7 and all(level[p] >= level[s] for p, s in edges)
    # equal costs: the same access pattern as empty tasks
    acc = och.accesses(T)
    tid = {tile: i for i, tile in enumerate(sorted({h for a in acc for h, _ in a}))}
    with b3t.Context(host_only=True) as c:
        _submit_accesses(c, [[(tid[h], m) for h, m in a] for a in acc], len(tid))
        rank_u, _ = c.dag_levels()
    t, steps = 0, 1
    while succ[t]:
        t = max(succ[t], key=lambda s: rank_u[s])
        steps += 1
    assert rank_u[0] == NOOP_COST * cp
    assert steps == cp == dag.critical_path(n, edges)


# ---- item chains (successor first at item granularity, Section 2)
def _chains_by_rule(kinds, bufs, edges, cap=32):
    """Item chains restated from the edge list: t links to s when both are
    vector-scaling tasks on one buffer, s is t's only successor and t is s's
    only predecessor; maximal runs of links are cut into chains of at most
    `cap` members after their head."""
    n = len(kinds)
    succ = [[] for _ in range(n)]
    npred = [0] * n
    for p, s in edges:
        succ[p].append(s)
        npred[s] += 1
    nxt = [-1] * n
    for t in range(n):
        if kinds[t] == "scal" and len(succ[t]) == 1:
            s = succ[t][0]
            if kinds[s] == "scal" and npred[s] == 1 and bufs[s] == bufs[t]:
                nxt[t] = s
    linked = {s for s in nxt if s >= 0}
    aux = [0] * n
    for t in range(n):
        if nxt[t] < 0 or t in linked:
            continue
        h = t
        while h >= 0 and nxt[h] >= 0:
            mem, m = [], nxt[h]
            while m >= 0 and len(mem) < cap:
                mem.append(m)
                m = nxt[m]
            aux[h] = len(mem)
            for x in mem:
                aux[x] = -1
            h = m
    return aux


@pytest.mark.parametrize("seed", range(6))
def test_item_chains_follow_the_rule(seed):
    # random mixes of RW scaling tasks and R / W / RW empty tasks on four
    # buffers, with long runs so that some chains are cut at 32 members
    rng = np.random.default_rng(seed)
    nb = 4
    kinds, bufs, accesses = [], [], []
    for _ in range(int(rng.integers(60, 160))):
        h = int(rng.integers(nb))
        r = rng.random()
        if r < 0.8:
            kinds.append("scal"); accesses.append([(h, RW)])
        else:
            kinds.append("noop"); accesses.append([(h, [R, W, RW][int(rng.integers(3))])])
        bufs.append(h)
    edges = dag.derive_edges(accesses)
    with b3t.Context(host_only=True, item_chains=True) as c:
        hs = [c.data_register(fake_ptr(i), 1 << 18, 4) for i in range(nb)]
        cs = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
        cn = {m: c.task_decl("t", b3t.NOOP, [m]) for m in (R, W, RW)}
        for k, acc in zip(kinds, accesses):
            h, m = acc[0]
            if k == "scal":
                c.task_submit(cs, [hs[h]], b3t.pack_f32(1.5))
            else:
                c.task_submit(cn[m], [hs[h]])
        assert sorted(c.dag_edges()) == sorted(edges)
        got = c.dag_item_chains()
    assert got == _chains_by_rule(kinds, bufs, edges)
    # with item chains off nothing is chained
    with b3t.Context(host_only=True) as c:
        hs = [c.data_register(fake_ptr(i), 1 << 18, 4) for i in range(nb)]
        cs = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
        for _ in range(5):
            c.task_submit(cs, [hs[0]], b3t.pack_f32(2.0))
        assert c.dag_item_chains() == [0] * 5


def test_item_chains_of_the_vector_configuration():
    # 256 blocks of 2^20 floats with 8 chained scaling tasks each form 256
    # chains: every block's first task heads its 7 successors
    with b3t.Context(host_only=True, item_chains=True) as c:
        cs = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
        hs = [c.data_register(fake_ptr(i), 1 << 20, 4) for i in range(256)]
        for k in range(8):
            for h in hs:
                c.task_submit(cs, [h], b3t.pack_f32(1.0))
        aux = c.dag_item_chains()
    assert aux[:256] == [7] * 256 and aux[256:] == [-1] * (7 * 256)


def test_item_chains_stay_off_beside_mixed_precision_kinds():
    # the tensor-memory kernel variant runs SCAL items through registers, not
    # the bulk-copy ring that applies a chain's factors: a batch that also
    # holds a mixed-precision factorisation forms no item chains
    T, b = 2, 128
    nt = och.ntiles(T)
    with b3t.Context(host_only=True, item_chains=True) as c:
        hs = [c.data_register(fake_ptr(3000 + i), 1 << 18, 4) for i in range(2)]
        cl = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
        for k in range(4):
            for h in hs:
                c.task_submit(cl, [h], b3t.pack_f32(2.0))
        assert c.dag_item_chains()[:2] == [3, 3]
        c.cholesky_mx_submit([fake_ptr(i) for i in range(nt)], [fake_ptr(100 + i) for i in range(nt)],
                             [fake_ptr(200 + i) for i in range(nt)], T, b, b3t.FMT_BF16)
        assert set(c.dag_item_chains()) == {0}
