"""Device executor against the oracle (GPU).  Every result is compared with
the sequential oracle run on the same seeded inputs: bit-exact for the
vector chains and integer-exact Cholesky, within a stated FP64 tolerance
otherwise (the device sums in another order and with FMA)."""
import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och, executor as oex, tiles as otl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]
R, W, RW = 1, 2, 3
FP64_TOL = 1e-12     # max |L_gpu - L_orc| / max |L_orc|


def run_chain_device(ctx, x, f, order="k"):
    nb, nk = f.shape
    n = x.size // nb
    xd = torch.from_numpy(x.copy()).cuda()
    blocks = [xd[i * n:(i + 1) * n] for i in range(nb)]
    hs = [ctx.data_register(bl.data_ptr(), n, 4) for bl in blocks]
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    seq = [(k, i) for k in range(nk) for i in range(nb)] if order == "k" else \
          [(k, i) for i in range(nb) for k in range(nk)]
    for k, i in seq:
        ctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
    ctx.task_wait()
    for h in hs:
        ctx.data_unregister(h)
    return xd.cpu().numpy()


def run_chain_oracle(x, f):
    nb, nk = f.shape
    n = x.size // nb
    y = x.copy()
    ex = oex.Executor()
    cl = ex.task_decl("scale_vector", oex.scal_body, [RW])
    hs = [ex.data_register(y[i * n:(i + 1) * n]) for i in range(nb)]
    for k in range(nk):
        for i in range(nb):
            ex.task_submit(cl, [hs[i]], scalars=(f[i, k],))
    return y


@pytest.mark.parametrize("nb,n,order", [(16, (1 << 16) + 4, "k"), (8, 3 * (1 << 16) + 12, "b"),
                                        (5, 1000, "k")])
def test_scal_chains_bit_exact(orc, gctx, nb, n, order):
    x = synth.vector_f32(nb * n, seed=1)
    x[:7] = np.array([1e-38, -3e-39, 5e-45, 0.0, -0.0, 3e38, -1.0], dtype=np.float32)
    f = synth.chain_factors(nb, 8, seed=2)
    y = run_chain_device(gctx, x, f, order)
    z = run_chain_oracle(x, f)
    assert np.array_equal(y.view(np.uint32), z.view(np.uint32))


@pytest.mark.parametrize("nb,n", [(8, 3 * (1 << 14) + 12), (4, (1 << 16) + 12), (1, 2 * (1 << 14) + 7)])
def test_scal_chains_successor_first_bit_exact(orc, nb, n):
    # under the successor-first order (a block's next task is claimed before
    # other blocks' first tasks) with a ragged last item, and a single block
    # with a tail of fewer than four elements (blocks start 16-byte aligned,
    # as submission requires): still exactly the in-order binary32 multiplies
    c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000,
                    prio_policy=b3t.PRIO_DEPTH)
    x = synth.vector_f32(nb * n, seed=21)
    x[:5] = np.array([1e-38, -3e-39, 5e-45, -0.0, 3e38], dtype=np.float32)
    f = synth.chain_factors(nb, 8, seed=22)
    y = run_chain_device(c, x, f, "b")
    c.close()
    z = run_chain_oracle(x, f)
    assert np.array_equal(y.view(np.uint32), z.view(np.uint32))


def test_scal_full_size_config(orc, gctx):
    # n = 2^28, 256 blocks x 8 chained tasks: compared element-wise against
    # in-order binary32 multiplies on sampled blocks (the whole vector fits
    # the oracle only slowly)
    nb, nk, n = 256, 8, 1 << 20
    x = synth.vector_f32(nb * n, seed=1)
    f = synth.chain_factors(nb, nk, seed=2)
    y = run_chain_device(gctx, x, f)
    for i in [0, 1, 77, 128, 255]:
        z = x[i * n:(i + 1) * n].copy()
        for k in range(nk):
            otl.scal_f32(z, f[i, k])
        assert np.array_equal(y[i * n:(i + 1) * n].view(np.uint32), z.view(np.uint32))


def factor_device(ctx, A, b, col0=0):
    N = A.shape[0]
    T = N // b
    t = torch.from_numpy(och.to_tiles(A, b)).cuda()
    ptrs = dt.tile_ptrs(t)
    ctx.cholesky_submit(ptrs, T, b, col0)
    ctx.task_wait()
    ctx.tiles_unregister(ptrs, T)
    return np.tril(och.from_tiles(t.cpu().numpy(), N, b))


def factor_oracle(A, b):
    N = A.shape[0]
    t = och.to_tiles(A, b)
    info = och.run(t, N // b, b)
    assert info == 0
    return np.tril(och.from_tiles(t, N, b))


@pytest.mark.parametrize("N,b", [(256, 64), (512, 128), (576, 192), (1024, 256)])
def test_cholesky_integer_exact(orc, gctx, N, b):
    A, L0 = synth.integer_spd(N, seed=N + b)
    L = factor_device(gctx, A, b)
    assert np.array_equal(L, L0)


@pytest.mark.parametrize("panels", [True, False])
def test_cholesky_config1_parity(orc, gctx, monkeypatch, panels):
    # N = 1024, tile 128 (8 x 8 tiles, 120 tile tasks), A = B B^T / N + I,
    # seed 0.  By default each diagonal POTRF runs as a DAG of 64-wide
    # panels (POTRF_D, PANEL_TRSM, PANEL_UPD, POTRF_D: 144 device tasks);
    # with the panels off, one POTRF task per diagonal tile (120)
    if not panels:
        monkeypatch.setenv("B3T_PANEL_WIDTH", "0")
    A = synth.spd_host(1024, seed=0, shift=1.0)
    L = factor_device(gctx, A, 128)
    Lo = factor_oracle(A, 128)
    assert np.max(np.abs(L - Lo)) / np.max(np.abs(Lo)) <= FP64_TOL
    assert och.rel_residual(L, A) <= 1e-12
    st = gctx.last_launch()
    assert st["ntasks"] == (144 if panels else 120)


@pytest.mark.parametrize("N,b", [(320, 64), (1536, 512)])
def test_cholesky_other_tiles(orc, gctx, N, b):
    A = synth.spd_host(N, seed=3, shift=0.1)
    L = factor_device(gctx, A, b)
    Lo = factor_oracle(A, b)
    assert np.max(np.abs(L - Lo)) / np.max(np.abs(Lo)) <= FP64_TOL
    assert och.rel_residual(L, A) <= 1e-12


@pytest.mark.parametrize("N,b", [(512, 128), (1024, 256)])
def test_cholesky_64_wide_panels(orc, gctx, monkeypatch, N, b):
    # diagonal tiles as 64-wide column panels: the 64 x 64 POTRF_D blocks
    # take the pipelined right-looking factorisation (a chain of two warps,
    # the trailing columns on four more)
    monkeypatch.setenv("B3T_PANEL_WIDTH", "64")
    A, L0 = synth.integer_spd(N, seed=N + b + 64)
    assert np.array_equal(factor_device(gctx, A, b), L0)
    A = synth.spd_host(N, seed=5, shift=0.1)
    L = factor_device(gctx, A, b)
    Lo = factor_oracle(A, b)
    assert np.max(np.abs(L - Lo)) / np.max(np.abs(Lo)) <= FP64_TOL
    assert och.rel_residual(L, A) <= 1e-12
    outs = [factor_device(gctx, A, b) for _ in range(2)]
    assert np.array_equal(outs[0], L) and np.array_equal(outs[1], L)
    # a pivot that fails inside a 64-wide panel is reported at its column
    A[300, 300] = -10.0
    with pytest.raises(b3t.B3TError) as e:
        factor_device(gctx, A, b, col0=0)
    assert e.value.code == b3t._lib.EDOM
    t = och.to_tiles(A, b)
    assert och.run(t, N // b, b) == gctx.last_error()[1] == 301


def test_cholesky_deterministic(orc, gctx):
    A = synth.spd_host(768, seed=8, shift=1.0)
    outs = [factor_device(gctx, A, 128) for _ in range(3)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_not_spd_reports_info(orc, gctx):
    A = synth.spd_host(512, seed=4, shift=1.0)
    A[300, 300] = -10.0
    with pytest.raises(b3t.B3TError) as e:
        factor_device(gctx, A, 128, col0=0)
    assert e.value.code == b3t._lib.EDOM
    task, info = gctx.last_error()
    # the oracle stops at the same column
    t = och.to_tiles(A, 128)
    assert och.run(t, 4, 128) == info == 301
    # the context stays usable
    A2, L0 = synth.integer_spd(256, seed=1)
    assert np.array_equal(factor_device(gctx, A2, 64), L0)


def test_single_tasks_against_oracle(orc, gctx):
    rng = np.random.default_rng(7)
    b = 128
    M = rng.standard_normal((b, b))
    Lk = np.tril(M) + b * np.eye(b)
    A = rng.standard_normal((b, b))
    B = rng.standard_normal((b, b))
    C = rng.standard_normal((b, b))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v.T)).cuda() for k, v in
           dict(L=Lk, A=A, B=B, C=C, S=C.copy()).items()}
    h = {k: gctx.data_register(v.data_ptr(), b * b, 8, b) for k, v in dev.items()}
    ct = gctx.task_decl("trsm", b3t.TRSM, [R, RW])
    cg = gctx.task_decl("gemm", b3t.GEMM, [R, R, RW])
    cs = gctx.task_decl("syrk", b3t.SYRK, [R, RW])
    gctx.task_submit(cg, [h["A"], h["B"], h["C"]])
    gctx.task_submit(cs, [h["A"], h["S"]])
    gctx.task_submit(ct, [h["L"], h["A"]])     # after GEMM / SYRK read A (WAR)
    gctx.task_wait()
    got = {k: v.cpu().numpy().T for k, v in dev.items()}
    X = np.asfortranarray(A.copy()); otl.trsm(np.asfortranarray(Lk), X)
    Cg = np.asfortranarray(C.copy()); otl.gemm(np.asfortranarray(A), np.asfortranarray(B), Cg)
    Cs = np.asfortranarray(C.copy()); otl.syrk(np.asfortranarray(A), Cs)
    assert np.max(np.abs(got["A"] - X)) <= 1e-13 * np.max(np.abs(X))
    assert np.max(np.abs(got["C"] - Cg)) <= 1e-13 * np.max(np.abs(Cg))
    assert np.max(np.abs(np.tril(got["S"]) - np.tril(Cs))) <= 1e-13 * np.max(np.abs(Cs))
    assert np.array_equal(np.triu(got["S"], 1), np.triu(C, 1))   # upper untouched


def test_graph_capture_replay(orc, gctx):
    N, b = 512, 128
    T = N // b
    A = synth.spd_host(N, seed=11, shift=1.0)
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    t = At.clone()
    ptrs = dt.tile_ptrs(t)
    gctx.graph_capture_begin()
    gctx.cholesky_submit(ptrs, T, b)
    g = gctx.graph_capture_end()
    outs = []
    for _ in range(3):
        t.copy_(At)
        gctx.graph_replay(g)
        gctx.task_wait()
        outs.append(np.tril(och.from_tiles(t.cpu().numpy(), N, b)))
    ref = factor_device(gctx, A, b)
    for o in outs:
        assert np.array_equal(o, ref)
    gctx.graph_destroy(g)


def test_timeout_is_bounded_and_recoverable(orc):
    # a task whose dependency counter never reaches zero: the launch must end
    # through the device-side timeout, and the context must stay usable
    c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=50_000_000)
    x = torch.ones(1 << 16, device="cuda")
    h = c.data_register(x.data_ptr(), x.numel(), 4)
    cl = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    c.task_submit(cl, [h], b3t.pack_f32(2.0))
    c.task_submit(cl, [h], b3t.pack_f32(2.0))
    c.debug_block_task(1)
    with pytest.raises(b3t.B3TError) as e:
        c.task_wait()
    assert e.value.code == b3t._lib.ETIMEDOUT
    assert float(x[0]) == 2.0             # the first task ran, the second never
    c.task_submit(cl, [h], b3t.pack_f32(3.0))
    c.task_wait()
    assert float(x[-1]) == 6.0
    c.close()


def test_noop_dags_and_partitions(orc, gctx):
    # many tiny tasks: chains, fan-out / fan-in through a partitioned buffer
    x = torch.zeros(1 << 12, device="cuda")
    hp = gctx.data_register(x.data_ptr(), x.numel(), 4)
    parts = gctx.data_partition(hp, 64, 64)
    c1 = gctx.task_decl("touch", b3t.NOOP, [RW])
    call = gctx.task_decl("all", b3t.NOOP, [R])
    for rep in range(20):
        for p in parts:
            gctx.task_submit(c1, [p])
        gctx.task_submit(call, [hp])
    nt, ne = gctx.dag_stats()
    assert nt == 20 * 65
    gctx.task_wait()
    assert gctx.last_launch()["ntasks"] == nt


def test_trace_records_every_item(gctx):
    # one record per finished work item: every (task, item) exactly once,
    # start <= end, kinds as submitted
    T, b = 4, 128
    A = torch.from_numpy(och.to_tiles(synth.spd_host(T * b, seed=11, shift=1.0), b)).cuda()
    gctx.trace_start(1 << 14)
    gctx.cholesky_submit(dt.tile_ptrs(A), T, b)
    gctx.task_wait()
    tr = gctx.trace_read()
    gctx.trace_stop()
    ntasks, nitems = gctx.last_launch()["ntasks"], gctx.last_launch()["nitems"]
    assert len(tr) == nitems
    pairs = set(zip(tr["task"].tolist(), tr["item"].tolist()))
    assert len(pairs) == nitems and {t for t, _ in pairs} == set(range(ntasks))
    assert np.all(tr["t_end_ns"] >= tr["t_start_ns"])
    assert set(tr["kind"].tolist()) <= {b3t.POTRF, b3t.TRSM, b3t.SYRK, b3t.GEMM, b3t.POTRF_D, b3t.PANEL_TRSM,
                                        b3t.PANEL_UPD}


def test_kernel_variant_covers_mixed_launch(orc, gctx):
    # one launch holding vector-scaling chains and a tiled Cholesky runs the
    # variant compiled with both families; each part matches the oracle.  The
    # grid shows the variant: three CTAs per SM for vector tasks alone, two
    # for a launch with FP64 tile tasks or with empty tasks only.
    import oracle
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, nb = 1 << 16, 3
    x = synth.vector_f32(nb * n, seed=3)
    f = synth.chain_factors(nb, 4, seed=4)
    xd = torch.from_numpy(x.copy()).cuda()
    hs = [gctx.data_register(xd[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
    cl = gctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    for k in range(4):
        for i in range(nb):
            gctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
    gctx.task_wait()
    assert gctx.last_launch()["nctas"] == 3 * sms          # vector variant alone
    N, b = 384, 128
    A = synth.spd_host(N, seed=9, shift=1.0)
    t = torch.from_numpy(och.to_tiles(A, b)).cuda()
    for k in range(4):
        for i in range(nb):
            gctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
    gctx.cholesky_submit(dt.tile_ptrs(t), N // b, b)
    gctx.task_wait()
    assert gctx.last_launch()["nctas"] == 2 * sms          # vector + FP64 tiles
    y = x.copy()
    for _ in range(2):
        for k in range(4):
            for i in range(nb):
                oracle.tiles.scal_f32(y[i * n:(i + 1) * n], f[i, k])
    assert np.array_equal(xd.cpu().numpy().view(np.uint32), y.view(np.uint32))
    L = np.tril(och.from_tiles(t.cpu().numpy(), N, b))
    to = och.to_tiles(A, b)
    assert och.run(to, N // b, b) == 0
    Lo = np.tril(och.from_tiles(to, N, b))
    assert np.max(np.abs(L - Lo)) / np.max(np.abs(Lo)) <= 1e-12
    cn = gctx.task_decl("noop", b3t.NOOP, [RW])
    gctx.task_submit(cn, [hs[0]])
    gctx.task_wait()
    assert gctx.last_launch()["nctas"] == 2 * sms          # empty tasks only


@pytest.mark.parametrize("shape", ["random", "fan", "cholesky"])
def test_execution_order_respects_every_edge(orc, gctx, shape):
    # The order the persistent kernel ran the tasks in is one the DAG allows
    # (Section 3: any order that keeps each access's predecessors first
    # gives the sequential program's result).  From the trace (the device's
    # global nanosecond timer): every task's first item started no earlier
    # than the last item of each of its predecessors ended.  The edges are
    # the oracle's, derived from the same accesses.
    from oracle import dag
    if shape == "cholesky":
        T, b = 6, 64      # one task per tile (from b = 128 the diagonal POTRF is a panel DAG)
        A = torch.from_numpy(och.to_tiles(synth.spd_host(T * b, seed=13, shift=1.0), b)).cuda()
        gctx.trace_start(1 << 16)
        gctx.cholesky_submit(dt.tile_ptrs(A), T, b)
        acc = och.accesses(T)
    else:
        if shape == "random":
            nh = 12
            acc = synth.random_accesses(3000, nhandles=nh, maxbuf=3, seed=77)
        else:
            # 20 rounds: one writer of buffer 0, then 63 readers of it that
            # each update a buffer of their own
            nh = 64
            acc = [a for _ in range(20) for a in [[(0, RW)]] + [[(0, R), (i, RW)] for i in range(1, nh)]]
        x = torch.zeros(nh * 64, device="cuda")
        hs = [gctx.data_register(x[i * 64:(i + 1) * 64].data_ptr(), 64, 4) for i in range(nh)]
        cls = {}
        gctx.trace_start(1 << 16)
        for a in acc:
            modes = tuple(m for _, m in a)
            if modes not in cls:
                cls[modes] = gctx.task_decl("empty", b3t.NOOP, list(modes))
            gctx.task_submit(cls[modes], [hs[h] for h, _ in a])
    edges = dag.derive_edges(acc)
    assert sorted(gctx.dag_edges()) == edges
    gctx.task_wait()
    tr = gctx.trace_read()
    gctx.trace_stop()
    ntasks = gctx.last_launch()["ntasks"]
    assert ntasks == len(acc) and len(tr) == gctx.last_launch()["nitems"]
    from paper_1304_0878_b300 import trace
    start, end = trace.task_spans(tr, ntasks)
    e = np.array(edges, dtype=np.int64).reshape(-1, 2)
    bad = np.nonzero(end[e[:, 0]] > start[e[:, 1]])[0]
    assert bad.size == 0, [(tuple(e[k]), int(end[e[k, 0]]), int(start[e[k, 1]])) for k in bad[:5]]
    if shape == "cholesky":
        L = np.tril(och.from_tiles(A.cpu().numpy(), T * b, b))
        Lo, info = och.dense_potrf(synth.spd_host(T * b, seed=13, shift=1.0))
        assert info == 0
        assert np.max(np.abs(L - np.tril(Lo))) / np.max(np.abs(Lo)) <= FP64_TOL
    else:
        for h in hs:
            gctx.data_unregister(h)


def test_acquire_makes_the_writers_result_visible(orc, gctx):
    # Section 3.4 (acquire): after acquire(h, R) returns, the host may read
    # the buffer.  A chain of 64 SCAL tasks per block keeps the device busy
    # for milliseconds; acquire is the only wait: right after it the
    # context's stream has nothing left to run, and the values are the
    # oracle's, bit for bit.
    nb, n, nk = 8, 1 << 18, 64
    x = synth.vector_f32(nb * n, seed=41)
    f = synth.chain_factors(nb, nk, seed=42)
    xd = torch.from_numpy(x.copy()).cuda()
    torch.cuda.synchronize()
    hs = [gctx.data_register(xd[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
    cl = gctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    for k in range(nk):
        for i in range(nb):
            gctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
    gctx.task_flush()
    gctx.data_acquire(hs[3], R)
    assert torch.cuda.current_stream().query()
    y = run_chain_oracle(x, f)
    got = xd[3 * n:4 * n].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), y[3 * n:4 * n].view(np.uint32))
    gctx.data_acquire(hs[5], RW)
    for h in hs:
        gctx.data_unregister(h)


# ---- item chains: successor first at item granularity (Section 2)
def run_chain_items(x, f, n, extra=None, trace=False):
    """Chains of scaling tasks (block-major submission) with item chains on;
    extra(ctx, hs) may submit more tasks in between.  Returns the result and
    the context's chain layout (and the trace when asked)."""
    nb, nk = f.shape
    c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000, item_chains=True)
    if trace:
        c.trace_start(1 << 16)      # before the submissions (a start waits for pending work)
    xd = torch.from_numpy(x.copy()).cuda()
    hs = [c.data_register(xd[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
    cl = c.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    for k in range(nk):
        for i in range(nb):
            c.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
            if extra:
                extra(c, hs, k, i)
    aux = c.dag_item_chains()
    ed = c.dag_edges()
    c.task_wait()
    tr = c.trace_read() if trace else None
    ll = c.last_launch()
    if trace:
        c.trace_stop()
    c.close()
    return xd.cpu().numpy(), aux, ed, tr, ll


@pytest.mark.parametrize("nb,n,nk", [(16, 3 * (1 << 16) + 12, 8), (3, 1000, 8), (4, (1 << 16) + 4, 40)])
def test_item_chains_bit_exact(orc, nb, n, nk):
    # each chunk takes every factor of its chain in order, one rounding each:
    # the oracle's in-order binary32 multiplies, bit for bit; a ragged last
    # item, tasks of one item, and runs of 40 cut into chains of 32 and 7
    x = synth.vector_f32(nb * n, seed=41)
    x[:7] = np.array([1e-38, -3e-39, 5e-45, 0.0, -0.0, 3e38, -1.0], dtype=np.float32)
    f = synth.chain_factors(nb, nk, seed=42)
    y, aux, _, _, _ = run_chain_items(x, f, n)
    heads = [a for a in aux if a > 0]
    assert len(heads) == nb * ((nk - 1 + 32) // 33 if nk > 33 else 1)
    assert sum(heads) + len(heads) == nb * nk
    z = run_chain_oracle(x, f)
    assert np.array_equal(y.view(np.uint32), z.view(np.uint32))


def test_item_chains_tail_of_a_single_block(orc):
    # one block whose length is not a multiple of four (elements after the
    # last full 16 bytes are scaled by the threads, not the bulk copies)
    n = 2 * (1 << 16) + 7
    x = synth.vector_f32(n, seed=43)
    f = synth.chain_factors(1, 8, seed=44)
    y, aux, _, _, _ = run_chain_items(x, f, n)
    assert aux[0] == 7
    assert np.array_equal(y.view(np.uint32), run_chain_oracle(x, f).view(np.uint32))


def test_item_chains_break_at_readers_and_release_successors(orc):
    # an empty task reading block 1 after step 3 ends that block's chain
    # (the reader must see the step-3 result) and a new chain starts after
    # it; every reader and the tasks after the chains run after them
    nb, n, nk = 4, (1 << 16) + 4, 8
    x = synth.vector_f32(nb * n, seed=45)
    f = synth.chain_factors(nb, nk, seed=46)
    cr = {}

    def extra(c, hs, k, i):
        if i == 1 and k == 3:
            if "r" not in cr:
                cr["r"] = c.task_decl("reader", b3t.NOOP, [R])
            c.task_submit(cr["r"], [hs[1]])
    y, aux, ed, tr, ll = run_chain_items(x, f, n, extra, trace=True)
    assert sum(1 for a in aux if a > 0) == nb + 1
    assert np.array_equal(y.view(np.uint32), run_chain_oracle(x, f).view(np.uint32))
    # the trace holds every (task, item) once; the edges that no chain
    # absorbed are respected task by task, the absorbed ones item by item
    assert len(tr) == ll["nitems"]
    pairs = set(zip(tr["task"].tolist(), tr["item"].tolist()))
    assert len(pairs) == ll["nitems"]
    member = {i for i, a in enumerate(aux) if a == -1}
    st = {}
    for t, it, s0, e0 in zip(tr["task"].tolist(), tr["item"].tolist(), tr["t_start_ns"].tolist(),
                             tr["t_end_ns"].tolist()):
        st[(t, it)] = (s0, e0)
    ntask = len(aux)
    ts = [min(v[0] for k, v in st.items() if k[0] == t) for t in range(ntask)]
    te = [max(v[1] for k, v in st.items() if k[0] == t) for t in range(ntask)]
    for p, s in ed:
        if s in member:
            items = [k[1] for k in st if k[0] == s]
            assert all(st[(s, it)][0] >= st[(p, it)][0] for it in items)
        else:
            assert te[p] <= ts[s], (p, s)


def test_item_chains_full_size_config(orc):
    # n = 2^28, 256 blocks x 8 chained tasks with item chains: sampled blocks
    # against in-order binary32 multiplies
    nb, nk, n = 256, 8, 1 << 20
    x = synth.vector_f32(nb * n, seed=1)
    f = synth.chain_factors(nb, nk, seed=2)
    y, aux, _, _, _ = run_chain_items(x, f, n)
    assert aux[:nb] == [7] * nb
    for i in [0, 1, 77, 128, 255]:
        z = x[i * n:(i + 1) * n].copy()
        for k in range(nk):
            otl.scal_f32(z, f[i, k])
        assert np.array_equal(y[i * n:(i + 1) * n].view(np.uint32), z.view(np.uint32))


def test_results_do_not_depend_on_the_queue_policy(orc):
    # the ready-queue order (critical path first, upward-rank buckets, depth)
    # changes when tasks run, never what they compute: the N = 1024
    # factorisation is bitwise the same under each, and the vector chains
    # too with item chains on or off
    A = synth.spd_host(1024, seed=0, shift=1.0)
    outs = []
    for pol in (b3t.PRIO_CRITICAL, b3t.PRIO_UPWARD, b3t.PRIO_DEPTH):
        c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000,
                        prio_policy=pol)
        outs.append(factor_device(c, A, 128))
        c.close()
    assert all(np.array_equal(o, outs[0]) for o in outs[1:])
    nb, n = 6, (1 << 16) + 4
    x = synth.vector_f32(nb * n, seed=47)
    f = synth.chain_factors(nb, 8, seed=48)
    ys = []
    for pol in (b3t.PRIO_CRITICAL, b3t.PRIO_UPWARD, b3t.PRIO_DEPTH):
        c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000,
                        prio_policy=pol)
        ys.append(run_chain_device(c, x, f, "b"))
        c.close()
    ys.append(run_chain_items(x, f, n)[0])
    z = run_chain_oracle(x, f)
    assert all(np.array_equal(y.view(np.uint32), z.view(np.uint32)) for y in ys)
