"""Stream mode (continuous submission into one resident kernel) on the GPU:
batches submitted while earlier ones run give the same results, bit for
bit, as the same work run alone; a failing request fails alone; waits are
bounded."""
import time

import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och, tiles as otl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]
RW = 3


_streams = []


def new_ctx(timeout_ns=20_000_000_000):
    # stream mode keeps a kernel resident on the context's stream for the
    # whole session: give it a stream of its own, so that torch's own work
    # (allocations, copies) on the current stream does not queue behind it
    s = torch.cuda.Stream()
    _streams.append(s)
    return b3t.Context(stream=s.cuda_stream, timeout_ns=timeout_ns)


def wait_batches(ctx, ids, limit_s=60.0):
    t0 = time.time()
    out = {}
    while len(out) < len(ids):
        for i in ids:
            if i not in out:
                done, info = ctx.stream_query(i)
                if done:
                    out[i] = info
        assert time.time() - t0 < limit_s, "batches did not finish"
        time.sleep(0.0005)
    return out


def factor_alone(A, b):
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    t = torch.from_numpy(och.to_tiles(A, b)).cuda()
    p = dt.tile_ptrs(t)
    ctx.cholesky_submit(p, A.shape[0] // b, b)
    ctx.task_wait()
    ctx.close()
    return t.cpu().numpy()


def test_stream_chains_bit_exact(orc):
    ctx = new_ctx()
    ctx.stream_open(1 << 16, 1 << 16, 64, 60_000_000_000)
    nb, n = 8, (1 << 16) + 8
    x = synth.vector_f32(nb * n, seed=3)
    f = synth.chain_factors(nb, 8, seed=4)
    xd = torch.from_numpy(x.copy()).cuda()
    hs = [ctx.data_register(xd[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    ids = []
    for i in range(nb):                        # one batch per chain
        for k in range(8):
            ctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
        ids.append(ctx.stream_submit())
    wait_batches(ctx, ids)
    ctx.stream_close()
    y = x.copy()
    for i in range(nb):
        for k in range(8):
            otl.scal_f32(y[i * n:(i + 1) * n], f[i, k])
    assert np.array_equal(xd.cpu().numpy().view(np.uint32), y.view(np.uint32))
    ctx.close()


def test_stream_mix_equals_alone(orc):
    sizes = [(512, 128), (768, 256), (384, 128), (1024, 256), (256, 64)]
    mats = [synth.spd_host(N, seed=40 + k, shift=1.0) for k, (N, b) in enumerate(sizes)]
    alone = [factor_alone(A, b) for A, (N, b) in zip(mats, sizes)]
    ctx = new_ctx()
    ctx.stream_open(1 << 18, 1 << 20, 64, 60_000_000_000)
    tiles = [torch.from_numpy(och.to_tiles(A, b)).cuda() for A, (N, b) in zip(mats, sizes)]
    ids = []
    for t, (N, b) in zip(tiles, sizes):       # each arrives while the earlier run
        ctx.cholesky_submit(dt.tile_ptrs(t), N // b, b)
        ids.append(ctx.stream_submit())
    infos = wait_batches(ctx, ids)
    ctx.stream_close()
    assert all(v == 0 for v in infos.values())
    for t, ref in zip(tiles, alone):
        assert np.array_equal(t.cpu().numpy(), ref)
    ctx.close()


def test_stream_failing_request_fails_alone(orc):
    ctx = new_ctx()
    ctx.stream_open(1 << 16, 1 << 18, 16, 60_000_000_000)
    good = synth.spd_host(512, seed=1, shift=1.0)
    bad = synth.spd_host(512, seed=2, shift=1.0)
    bad[300, 300] = -5.0
    tg = torch.from_numpy(och.to_tiles(good, 128)).cuda()
    tb = torch.from_numpy(och.to_tiles(bad, 128)).cuda()
    ctx.cholesky_submit(dt.tile_ptrs(tb), 4, 128, 1000)
    i_bad = ctx.stream_submit()
    ctx.cholesky_submit(dt.tile_ptrs(tg), 4, 128)
    i_good = ctx.stream_submit()
    infos = wait_batches(ctx, [i_bad, i_good])
    ctx.stream_close()
    assert infos[i_bad] == 1000 + 301 and infos[i_good] == 0
    assert np.array_equal(tg.cpu().numpy(), factor_alone(good, 128))
    ctx.close()


def test_stream_busy_buffer_and_deadline(orc):
    # batch 0 can never finish (phantom dependency), so a batch naming its
    # buffer is refused, and the resident kernel ends at its deadline
    ctx = new_ctx(timeout_ns=100_000_000)
    ctx.stream_open(1024, 1024, 8, 1_000_000_000)
    x = torch.ones(1 << 12, device="cuda")
    h = ctx.data_register(x.data_ptr(), x.numel(), 4)
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    ctx.task_submit(cl, [h], b3t.pack_f32(2.0))
    ctx.debug_block_task(0)
    b0 = ctx.stream_submit()
    ctx.task_submit(cl, [h], b3t.pack_f32(2.0))
    with pytest.raises(b3t.B3TError) as e:
        ctx.stream_submit()
    assert e.value.code == b3t._lib.EBUSY
    t0 = time.time()
    with pytest.raises(b3t.B3TError) as e:
        ctx.stream_close()
    assert e.value.code == b3t._lib.ETIMEDOUT and time.time() - t0 < 30
    ctx.close()


def test_stream_without_tensor_memory(orc):
    # an FP64-only stream runs the resident kernel without the tensor-memory
    # path (two CTAs per SM): factorisations in it equal the same work alone
    sizes = [(512, 128), (768, 256), (384, 128)]
    mats = [synth.spd_host(N, seed=60 + k, shift=1.0) for k, (N, b) in enumerate(sizes)]
    alone = [factor_alone(A, b) for A, (N, b) in zip(mats, sizes)]
    s = torch.cuda.Stream()
    _streams.append(s)
    ctx = b3t.Context(stream=s.cuda_stream, timeout_ns=20_000_000_000, stream_no_mx=True)
    ctx.stream_open(1 << 16, 1 << 18, 16, 60_000_000_000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ctx.last_launch()["nctas"] == 2 * (sms - 8)     # 8 SMs left free
    tiles, ids = [], []
    for A, (N, b) in zip(mats, sizes):
        t = torch.from_numpy(och.to_tiles(A, b)).cuda()
        tiles.append(t)
        ctx.cholesky_submit(dt.tile_ptrs(t), N // b, b)
        ids.append(ctx.stream_submit())
    infos = wait_batches(ctx, ids)
    ctx.stream_close()
    assert all(v == 0 for v in infos.values())
    for t, ref in zip(tiles, alone):
        assert np.array_equal(t.cpu().numpy(), ref)
    ctx.close()
