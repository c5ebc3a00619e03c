"""The allocation-free entry point b3t_scal_chains_noalloc, for callers that
cannot let a library call cudaMalloc (their GPU memory is owned by a
framework's allocator, or they cannot afford the synchronisation an
allocation may imply).  Its output must equal, bit for bit, what the
ordinary entry point (the task executor, fed B3T_SCAL_F32 tasks through
b3t_task_submit) produces, on two calls in a row: the second call reuses
the scratch array the first one left behind.  The oracle's in-order
binary32 multiplies give the same bits, and a call leaves the device's free
memory unchanged.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1304_0878_b300 as b3t

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]
RW = 3


def reference_chains(x0, f):
    """The existing entry point: SCAL tasks submitted to a context."""
    nb, nk = f.shape
    n = x0.numel() // nb
    x = x0.clone()
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    hs = [ctx.data_register(x[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
    cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [RW], 4)
    for k in range(nk):
        for i in range(nb):
            ctx.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
    ctx.task_wait()
    ctx.close()
    return x


def noalloc_chains(x0, fd, nb, nk):
    x = x0.clone()
    n = x.numel() // nb
    rc = b3t.lib().b3t_scal_chains_noalloc(ctypes.c_void_p(x.data_ptr()), n, nb, nk,
                                           ctypes.c_void_p(fd.data_ptr()), 20_000_000_000,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, b3t.strerror(rc)
    return x


@pytest.mark.parametrize("nb,n,nk", [(64, (1 << 16) + 1024, 8), (7, 4 * 1000, 5)])
def test_noalloc_matches_executor_twice(nb, n, nk):
    torch.cuda.set_device(0)
    x0 = torch.from_numpy(synth.vector_f32(nb * n, seed=31)).cuda()
    f = synth.chain_factors(nb, nk, seed=32)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    ref = reference_chains(x0, f)
    for _ in range(2):
        got = noalloc_chains(x0, fd, nb, nk)
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
    # the oracle: each task multiplies its block once, in chain order
    y = x0.cpu().numpy().copy()
    for k in range(nk):
        for i in range(nb):
            oracle.tiles.scal_f32(y[i * n:(i + 1) * n], f[i, k])
    assert np.array_equal(got.cpu().numpy().view(np.uint32), y.view(np.uint32))


def test_noalloc_leaves_free_memory_unchanged():
    torch.cuda.set_device(0)
    nb, n, nk = 16, 1 << 16, 4
    x = torch.from_numpy(synth.vector_f32(nb * n, seed=33)).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(synth.chain_factors(nb, nk, seed=34))).cuda()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = b3t.lib()

    def call():
        rc = L.b3t_scal_chains_noalloc(ctypes.c_void_p(x.data_ptr()), n, nb, nk,
                                       ctypes.c_void_p(fd.data_ptr()), 0, st)
        assert rc == 0, b3t.strerror(rc)

    call()                       # first call on the device: one-time set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversize_and_misaligned():
    x = torch.zeros(1 << 12, device="cuda")
    fd = torch.ones(1, device="cuda")
    L = b3t.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.b3t_scal_chains_noalloc(ctypes.c_void_p(x.data_ptr()), 4, 65537, 1,
                                   ctypes.c_void_p(fd.data_ptr()), 0, st)
    assert rc == b3t._lib.E2BIG
    rc = L.b3t_scal_chains_noalloc(ctypes.c_void_p(x.data_ptr() + 4), 8, 1, 1,
                                   ctypes.c_void_p(fd.data_ptr()), 0, st)
    assert rc == b3t._lib.EINVAL
