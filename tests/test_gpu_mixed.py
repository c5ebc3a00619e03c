"""Mixed-precision tasks against the oracle (GPU): quantisation bit-exact
(both sides round once, FP64 -> format, ties to even; crafted tiles hold
values just off the format's midpoints, where a rounding through binary32
would break the tie the other way), tensor-core updates exact when every
product and partial sum is representable, and within the binary32
accumulation bound otherwise."""
import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och, mixed as omx, tiles as otl
from fpgrid import chain_round, grid_midpoints, ulp32
from qlayout import decode

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]
R, W, RW = 1, 2, 3
FMTS = {"bf16": b3t.FMT_BF16, "e4m3": b3t.FMT_E4M3}
U32 = 2.0 ** -24


def dev_tile(M, dtype=torch.float64):
    """(r, c) matrix -> device tile (column-major)."""
    return torch.from_numpy(np.ascontiguousarray(M.T)).to(dtype).cuda()


def quantise_dev(ctx, Lm, fmt, b):
    L = dev_tile(Lm)
    Q = torch.zeros(b3t.q_bytes(b, FMTS[fmt]), dtype=torch.uint8, device="cuda")
    hl = ctx.data_register(L.data_ptr(), b * b, 8, b)
    hq = ctx.data_register(Q.data_ptr(), Q.numel(), 1, b)
    cq = ctx.task_decl("quant", b3t.QUANT, [R, W], 4)
    ctx.task_submit(cq, [hl, hq], b3t.pack_i32(FMTS[fmt]))
    ctx.task_wait()
    ctx.data_unregister(hl)
    return Q, hq


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("b", [128, 256])
def test_quant_bit_exact(orc, gctx, fmt, b):
    rng = np.random.default_rng(b)
    Lm = rng.standard_normal((b, b)) * 10.0 ** rng.integers(-3, 3)
    Lm[0, 0] = 1e-30
    Q, hq = quantise_dev(gctx, Lm, fmt, b)
    vals, e = decode(Q.cpu().numpy(), b, FMTS[fmt])
    qo, eo = otl.quantise(Lm, fmt)
    assert e == eo
    assert np.array_equal(vals, qo)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_quant_one_rounding_crafted(orc, gctx, fmt):
    # tile maximum 448 * 2^3 (E4M3 scale e = 3); a quarter of the tile are
    # format midpoints (after the scale) nudged by less than half a binary32
    # ulp, up or down, and their negatives
    b = 128
    rng = np.random.default_rng(7)
    Lm = rng.standard_normal((b, b))
    Lm = Lm / np.max(np.abs(Lm)) * 448.0 * 8.0 * 0.99
    Lm[3, 100] = 448.0 * 8.0
    n = b * 32
    mids = grid_midpoints(fmt, rng, n)
    if fmt == "e4m3":
        mids = mids * 8.0
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    Lm[:, :32] = (sign * (mids + side * ulp32(mids) * 2.0 ** -9)).reshape(b, 32, order="F")
    Q, hq = quantise_dev(gctx, Lm, fmt, b)
    vals, e = decode(Q.cpu().numpy(), b, FMTS[fmt])
    qo, eo = otl.quantise(Lm, fmt)
    assert e == eo == (3 if fmt == "e4m3" else 0)
    assert np.array_equal(vals, qo)
    # the crafted block separates one rounding from the binary32 chain
    chain = chain_round(Lm[:, :32].ravel(order="F") * 2.0 ** -e, fmt)
    assert np.sum(chain != qo[:, :32].ravel(order="F")) >= n // 8


def mx_update_dev(ctx, QA_m, QB_m, W0, fmt, b, syrk):
    """Run SYRK_MX / GEMM_MX with Q tiles produced by QUANT from exact
    values (so the device operands equal the oracle's)."""
    QA, ha = quantise_dev(ctx, QA_m, fmt, b)
    if not syrk:
        QB, hb = quantise_dev(ctx, QB_m, fmt, b)
    Wd = dev_tile(W0, torch.float32)
    hw = ctx.data_register(Wd.data_ptr(), b * b, 4, b)
    if syrk:
        cs = ctx.task_decl("syrk_mx", b3t.SYRK_MX, [R, RW], 4)
        ctx.task_submit(cs, [ha, hw], b3t.pack_i32(FMTS[fmt]))
    else:
        cg = ctx.task_decl("gemm_mx", b3t.GEMM_MX, [R, R, RW], 4)
        ctx.task_submit(cg, [ha, hb, hw], b3t.pack_i32(FMTS[fmt]))
    ctx.task_wait()
    for h in ([ha, hw] if syrk else [ha, hb, hw]):
        ctx.data_unregister(h)
    return Wd.cpu().numpy().T


@pytest.mark.parametrize("fmt,lim", [("bf16", 32), ("e4m3", 8)])
@pytest.mark.parametrize("syrk", [False, True])
def test_mx_update_exact_on_integers(orc, gctx, fmt, lim, syrk):
    b = 256
    rng = np.random.default_rng(3)
    A = rng.integers(-lim, lim + 1, (b, b)).astype(np.float64)
    B = rng.integers(-lim, lim + 1, (b, b)).astype(np.float64)
    W0 = rng.integers(-4096, 4096, (b, b)).astype(np.float32)
    got = mx_update_dev(gctx, A, B, W0, fmt, b, syrk)
    qa, ea = otl.quantise(A, fmt)
    qb, eb = otl.quantise(A if syrk else B, fmt)
    ref = np.asfortranarray(W0.copy())
    otl.gemm_lowp(qa, qb, 2.0 ** (ea + eb), ref, lower=syrk)
    if syrk:
        assert np.array_equal(np.tril(got), np.tril(ref))
        assert np.array_equal(np.triu(got, 1), np.triu(W0, 1))
    else:
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_mx_update_within_fp32_bound(orc, gctx, fmt):
    b = 384
    rng = np.random.default_rng(4)
    A = rng.standard_normal((b, b)) * 0.3
    B = rng.standard_normal((b, b)) * 0.3
    W0 = rng.standard_normal((b, b)).astype(np.float32)
    got = mx_update_dev(gctx, A, B, W0, fmt, b, False)
    qa, ea = otl.quantise(A, fmt)
    qb, eb = otl.quantise(B, fmt)
    s = 2.0 ** (ea + eb)
    ref = np.asfortranarray(W0.copy())
    otl.gemm_lowp(qa, qb, s, ref)
    # binary32 accumulation of b products plus the final rounding
    bound = (b + 2) * U32 * (s * otl.gemm_abs(qa, qb) + np.abs(W0)) + U32 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)


def factor_mx_dev(ctx, A, b, fmt):
    N = A.shape[0]
    T = N // b
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Wt = At.float()
    Lt = torch.zeros_like(At)
    Qt = dt.q_tiles(T, b, FMTS[fmt], "cuda")
    wp, lp, qp = dt.tile_ptrs(Wt), dt.tile_ptrs(Lt), dt.tile_ptrs(Qt)
    ctx.cholesky_mx_submit(wp, lp, qp, T, b, FMTS[fmt])
    ctx.task_wait()
    for p in (wp, lp, qp):
        ctx.tiles_unregister(p, T)
    return np.tril(och.from_tiles(Lt.cpu().numpy(), N, b))


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("N,b", [(512, 128), (768, 256)])
def test_mixed_factor_exact_on_integer_matrix(orc, gctx, fmt, N, b):
    A, L0 = synth.integer_spd(N, seed=N + 7)
    L = factor_mx_dev(gctx, A, b, fmt)
    assert np.array_equal(L, L0)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_mixed_factor_matches_mixed_oracle(orc, gctx, fmt):
    N, b = 1024, 128
    A = synth.spd_host(N, seed=0, shift=1.0)
    L = factor_mx_dev(gctx, A, b, fmt)
    Lt, info = omx.factor(och.to_tiles(A, b), N // b, b, fmt)
    Lo = np.tril(och.from_tiles(Lt, N, b))
    r_dev, r_orc = och.rel_residual(L, A), och.rel_residual(Lo, A)
    # the same low-precision factor up to the order of the binary32 sums: a
    # residual of the same size (the element-level parity is
    # test_mixed_factor_every_task_within_its_bound)
    assert r_dev <= 2.0 * r_orc and r_orc <= 2.0 * r_dev


# ---- the panel solve as a product with the inverted diagonal tile

def trmm_dev(ctx, Lkk, Wik, b):
    """TRTRI(L_kk -> U) then TRMM_MX(U, W_ik -> L_ik) on the device."""
    L = dev_tile(Lkk)
    Wd = dev_tile(Wik, torch.float32)
    U = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    X = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    hl = ctx.data_register(L.data_ptr(), b * b, 8, b)
    hu = ctx.data_register(U.data_ptr(), b * b, 8, b)
    hw = ctx.data_register(Wd.data_ptr(), b * b, 4, b)
    hx = ctx.data_register(X.data_ptr(), b * b, 8, b)
    ci = ctx.task_decl("trtri", b3t.TRTRI, [R, W])
    cm = ctx.task_decl("trmm_mx", b3t.TRMM_MX, [R, R, W])
    ctx.task_submit(ci, [hl, hu])
    ctx.task_submit(cm, [hu, hw, hx])
    ctx.task_wait()
    for h in (hl, hu, hw, hx):
        ctx.data_unregister(h)
    return X.cpu().numpy().T


@pytest.mark.parametrize("b", [128, 256, 512])
def test_trmm_mx_matches_substitution(orc, gctx, b):
    # L_ik = fp64(W_ik) L_kk^{-T}: the oracle substitutes row by row
    # (oracle.tiles.trsm); the device multiplies by U = L_kk^{-T}.  Both are
    # FP64; an explicit inverse rounds differently, so the bound is relative
    rng = np.random.default_rng(b + 1)
    A = synth.spd_host(b, seed=b, shift=1.0)
    Lkk = np.asfortranarray(np.tril(A))
    assert otl.potrf(Lkk) == 0
    Lkk = np.asfortranarray(np.tril(Lkk))
    Wik = (rng.standard_normal((b, b)) * 0.5).astype(np.float32)
    got = trmm_dev(gctx, Lkk, Wik, b)
    ref = np.asfortranarray(Wik.astype(np.float64))
    otl.trsm(Lkk, ref)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-12, err


def factor_mx_inv_dev(ctx, A, b, fmt):
    N = A.shape[0]
    T = N // b
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Wt = At.float()
    Lt = torch.zeros_like(At)
    Qt = dt.q_tiles(T, b, FMTS[fmt], "cuda")
    Ut = torch.zeros((T, b, b), dtype=torch.float64, device="cuda")
    wp, lp, qp, up = dt.tile_ptrs(Wt), dt.tile_ptrs(Lt), dt.tile_ptrs(Qt), dt.tile_ptrs(Ut)
    ctx.cholesky_mx_inv_submit(wp, lp, qp, up, T, b, FMTS[fmt])
    ctx.task_wait()
    for p, n in ((wp, T), (lp, T), (qp, T)):
        ctx.tiles_unregister(p, n)
    for p in up:
        ctx.data_unregister(ctx.data_lookup(p))
    return np.tril(och.from_tiles(Lt.cpu().numpy(), N, b))


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("N,b", [(512, 128), (768, 256)])
def test_mixed_inv_factor_on_integer_matrix(orc, gctx, fmt, N, b):
    # integer L0: the panel tiles carry the inverse's FP64 rounding (an
    # explicit inverse is only as accurate as the diagonal tile is well
    # conditioned: random integer triangles with small diagonals have inverses
    # of 1e15 and more, so this L0 has entries in [-1, 1] and diagonal 8, max
    # |L_kk^-1| about 0.2).  Entries that are 0 in L0 come out as residues of
    # up to ~1e-14: E4M3 (smallest step 2^-9 times the tile scale) rounds them
    # to 0, so its operands and updates, hence the diagonal factors, are
    # exact; bf16 keeps them (binary32's exponent range), and whether they
    # survive the binary32 sums depends on the summation order, so there the
    # diagonal blocks meet the same relative bound as the rest
    A, L0 = synth.integer_spd(N, seed=N + 7, lo=-1, hi=1, dlo=8, dhi=8)
    L = factor_mx_inv_dev(gctx, A, b, fmt)
    assert np.max(np.abs(L - L0)) / np.max(np.abs(L0)) <= 1e-13
    T = N // b
    for k in range(T):
        blk = slice(k * b, (k + 1) * b)
        if fmt == "e4m3":
            assert np.array_equal(L[blk, blk], L0[blk, blk])
        else:
            assert np.max(np.abs(L[blk, blk] - L0[blk, blk])) <= 1e-13 * np.max(np.abs(L0))


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_mixed_inv_factor_matches_mixed_oracle(orc, gctx, fmt):
    N, b = 1024, 128
    A = synth.spd_host(N, seed=0, shift=1.0)
    L = factor_mx_inv_dev(gctx, A, b, fmt)
    Lt, info = omx.factor(och.to_tiles(A, b), N // b, b, fmt)
    Lo = np.tril(och.from_tiles(Lt, N, b))
    r_dev, r_orc = och.rel_residual(L, A), och.rel_residual(Lo, A)
    assert r_dev <= 2.0 * r_orc and r_orc <= 2.0 * r_dev


# ---- every task of the factorisation against its own rounding bound

def factor_state_dev(ctx, A, b, fmt, inv):
    """Run the mixed factorisation; return what it leaves on the device: W
    and L tiles (packed), the decoded panel tiles {(i, k): (values, e)} and
    the inverted diagonal tiles (product form) or None."""
    N = A.shape[0]
    T = N // b
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Wt = At.float()
    Lt = torch.zeros_like(At)
    Qt = dt.q_tiles(T, b, FMTS[fmt], "cuda")
    Ut = torch.zeros((T, b, b), dtype=torch.float64, device="cuda")
    wp, lp, qp, up = dt.tile_ptrs(Wt), dt.tile_ptrs(Lt), dt.tile_ptrs(Qt), dt.tile_ptrs(Ut)
    if inv:
        ctx.cholesky_mx_inv_submit(wp, lp, qp, up, T, b, FMTS[fmt])
    else:
        ctx.cholesky_mx_submit(wp, lp, qp, T, b, FMTS[fmt])
    ctx.task_wait()
    for p in (wp, lp, qp):
        ctx.tiles_unregister(p, T)
    if inv:
        for p in up:
            ctx.data_unregister(ctx.data_lookup(p))
    Qh = Qt.cpu().numpy()
    Q = {}
    for k in range(T):
        for i in range(k + 1, T):
            Q[(i, k)] = decode(Qh[och.tile_index(i, k, T)], b, FMTS[fmt])
    return Wt.cpu().numpy(), Lt.cpu().numpy(), Q, (Ut.cpu().numpy() if inv else None)


@pytest.mark.parametrize("inv", [False, True])
@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("N,b", [(1024, 128), (1024, 256)])
def test_mixed_factor_every_task_within_its_bound(orc, gctx, fmt, inv, N, b):
    # each task's output against that task's inputs as the device left them:
    # QUANT bit for bit, the tensor-core updates within the binary32
    # accumulation bound carried over a tile's updates, POTRF / TRSM / TRTRI /
    # TRMM within the FP64 backward-error bounds (tests/mixed_steps.py); b =
    # 256 takes the diagonal-panel DAG (CVT, POTRF_D, PANEL_TRSM, PANEL_UPD)
    from mixed_steps import check_factor
    A = synth.spd_host(N, seed=N + b, shift=1.0)
    Wt, Lt, Q, Ut = factor_state_dev(gctx, A, b, fmt, inv)
    r = check_factor(A, Wt, Lt, Q, N // b, b, fmt, Ut)
    assert r["quant"] == 0.0, r
    assert all(v <= 1.0 for v in r.values()), r
