"""The sliced FP64 residual on the device (GPU): the slices SLICE_A and
SLICE_X write are the host restatement's digits bit for bit (every value's
integer V, the scale exponents, the row sums of |A| and the max|x| the norm
uses); RESID_SL's residual and its per-16-row maxima equal the host
restatement of the same arithmetic (tests/sliced_ref.py) bit for bit and lie
within the a-priori bound of the exact residual; the sliced refinement
reaches the same backward error as the FP64 one."""
import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och
import sliced_ref as sr

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]
R, W = 1, 2


def e4m3_ints(raw):
    v = torch.from_numpy(np.ascontiguousarray(raw)).view(torch.float8_e4m3fn).to(torch.float32).numpy()
    return v.astype(np.int64)


def decode_a_part(p, b):
    """A slice part -> (digits (12, b, b), row sums (b), exponent)."""
    nk = b // 128
    vals = e4m3_ints(p[:12 * b * b]).reshape(nk, nk, 12, 128, 8, 16)
    rows = np.arange(128)
    out = np.empty((12, b, b), dtype=np.int64)
    for g in range(8):
        grp = vals[:, :, :, rows, g ^ (rows % 8), :]          # (nk, nk, 12, 128, 16)
        for rb in range(nk):
            for kc in range(nk):
                out[:, rb * 128:(rb + 1) * 128, kc * 128 + 16 * g:kc * 128 + 16 * g + 16] = grp[rb, kc]
    o = 12 * b * b
    P = p[o:o + 8 * b].view(np.float64)
    e = int(p[o + 8 * b:o + 8 * b + 4].view(np.int32)[0])
    return out, P, e


def decode_x_part(p, b):
    """X slice part -> (digits (12, 16, b), exponents (16), max|x| (b/16, 16))."""
    nk = b // 128
    vals = e4m3_ints(p[:12 * nk * 2048]).reshape(nk, 12, 16, 8, 16)
    rows = np.arange(16)
    out = np.empty((12, 16, b), dtype=np.int64)
    for g in range(8):
        grp = vals[:, :, rows, g ^ (rows % 8), :]            # (nk, 12, 16, 16)
        for kc in range(nk):
            out[:, :, kc * 128 + 16 * g:kc * 128 + 16 * g + 16] = grp[kc]
    o = 12 * nk * 2048
    ex = p[o:o + 64].view(np.int32).astype(np.int64)
    xm = p[o + 64:o + 64 + (b // 16) * 16 * 8].view(np.float64).reshape(b // 16, 16)
    return out, ex, xm


def parts_from(M, b):
    N, nrhs = M.shape
    T = N // b
    return torch.from_numpy(np.ascontiguousarray(M.reshape(T, b, nrhs).transpose(0, 2, 1))).cuda()


def run_sliced(ctx, A, X, Bm, b, nrhs):
    """SLICE_A on every stored tile, SLICE_X on every part, RESID_SL per part;
    returns (R parts host (T, PR), AS bytes, XS bytes)."""
    N = A.shape[0]
    T = N // b
    PB, XB, PR = b3t.slice_a_part_bytes(b), b3t.slice_x_part_bytes(b), b3t.resid_part_elems(b, nrhs)
    Ap = torch.from_numpy(och.to_tiles(A, b)).cuda()
    AS = torch.zeros(T * T * PB, dtype=torch.uint8, device="cuda")
    XS = torch.zeros(T * XB, dtype=torch.uint8, device="cuda")
    Xd, Bd = parts_from(X, b), parts_from(Bm, b)
    Rd = torch.full((T, PR), float("nan"), dtype=torch.float64, device="cuda")
    hA = ctx.data_register(Ap.data_ptr(), Ap.numel(), 8)
    hAS = ctx.data_register(AS.data_ptr(), AS.numel(), 1)
    pAS = ctx.data_partition(hAS, T * T, PB)
    hXS = ctx.data_register(XS.data_ptr(), XS.numel(), 1)
    pXS = ctx.data_partition(hXS, T, XB)
    hX = ctx.data_register(Xd.data_ptr(), Xd.numel(), 8)
    pX = ctx.data_partition(hX, T, b * nrhs)
    hB = ctx.data_register(Bd.data_ptr(), Bd.numel(), 8)
    hR = ctx.data_register(Rd.data_ptr(), Rd.numel(), 8)
    pR = ctx.data_partition(hR, T, PR)
    ca = ctx.task_decl("slice_a", b3t.SLICE_A, [R, W, W], 20)
    cx = ctx.task_decl("slice_x", b3t.SLICE_X, [R, W], 20)
    cr = ctx.task_decl("resid_sl", b3t.RESID_SL, [R, R, R, W], 20)
    for j in range(T):
        for i in range(j, T):
            ctx.task_submit(ca, [hA, pAS[i * T + j], pAS[j * T + i]], b3t.slice_args(i, j, T, b, 0))
    for J in range(T):
        ctx.task_submit(cx, [pX[J], pXS[J]], b3t.slice_args(J, 0, T, b, nrhs))
    for i in range(T):
        ctx.task_submit(cr, [hAS, hXS, hB, pR[i]], b3t.slice_args(i, 0, T, b, nrhs))
    ctx.task_wait()
    for h in (hA, hAS, hXS, hX, hB, hR):
        ctx.data_unregister(h)
    return Rd.cpu().numpy(), AS.cpu().numpy(), XS.cpu().numpy()


CASES = [(512, 128, 16), (768, 256, 5), (512, 128, 1)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "N%d_b%d_r%d" % c)
def sliced_run(request):
    N, b, nrhs = request.param
    A = synth.spd_host(N, seed=N + nrhs, shift=0.1)
    X = synth.rhs(N, nrhs, seed=7) * 0.5
    X[5, 0] = 0.0
    Bm = A @ X + 1e-4 * synth.rhs(N, nrhs, seed=8)
    torch.cuda.set_device(0)
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    try:
        out = run_sliced(ctx, A, X, Bm, b, nrhs)
    finally:
        ctx.close()
    return (N, b, nrhs, A, X, Bm) + out


def test_a_slices_bit_exact(orc, sliced_run):
    N, b, nrhs, A, X, Bm, Rh, AS, XS = sliced_run
    T = N // b
    PB = b3t.slice_a_part_bytes(b)
    for I in range(T):
        for J in range(T):
            D, P, e = decode_a_part(AS[(I * T + J) * PB:(I * T + J + 1) * PB], b)
            Au = sr.use_tile(A, I, J, b)
            e0 = sr.scale_exp(float(np.max(np.abs(Au))))
            assert e == e0, (I, J)
            assert D.min() >= -16 and D.max() <= 15
            assert np.array_equal(sr.from_digits(D), sr.to_int(Au, e0)), (I, J)
            assert np.array_equal(P, sr.row_sums_of_use(A, I, J, b)), (I, J)


def test_x_slices_bit_exact(orc, sliced_run):
    N, b, nrhs, A, X, Bm, Rh, AS, XS = sliced_run
    T = N // b
    XB = b3t.slice_x_part_bytes(b)
    for J in range(T):
        D, ex, xm = decode_x_part(XS[J * XB:(J + 1) * XB], b)
        Xj = np.zeros((b, 16))
        Xj[:, :nrhs] = X[J * b:(J + 1) * b]
        e0 = sr.x_exps(Xj, nrhs)
        assert np.array_equal(ex, e0)
        assert np.array_equal(sr.from_digits(D), sr.to_int(Xj, e0[None, :]).T)
        want = np.max(np.abs(Xj).reshape(b // 16, 16, 16), axis=1)
        assert np.array_equal(xm, want)


def test_residual_bit_exact_and_within_bound(orc, sliced_run):
    N, b, nrhs, A, X, Bm, Rh, AS, XS = sliced_run
    T = N // b
    PR = b3t.resid_part_elems(b, nrhs)
    Rref, eA, eX = sr.resid_sliced(A, X, Bm, b, nrhs)
    got = Rh[:, :b * nrhs].reshape(T, nrhs, b).transpose(0, 2, 1).reshape(N, nrhs)
    assert np.array_equal(got, Rref)
    # the per-16-row maxima NRM reads
    nit = b // 16
    for i in range(T):
        Rn = Rh[i, b * nrhs:PR]
        blk = slice(i * b, (i + 1) * b)
        r16 = np.abs(Rref[blk]).reshape(nit, 16, nrhs).max(axis=1)
        x16 = np.abs(X[blk]).reshape(nit, 16, nrhs).max(axis=1)
        b16 = np.abs(Bm[blk]).reshape(nit, 16, nrhs).max(axis=1)
        assert np.array_equal(Rn[:nit * nrhs].reshape(nit, nrhs), r16)
        assert np.array_equal(Rn[nit * nrhs:2 * nit * nrhs].reshape(nit, nrhs), x16)
        assert np.array_equal(Rn[2 * nit * nrhs:3 * nit * nrhs].reshape(nit, nrhs), b16)
        rs = np.zeros(b)
        for J in range(T):
            rs = rs + sr.row_sums_of_use(A, i, J, b)
        assert np.array_equal(Rn[3 * nit * nrhs:], rs.reshape(nit, 16).max(axis=1))
    rows = list(range(0, N, 29)) + [N - 1]
    Rex = sr.exact_resid_rows(A, X, Bm, rows, b)
    assert np.all(np.abs(got[rows] - Rex) <= sr.resid_bound(eA, eX, rows, Rex, b, T, nrhs))


@pytest.mark.parametrize("fmt", [b3t.FMT_BF16, b3t.FMT_E4M3])
def test_sliced_refinement_matches_fp64_refinement(orc, gctx, fmt):
    # the mixed factor refined with the FP64 residual and with the sliced
    # one: both reach eta <= 1e-12 in the same number of steps (+-1), and the
    # exact residual of the sliced solution meets the target
    N, b, nrhs = 1024, 128, 16
    T = N // b
    A = synth.spd_host(N, seed=9, shift=0.1)
    Bm = synth.rhs(N, nrhs, seed=4)
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Wt = At.float()
    Lt = torch.zeros_like(At)
    Qt = dt.q_tiles(T, b, fmt, "cuda")
    Ut = torch.zeros((T, b, b), dtype=torch.float64, device="cuda")
    wp, lp, qp, up = dt.tile_ptrs(Wt), dt.tile_ptrs(Lt), dt.tile_ptrs(Qt), dt.tile_ptrs(Ut)
    gctx.cholesky_mx_inv_submit(wp, lp, qp, up, T, b, fmt)
    gctx.task_wait()
    Bd = parts_from(Bm, b)
    Rw = torch.zeros(b3t.ir_work_elems(T, b, nrhs), dtype=torch.float64, device="cuda")
    S = torch.empty(b3t.ir_slice_bytes(T, b) + 256, dtype=torch.uint8, device="cuda")
    s_ptr = (S.data_ptr() + 255) // 256 * 256
    eta = torch.zeros(nrhs + 1, dtype=torch.float64, device="cuda")
    X64 = torch.zeros_like(Bd)
    Xsl = torch.zeros_like(Bd)
    rc1, it1, e1 = gctx.ir_solve(At.data_ptr(), lp, Bd.data_ptr(), X64.data_ptr(), Rw.data_ptr(), eta.data_ptr(),
                                 T, b, nrhs, b3t.VEC_F32, 1e-12, 30)
    rc2, it2, e2 = gctx.ir_solve_sliced(At.data_ptr(), lp, Bd.data_ptr(), Xsl.data_ptr(), Rw.data_ptr(), s_ptr,
                                        eta.data_ptr(), T, b, nrhs, b3t.VEC_F32, 1e-12, 30)
    assert rc1 == 0 and rc2 == 0, (rc1, rc2, e1[-1], e2[-1])
    assert abs(it1 - it2) <= 1
    assert e2[-1] <= 1e-12
    Xh = Xsl.cpu().numpy().transpose(0, 2, 1).reshape(N, nrhs)
    rows = list(range(0, N, 61))
    Rex = sr.exact_resid_rows(A, Xh, Bm, rows, b)
    anorm = np.max(np.sum(np.abs(A), axis=1))
    eta_h = np.max(np.abs(Rex), axis=0) / (anorm * np.max(np.abs(Xh), axis=0) + np.max(np.abs(Bm), axis=0))
    assert np.max(eta_h) <= 1e-12
    gctx.ir_release(Rw.data_ptr(), T, b, nrhs)
    for p in (wp, lp, qp):
        gctx.tiles_unregister(p, T)
    for p in up:
        gctx.data_unregister(gctx.data_lookup(p))


# ---- the sliced panel product of the mixed factorisation

def decode_w(p, b):
    """W slices -> (digits (12, b rows, b K), row exponents (b))."""
    nk = b // 128
    vals = e4m3_ints(p[:12 * b * b]).reshape(nk, nk, 12, 128, 8, 16)
    rows = np.arange(128)
    out = np.empty((12, b, b), dtype=np.int64)
    for g in range(8):
        grp = vals[:, :, :, rows, g ^ (rows % 8), :]
        for rb in range(nk):
            for kc in range(nk):
                out[:, rb * 128:(rb + 1) * 128, kc * 128 + 16 * g:kc * 128 + 16 * g + 16] = grp[rb, kc]
    return out, p[12 * b * b:12 * b * b + 4 * b].view(np.int32).astype(np.int64)


def decode_u(p, b):
    """U slices -> (digits (12, b K, b columns), column exponents (b))."""
    nk, ncb = b // 128, b // 32
    vals = e4m3_ints(p[:12 * b * b]).reshape(ncb, nk, 12, 32, 8, 16)
    rows = np.arange(32)
    out = np.empty((12, b, b), dtype=np.int64)
    for g in range(8):
        grp = vals[:, :, :, rows, g ^ (rows % 8), :]       # (ncb, nk, 12, 32, 16): [.., column, K]
        for cb in range(ncb):
            for kc in range(nk):
                out[:, kc * 128 + 16 * g:kc * 128 + 16 * g + 16, cb * 32:(cb + 1) * 32] = \
                    grp[cb, kc].transpose(0, 2, 1)
    return out, p[12 * b * b:12 * b * b + 4 * b].view(np.int32).astype(np.int64)


def dev_tile(M, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(M.T)).to(dtype).cuda()


def sliced_panel_dev(ctx, Lkk, Wik, b):
    """TRTRI(L_kk -> U), SLICE_U, SLICE_W, TRMM_SL on the device; returns
    (U, L_ik, WS bytes, US bytes) on the host."""
    L = dev_tile(Lkk)
    Wd = dev_tile(Wik, torch.float32)
    U = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    X = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    WS = torch.zeros(b3t.slice_w_bytes(b), dtype=torch.uint8, device="cuda")
    US = torch.zeros(b3t.slice_u_bytes(b), dtype=torch.uint8, device="cuda")
    hl = ctx.data_register(L.data_ptr(), b * b, 8, b)
    hu = ctx.data_register(U.data_ptr(), b * b, 8, b)
    hw = ctx.data_register(Wd.data_ptr(), b * b, 4, b)
    hx = ctx.data_register(X.data_ptr(), b * b, 8, b)
    hws = ctx.data_register(WS.data_ptr(), WS.numel(), 1)
    hus = ctx.data_register(US.data_ptr(), US.numel(), 1)
    ci = ctx.task_decl("trtri", b3t.TRTRI, [R, W])
    cu = ctx.task_decl("slice_u", b3t.SLICE_U, [R, W])
    cw = ctx.task_decl("slice_w", b3t.SLICE_W, [R, W])
    cm = ctx.task_decl("trmm_sl", b3t.TRMM_SL, [R, R, W])
    ctx.task_submit(ci, [hl, hu])
    ctx.task_submit(cu, [hu, hus])
    ctx.task_submit(cw, [hw, hws])
    ctx.task_submit(cm, [hus, hws, hx])
    ctx.task_wait()
    for h in (hl, hu, hw, hx, hws, hus):
        ctx.data_unregister(h)
    return U.cpu().numpy().T, X.cpu().numpy().T, WS.cpu().numpy(), US.cpu().numpy()


@pytest.mark.parametrize("b", [128, 256, 512])
def test_sliced_panel_product_bit_exact_and_within_bound(orc, gctx, b):
    from oracle import tiles as otl
    rng = np.random.default_rng(b + 3)
    A = synth.spd_host(b, seed=b, shift=1.0)
    Lkk = np.asfortranarray(np.tril(A))
    assert otl.potrf(Lkk) == 0
    Lkk = np.tril(Lkk)
    Wik = (rng.standard_normal((b, b)) * 10.0 ** rng.integers(-2, 3, (b, 1))).astype(np.float32)
    Wik[3, :] = 0.0
    U, X, WS, US = sliced_panel_dev(gctx, Lkk, Wik, b)
    Xref, eW, eU = sr.trmm_sliced(Wik, U)
    # the slices, then the product, bit for bit
    DW, eWd = decode_w(WS, b)
    DU, eUd = decode_u(US, b)
    assert np.array_equal(eWd, eW) and np.array_equal(eUd, eU)
    assert np.array_equal(sr.from_digits(DW), sr.to_int(Wik.astype(np.float64), eW[:, None]))
    assert np.array_equal(sr.from_digits(DU), sr.to_int(U, eU[None, :]))
    assert np.array_equal(X, Xref)
    # against the exact product: b terms of the truncation bound plus one rounding
    ent = [(int(r), int(c)) for r, c in zip(rng.integers(0, b, 64), rng.integers(0, b, 64))] + [(b - 1, b - 1)]
    ex = sr.exact_product_entries(Wik.astype(np.float64), U, ent)
    got = np.array([X[r, c] for r, c in ent])
    bound = np.array([b * sr.term_error() * 2.0 ** float(eW[r] + eU[c]) for r, c in ent]) + 2 * sr.U64 * np.abs(ex)
    assert np.all(np.abs(got - ex) <= bound)


def factor_sliced_dev(ctx, A, b, fmt):
    N = A.shape[0]
    T = N // b
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Wt = At.float()
    Lt = torch.zeros_like(At)
    Qt = dt.q_tiles(T, b, fmt, "cuda")
    Ut = torch.zeros((T, b, b), dtype=torch.float64, device="cuda")
    nt = T * (T + 1) // 2
    WSt = torch.zeros((nt, b3t.slice_w_bytes(b)), dtype=torch.uint8, device="cuda")
    USt = torch.zeros((T, b3t.slice_u_bytes(b)), dtype=torch.uint8, device="cuda")
    wp, lp, qp, up = dt.tile_ptrs(Wt), dt.tile_ptrs(Lt), dt.tile_ptrs(Qt), dt.tile_ptrs(Ut)
    ctx.cholesky_mx_sliced_submit(wp, lp, qp, up, dt.tile_ptrs(WSt), dt.tile_ptrs(USt), T, b, fmt)
    ctx.task_wait()
    for p in (wp, lp, qp):
        ctx.tiles_unregister(p, T)
    for p in up[:-1] + dt.tile_ptrs(USt)[:-1]:
        ctx.data_unregister(ctx.data_lookup(p))
    ctx.data_unregister(ctx.data_lookup(up[-1]))
    for j in range(T):
        for i in range(j + 1, T):
            ctx.data_unregister(ctx.data_lookup(dt.tile_ptrs(WSt)[och.tile_index(i, j, T)]))
    return Wt, Lt, Qt, Ut


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("N,b", [(1024, 128), (1024, 256)])
def test_sliced_factor_every_task_within_its_bound(orc, gctx, fmt, N, b):
    from mixed_steps import check_factor
    from qlayout import decode
    FM = {"bf16": b3t.FMT_BF16, "e4m3": b3t.FMT_E4M3}[fmt]
    A = synth.spd_host(N, seed=N + b + 1, shift=1.0)
    Wt, Lt, Qt, Ut = factor_sliced_dev(gctx, A, b, FM)
    T = N // b
    Qh = Qt.cpu().numpy()
    Q = {(i, k): decode(Qh[och.tile_index(i, k, T)], b, FM) for k in range(T) for i in range(k + 1, T)}
    r = check_factor(A, Wt.cpu().numpy(), Lt.cpu().numpy(), Q, T, b, fmt, Ut.cpu().numpy(), sliced=True)
    assert r["quant"] == 0.0, r
    assert all(v <= 1.0 for v in r.values()), r


@pytest.mark.parametrize("b", [128, 256, 512])
def test_trtri_by_column_blocks_equals_trtri(orc, gctx, b):
    # U_k = L_kk^{-T} one 64-column block at a time (TRTRI_COL, each block
    # from the blocks before it) is TRTRI's result bit for bit
    from oracle import tiles as otl
    A = synth.spd_host(b, seed=b + 11, shift=1.0)
    Lkk = np.asfortranarray(np.tril(A))
    assert otl.potrf(Lkk) == 0
    L = dev_tile(np.tril(Lkk))
    U1 = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    U2 = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    hl = gctx.data_register(L.data_ptr(), b * b, 8, b)
    h1 = gctx.data_register(U1.data_ptr(), b * b, 8, b)
    h2 = gctx.data_register(U2.data_ptr(), b * b, 8, b)
    ci = gctx.task_decl("trtri", b3t.TRTRI, [R, W])
    gctx.task_submit(ci, [hl, h1])
    gctx.task_wait()
    pl = gctx.data_partition(hl, b // 64, b * 64)
    pu = gctx.data_partition(h2, b // 64, b * 64)
    cc = gctx.task_decl("trtri_col", b3t.TRTRI_COL, [R, R, W], 20)
    for cb in range(b // 64):
        gctx.task_submit(cc, [pl[cb], pu[cb - 1 if cb else 0], pu[cb]], struct_panel(b, 64, cb))
    gctx.task_wait()
    for h in (hl, h1, h2):
        gctx.data_unregister(h)
    assert np.array_equal(U1.cpu().numpy(), U2.cpu().numpy())


def struct_panel(b, pw, kk, jj=0, col0=0):
    import struct
    return struct.pack("<5i", b, pw, kk, jj, col0)
