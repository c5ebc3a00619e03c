"""Solve and refinement tasks against the oracle (GPU): triangular solves
with a tiled factor (FP64 and binary32 arithmetic), the FP64 residual and
backward error, and iterative refinement with a low-precision factor."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och, ir as oir, mixed as omx

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


def parts_from(M, b):
    """Dense (N, nrhs) -> (T, nrhs, b) device tensor (part k column-major)."""
    N, nrhs = M.shape
    T = N // b
    return torch.from_numpy(np.ascontiguousarray(M.reshape(T, b, nrhs).transpose(0, 2, 1))).cuda()


def dense_from(P):
    T, nrhs, b = P.shape
    return P.cpu().numpy().transpose(0, 2, 1).reshape(T * b, nrhs)


@pytest.mark.parametrize("nrhs", [1, 5, 16, 32])
@pytest.mark.parametrize("f32", [False, True])
def test_chol_solve_against_substitution(orc, gctx, nrhs, f32):
    N, b = 512, 128
    T = N // b
    A = synth.spd_host(N, seed=nrhs, shift=1.0)
    L = sla.cholesky(A, lower=True)
    Bm = synth.rhs(N, nrhs, seed=2)
    Lt = torch.from_numpy(och.to_tiles(L, b)).cuda()
    Y = parts_from(Bm, b)
    gctx.chol_solve_submit(dt.tile_ptrs(Lt), Y.data_ptr(), T, b, nrhs, b * nrhs,
                           b3t.VEC_F32 if f32 else 0)
    gctx.task_wait()
    got = dense_from(Y)
    ref = oir.chol_solve(L, Bm)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= (1e-5 if f32 else 1e-13), err


@pytest.mark.parametrize("nrhs", [1, 7, 16, 32])
@pytest.mark.parametrize("f32", [False, True])
def test_chol_solve_with_inverted_diagonal(orc, gctx, nrhs, f32):
    # TRTRI: U_k = L_kk^{-T}, checked against forward substitution on the
    # identity; then the inverse-based solve against substitution
    N, b = 640, 128
    T = N // b
    A = synth.spd_host(N, seed=nrhs + 3, shift=1.0)
    L = sla.cholesky(A, lower=True)
    Bm = synth.rhs(N, nrhs, seed=4)
    Lt = torch.from_numpy(och.to_tiles(L, b)).cuda()
    U = torch.full((T, b, b), float("nan"), dtype=torch.float64, device="cuda")
    Y = parts_from(Bm, b)
    Z = torch.zeros_like(Y)
    gctx.chol_inv_submit(dt.tile_ptrs(Lt), dt.tile_ptrs(U), T, b)
    gctx.chol_solve_inv_submit(dt.tile_ptrs(Lt), dt.tile_ptrs(U), Y.data_ptr(), Z.data_ptr(), T, b, nrhs,
                               b * nrhs, b3t.VEC_F32 if f32 else 0)
    gctx.task_wait()
    Uh = U.cpu().numpy()
    for k in range(T):
        Lkk = L[k * b:(k + 1) * b, k * b:(k + 1) * b]
        Uk = Uh[k].T                                   # tile memory is column-major
        Linv = oir.forward_sub(Lkk, np.eye(b))
        assert np.all(np.tril(Uk, -1) == 0.0)
        assert np.max(np.abs(Uk - Linv.T)) / np.max(np.abs(Linv)) <= 1e-13
    got = dense_from(Y)
    ref = oir.chol_solve(L, Bm)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= (1e-5 if f32 else 1e-12), err


def test_residual_and_backward_error(orc, gctx):
    N, b, nrhs = 768, 256, 3
    T = N // b
    A = synth.spd_host(N, seed=5, shift=1.0)
    As = oir.symmetric_from_lower(A)
    Bm = synth.rhs(N, nrhs, seed=6)
    X = np.linalg.solve(As, Bm) * (1.0 + 1e-3 * synth.gaussian((N, nrhs), 7))   # eta ~ 1e-3
    Ap = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Xd, Bd = parts_from(X, b), parts_from(Bm, b)
    PR = b3t.resid_part_elems(b, nrhs)             # residual part: values, then per-item maxima
    R = torch.zeros(T * PR, dtype=torch.float64, device="cuda")
    eta = torch.zeros(nrhs + 1, dtype=torch.float64, device="cuda")
    ha = gctx.data_register(Ap.data_ptr(), Ap.numel(), 8)
    hx = gctx.data_register(Xd.data_ptr(), Xd.numel(), 8)
    hb = gctx.data_register(Bd.data_ptr(), Bd.numel(), 8)
    hr = gctx.data_register(R.data_ptr(), R.numel(), 8)
    pr = gctx.data_partition(hr, T, PR)
    he = gctx.data_register(eta.data_ptr(), eta.numel(), 8)
    cres = gctx.task_decl("resid", b3t.RESID, [1, 1, 1, 2], 20)
    cnrm = gctx.task_decl("nrm", b3t.NRM, [1, 1, 2], 20)
    for i in range(T):
        gctx.task_submit(cres, [ha, hx, hb, pr[i]], b3t.vec_args(nrhs, 0, i, T, b))
    gctx.task_submit(cnrm, [hr, hb, he], b3t.vec_args(nrhs, 0, 0, T, b))
    gctx.task_wait()
    Rv = R.view(T, PR)[:, : b * nrhs].reshape(T, nrhs, b)
    ref = Bm - As @ X
    assert np.max(np.abs(dense_from(Rv) - ref)) <= 1e-13 * np.max(np.abs(As)) * np.max(np.abs(X))
    e = eta.cpu().numpy()
    for j in range(nrhs):
        ej = oir.backward_error(As, X[:, j:j + 1], Bm[:, j:j + 1])
        assert abs(e[j] - ej) <= 1e-10 * ej
    assert e[nrhs] == max(e[:nrhs])


def run_ir(ctx, A, Lt, Bm, b, f32, tol=1e-12, max_iter=30):
    N, nrhs = Bm.shape
    T = N // b
    Ap = torch.from_numpy(och.to_tiles(A, b)).cuda()
    Bd = parts_from(Bm, b)
    Xd = torch.zeros_like(Bd)
    R = torch.zeros(b3t.ir_work_elems(T, b, nrhs), dtype=torch.float64, device="cuda")
    eta = torch.zeros(nrhs + 1, dtype=torch.float64, device="cuda")
    rc, its, e = ctx.ir_solve(Ap.data_ptr(), dt.tile_ptrs(Lt), Bd.data_ptr(), Xd.data_ptr(), R.data_ptr(),
                              eta.data_ptr(), T, b, nrhs, b3t.VEC_F32 if f32 else 0, tol, max_iter)
    return rc, its, e, dense_from(Xd)


def test_ir_with_fp64_factor_one_step(orc, gctx):
    N, b, nrhs = 1024, 128, 4
    A = synth.spd_host(N, seed=0, shift=1.0)
    L = sla.cholesky(A, lower=True)
    Bm = synth.rhs(N, nrhs, seed=4)
    rc, its, e, X = run_ir(gctx, A, torch.from_numpy(och.to_tiles(L, b)).cuda(), Bm, b, False,
                           tol=1e-14, max_iter=1)
    As = oir.symmetric_from_lower(A)
    assert rc == 0 and its == 1
    # both sides see only rounding noise here (~1e-16): bound both
    assert oir.backward_error(As, X, Bm) <= 1e-14
    assert e[nrhs] <= 1e-14


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_ir_with_mixed_factor(orc, gctx, fmt):
    N, b, nrhs = 1024, 128, 4
    A = synth.spd_host(N, seed=0, shift=1.0)
    Lt, info = omx.factor(och.to_tiles(A, b), N // b, b, fmt)
    Bm = synth.rhs(N, nrhs, seed=4)
    rc, its, e, X = run_ir(gctx, A, torch.from_numpy(Lt).cuda(), Bm, b, True)
    As = oir.symmetric_from_lower(A)
    eta_orc = oir.backward_error(As, X, Bm)
    if rc == 0:
        assert eta_orc <= 1e-12 and e[nrhs] <= 1e-12
        Xs = sla.cho_solve(sla.cho_factor(A, lower=True), Bm)
        assert np.max(np.abs(X - Xs)) / np.max(np.abs(Xs)) <= np.linalg.cond(As) * 1e-12
    else:
        # E4M3 may stagnate (kappa * u_e4m3 close to 1): then it must say so
        assert fmt == "e4m3" and rc == b3t._lib.ERANGE


def test_mixed_factor_then_refinement_end_to_end(orc, gctx):
    # device mixed-precision factorisation, then device refinement: the
    # solution reaches eta <= 1e-12 and agrees with the FP64 solution
    N, b, nrhs = 1024, 128, 8
    T = N // b
    A = synth.spd_host(N, seed=0, shift=1.0)
    At = torch.from_numpy(och.to_tiles(A, b)).cuda()
    W = At.float()
    Lm = torch.zeros_like(At)
    Q = dt.q_tiles(T, b, b3t.FMT_BF16, "cuda")
    gctx.cholesky_mx_submit(dt.tile_ptrs(W), dt.tile_ptrs(Lm), dt.tile_ptrs(Q), T, b, b3t.FMT_BF16)
    gctx.task_wait()
    Bm = synth.rhs(N, nrhs, seed=9)
    rc, its, e, X = run_ir(gctx, A, Lm, Bm, b, True)
    As = oir.symmetric_from_lower(A)
    assert rc == 0 and its <= 30
    assert oir.backward_error(As, X, Bm) <= 1e-12
    Xs = sla.cho_solve(sla.cho_factor(A, lower=True), Bm)
    assert np.max(np.abs(X - Xs)) / np.max(np.abs(Xs)) <= np.linalg.cond(As) * 1e-12
