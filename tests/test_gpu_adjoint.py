"""Gradient of a validation loss through the solve (adjoint PCG) against the
FP64 oracle's adjoint formula, which is itself pinned to central finite
differences (tests/test_oracle_pins.py)."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("modes", ["exact", "default"])
@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE])
def test_val_loss_gradient_n2048(kind, modes):
    wl = W.krr_rbf_hyper(seed=0, n=2048, nval=512, d=32)
    bw, lam = wl.bandwidth, 1e-4 * 2048
    Xt = torch.from_numpy(wl.X).cuda()
    Xv = torch.from_numpy(wl.Xval).cuda()
    y = torch.from_numpy(wl.B[:, 0].copy()).cuda()
    yv = torch.from_numpy(wl.yval).cuda()
    op = ops.KernelOperator(Xt, kind, bw)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(2048, 100, seed=0)).cuda())
    # the loss, the adjoint solve and both derivatives run in the library
    # (pcg_adjoint_val); the default modes take the cross and derivative
    # products with the direct-difference FP32 operator (error-free sums)
    kw = dict(refine_mode=ops.EXACT, check_mode=ops.EXACT) if modes == "exact" else dict()
    loss, g_bw, g_lam = ops.krr_val_loss_and_grad(op, ny, y, Xv, yv, lam, tol=1e-8 if modes == "exact" else 1e-6,
                                                  **kw)
    L_o, dbw_o, dlam_o, _ = O.krr_val_grad(kind, wl.X, wl.B[:, 0], wl.Xval, wl.yval, bw, lam)
    rt = 1e-4 if modes == "exact" else 1e-3
    assert abs(loss - L_o) <= 1e-5 * abs(L_o)
    assert abs(g_lam - dlam_o) <= rt * abs(dlam_o)
    assert abs(g_bw - dbw_o) <= rt * abs(dbw_o)


def test_autograd_function_matches_adjoint():
    wl = W.krr_rbf_hyper(seed=1, n=700, nval=200, d=8)
    lam = 0.5
    Xt = torch.from_numpy(wl.X).cuda()
    op = ops.KernelOperator(Xt, ops.RBF, wl.bandwidth)
    y = torch.from_numpy(wl.B[:, 0].copy()).cuda().requires_grad_(True)
    bw_t = torch.tensor(wl.bandwidth, dtype=torch.float64, requires_grad=True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    x = ops.krr_solve(op, y, bw_t, lam_t, None, tol=1e-8, refine_mode=ops.EXACT, check_mode=ops.EXACT)
    w = torch.from_numpy(W.random_block(700, 1, seed=4)[:, 0]).cuda()
    (x * w).sum().backward()
    # d/dy (w^T x) = (K + lam I)^{-1} w ; d/dlam = -g^T x
    K = O.kernel_matrix(O.RBF, wl.X, wl.X, wl.bandwidth)
    A = K + lam * np.eye(700)
    g = np.linalg.solve(A, w.cpu().numpy().astype(np.float64))
    xs = np.linalg.solve(A, wl.B[:, 0].astype(np.float64))
    np.testing.assert_allclose(y.grad.cpu().numpy(), g, rtol=2e-4, atol=1e-6 * np.abs(g).max())
    assert abs(lam_t.grad.item() - (-g @ xs)) <= 1e-4 * abs(g @ xs)
    dK = O.dkernel_dbw_from_sqdist(O.RBF, O.sqdist(wl.X, wl.X), wl.bandwidth)
    assert abs(bw_t.grad.item() - (-g @ dK @ xs)) <= 1e-4 * abs(g @ dK @ xs)


def test_autograd_backward_uses_its_own_bandwidth():
    # two forwards at different bandwidths on one operator, then the first
    # forward's backward: its gradient is the one at its own bandwidth
    wl = W.krr_rbf_hyper(seed=2, n=600, nval=100, d=8)
    lam = 0.5
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    bw1, bw2 = wl.bandwidth, 1.7 * wl.bandwidth
    kw = dict(tol=1e-8, refine_mode=ops.EXACT, check_mode=ops.EXACT)
    w = torch.from_numpy(W.random_block(600, 1, seed=9)[:, 0]).cuda()
    y = torch.from_numpy(wl.B[:, 0].copy()).cuda()
    bw_t1 = torch.tensor(bw1, dtype=torch.float64, requires_grad=True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    x1 = ops.krr_solve(op, y, bw_t1, lam_t, None, **kw)
    x2 = ops.krr_solve(op, y, torch.tensor(bw2, dtype=torch.float64), torch.tensor(lam, dtype=torch.float64),
                       None, **kw)
    assert torch.max(torch.abs(x1 - x2)).item() > 1e-3
    (x1 * w).sum().backward()
    K = O.kernel_matrix(O.RBF, wl.X, wl.X, bw1)
    A = K + lam * np.eye(600)
    g = np.linalg.solve(A, w.cpu().numpy().astype(np.float64))
    xs = np.linalg.solve(A, wl.B[:, 0].astype(np.float64))
    dK = O.dkernel_dbw_from_sqdist(O.RBF, O.sqdist(wl.X, wl.X), bw1)
    assert abs(bw_t1.grad.item() - (-g @ dK @ xs)) <= 1e-4 * abs(g @ dK @ xs)
    assert abs(lam_t.grad.item() - (-g @ xs)) <= 1e-4 * abs(g @ xs)


def test_unconverged_differentiable_solve_warns():
    wl = W.krr_rbf_hyper(seed=3, n=300, nval=50, d=4)
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    y = torch.from_numpy(wl.B[:, 0].copy()).cuda()
    with pytest.warns(ops.NotConvergedWarning):
        ops.krr_solve(op, y, torch.tensor(wl.bandwidth, dtype=torch.float64), torch.tensor(1e-3, dtype=torch.float64),
                      None, tol=1e-12, maxit=2)
