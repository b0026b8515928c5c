"""Point gradient d(a^T K(X) b)/dX (kop_grad_points) against the FP64 oracle
(oracle.kop_oracle.kernel_grad_points), three kernels, the three modes.
Errors are Frobenius-relative over the whole n x d gradient."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu

# FP64 direct differences (FP32 output); the accurate operator (FP32 kernel
# values, error-free contraction); the fast one (BF16 hi/lo kernel values and
# V on the tensor cores, about 2^-16 per term).  Measured at n = 1500 on a
# B300: 2.5e-8, 0.9-1.6e-7 and 7e-6; the bounds leave about 10x.
TOL = {ops.EXACT: 1e-6, ops.ACCURATE: 2e-6, ops.FAST: 1e-4}


@pytest.mark.parametrize("kind,bw", [(ops.RBF, 4.0), (ops.LAPLACE, 6.0), (ops.MATERN52, 4.0)])
@pytest.mark.parametrize("mode", [ops.EXACT, ops.ACCURATE, ops.FAST])
def test_grad_points_matches_oracle(kind, bw, mode):
    n, d = 1500, 16
    X = W.random_points(n, d, seed=41, shift=1.5)
    a = W.random_block(n, 1, seed=42)[:, 0]
    b = W.random_block(n, 1, seed=43)[:, 0]
    Go = O.kernel_grad_points(kind, X, a, b, bw)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    G = op.grad_points(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), mode=mode).cpu().numpy()
    err = np.linalg.norm(G - Go) / np.linalg.norm(Go)
    assert err <= TOL[mode], err


def test_grad_points_full_size_sampled_rows():
    # the benchmark's point set (n = 200000, d = 64, Laplace), in the fast mode,
    # on 48 sampled rows computed one by one by the oracle
    wl = W.krr_laplace_mix(seed=0)
    n = wl.n
    a = W.random_block(n, 1, seed=44)[:, 0]
    b = W.random_block(n, 1, seed=45)[:, 0]
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.LAPLACE, wl.bandwidth)
    G = op.grad_points(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), mode=ops.FAST).cpu().numpy()
    rows = np.random.default_rng(46).choice(n, 48, replace=False)
    Go = O.kernel_grad_points(O.LAPLACE, wl.X, a, b, wl.bandwidth, rows_per_block=8, rows=rows)
    err = np.linalg.norm(G[rows] - Go) / np.linalg.norm(Go)
    # measured 7.4e-4: 200000-term sums of BF16-split products
    assert err <= 3e-3, err


def test_solve_gradient_matches_finite_differences():
    # L(X) = w^T x with x = (K(X) + lam I)^-1 y: the adjoint solve plus the point
    # gradient against central differences of the FP64 dense solve
    n, d, bw, lam = 300, 3, 1.0, 1.0
    X = W.random_points(n, d, seed=47)
    y = W.random_block(n, 1, seed=48)
    w = W.random_block(n, 1, seed=49)[:, 0].astype(np.float64)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, bw)
    res = ops.pcg_solve(op, torch.from_numpy(y).cuda(), [lam], tol=1e-8, maxit=2000,
                        refine_mode=ops.EXACT, check_mode=ops.EXACT)
    assert res.converged
    g, _, _, _ = ops.pcg_adjoint(op, res.x[:, 0], torch.from_numpy(w).cuda(), lam, tol=1e-8, maxit=2000,
                                 refine_mode=ops.EXACT, check_mode=ops.EXACT)
    G = ops.solve_grad_points(op, res.x[:, 0], g, mode=ops.EXACT).cpu().numpy()

    X64 = X.astype(np.float64)

    def loss(Y):
        return w @ np.linalg.solve(O.kernel_matrix(O.RBF, Y, Y, bw) + lam * np.eye(n), y[:, 0].astype(np.float64))

    eps = 1e-5
    for i, k in [(0, 0), (57, 2), (150, 1), (299, 0)]:
        Xp, Xm = X64.copy(), X64.copy()
        Xp[i, k] += eps
        Xm[i, k] -= eps
        fd = (loss(Xp) - loss(Xm)) / (2 * eps)
        assert abs(G[i, k] - fd) <= 1e-4 * np.abs(G).max(), (i, k, G[i, k], fd)
