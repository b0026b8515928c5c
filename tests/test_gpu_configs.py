"""The other workload shapes at sizes the FP64 oracle finishes in seconds:
the Matern workload (z-scored uniform points, lengthscale 1 and the flagged
sqrt(d) variant), the block workload (d = 128, right-hand sides x shifts,
whose PCG products run on the tensor-core contraction path), and the
hyper-parameter workload's solve.  Acceptance as in test_gpu_solver.py: FP64
relative residual <= 1e-6 per column and ||x - x*|| / ||x*|| <= 1e-4, with
the FP64 operator for refinement and checks and with the library defaults.
The benchmark's own mode mix (fast inner products and sketch, direct-
difference refinement and checks, rank 500) runs on the benchmark's data
generator at n = 16384 against a dense FP64 Cholesky solve."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import cmatvec
from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


MODES = {"exact": dict(refine_mode=ops.EXACT, check_mode=ops.EXACT), "default": dict()}


def _accept(kind, X, bw, lams, B, Xg, dense=True):
    n = len(X)
    if dense:
        K = O.kernel_matrix(kind, X, X, bw)
    for c in range(Xg.shape[1]):
        lam = lams[c]
        b = B[:, c % B.shape[1]].astype(np.float64)
        x = Xg[:, c]
        kx = K @ x if dense else cmatvec.kernel_matvec(kind, X, x, bw)
        rr = np.linalg.norm(kx + lam * x - b) / np.linalg.norm(b)
        assert rr <= 1e-6, (c, rr)
        if dense:
            xs = sla.cho_solve(sla.cho_factor(K + lam * np.eye(n)), b)
            assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-4, c


@pytest.mark.parametrize("modes", ["exact", "default"])
@pytest.mark.parametrize("lengthscale", [1.0, float(np.sqrt(32))])
def test_matern_workload_scaled(lengthscale, modes):
    wl = W.krr_matern_large(seed=0, n=6000, lengthscale=lengthscale, rank=200)
    lam = 1e-7 * 1_000_000  # the full-size shift
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.MATERN52, lengthscale)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(wl.n, 200, seed=0)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=400,
                        **MODES[modes])
    assert res.converged
    _accept(O.MATERN52, wl.X, lengthscale, [lam], wl.B, res.x.cpu().numpy())


@pytest.mark.parametrize("modes", ["exact", "default"])
def test_block_workload_scaled(modes):
    # d = 128 RBF, 8 right-hand sides x 4 shifts = 32 columns: the PCG products
    # use the tensor-core contraction kernel, the preconditioner the FP32 block
    # products
    n, nrhs, n_shifts = 3000, 8, 4
    wl = W.krr_rbf_block(seed=0, n=n, nrhs=nrhs, n_shifts=n_shifts, rank=150)
    lams = list(np.logspace(-4, -2, n_shifts) * n)
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 150, seed=0)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), lams, nys=ny, tol=1e-6, maxit=500,
                        **MODES[modes])
    assert res.converged
    cols_lam = [lams[c // nrhs] for c in range(nrhs * n_shifts)]
    _accept(O.RBF, wl.X, wl.bandwidth, cols_lam, wl.B, res.x.cpu().numpy())


@pytest.mark.parametrize("modes", ["exact", "default"])
def test_hyper_workload_solve_scaled(modes):
    wl = W.krr_rbf_hyper(seed=0, n=5000, nval=1000)
    lam = 1e-4 * 100_000
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(wl.n, 100, seed=0)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=300,
                        **MODES[modes])
    assert res.converged
    _accept(O.RBF, wl.X, wl.bandwidth, [lam], wl.B, res.x.cpu().numpy())


def test_laplace_mixture_full_size_sampled_rows():
    # the benchmark workload at its full size, in the launch configuration the
    # benchmark times: FP64 residual on sampled rows (host oracle), and the
    # preconditioner's eigenvalues are positive and descending
    wl = W.krr_laplace_mix(seed=0)
    lam = float(wl.lambdas[0])
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.LAPLACE, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(wl.n, wl.rank, seed=0)).cuda())
    lam_hat, _ = ny.eigs()
    assert np.all(np.diff(lam_hat.numpy()) <= 0) and lam_hat[0] > 0
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=500)
    assert res.converged
    x = res.x.cpu().numpy()[:, 0]
    b = wl.B[:, 0].astype(np.float64)
    # the host oracle's FP64 residual on 512 random rows (other rows than the
    # solver's stride sample) agrees with the solver's certified estimate
    rows = np.random.default_rng(3).choice(wl.n, 512, replace=False)
    kx = cmatvec.kernel_matvec(O.LAPLACE, wl.X, x, wl.bandwidth, Z=wl.X[rows])
    r_s = b[rows] - kx - lam * x[rows]
    est = np.sqrt(wl.n / len(rows)) * np.linalg.norm(r_s) / np.linalg.norm(b)
    assert est <= 1e-6, est
    assert abs(est - res.true_relres[0]) <= 0.25 * est, (est, res.true_relres[0])


def test_benchmark_path_scaled_n16384():
    # the benchmark's mode mix on its generator at n = 16384 (same sigma, lam / n
    # and rank): FP64 residual on every row and the error against a dense FP64
    # Cholesky solve
    n = 16384
    wl = W.krr_laplace_mix(seed=0, n=n, rank=500)
    lam = 1e-6 * n
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.LAPLACE, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 500, seed=0)).cuda(), mode=ops.FAST)
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=500, refine_every=30,
                        inner_mode=ops.FAST, refine_mode=ops.PLAIN, check_mode=ops.PLAIN)
    assert res.converged
    _accept(O.LAPLACE, wl.X, wl.bandwidth, [lam], wl.B, res.x.cpu().numpy())


def test_block_workload_all_columns_n8000():
    """The block workload's full shape at n = 8000: d = 128, RBF sigma =
    sqrt(128), 64 right-hand sides x 16 shifts lam in logspace(-8, -3) n
    (1024 columns, one solve), rank 800, the library's default modes.  Every
    column must meet the paper's acceptance test (FP64 relative residual
    <= 1e-6, against the oracle's dense K), and for the smallest and the
    largest shift the first right-hand side must match a dense Cholesky
    solve to 1e-4."""
    n, nrhs, n_shifts, r = 8000, 64, 16, 800
    wl = W.krr_rbf_block(seed=0, n=n, nrhs=nrhs, n_shifts=n_shifts, rank=r)
    lams = [float(x) for x in wl.lambdas]
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=0)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), lams, nys=ny, tol=1e-6, maxit=500)
    assert res.converged
    Xg = res.x.cpu().numpy()
    K = O.kernel_matrix(O.RBF, wl.X, wl.X, wl.bandwidth)
    lam_col = np.repeat(np.asarray(lams), nrhs)
    Bc = np.tile(wl.B.astype(np.float64), (1, n_shifts))
    R = K @ Xg + lam_col[None, :] * Xg - Bc
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bc, axis=0)
    assert np.all(rel <= 1e-6), (int(np.argmax(rel)), rel.max())
    for s in (0, n_shifts - 1):
        xs = sla.cho_solve(sla.cho_factor(K + lams[s] * np.eye(n)), wl.B[:, 0].astype(np.float64))
        x = Xg[:, s * nrhs]
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-4, s
