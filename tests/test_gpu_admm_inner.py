"""Warm-started PCG (pcg_solve x0) and the NysADMM linear solve
(ops.NysADMMLinearSolver) on the ridge normal operator, against dense FP64
solves."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _ridge(n=4096, p=1024, alpha=1.0):
    wl = W.ridge_spectral(seed=2, n=n, p=p, alpha=alpha)
    X64 = wl.X.astype(np.float64)
    return wl, X64.T @ X64, ops.RidgeOperator(torch.from_numpy(wl.X).cuda())


def test_warm_start_from_the_solution_takes_no_iterations():
    wl, A, op = _ridge()
    b = O.ridge_rhs(wl.X, wl.y).astype(np.float32)
    lam = 1e-3
    xs = O.shifted_solve(A, b.astype(np.float64), lam)
    bd = torch.from_numpy(b[:, None]).cuda()
    res = ops.pcg_solve(op, bd, [lam], tol=1e-6, maxit=500, refine_mode=ops.EXACT, check_mode=ops.EXACT,
                        x0=torch.from_numpy(xs[:, None]).cuda())
    assert res.converged and res.iters[0] == 0
    assert np.allclose(res.x.cpu().numpy()[:, 0], xs)
    # a perturbed start needs fewer iterations than x0 = 0
    cold = ops.pcg_solve(op, bd, [lam], tol=1e-8, maxit=2000, refine_mode=ops.EXACT, check_mode=ops.EXACT)
    x0 = xs * (1 + 1e-3 * np.random.default_rng(3).standard_normal(len(xs)))
    warm = ops.pcg_solve(op, bd, [lam], tol=1e-8, maxit=2000, refine_mode=ops.EXACT, check_mode=ops.EXACT,
                         x0=torch.from_numpy(x0[:, None]).cuda())
    assert cold.converged and warm.converged and warm.iters[0] < cold.iters[0]
    for r in (cold, warm):
        x = r.x.cpu().numpy()[:, 0]
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8 * (1 + lam) / (1024 ** -1.0 + lam) * 10


def test_nysadmm_linear_solves_with_changing_rho():
    wl, A, op = _ridge()
    p = A.shape[0]
    Om = torch.from_numpy(W.gaussian_sketch(p, 64, seed=1)).cuda()
    # gamma = 6 makes the later solves tight (k = 7: 8.5e-6) so that the check bites
    solver = ops.NysADMMLinearSolver(op, Om, update_freq=3, sigma=1e-6, gamma=6.0, tol_min=1e-9, maxit=2000,
                                     refine_mode=ops.ACCURATE, check_mode=ops.EXACT)
    rng = np.random.default_rng(4)
    base = O.ridge_rhs(wl.X, wl.y)
    rhs = base.copy()
    for k, rho in enumerate([1.0, 1.0, 0.5, 0.5, 0.25, 2.0, 2.0], start=1):
        rhs = rhs + 0.05 * np.linalg.norm(base) / np.sqrt(p) * rng.standard_normal(p)
        rf = rhs.astype(np.float32)
        x = solver.solve(torch.from_numpy(rf).cuda(), rho).cpu().numpy()
        assert solver.last.converged
        xs = O.shifted_solve(A, rf.astype(np.float64), rho + 1e-6)
        tol = max(1e-9, k ** -6.0)
        # the solve stops at relres <= tol; the error is at most cond times that
        kappa = (1 + rho) / (p ** -1.0 + rho)
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 2 * kappa * tol, (k, rho)
    assert solver.builds == 3  # calls 1, 4 and 7
