"""Rank adaptation of the Nystrom approximation (nys_build_adaptive) against
the FP64 oracle (oracle.kop_oracle.nystrom_adaptive): the same test matrix,
start vector, power iterations and tolerance.  The GPU side runs the build and
the error estimate's products with the accurate operator."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu

NU_REL = 2.0 ** -21


def _case(n=3000, d=8, bw_factor=2.0, rmax=256):
    X = W.random_points(n, d, seed=21)
    bw = bw_factor * float(np.sqrt(d))
    Om = W.gaussian_sketch(n, rmax, seed=0)
    g0 = W.random_block(n, 1, seed=5)[:, 0]
    return X, bw, Om, g0


def test_adaptive_rank_matches_oracle():
    X, bw, Om, g0 = _case()
    K = O.kernel_matrix(O.RBF, X, X, bw)
    A = lambda V: K @ V
    # tolerance halfway (geometrically) between the ratios est / lam_hat_1 of
    # ranks 32 and 64 of the oracle, so that the accepted rank is 64 with margin
    *_, hist_all = O.nystrom_adaptive(A, Om, 8, 256, 10, 0.0, g0, nu_rel=NU_REL)
    lam1 = {}
    for rk, _ in hist_all:
        lam1[rk] = O.nystrom(A(Om[:, :rk]), Om[:, :rk], NU_REL)[1][0]
    ratio = {rk: e / lam1[rk] for rk, e in hist_all}
    tol = float(np.sqrt(ratio[32] * ratio[64]))
    assert ratio[32] > 2 * tol and ratio[64] < tol / 2
    U, lam_o, _, r_o, est_o, hist_o = O.nystrom_adaptive(A, Om, 8, 256, 10, tol, g0, nu_rel=NU_REL)
    assert r_o == 64

    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, bw)
    ny = ops.Nystrom.adaptive(op, torch.from_numpy(Om).cuda(), 8, 256, g0=torch.from_numpy(g0).cuda(),
                              power_iters=10, err_tol=tol, nu_rel=NU_REL, mode=ops.ACCURATE)
    assert ny.r == 64
    assert [h[0] for h in ny.hist] == [h[0] for h in hist_o] == [8, 16, 32, 64]
    for (rk, e_g), (_, e_o) in zip(ny.hist, hist_o):
        assert abs(e_g - e_o) <= 2e-3 * e_o, (rk, e_g, e_o)
    assert abs(ny.err_est - est_o) <= 2e-3 * est_o
    lam_g, _ = ny.eigs()
    lam_g = lam_g.numpy()
    assert len(lam_g) == 64
    assert np.all(np.abs(lam_g - lam_o) <= 2e-6 * lam_o[0] + 1e-5 * lam_o), np.max(np.abs(lam_g - lam_o))


def test_adaptive_rank_doubles_and_caps():
    X, bw, Om, g0 = _case(n=2000, rmax=100)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, bw)
    ny = ops.Nystrom.adaptive(op, torch.from_numpy(Om).cuda(), 24, 100, g0=torch.from_numpy(g0).cuda(),
                              power_iters=3, err_tol=0.0, nu_rel=NU_REL, mode=ops.ACCURATE)
    assert [h[0] for h in ny.hist] == [24, 48, 96, 100] and ny.r == 100
    # each rank's estimate (3 power iterations from g0) as in the oracle
    K = O.kernel_matrix(O.RBF, X, X, bw)
    *_, hist_o = O.nystrom_adaptive(lambda V: K @ V, Om, 24, 100, 3, 0.0, g0, nu_rel=NU_REL)
    assert [h[0] for h in hist_o] == [24, 48, 96, 100]
    for (rk, e_g), (_, e_o) in zip(ny.hist, hist_o):
        assert abs(e_g - e_o) <= 2e-3 * e_o, (rk, e_g, e_o)


def test_adaptive_preconditioner_solves():
    # the accepted approximation preconditions the solve: FP64 relres <= 1e-6
    X, bw, Om, g0 = _case(n=3000, rmax=128)
    y = np.sin(X @ (np.ones(X.shape[1]) / np.sqrt(X.shape[1]))).astype(np.float32)[:, None]
    lam = 1e-3 * X.shape[0]
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, bw)
    ny = ops.Nystrom.adaptive(op, torch.from_numpy(Om).cuda(), 16, 128, g0=torch.from_numpy(g0).cuda(),
                              power_iters=10, err_tol=1e-3, nu_rel=NU_REL, mode=ops.ACCURATE)
    res = ops.pcg_solve(op, torch.from_numpy(y).cuda(), [lam], nys=ny, tol=5e-7, maxit=300,
                        refine_mode=ops.EXACT, check_mode=ops.EXACT)
    assert res.converged
    K = O.kernel_matrix(O.RBF, X, X, bw)
    x = res.x.cpu().numpy()[:, 0]
    b = y[:, 0].astype(np.float64)
    assert np.linalg.norm(K @ x + lam * x - b) / np.linalg.norm(b) <= 1e-6
