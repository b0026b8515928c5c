"""Ridge normal operator X^T X (kop_create_ridge) and NysPCG on the paper's
ridge data (Sec. 5.1: X = U Sigma_alpha V^T, y = U g / ||g||) against the FP64
oracle."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


# FP32 sums; error-free sums (their only error is the FP32 output rounding,
# 2^-24 of |O| <= the scale below)
@pytest.mark.parametrize("mode,tol", [(ops.FAST, 1e-5), (ops.ACCURATE, 1e-7), (ops.PLAIN, 1e-7)])
def test_ridge_matvec_matches_oracle(mode, tol):
    wl = W.ridge_spectral(seed=1, n=3000, p=700, alpha=1.0)
    V = W.random_block(700, 11, seed=2)
    want = O.ridge_normal_matvec(wl.X, V)
    op = ops.RidgeOperator(torch.from_numpy(wl.X).cuda())
    got = op.matvec(torch.from_numpy(V).cuda(), mode=mode).cpu().numpy()
    # relative to the sum of |terms|: |X|^T |X| |V|
    Xa = np.abs(wl.X.astype(np.float64))
    scale = Xa.T @ (Xa @ np.abs(V.astype(np.float64)))
    err = np.max(np.abs(got - want) / scale)
    assert err <= tol, err
    got64 = op.matvec_f64(torch.from_numpy(V.astype(np.float64)).cuda()).cpu().numpy()
    assert np.max(np.abs(got64 - want) / scale) <= 1e-13


@pytest.mark.parametrize("alpha,lam", [(1.0, 1e-4), (2.0, 1e-6), (0.5, 1e-2)])
def test_ridge_nystrom_pcg(alpha, lam):
    n, p, r = 4096, 1024, 128
    wl = W.ridge_spectral(seed=0, n=n, p=p, alpha=alpha, lam=lam)
    X64 = wl.X.astype(np.float64)
    b = O.ridge_rhs(X64, wl.y)
    op = ops.RidgeOperator(torch.from_numpy(wl.X).cuda())
    Om = torch.from_numpy(W.gaussian_sketch(p, r, seed=0)).cuda()
    ny = ops.Nystrom(op, Om, mode=ops.FAST)
    res = ops.pcg_solve(op, torch.from_numpy(b.astype(np.float32)[:, None]).cuda(), [lam], nys=ny, tol=5e-7,
                        maxit=500, refine_mode=ops.ACCURATE, check_mode=ops.EXACT)
    assert res.converged
    w = res.x.cpu().numpy()[:, 0]
    bf = b.astype(np.float32).astype(np.float64)
    rr = np.linalg.norm(X64.T @ (X64 @ w) + lam * w - bf) / np.linalg.norm(bf)
    assert rr <= 1e-6, rr
    wd = np.linalg.solve(X64.T @ X64 + lam * np.eye(p), bf)
    kappa = (1 + lam) / (p ** -alpha + lam)
    assert np.linalg.norm(w - wd) / np.linalg.norm(wd) <= 2e-6 * kappa
    # the preconditioner's eigenvalues are the oracle's for the same test matrix
    # and shift (Weyl: within the FP32 sketch error), and never above the true
    # spectrum i^-alpha (a Nystrom approximation is below A)
    lam_hat = ny.eigs()[0].numpy()
    Omn = W.gaussian_sketch(p, r, seed=0).astype(np.float64)
    _, lam_o, _ = O.nystrom(O.ridge_normal_matvec(X64, Omn), Omn, nu_rel=2.0 ** -16)
    assert np.all(np.abs(lam_hat - lam_o) <= 1e-5 * lam_o[0] + 1e-4 * lam_o)
    assert np.all(lam_hat[:10] <= np.arange(1, 11, dtype=np.float64) ** -alpha * (1 + 1e-4))
    assert res.iters[0] < 120
