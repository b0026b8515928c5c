"""Parity of the Nystrom preconditioner and of block PCG with the FP64 oracle.

Acceptance per solved column (the paper's accuracy check, App. B.2): the true
relative residual ||(K + lam I) x - b|| / ||b||, computed by the oracle in
FP64, is <= 1e-6, and ||x - x*|| / ||x*|| <= 1e-4 against a dense FP64
Cholesky solve.  These problems are small and badly conditioned (kappa up to
4e3), where FP32 kernel values alone leave an FP64 residual floor near 1e-6.
Each solve runs twice: with the FP64 operator (KOP_EXACT) for refinement and
checks, and with the library's defaults (direct-difference FP32 checks whose
candidate stops the solver certifies with a sampled FP64 residual); both must
meet the FP64 acceptance on every row."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _dense_solve(kind, X, bw, lam, B):
    K = O.kernel_matrix(kind, X, X, bw)
    cf = sla.cho_factor(K + lam * np.eye(len(X)))
    return K, sla.cho_solve(cf, B.astype(np.float64))


# refinement / check operators: the FP64 operator, or the library defaults
MODES = {"exact": dict(refine_mode=ops.EXACT, check_mode=ops.EXACT), "default": dict()}


def _check_cols(K, lam_cols, B, Xg, xs):
    for c in range(Xg.shape[1]):
        b = B[:, c % B.shape[1]].astype(np.float64)
        x = Xg[:, c].astype(np.float64)
        rr = np.linalg.norm(K @ x + lam_cols[c] * x - b) / np.linalg.norm(b)
        err = np.linalg.norm(x - xs[c]) / np.linalg.norm(xs[c])
        assert rr <= 1e-6, (c, rr)
        assert err <= 1e-4, (c, err)


def test_nystrom_matches_oracle():
    n, d, r = 1500, 16, 60
    wl = W.krr_rbf_small(seed=1, n=n, d=d)
    X = torch.from_numpy(wl.X).cuda()
    Om = W.gaussian_sketch(n, r, seed=1)
    op = ops.KernelOperator(X, ops.RBF, wl.bandwidth)
    nu_rel = 1e-5
    ny = ops.Nystrom(op, torch.from_numpy(Om).cuda(), nu_rel=nu_rel, mode=ops.ACCURATE)
    lam_g, nu_g = ny.eigs()
    K = O.kernel_matrix(O.RBF, wl.X, wl.X, wl.bandwidth)
    U_o, lam_o, nu_o = O.nystrom(K @ Om.astype(np.float64), Om, nu_rel=nu_rel)
    assert abs(nu_g - nu_o) <= 1e-6 * nu_o
    # Weyl: |lam_gpu - lam_oracle| <= ||E||, E the sketch's operator error
    # (FP32-level, ~1e-6 of ||K||), so the bound is absolute in lam_1
    big = lam_o > 1e3 * nu_o
    np.testing.assert_allclose(lam_g.numpy()[big], lam_o[big], rtol=1e-5, atol=2e-6 * lam_o[0])
    U = ny.factor().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(U.T @ U - np.eye(r)) < 1e-5
    # preconditioner action against the oracle's, both damping modes
    V = W.random_block(n, 3, seed=2)
    for adaptive in (True, False):
        mu = 0.15
        got = ny.apply(torch.from_numpy(V).cuda(), [mu] * 3, adaptive=adaptive).cpu().numpy()
        rho = O.nystrom_rho(lam_o, mu, adaptive)
        ref = O.precond_apply(U_o, lam_o, mu, rho, V.astype(np.float64))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4


def test_preconditioner_spd_small():
    n, r = 384, 24
    X = W.random_points(n, 8, seed=5)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.LAPLACE, 3.0)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=5)).cuda())
    lam, _ = ny.eigs()
    mu = 0.05
    Pm = ny.apply(torch.eye(n, device="cuda"), [mu] * n).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Pm - Pm.T)) < 1e-5 * np.max(np.abs(Pm))
    ev = np.linalg.eigvalsh(0.5 * (Pm + Pm.T))
    lo = 1.0 / (lam[0].item() + mu)
    assert ev[0] > 0.99 * lo and ev[-1] < 1.01 / mu


@pytest.mark.parametrize("modes", ["exact", "default"])
@pytest.mark.parametrize("inner", [ops.FAST, ops.PLAIN, ops.ACCURATE])
def test_krr_rbf_small_full_size(inner, modes):
    # the 4096 x 16 RBF workload at its full size, direct FP64 solve as reference
    wl = W.krr_rbf_small(seed=0)
    lam = float(wl.lambdas[0])
    K, xs = _dense_solve(O.RBF, wl.X, wl.bandwidth, lam, wl.B[:, 0])
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.RBF, wl.bandwidth)
    Om = torch.from_numpy(W.gaussian_sketch(wl.n, wl.rank, seed=0)).cuda()
    ny = ops.Nystrom(op, Om, mode=inner if inner != ops.ACCURATE else ops.FAST)
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=500, refine_every=20,
                        inner_mode=inner, **MODES[modes])
    assert res.converged
    _check_cols(K, [lam], wl.B, res.x.cpu().numpy(), [xs])
    # the reported residual is the FP64 one (every row is sampled at this n)
    rr = np.linalg.norm(K @ res.x.cpu().numpy()[:, 0] + lam * res.x.cpu().numpy()[:, 0] - wl.B[:, 0]) / \
        np.linalg.norm(wl.B[:, 0].astype(np.float64))
    assert abs(res.true_relres[0] - rr) <= 1e-3 * rr + 1e-12
    # preconditioning pays off: plain CG needs more iterations
    cg = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=None, tol=1e-6, maxit=3000, **MODES[modes])
    assert cg.converged and cg.iters[0] > res.iters[0]


@pytest.mark.parametrize("modes", ["exact", "default"])
@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE, ops.MATERN52])
def test_block_shifts_ragged(kind, modes):
    n, d, nrhs = 1000, 20, 3
    X = W.random_points(n, d, seed=11)
    B = W.random_block(n, nrhs, seed=12)
    bw = float(np.sqrt(d))
    lams = [0.05, 0.5]
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 50, seed=3)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(B).cuda(), lams, nys=ny, tol=1e-6, maxit=800, **MODES[modes])
    assert res.converged
    Xg = res.x.cpu().numpy()
    K = O.kernel_matrix(kind, X, X, bw)
    cols_lam = [lams[c // nrhs] for c in range(len(lams) * nrhs)]
    xs = [sla.cho_solve(sla.cho_factor(K + cols_lam[c] * np.eye(n)), B[:, c % nrhs].astype(np.float64))
          for c in range(len(cols_lam))]
    _check_cols(K, cols_lam, B, Xg, xs)


def test_identity_preconditioner_is_cg_and_edge_cases():
    n = 129
    X = W.random_points(n, 3, seed=2)
    B = W.random_block(n, 2, seed=3)
    B[:, 1] = 0.0
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, 1.0)
    res = ops.pcg_solve(op, torch.from_numpy(B).cuda(), [0.3], nys=None, tol=1e-7, maxit=600,
                        refine_mode=ops.EXACT, check_mode=ops.EXACT)
    assert res.converged
    assert res.iters[1] == 0 and np.all(res.x.cpu().numpy()[:, 1] == 0.0)
    K = O.kernel_matrix(O.RBF, X, X, 1.0)
    xo, _, _ = O.pcg(lambda v: K @ v + 0.3 * v, B[:, 0].astype(np.float64), None, tol=1e-10, maxit=500)
    x = res.x.cpu().numpy()[:, 0]
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-5
    # maxit reached: warning status, iterate written
    r1 = ops.pcg_solve(op, torch.from_numpy(B[:, :1].copy()).cuda(), [0.3], tol=1e-12, maxit=2,
                       refine_mode=ops.EXACT, check_mode=ops.EXACT)
    assert r1.status == 1 and r1.iters[0] == 2
    assert np.all(np.isfinite(r1.x.cpu().numpy()))


def test_single_point():
    X = np.array([[0.5, -1.0]], dtype=np.float32)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.MATERN52, 1.0)
    res = ops.pcg_solve(op, torch.tensor([[2.0]], device="cuda"), [1.0], tol=1e-6, maxit=5)
    assert res.converged
    assert abs(res.x.cpu().item() - 1.0) < 1e-6  # (1 + 1) x = 2


def test_laplace_mixture_accurate_refinement_n20000():
    # the benchmark workload's distribution at n = 20000 (same lam): the FP32
    # accurate operator with compensated sums is enough for the true residual;
    # the FP64 residual is checked with the host oracle on all rows
    from oracle import cmatvec
    wl = W.krr_laplace_mix(seed=0, n=20000, rank=200)
    lam = 1e-6 * 200000
    op = ops.KernelOperator(torch.from_numpy(wl.X).cuda(), ops.LAPLACE, wl.bandwidth)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(wl.n, 200, seed=0)).cuda())
    res = ops.pcg_solve(op, torch.from_numpy(wl.B).cuda(), [lam], nys=ny, tol=1e-6, maxit=500,
                        inner_mode=ops.FAST, refine_mode=ops.ACCURATE)
    assert res.converged
    x = res.x.cpu().numpy()[:, 0]
    b = wl.B[:, 0].astype(np.float64)
    kx = cmatvec.kernel_matvec(O.LAPLACE, wl.X, x, wl.bandwidth)
    rr = np.linalg.norm(kx + lam * x - b) / np.linalg.norm(b)
    assert rr <= 1e-6
    # the solver's own certified estimate (1024 sampled FP64 rows) of that residual
    assert abs(res.true_relres[0] - rr) <= 0.1 * rr
