"""Solves with the kernel matrix of the checks kept in device memory
(kop_set_check_cache) against the same solves without it.  The first check
product of a solve stores K(X, X) as the direct-difference operator computes
it; later checks of that solve multiply the stored matrix with the same
error-free contraction.  So the solver takes the same decisions, its outputs
agree up to the order of the compensated sums, the residual it reports is
the certified FP64 residual, which matches the oracle's, and the oracle's
FP64 residual of every accepted iterate meets the tolerance (the paper's
acceptance test, App. B.2)."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W
from paper_2609_08136_b300._ffi import KopError

pytestmark = pytest.mark.gpu

_KIND = {ops.RBF: O.RBF, ops.LAPLACE: O.LAPLACE, ops.MATERN52: O.MATERN52}


def _solve(op, B, lams, ny, cache, **kw):
    if cache == "library":
        op.set_check_cache(True)
    elif cache == "buffer":
        # caller-owned memory, one float past the end to spare
        op.set_check_cache(True, torch.empty(op.check_cache_floats() + 1, device="cuda"))
    try:
        return ops.pcg_solve(op, torch.from_numpy(B).cuda(), lams, nys=ny, **kw)
    finally:
        op.set_check_cache(False)


# n ragged against the 32-key tiles and the 128-point row blocks, odd and even
# numbers of row blocks (24, 16, 12, 1); 2 x cols = 2, 6 and 10 columns cover
# one, one and two column blocks of the stored product
@pytest.mark.parametrize("kind,n,nrhs,lams", [
    (ops.LAPLACE, 3001, 1, [1e-3]),
    (ops.RBF, 2000, 3, [1e-3]),
    (ops.MATERN52, 1500, 1, [1e-3, 3e-3, 1e-2, 3e-2, 1e-1]),
    (ops.LAPLACE, 37, 2, [1e-2]),
])
def test_cached_checks_match_direct_checks(kind, n, nrhs, lams):
    d = 8
    X = W.random_points(n, d, seed=n)
    bw = 2.0 * np.sqrt(d)
    B = W.random_block(n, nrhs, seed=n + 1)
    lam_abs = [l * n for l in lams]
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    r = min(64, n)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=n)).cuda())
    # refinement every 5 iterations: many check products per solve
    kw = dict(tol=1e-6, maxit=400, refine_every=5)
    a = _solve(op, B, lam_abs, ny, None, **kw)
    b = _solve(op, B, lam_abs, ny, "library", **kw)
    c = _solve(op, B, lam_abs, ny, "buffer", **kw)
    assert a.converged and b.converged and c.converged
    assert a.iters == b.iters == c.iters
    xa, xb, xc = a.x.cpu().numpy(), b.x.cpu().numpy(), c.x.cpu().numpy()
    assert np.max(np.abs(xa - xb)) <= 1e-6 * np.max(np.abs(xa))
    assert np.max(np.abs(xc - xb)) <= 1e-6 * np.max(np.abs(xa))
    # the stored matrix is multiplied in another order (each stored tile used
    # for its row and its column contributions), so each refinement replaces
    # the residual by one that differs in the last bits and the iterates drift
    # apart (to ~1e-7 of max |x| here); near the tolerance that moves the final
    # FP64 residual by up to ~20% of it, so the direct and stored runs are each
    # checked against the oracle below rather than against each other.  The
    # library's and the caller's memory run the same code; the solver's FP64
    # reductions add their block sums atomically in any order, which moves the
    # reported residual by ~1e-8 of itself.
    np.testing.assert_allclose(c.true_relres, b.true_relres, rtol=1e-5, atol=0.0)
    assert max(a.true_relres) <= kw["tol"] and max(b.true_relres) <= kw["tol"]
    # the oracle's FP64 residual of each accepted iterate meets the tolerance,
    # and the reported residual is that FP64 residual: exact here (n <= 4096,
    # so the solver's FP64 certification covers every row) up to the FP64
    # rounding of the two products
    K = O.kernel_matrix(_KIND[kind], X, X, bw)
    xb2 = xb.reshape(n, -1)
    for col in range(xb2.shape[1]):
        bc = B[:, col % nrhs].astype(np.float64)
        lam = lam_abs[col // nrhs]
        nb = np.linalg.norm(bc)
        for res, xx in ((a, xa.reshape(n, -1)), (b, xb2)):
            rr = np.linalg.norm(K @ xx[:, col] + lam * xx[:, col] - bc) / nb
            assert rr <= 1e-6, (col, rr)
            assert abs(res.true_relres[col] - rr) <= 1e-3 * rr, (col, res.true_relres[col], rr)


def test_cached_checks_in_the_adjoint():
    n, d = 2500, 8
    X = W.random_points(n, d, seed=3)
    bw = 2.0 * np.sqrt(d)
    lam = 1e-3 * n
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, bw)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 64, seed=3)).cuda())
    x = torch.from_numpy(W.random_block(n, 1, seed=4)[:, 0].astype(np.float64)).cuda()
    dl = torch.from_numpy(W.random_block(n, 1, seed=5)[:, 0].astype(np.float64)).cuda()
    kw = dict(tol=1e-6, maxit=400, refine_every=5)
    g0, dlam0, dbw0, it0 = ops.pcg_adjoint(op, x, dl, lam, nys=ny, **kw)
    op.set_check_cache(True)
    try:
        g1, dlam1, dbw1, it1 = ops.pcg_adjoint(op, x, dl, lam, nys=ny, **kw)
    finally:
        op.set_check_cache(False)
    assert it0 == it1
    assert torch.max(torch.abs(g0 - g1)).item() <= 1e-6 * torch.max(torch.abs(g0)).item()
    assert abs(dlam1 - dlam0) <= 1e-6 * abs(dlam0) and abs(dbw1 - dbw0) <= 1e-6 * abs(dbw0)


def test_cache_reserves_and_frees_memory():
    n = 3001
    op = ops.KernelOperator(torch.from_numpy(W.random_points(n, 4, seed=1)).cuda(), ops.RBF, 2.0)
    need = 24 * 13 * 128 * 128 * 4  # 24 row blocks x 13 band tiles of 128 x 128 floats
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    op.set_check_cache(True)
    op.set_check_cache(True)  # already reserved: no second buffer
    f1 = torch.cuda.mem_get_info()[0]
    op.set_check_cache(False)
    f2 = torch.cuda.mem_get_info()[0]
    assert need <= f0 - f1 <= need + (64 << 20)
    assert f2 - f1 >= need


def test_cache_refused_when_it_does_not_fit_and_for_ridge():
    # 3125 row blocks x 1563 band tiles x 64 KB = 320 GB: more than the device
    # holds, nothing reserved
    n = 400_000
    op = ops.KernelOperator(torch.from_numpy(W.random_points(n, 1, seed=2)).cuda(), ops.RBF, 1.0)
    f0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(KopError, match="not enough free device memory"):
        op.set_check_cache(True)
    assert torch.cuda.mem_get_info()[0] >= f0 - (64 << 20)
    rop = ops.RidgeOperator(torch.from_numpy(W.random_block(50, 8, seed=1)).cuda())
    with pytest.raises(KopError, match="ridge"):
        rop.set_check_cache(True)


def test_caller_buffer_checked():
    n = 500
    op = ops.KernelOperator(torch.from_numpy(W.random_points(n, 4, seed=6)).cuda(), ops.RBF, 2.0)
    need = op.check_cache_floats()
    assert need == 4 * 3 * 128 * 128  # 4 row blocks x 3 band tiles
    with pytest.raises(KopError, match="buffer smaller"):
        op.set_check_cache(True, torch.empty(need - 1, device="cuda"))
    buf = torch.empty(need + 4, device="cuda")
    with pytest.raises(KopError, match="aligned"):
        op.set_check_cache(True, buf[1:])
    op.set_check_cache(True, buf)
    op.set_check_cache(False)


@pytest.mark.parametrize("kind,n,nrhs", [(ops.LAPLACE, 6001, 1), (ops.MATERN52, 5000, 3)])
def test_computed_checks_match_stored_checks(kind, n, nrhs):
    """Beyond 4096 rows the solver's checks run the direct-difference
    operator: from the stored matrix, or (no stored matrix) with each pair of
    row blocks computed once in shared memory by the build's arithmetic and
    used for both of its contributions.  The two forms give the same check
    products, so the solves take the same decisions, and the oracle's FP64
    residual of the accepted iterates meets the tolerance."""
    d = 8
    X = W.random_points(n, d, seed=n)
    bw = 2.0 * np.sqrt(d)
    B = W.random_block(n, nrhs, seed=n + 1)
    lam = 1e-3 * n
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 64, seed=n)).cuda())
    # refinements with the check operator every 5 iterations, stops certified
    # by the FP64 operator: every check product is a plain refinement
    kw = dict(tol=1e-6, maxit=400, refine_every=5, refine_mode=ops.PLAIN, check_mode=ops.EXACT)
    a = _solve(op, B, [lam], ny, None, **kw)
    b = _solve(op, B, [lam], ny, "library", **kw)
    assert a.converged and b.converged
    assert a.iters == b.iters
    xa, xb = a.x.cpu().numpy(), b.x.cpu().numpy()
    assert np.allclose(xa, xb, rtol=0, atol=1e-9 * np.abs(xb).max())
    K = O.kernel_matrix(_KIND[kind], X.astype(np.float64), X.astype(np.float64), bw)
    for c in range(nrhs):
        r = B[:, c] - (K @ xa[:, c] + lam * xa[:, c])
        assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(B[:, c]) * (1 + 1e-9)
