"""The preconditioner apply against its defining formula, evaluated in FP64 on
the factors the build stored:

    P^-1 V = V / rho + U [ (diag(lam_hat) + mu)^-1 - 1 / rho ] U^T V

(the randomized Nystrom preconditioner, Sec. 2.3; damping rho of App. A.5).
This is a property of the apply kernels alone: U and lam_hat are read back
from the device and the formula is written out here with numpy, so the check
needs no oracle.  For up to 8 columns the apply sums error-free (float-float
pairs), so what is left is the rounding of the FP32 output,
|got - ref| <= 2^-24 |ref|, plus 1e-11 of the magnitudes summed (float-float
sums carry about 2^-44 of them; the factor covers the growth of the FP32 error
word).  One input block lies along the leading eigen-directions and mu is
small, so with rho = mu the terms V / rho and U d U^T V cancel by about
lam_k / mu: FP32 sums would miss the bound by orders of magnitude.  A generic
block is checked too."""
import numpy as np
import pytest
import torch

from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu

_CACHE = {}


def _nystrom(n, r):
    key = (n, r)
    if key not in _CACHE:
        X = W.random_points(n, 16, seed=n + r)
        op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, 4.0)
        ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=r)).cuda(), nu_rel=1e-6)
        U = ny.factor().cpu().numpy().astype(np.float64)
        lam = ny.eigs()[0].numpy()
        _CACHE[key] = (op, ny, U, lam)
    return _CACHE[key]


def _formula(U, lam, mu, adaptive, V):
    """Reference in FP64 and the magnitude of the terms it sums."""
    rho = lam[-1] + mu if adaptive else mu
    d = 1.0 / (lam + mu) - 1.0 / rho
    ref = V / rho + U @ (d[:, None] * (U.T @ V))
    mag = np.abs(V) / rho + np.abs(U) @ (np.abs(d)[:, None] * (np.abs(U).T @ np.abs(V)))
    return ref, mag


def _check(n, r, m, adaptive, seed):
    op, ny, U, lam = _nystrom(n, r)
    rng = np.random.default_rng(seed)
    # along the leading eigen-directions (lam_k >= lam_1 / 10), where V / rho
    # and the projected part cancel by (lam_k + mu) / rho, and a generic block
    kt = max(1, int(np.sum(lam >= 0.1 * lam[0])))
    Vc = U[:, :kt] @ rng.standard_normal((kt, m)) + 1e-6 * rng.standard_normal((n, m))
    Vg = rng.standard_normal((n, m))
    mus = [1e-4 * lam[0] * (1 + c) for c in range(m)]
    for V, cancelling in ((Vc.astype(np.float32), True), (Vg.astype(np.float32), False)):
        got = ny.apply(torch.from_numpy(V).cuda(), mus, adaptive=adaptive).cpu().numpy().astype(np.float64)
        for c in range(m):
            ref, mag = _formula(U, lam, mus[c], adaptive, V[:, c:c + 1].astype(np.float64))
            err = np.abs(got[:, c:c + 1] - ref)
            bound = 2.0 ** -24 * np.abs(ref) * (1 + 2.0 ** -20) + 1e-11 * mag
            worst = int(np.argmax(err - bound))
            assert np.all(err <= bound), (n, r, m, adaptive, c, worst, err.flat[worst], bound.flat[worst])
            if cancelling and not adaptive:
                # the cancellation the inputs were chosen for (rho = mu here)
                assert np.median(mag / np.maximum(np.abs(ref), 1e-300)) > 1e2


@pytest.mark.parametrize("r", [24, 500, 512, 700])
@pytest.mark.parametrize("m", [1, 2, 3, 8])
def test_apply_matches_formula_to_output_rounding(r, m):
    for adaptive in (False, True):
        _check(3001, r, m, adaptive, seed=r * 10 + m)


@pytest.mark.parametrize("n,r,m", [(37, 8, 1), (37, 8, 2), (17, 16, 5), (600, 513, 1)])
def test_apply_small_and_ragged(n, r, m):
    _check(n, r, m, False, seed=n + r + m)


def test_apply_one_and_two_columns_agree():
    # the one- and two-column forms of the apply are the same operator: on
    # [v, 2 v] and on v alone they agree to the output rounding
    op, ny, U, lam = _nystrom(3001, 500)
    v = W.random_block(3001, 1, seed=9)
    V = np.concatenate([v, 2 * v], axis=1)
    mu = 1e-3 * lam[0]
    got = ny.apply(torch.from_numpy(V).cuda(), [mu, mu], adaptive=True).cpu().numpy().astype(np.float64)
    one = ny.apply(torch.from_numpy(v).cuda(), [mu], adaptive=True).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got[:, 1] - 2 * got[:, 0]) <= 2.0 ** -22 * np.abs(got[:, 1]))
    assert np.all(np.abs(got[:, :1] - one) <= 2.0 ** -22 * np.abs(one))


def _check_block(n, r, m, adaptive, seed):
    """More than 8 columns: U^T V and U W run on the tensor cores with every
    FP32 operand split exactly into three BF16 terms and FP32 sums, so each
    entry is an FP32-accurate sum: its error is a few 2^-24 of the magnitudes
    summed (chunks of 256 rows in FP32, FP64 across chunks).  The bound
    2^-17 of the summed magnitudes leaves room for that and fails for a
    missing split term (2^-8) or a misplaced tile (order 1); the error is also
    compared with a plain FP32 evaluation of the same formula."""
    op, ny, U, lam = _nystrom(n, r)
    rng = np.random.default_rng(seed)
    kt = max(1, int(np.sum(lam >= 0.1 * lam[0])))
    Vc = U[:, :kt] @ rng.standard_normal((kt, m)) + 1e-6 * rng.standard_normal((n, m))
    Vg = rng.standard_normal((n, m))
    mus = [1e-4 * lam[0] * (1 + 0.01 * c) for c in range(m)]
    U32 = U.astype(np.float32)
    for V in (Vc.astype(np.float32), Vg.astype(np.float32)):
        got = ny.apply(torch.from_numpy(V).cuda(), mus, adaptive=adaptive).cpu().numpy().astype(np.float64)
        V64 = V.astype(np.float64)
        mu = np.asarray(mus)
        rho = lam[-1] + mu if adaptive else mu
        d = 1.0 / (lam[:, None] + mu[None, :]) - 1.0 / rho[None, :]
        ref = V64 / rho + U @ (d * (U.T @ V64))
        mag = np.abs(V64) / rho + np.abs(U) @ (np.abs(d) * (np.abs(U).T @ np.abs(V64)))
        err = np.abs(got - ref)
        bound = 2.0 ** -24 * np.abs(ref) + 2.0 ** -17 * mag
        worst = np.unravel_index(int(np.argmax(err - bound)), err.shape)
        assert np.all(err <= bound), (n, r, m, adaptive, worst, err[worst], bound[worst], mag[worst])
        # plain FP32 evaluation of the same formula
        f32 = V / rho.astype(np.float32) + U32 @ (d.astype(np.float32) * (U32.T @ V))
        e32 = np.linalg.norm(f32.astype(np.float64) - ref)
        assert np.linalg.norm(got - ref) <= 8.0 * e32 + 2.0 ** -24 * np.linalg.norm(ref), (
            np.linalg.norm(got - ref), e32)


@pytest.mark.parametrize("n,r,m", [(3001, 500, 9), (3001, 700, 130), (600, 513, 16), (37, 8, 12), (5000, 24, 257)])
def test_apply_block_tensor_core(n, r, m):
    for adaptive in (False, True):
        _check_block(n, r, m, adaptive, seed=n + 7 * r + m)
