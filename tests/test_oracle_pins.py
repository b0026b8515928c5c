"""Pins of the FP64 oracle against things other than itself: closed forms,
brute force, library direct solves, exact-recovery and finite-termination
properties.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import kop_oracle as O
from oracle import cmatvec
from paper_2609_08136_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = {"rbf": O.RBF, "laplace": O.LAPLACE, "matern52": O.MATERN52}


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "kernel_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, bw, r2, val = line.split()[:4]
            rows.append((KINDS[k], float(bw), float(r2), float(val)))
    return rows


@pytest.mark.parametrize("kind,bw,r2,val", _golden_rows())
def test_kernel_closed_forms(kind, bw, r2, val):
    # through the distance routine too: x = (0, 0), z = (3, 4) has r^2 = 25
    pts = {25.0: np.array([[3.0, 4.0]]), 0.0: np.array([[0.0, 0.0]])}
    k = O.kernel_matrix(kind, np.zeros((1, 2)), pts[r2], bw)[0, 0]
    assert abs(k - val) <= 1e-15 * max(1.0, val)


def test_sqdist_brute_force():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((7, 5))
    B = rng.standard_normal((9, 5))
    D = O.sqdist(A, B)
    for i in range(7):
        for j in range(9):
            s = 0.0
            for k in range(5):
                s += (A[i][k] - B[j][k]) ** 2
            assert abs(D[i, j] - s) <= 1e-13 * s


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_kernel_matrix_invariants(kind):
    X = W.random_points(300, 6, seed=1).astype(np.float64)
    K = O.kernel_matrix(kind, X, X, 2.0)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-12 * ev[-1]          # psd (all three kernels are pd)
    # translation invariance: K(X + c) == K(X)
    K2 = O.kernel_matrix(kind, X + 3.0, X + 3.0, 2.0)
    assert np.max(np.abs(K - K2)) < 1e-12


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_kernel_derivative_matches_finite_difference(kind):
    D2 = np.linspace(0.0, 30.0, 61)
    bw, h = 2.7, 1e-5
    fd = (O.kernel_from_sqdist(kind, D2, bw + h) - O.kernel_from_sqdist(kind, D2, bw - h)) / (2 * h)
    an = O.dkernel_dbw_from_sqdist(kind, D2, bw)
    assert np.max(np.abs(fd - an)) < 1e-9


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_matrix_free_and_host_c_matvec(kind):
    X = W.random_points(257, 9, seed=2)
    Z = W.random_points(33, 9, seed=4)
    V = W.random_block(257, 3, seed=5).astype(np.float64)
    ref = O.kernel_matrix(kind, Z, X, 1.7) @ V
    mf = O.kernel_matvec(kind, X, V, 1.7, Z=Z, rows_per_block=5)
    c = cmatvec.kernel_matvec(kind, X, V, 1.7, Z=Z)
    assert np.max(np.abs(mf - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(c - ref)) < 1e-12 * np.max(np.abs(ref))
    dref = O.dkernel_dbw_from_sqdist(kind, O.sqdist(Z, X), 1.7) @ V
    dc = cmatvec.kernel_matvec(kind, X, V, 1.7, Z=Z, deriv=True)
    assert np.max(np.abs(dc - dref)) < 1e-12 * np.max(np.abs(dref))


def _spd_with_spectrum(ev, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(ev), len(ev))))
    return (Q * ev) @ Q.T


def test_cg_finite_termination_three_eigenvalues():
    # CG on a matrix with k distinct eigenvalues converges in at most k steps
    # in exact arithmetic; any dropped term or wrong sign in the recurrences
    # breaks this.
    ev = np.repeat([1.0, 10.0, 100.0], [40, 30, 30])
    A = _spd_with_spectrum(ev, 0)
    b = np.random.default_rng(1).standard_normal(100)
    x, it, hist = O.pcg(lambda v: A @ v, b, None, tol=1e-12, maxit=50)
    assert it == 3
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-11
    assert len(hist) == it + 1


def test_pcg_exact_preconditioner_one_step():
    A = _spd_with_spectrum(np.logspace(0, 6, 80), 2)
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(3).standard_normal(80)
    x, it, _ = O.pcg(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-10, maxit=20)
    assert it == 1


def test_pcg_preconditioner_scale_invariance():
    # iterates under P^{-1} and c P^{-1} agree (alpha scales by 1/c, beta is
    # unchanged); checked over the first iterations, before rounding drifts.
    A = _spd_with_spectrum(np.logspace(0, 2, 60), 4)
    D = np.diag(1.0 / np.linspace(1, 5, 60))
    b = np.random.default_rng(5).standard_normal(60)
    x1, i1, h1 = O.pcg(lambda v: A @ v, b, lambda v: D @ v, tol=1e-30, maxit=12)
    x2, i2, h2 = O.pcg(lambda v: A @ v, b, lambda v: 7.5 * (D @ v), tol=1e-30, maxit=12)
    assert i1 == i2 == 12
    np.testing.assert_allclose(h1, h2, rtol=1e-9)
    np.testing.assert_allclose(x1, x2, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_krr_solution_matches_direct_cholesky(kind):
    wl = W.krr_rbf_small(seed=0, n=1024, d=8)
    X = wl.X
    b = wl.B[:, 0].astype(np.float64)
    lam = 1e-2 * 1024
    K = O.kernel_matrix(kind, X, X, wl.bandwidth)
    x_direct = np.linalg.solve(K + lam * np.eye(1024), b)
    Om = W.gaussian_sketch(1024, 40, seed=0)
    xs, its, hists, _ = O.krr_solve(kind, X, b, wl.bandwidth, [lam], Omega=Om, tol=1e-13, maxit=500)
    kappa = np.linalg.cond(K + lam * np.eye(1024))
    assert np.linalg.norm(xs[:, 0] - x_direct) / np.linalg.norm(x_direct) < kappa * 1e-13
    assert O.true_relres(kind, X, wl.bandwidth, lam, xs[:, 0], b, K=K) < 1e-12
    # the preconditioner must pay off against plain CG on this problem
    _, its_cg, _, _ = O.krr_solve(kind, X, b, wl.bandwidth, [lam], Omega=None, tol=1e-8, maxit=2000)
    _, its_p, _, _ = O.krr_solve(kind, X, b, wl.bandwidth, [lam], Omega=Om, tol=1e-8, maxit=2000)
    assert its_p[0] < its_cg[0]


def _planted(n, k, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, k)) * np.linspace(3.0, 1.0, k)
    return G @ G.T


@pytest.mark.parametrize("r_extra", [5, 0])
def test_nystrom_exact_recovery_planted_low_rank(r_extra):
    n, k = 400, 12
    K = _planted(n, k, 7)
    r = k + r_extra
    Om = W.gaussian_sketch(n, r, seed=3).astype(np.float64)
    U, lam_hat, nu = O.nystrom(K @ Om, Om)
    assert np.linalg.norm(U.T @ U - np.eye(r)) < 1e-12
    A_nys = (U * lam_hat) @ U.T
    assert np.linalg.norm(A_nys - K) / np.linalg.norm(K) < 1e-10
    ev = np.sort(np.linalg.eigvalsh(K))[::-1][:k]
    np.testing.assert_allclose(lam_hat[:k], ev, rtol=1e-10)
    assert np.all(np.diff(lam_hat) <= 0)
    # PCG on (K + mu I) with the exact Nystrom preconditioner
    mu = 0.37
    rho = O.nystrom_rho(lam_hat, mu, adaptive=True)
    b = np.random.default_rng(8).standard_normal(n)
    _, it, _ = O.pcg(lambda v: K @ v + mu * v, b,
                     lambda v: O.precond_apply(U, lam_hat, mu, rho, v), tol=1e-8, maxit=50)
    # r > rank: lam_hat_r = 0 so P^{-1}(K + mu I) = I (one step);
    # r = rank: two distinct eigenvalues {1, mu/rho} (at most two steps).
    assert it == (1 if r_extra > 0 else 2)


def test_nystrom_omega_invariance():
    n, r = 300, 20
    X = W.random_points(n, 5, seed=9)
    K = O.kernel_matrix(O.RBF, X, X, 1.5)
    Om = W.gaussian_sketch(n, r, seed=4).astype(np.float64)
    R = np.triu(np.random.default_rng(5).standard_normal((r, r))) + 4 * np.eye(r)
    U1, l1, _ = O.nystrom(K @ Om, Om, nu_rel=1e-15)
    Om2 = Om @ R
    U2, l2, _ = O.nystrom(K @ Om2, Om2, nu_rel=1e-15)
    A1 = (U1 * l1) @ U1.T
    A2 = (U2 * l2) @ U2.T
    assert np.linalg.norm(A1 - A2) / np.linalg.norm(A1) < 1e-6


@pytest.mark.parametrize("adaptive", [True, False])
def test_preconditioner_spectrum_and_symmetry(adaptive):
    n, r = 200, 15
    X = W.random_points(n, 4, seed=11)
    K = O.kernel_matrix(O.LAPLACE, X, X, 2.0)
    Om = W.gaussian_sketch(n, r, seed=6).astype(np.float64)
    U, lam_hat, _ = O.nystrom(K @ Om, Om)
    mu = 0.05
    rho = O.nystrom_rho(lam_hat, mu, adaptive)
    Pinv = O.precond_apply(U, lam_hat, mu, rho, np.eye(n))
    assert np.max(np.abs(Pinv - Pinv.T)) < 1e-12
    ev = np.sort(np.linalg.eigvalsh(Pinv))
    expect = np.sort(np.concatenate([1.0 / (lam_hat + mu), np.full(n - r, 1.0 / rho)]))
    np.testing.assert_allclose(ev, expect, rtol=1e-9)
    assert ev[0] > 0
    assert ev[0] >= 1.0 / (lam_hat[0] + mu) * (1 - 1e-12) and ev[-1] <= 1.0 / mu * (1 + 1e-12)


def test_adjoint_gradient_two_points_closed_form():
    # n = 2, RBF, points at distance r: K = [[1, c], [c, 1]], c = exp(-r^2/(2 s^2)).
    # With y = (1, 0) and a single validation point equal to x_1 with target 0:
    # x = (K + l I)^{-1} y = (1 + l, -c) / ((1 + l)^2 - c^2),
    # prediction p = x_1 + c x_2 = ((1 + l) - c^2) / ((1 + l)^2 - c^2), L = p^2.
    s, l, r = 1.3, 0.4, 1.1
    X = np.array([[0.0], [r]])
    y = np.array([1.0, 0.0])
    Xv = np.array([[0.0]])
    yv = np.array([0.0])

    def closed(s, l):
        c = math.exp(-r * r / (2 * s * s))
        p = ((1 + l) - c * c) / ((1 + l) ** 2 - c * c)
        return p * p

    L, dbw, dlam, _ = O.krr_val_grad(O.RBF, X, y, Xv, yv, s, l)
    h = 1e-6
    assert abs(L - closed(s, l)) < 1e-14
    assert abs(dlam - (closed(s, l + h) - closed(s, l - h)) / (2 * h)) < 1e-8
    assert abs(dbw - (closed(s + h, l) - closed(s - h, l)) / (2 * h)) < 1e-8


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_adjoint_gradient_matches_finite_differences(kind):
    wl = W.krr_rbf_hyper(seed=0, n=256, nval=64, d=4)
    X, y, Xv, yv = wl.X, wl.B[:, 0], wl.Xval, wl.yval
    bw, lam = 1.9, 0.3
    L, dbw, dlam, _ = O.krr_val_grad(kind, X, y, Xv, yv, bw, lam)
    hb, hl = 1e-4 * bw, 1e-4 * lam
    fdb = (O.krr_val_loss(kind, X, y, Xv, yv, bw + hb, lam)[0]
           - O.krr_val_loss(kind, X, y, Xv, yv, bw - hb, lam)[0]) / (2 * hb)
    fdl = (O.krr_val_loss(kind, X, y, Xv, yv, bw, lam + hl)[0]
           - O.krr_val_loss(kind, X, y, Xv, yv, bw, lam - hl)[0]) / (2 * hl)
    assert abs(dbw - fdb) <= 1e-6 * abs(fdb)
    assert abs(dlam - fdl) <= 1e-6 * abs(fdl)


def test_adjoint_gradient_n2048_rbf():
    # the size at which the hyper-parameter workload's gradient is checked
    wl = W.krr_rbf_hyper(seed=0, n=2048, nval=512, d=32)
    X, y, Xv, yv = wl.X, wl.B[:, 0], wl.Xval, wl.yval
    bw, lam = wl.bandwidth, 1e-4 * 2048
    L, dbw, dlam, _ = O.krr_val_grad(O.RBF, X, y, Xv, yv, bw, lam)
    hb, hl = 1e-4 * bw, 1e-4 * lam
    fdb = (O.krr_val_loss(O.RBF, X, y, Xv, yv, bw + hb, lam)[0]
           - O.krr_val_loss(O.RBF, X, y, Xv, yv, bw - hb, lam)[0]) / (2 * hb)
    fdl = (O.krr_val_loss(O.RBF, X, y, Xv, yv, bw, lam + hl)[0]
           - O.krr_val_loss(O.RBF, X, y, Xv, yv, bw, lam - hl)[0]) / (2 * hl)
    assert abs(dbw - fdb) <= 1e-6 * abs(fdb)
    assert abs(dlam - fdl) <= 1e-6 * abs(fdl)


def test_true_relres_definition():
    A = _spd_with_spectrum(np.linspace(1, 2, 30), 12)
    X = np.zeros((30, 1))
    x = np.random.default_rng(0).standard_normal(30)
    b = A @ x + 0.25 * x
    assert O.true_relres(O.RBF, X, 1.0, 0.25, x, b, K=A) < 1e-15
    b2 = b.copy()
    b2[0] += 1e-3 * np.linalg.norm(b)
    assert abs(O.true_relres(O.RBF, X, 1.0, 0.25, x, b2, K=A)
               - 1e-3 * np.linalg.norm(b) / np.linalg.norm(b2)) < 1e-12


# ---------------------------------------------------------------- rank adaptation
def _planted_psd(n, lam, seed):
    """A = Q diag(lam) Q^T with a random orthonormal Q (n x len(lam))."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, len(lam))))
    return Q, (Q * lam) @ Q.T


def test_error_estimate_closed_form_exact_eigenvectors():
    # Omega spanning the top r eigenvectors makes the Nystrom approximation the
    # truncated eigendecomposition, so ||A - A_nys||_2 = lam_{r+1} exactly; the
    # power method from a generic start converges to it (gap lam_{r+1} / lam_{r+2} = 4)
    n, r = 200, 6
    lam = np.array([50.0, 30.0, 20.0, 10.0, 8.0, 6.0, 4.0, 1.0, 0.5, 0.25])
    Q, A = _planted_psd(n, lam, 11)
    U, lam_hat, _ = O.nystrom(A @ Q[:, :r], Q[:, :r], nu_rel=1e-14)
    assert np.allclose(lam_hat, lam[:r], rtol=1e-10)
    g0 = np.random.default_rng(12).standard_normal(n)
    est = O.nystrom_error_estimate(lambda v: A @ v, U, lam_hat, g0, 60)
    assert abs(est - lam[r]) <= 1e-9 * lam[r]


def test_error_estimate_bounded_by_largest_eigenvalue_of_error():
    # for unit v, ||E v|| <= lambda_max(E): every iterate is a lower bound, and it
    # reaches lambda_max(E) (computed by a dense symmetric eigensolver) as q grows
    n, r = 300, 12
    X = W.random_points(n, 4, seed=13)
    A = O.kernel_matrix(O.RBF, X, X, 2.0)
    Om = W.gaussian_sketch(n, r, seed=2)
    U, lam_hat, _ = O.nystrom(A @ Om, Om, nu_rel=1e-14)
    lmax = np.linalg.eigvalsh(A - (U * lam_hat) @ U.T)[-1]
    g0 = np.random.default_rng(14).standard_normal(n)
    prev = 0.0
    for q in (1, 3, 10, 400):
        est = O.nystrom_error_estimate(lambda v: A @ v, U, lam_hat, g0, q)
        assert est <= lmax * (1 + 1e-12)
        prev = est
    assert prev >= lmax * (1 - 1e-6)


def test_rank_adaptation_stops_at_planted_rank():
    # exact rank 12: ranks 4 and 8 leave an error of at least lam_{r+1} (Eckart-
    # Young: no rank-r matrix does better), rank 16 recovers A exactly
    n = 256
    lam = np.geomspace(100.0, 1.0, 12)
    _, A = _planted_psd(n, lam, 15)
    Om = np.random.default_rng(16).standard_normal((n, 64)) / np.sqrt(n)
    g0 = np.random.default_rng(17).standard_normal(n)
    U, lam_hat, _, r, est, hist = O.nystrom_adaptive(lambda V: A @ V, Om, 4, 64, 200, 1e-8, g0, nu_rel=1e-14)
    assert [h[0] for h in hist] == [4, 8, 16] and r == 16
    assert est <= 1e-8 * lam_hat[0]
    for rk, e in hist[:-1]:
        assert e >= lam[rk] * (1 - 1e-6)
    assert np.allclose(lam_hat[:12], lam, rtol=1e-9)


def test_rank_adaptation_doubles_and_caps():
    n = 128
    _, A = _planted_psd(n, np.geomspace(10.0, 0.1, 40), 18)
    Om = np.random.default_rng(19).standard_normal((n, 12)) / np.sqrt(n)
    g0 = np.ones(n)
    *_, r, est, hist = O.nystrom_adaptive(lambda V: A @ V, Om, 5, 12, 5, 0.0, g0, nu_rel=1e-14)
    assert [h[0] for h in hist] == [5, 10, 12] and r == 12


# ---------------------------------------------------------------- point gradient
@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACE, O.MATERN52])
def test_point_gradient_matches_finite_differences(kind):
    rng = np.random.default_rng(31)
    n, d, bw = 30, 3, 1.3
    X = rng.standard_normal((n, d))
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    f = lambda Y: a @ O.kernel_matrix(kind, Y, Y, bw) @ b
    G = O.kernel_grad_points(kind, X, a, b, bw, rows_per_block=7)
    eps = 1e-6
    for i, k in [(0, 0), (3, 2), (17, 1), (29, 0), (11, 2)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] += eps
        Xm[i, k] -= eps
        fd = (f(Xp) - f(Xm)) / (2 * eps)
        assert abs(G[i, k] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, k, G[i, k], fd)


def test_point_gradient_translation_invariance_and_two_points():
    # a^T K b does not change when all points move together: the gradients sum to 0
    rng = np.random.default_rng(32)
    X = rng.standard_normal((50, 4))
    a, b = rng.standard_normal(50), rng.standard_normal(50)
    for kind in (O.RBF, O.LAPLACE, O.MATERN52):
        G = O.kernel_grad_points(kind, X, a, b, 2.0)
        assert np.abs(G.sum(axis=0)).max() <= 1e-12 * np.abs(G).max()
    # two RBF points at distance 1 along x, bw = 2: the diagonal terms a_i b_i k(0)
    # do not depend on X, so only (a1 b2 + a2 b1) k(x1, x2) moves, and
    # d k / d x1 = -k (x1 - x2) / bw^2 = -e^{-1/8} (1, 0) / 4
    X2 = np.array([[1.0, 0.0], [0.0, 0.0]])
    a2, b2 = np.array([0.5, -2.0]), np.array([3.0, 1.5])
    G2 = O.kernel_grad_points(O.RBF, X2, a2, b2, 2.0)
    c = a2[0] * b2[1] + a2[1] * b2[0]
    assert np.allclose(G2[0], [-c * math.exp(-1.0 / 8.0) / 4.0, 0.0], rtol=1e-14, atol=1e-15)
    assert np.allclose(G2[1], -G2[0], rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- ridge workload
def test_ridge_spectrum_is_the_constructed_one():
    # X^T X + lam I has eigenvalues i^-alpha + lam (the paper's statement of its
    # construction), so condition number (1 + lam) / (p^-alpha + lam)
    wl = W.ridge_spectral(seed=3, n=400, p=96, alpha=2.0, lam=1e-4)
    X = wl.X.astype(np.float64)
    ev = np.sort(np.linalg.eigvalsh(X.T @ X + wl.lam * np.eye(96)))[::-1]
    want = np.arange(1, 97, dtype=np.float64) ** -2.0 + 1e-4
    assert np.allclose(ev, want, rtol=1e-5, atol=1e-7)


def test_ridge_nystrom_pcg_reaches_the_closed_form_solution():
    wl = W.ridge_spectral(seed=4, n=600, p=200, alpha=1.0, lam=1e-4)
    X = wl.X.astype(np.float64)
    b = O.ridge_rhs(X, wl.y)
    A = lambda v: O.ridge_normal_matvec(X, v) + wl.lam * v
    Om = np.random.default_rng(5).standard_normal((200, 40)) / np.sqrt(200)
    U, lam_hat, _ = O.nystrom(O.ridge_normal_matvec(X, Om), Om)
    rho = O.nystrom_rho(lam_hat, wl.lam)
    Pinv = lambda v: O.precond_apply(U, lam_hat, wl.lam, rho, v)
    w, it, _ = O.pcg(A, b, Pinv, tol=1e-10, maxit=400)
    # the closed form uses the float64 U, V of the construction while X is its
    # float32 rounding: agreement to the rounding of X amplified by the condition
    ws = O.ridge_exact_solution(wl.V, wl.g, wl.alpha, wl.lam)
    assert np.linalg.norm(w - ws) / np.linalg.norm(ws) <= 2e-3
    # and exactly the solution of the float32 X
    wd = np.linalg.solve(X.T @ X + wl.lam * np.eye(200), b)
    assert np.linalg.norm(w - wd) / np.linalg.norm(wd) <= 1e-8
    assert it < 60


def test_shifted_solve_spectral_closed_form():
    # (Q diag(a) Q^T + s I)^-1 b = Q diag(1 / (a + s)) Q^T b
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    a = np.logspace(-3, 2, 50)
    A = (Q * a) @ Q.T
    b = rng.standard_normal(50)
    for s in (1e-4, 0.3, 7.0):
        ref = Q @ ((Q.T @ b) / (a + s))
        np.testing.assert_allclose(O.shifted_solve(A, b, s), ref, rtol=1e-9, atol=1e-12)


def test_pcg_warm_start():
    # the warm start begins from r = b - A x0: (i) an exact x0 stops after 0
    # products; (ii) on a matrix with 3 distinct eigenvalues CG terminates in
    # 3 steps from any x0 (the initial error spans at most 3 eigenspaces);
    # (iii) a warm run equals x0 plus a cold run on b - A x0 (same Krylov
    # space), over a fixed number of steps.  Starting from r = b instead
    # fails (ii) and (iii).
    ev = np.repeat([1.0, 10.0, 100.0], [40, 30, 30])
    A = _spd_with_spectrum(ev, 7)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(100)
    xs = np.linalg.solve(A, b)
    x, it, hist = O.pcg(lambda v: A @ v, b, None, tol=1e-10, maxit=50, x0=xs)
    assert it == 0 and hist[0] <= 1e-10
    x0 = xs + rng.standard_normal(100)
    x, it, _ = O.pcg(lambda v: A @ v, b, None, tol=1e-30, maxit=3, x0=x0)
    assert it == 3
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-9
    B2 = _spd_with_spectrum(np.logspace(0, 3, 100), 9)
    D = np.diag(1.0 / np.linspace(1, 4, 100))
    x0 = rng.standard_normal(100)
    xw, iw, _ = O.pcg(lambda v: B2 @ v, b, lambda v: D @ v, tol=1e-30, maxit=8, x0=x0)
    dc, ic, _ = O.pcg(lambda v: B2 @ v, b - B2 @ x0, lambda v: D @ v, tol=1e-30, maxit=8)
    assert iw == ic == 8
    np.testing.assert_allclose(xw, x0 + dc, rtol=1e-10, atol=1e-10)
