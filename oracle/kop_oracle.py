"""FP64 CPU oracle for Nystrom-preconditioned CG on (K + lam I) x = b.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg call
it.  It shares no code with the CUDA path: it works from the FP32 input arrays
promoted to FP64, with plain numpy/scipy primitives and no blocking or fusion
beyond bounding memory.

What it computes, and where the paper defines it:

* the regularized positive-definite system (K + lam I) x = b with
  K_ij = k(x_i, x_j) (Sec. 2.1, Eqs. "rlaopt-regularized-linear-system" and
  "rlaopt-krr");
* the kernel functions k.  The paper names only k(x_i, x_j); the RBF, Laplace
  and Matern-5/2 forms used here follow Rasmussen & Williams, which the paper
  cites for GP inference (Sec. 2.1);
* the randomized Nystrom approximation of Frangella, Tropp & Udell (cited in
  Sec. 1, Sec. 2.3 and Sec. 4.3) with damping per the NystromConfig table
  (App. A.5, "damping_mode"), and its rank adaptation (same table:
  rank_init, rank_max, num_power_iters, error_tolerance);
* preconditioned CG (Hestenes & Stiefel, cited in Sec. 5.1) with the stopping
  rule ||r_k|| <= tol ||b|| checked per right-hand side (App. A.1,
  PCGStoppingCriteria);
* the adjoint gradient of a validation loss through the solve (Sec. 3.2,
  Eq. "rlaopt-bilevel"; computed here by an adjoint solve instead of unrolled
  backpropagation, which gives the same gradient at convergence), and the
  gradient of a^T K(X) b with respect to the points X;
* the ridge normal operator X^T X, the right-hand side X^T y and the closed-form
  solution of the ridge data construction (Sec. 5.1, Eqs. "experiment-ridge"
  and "experiment-ridge-data"), and the dense shifted solve of an ADMM
  x-update (App. A.4).

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, brute force, library direct solves, exact-recovery and
finite-termination properties.  Iteration counts of PCG are not pinned
(rounding changes them).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

RBF, LAPLACE, MATERN52 = 0, 1, 2
SQRT5 = np.sqrt(5.0)
EPS64 = np.finfo(np.float64).eps


# --------------------------------------------------------------------------
# Kernel entries (Sec. 2.1: K_ij = k(x_i, x_j)).
# --------------------------------------------------------------------------
def sqdist(A, B):
    """Squared Euclidean distances D2_ij = sum_k (a_ik - b_jk)^2 by direct
    differences (no norm identity, so no cancellation).  FP64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.empty((A.shape[0], B.shape[0]))
    step = max(1, int(2_000_000 // max(1, B.shape[0] * A.shape[1])))
    for i0 in range(0, A.shape[0], step):
        diff = A[i0:i0 + step, None, :] - B[None, :, :]
        out[i0:i0 + step] = np.einsum("ijk,ijk->ij", diff, diff)
    return out


def kernel_from_sqdist(kind, D2, bw):
    """k as a function of the squared distance.
    RBF: exp(-r^2 / (2 s^2)); Laplace: exp(-r / s) with Euclidean r;
    Matern-5/2: (1 + sqrt5 r/l + 5 r^2/(3 l^2)) exp(-sqrt5 r/l)."""
    D2 = np.asarray(D2, dtype=np.float64)
    if kind == RBF:
        return np.exp(-D2 / (2.0 * bw * bw))
    r = np.sqrt(D2)
    if kind == LAPLACE:
        return np.exp(-r / bw)
    if kind == MATERN52:
        a = SQRT5 * r / bw
        return (1.0 + a + a * a / 3.0) * np.exp(-a)
    raise ValueError(kind)


def dkernel_dbw_from_sqdist(kind, D2, bw):
    """Derivative of k with respect to the bandwidth (sigma or lengthscale)."""
    D2 = np.asarray(D2, dtype=np.float64)
    if kind == RBF:
        return np.exp(-D2 / (2.0 * bw * bw)) * D2 / bw ** 3
    r = np.sqrt(D2)
    if kind == LAPLACE:
        return np.exp(-r / bw) * r / (bw * bw)
    if kind == MATERN52:
        a = SQRT5 * r / bw
        # dk/da = -(a/3)(1+a) e^{-a},  da/dl = -a/l
        return np.exp(-a) * (a * a / 3.0) * (1.0 + a) / bw
    raise ValueError(kind)


def radial_derivative_from_sqdist(kind, D2, bw):
    """h(r) = -k'(r) / r, the factor of d k(x_i, x_j) / d x_i = -h (x_i - x_j)
    (0 for Laplace at r = 0, where that kernel has no derivative)."""
    D2 = np.asarray(D2, dtype=np.float64)
    if kind == RBF:
        # k = exp(-r^2 / 2 bw^2):  k' = -(r / bw^2) k
        return np.exp(-D2 / (2.0 * bw * bw)) / (bw * bw)
    r = np.sqrt(D2)
    if kind == LAPLACE:
        # k = exp(-r / bw):  k' = -k / bw
        with np.errstate(divide="ignore", invalid="ignore"):
            h = np.exp(-r / bw) / (bw * r)
        return np.where(r > 0.0, h, 0.0)
    if kind == MATERN52:
        # k = (1 + a + a^2/3) e^-a, a = sqrt(5) r / bw:  dk/da = -(a/3)(1 + a) e^-a
        a = SQRT5 * r / bw
        return (5.0 / (3.0 * bw * bw)) * (1.0 + a) * np.exp(-a)
    raise ValueError(kind)


def kernel_grad_points(kind, X, a, b, bw, rows_per_block=256, rows=None):
    """d(a^T K(X) b) / dX (n x d; only the given rows when `rows` is set): row i
    is sum_j (a_i b_j + a_j b_i) d k(x_i, x_j) / d x_i = -sum_j c_ij h_ij (x_i - x_j),
    the backward product of the operator for its inputs (differentiation
    through the solve, Sec. 3.2), written out from that definition."""
    X = np.asarray(X, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    idx = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    G = np.zeros((len(idx), X.shape[1]))
    for s0 in range(0, len(idx), rows_per_block):
        I = idx[s0:s0 + rows_per_block]
        Dif = X[I, None, :] - X[None, :, :]
        h = radial_derivative_from_sqdist(kind, np.einsum("ijk,ijk->ij", Dif, Dif), bw)
        c = a[I, None] * b[None, :] + b[I, None] * a[None, :]
        G[s0:s0 + len(I)] = -np.einsum("ij,ijk->ik", c * h, Dif)
    return G


def kernel_matrix(kind, A, B, bw):
    return kernel_from_sqdist(kind, sqdist(A, B), bw)


def kernel_matvec(kind, X, V, bw, Z=None, deriv=False, rows_per_block=None):
    """O = K(Z, X) V (Z defaults to X), matrix-free over row blocks.
    With deriv=True, O = (dK(Z, X)/d bw) V."""
    X = np.asarray(X, dtype=np.float64)
    Z = X if Z is None else np.asarray(Z, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = V[:, None] if vec else V
    f = dkernel_dbw_from_sqdist if deriv else kernel_from_sqdist
    if rows_per_block is None:
        rows_per_block = max(1, int(4_000_000 // max(1, X.shape[0])))
    out = np.empty((Z.shape[0], V2.shape[1]))
    for i0 in range(0, Z.shape[0], rows_per_block):
        out[i0:i0 + rows_per_block] = f(kind, sqdist(Z[i0:i0 + rows_per_block], X), bw) @ V2
    return out[:, 0] if vec else out


# --------------------------------------------------------------------------
# Randomized Nystrom approximation (Frangella-Tropp-Udell; cited Sec. 1, 2.3).
# --------------------------------------------------------------------------
def nystrom(Y, Omega, nu_rel=None):
    """Rank-r Nystrom approximation A_nys = U diag(lam_hat) U^T of a psd A from
    the sketch Y = A Omega.

    Steps, in the published order:
      nu = nu_rel * ||Y||_2 (default nu_rel = sqrt(n) * eps64),
      Y_nu = Y + nu Omega,
      C = chol((Omega^T Y_nu + Y_nu^T Omega) / 2)  (upper, C^T C = ...),
      B = Y_nu C^{-1},
      B = U Sigma V^T (thin SVD),
      lam_hat = max(0, Sigma^2 - nu).
    Omega is used as given (no QR): the approximation Y (Omega^T Y)^+ Y^T is
    invariant under Omega -> Omega R.  Returns (U, lam_hat descending, nu)."""
    Y = np.asarray(Y, dtype=np.float64)
    Om = np.asarray(Omega, dtype=np.float64)
    n = Y.shape[0]
    if nu_rel is None:
        nu_rel = np.sqrt(n) * EPS64
    nu = nu_rel * np.linalg.norm(Y, 2)
    Ynu = Y + nu * Om
    M = Om.T @ Ynu
    C = np.linalg.cholesky(0.5 * (M + M.T)).T          # upper: M = C^T C
    Bm = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T   # Y_nu C^{-1}
    U, s, _ = np.linalg.svd(Bm, full_matrices=False)
    lam_hat = np.maximum(0.0, s * s - nu)
    return U, lam_hat, nu


def nystrom_error_estimate(apply_A, U, lam_hat, g0, power_iters):
    """Power-iteration estimate of ||A - U diag(lam_hat) U^T||_2, the error of a
    Nystrom approximation (NystromConfig num_power_iters, App. A.5).

    E = A - A_nys is symmetric positive semidefinite for a Nystrom
    approximation, so the power method from v_0 = g0 / ||g0|| converges to its
    largest eigenvalue:  w = E v_{i-1},  est_i = ||w||,  v_i = w / est_i, for
    i = 1 .. power_iters; returns est_q (0 if E v vanishes).  g0 is the start
    vector the caller draws."""
    v = np.asarray(g0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(power_iters):
        w = np.asarray(apply_A(v), dtype=np.float64) - U @ (lam_hat * (U.T @ v))
        est = float(np.linalg.norm(w))
        if est == 0.0:
            break
        v = w / est
    return est


def nystrom_adaptive(apply_A, Omega, rank_init, rank_max, power_iters, err_tol, g0, nu_rel=None):
    """Nystrom approximation with rank adaptation (NystromConfig rank_init,
    rank_max, num_power_iters, error_tolerance; App. A.5).

    The paper lists the parameters only.  Reading (Frangella-Tropp-Udell's
    adaptive scheme): r = rank_init; the approximation of rank r uses the first
    r columns of Omega; its error is estimated by nystrom_error_estimate; stop
    when est <= err_tol * lam_hat_1 (the largest approximate eigenvalue) or
    r == rank_max, else r = min(2 r, rank_max).  Returns
    (U, lam_hat, nu, r, est, [(rank, est), ...])."""
    Om_all = np.asarray(Omega, dtype=np.float64)
    r = int(rank_init)
    hist = []
    while True:
        Om = Om_all[:, :r]
        Y = np.asarray(apply_A(Om), dtype=np.float64)
        U, lam_hat, nu = nystrom(Y, Om, nu_rel)
        est = nystrom_error_estimate(apply_A, U, lam_hat, g0, power_iters)
        hist.append((r, est))
        if est <= err_tol * lam_hat[0] or r >= rank_max:
            return U, lam_hat, nu, r, est, hist
        r = min(2 * r, int(rank_max))


def ridge_normal_matvec(X, V):
    """(X^T X) V without forming X^T X (the ridge normal operator, Sec. 5.1,
    Eq. "experiment-ridge")."""
    X = np.asarray(X, dtype=np.float64)
    return X.T @ (X @ np.asarray(V, dtype=np.float64))


def ridge_rhs(X, y):
    """b = X^T y of (X^T X + lam I) w = X^T y."""
    return np.asarray(X, dtype=np.float64).T @ np.asarray(y, dtype=np.float64)


def ridge_exact_solution(V, g, alpha, lam):
    """w* for the constructed data X = U diag(s) V^T, y = U g / ||g||,
    s_i = i^(-alpha/2) (Eq. "experiment-ridge-data"):
    w* = (X^T X + lam I)^-1 X^T y = V diag(s / (s^2 + lam)) g / ||g||."""
    p = V.shape[1]
    s = np.arange(1, p + 1, dtype=np.float64) ** (-alpha / 2.0)
    return V @ ((s / (s * s + lam)) * (g / np.linalg.norm(g)))


def shifted_solve(A, rhs, shift):
    """x = (A + shift I)^-1 rhs for a dense symmetric A (the linear system of an
    ADMM x-update, App. A.4), by a dense FP64 solve."""
    A = np.asarray(A, dtype=np.float64)
    return np.linalg.solve(A + shift * np.eye(A.shape[0]), np.asarray(rhs, dtype=np.float64))


def nystrom_rho(lam_hat, mu, adaptive=True):
    """Damping of the complement subspace (App. A.5 NystromConfig):
    adaptive adds the smallest retained eigenvalue lam_hat_r to mu."""
    return (lam_hat[-1] + mu) if adaptive else mu


def precond_apply(U, lam_hat, mu, rho, V):
    """P^{-1} V = V / rho + U [ (diag(lam_hat) + mu I)^{-1} - I / rho ] U^T V."""
    V = np.asarray(V, dtype=np.float64)
    W = U.T @ V
    scale = 1.0 / (lam_hat + mu) - 1.0 / rho
    W = (scale[:, None] * W) if W.ndim == 2 else scale * W
    return V / rho + U @ W


# --------------------------------------------------------------------------
# Preconditioned CG (Hestenes-Stiefel; stopping rule App. A.1).
# --------------------------------------------------------------------------
def pcg(apply_A, b, apply_Pinv=None, tol=1e-6, maxit=1000, x0=None):
    """Textbook PCG for one right-hand side.

    x0 = 0 unless given; r = b - A x0; z = P^{-1} r; p = z; then repeat
      q = A p; alpha = r^T z / p^T q; x += alpha p; r -= alpha q;
      stop if ||r|| <= tol ||b||;  z = P^{-1} r;  beta = r^T z_new / r^T z_old;
      p = z + beta p.
    Returns x, the number of A-products, and the recursive relative residual
    history ||r_k|| / ||b|| (entry 0 is the initial residual)."""
    b = np.asarray(b, dtype=np.float64)
    P = apply_Pinv if apply_Pinv is not None else (lambda v: v)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[0] <= tol:
        return x, 0, hist
    z = P(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = apply_A(p)
        pq = p @ q
        if not pq > 0:
            raise FloatingPointError("PCG breakdown: p^T A p <= 0")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
        z = P(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist


def krr_solve(kind, X, B, bw, lambdas, Omega=None, mu=None, adaptive=True, tol=1e-6,
              maxit=1000, nu_rel=None, explicit=True):
    """Nystrom PCG over all columns of B and all shifts (column c = rhs j,
    shift s with c = s * nrhs + j); each column runs its own CG (App. A.1:
    the stopping condition must hold for each right-hand side).  mu defaults
    to each column's lam.  Returns X_sol (n x cols), iteration counts and
    histories, plus the Nystrom factors."""
    X = np.asarray(X, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    K = kernel_matrix(kind, X, X, bw) if explicit else None
    apply_K = (lambda v: K @ v) if explicit else (lambda v: kernel_matvec(kind, X, v, bw))
    U = lam_hat = None
    if Omega is not None:
        Y = apply_K(np.asarray(Omega, dtype=np.float64))
        U, lam_hat, _ = nystrom(Y, Omega, nu_rel)
    cols, iters, hists = [], [], []
    for lam in np.atleast_1d(lambdas):
        m = lam if mu is None else mu
        Pinv = None
        if U is not None:
            rho = nystrom_rho(lam_hat, m, adaptive)
            Pinv = (lambda v, m=m, rho=rho: precond_apply(U, lam_hat, m, rho, v))
        for j in range(B.shape[1]):
            x, it, h = pcg(lambda v, lam=lam: apply_K(v) + lam * v, B[:, j], Pinv, tol, maxit)
            cols.append(x)
            iters.append(it)
            hists.append(h)
    return np.stack(cols, axis=1), iters, hists, (U, lam_hat)


def true_relres(kind, X, bw, lam, x, b, K=None):
    """||(K + lam I) x - b|| / ||b|| in FP64 (App. B.2, relative-residual check)."""
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    Kx = (K @ x) if K is not None else kernel_matvec(kind, X, x, bw)
    return np.linalg.norm(Kx + lam * x - b) / np.linalg.norm(b)


# --------------------------------------------------------------------------
# Gradient of a validation loss through the solve (Sec. 3.2).
# --------------------------------------------------------------------------
def krr_val_loss(kind, X, y, Xv, yv, bw, lam):
    """L(bw, lam) = (1/n_val) ||K(Xv, X) x - yv||^2, x = (K + lam I)^{-1} y,
    by a dense Cholesky solve (for finite-difference checks)."""
    K = kernel_matrix(kind, X, X, bw)
    A = K + lam * np.eye(K.shape[0])
    x = sla.cho_solve(sla.cho_factor(A), np.asarray(y, dtype=np.float64))
    e = kernel_matrix(kind, Xv, X, bw) @ x - np.asarray(yv, dtype=np.float64)
    return float(e @ e / len(e)), x


def krr_val_grad(kind, X, y, Xv, yv, bw, lam, x=None, solve=None):
    """Adjoint gradient of L with respect to (bw, lam).

    e = K_v x - yv;  dL/dx = (2/n_val) K_v^T e;  g = (K + lam I)^{-1} dL/dx;
    dL/dlam = -g^T x;
    dL/dbw  = (2/n_val) e^T (dK_v/dbw) x - g^T (dK/dbw) x.
    ``solve`` maps a right-hand side to (K + lam I)^{-1} rhs (dense Cholesky
    by default)."""
    X = np.asarray(X, dtype=np.float64)
    Xv = np.asarray(Xv, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    yv = np.asarray(yv, dtype=np.float64)
    if solve is None:
        K = kernel_matrix(kind, X, X, bw)
        cf = sla.cho_factor(K + lam * np.eye(K.shape[0]))
        solve = lambda rhs: sla.cho_solve(cf, rhs)
    if x is None:
        x = solve(y)
    nv = Xv.shape[0]
    e = kernel_matvec(kind, X, x, bw, Z=Xv) - yv
    dLdx = (2.0 / nv) * kernel_matvec(kind, Xv, e, bw, Z=X)
    g = solve(dLdx)
    dlam = -g @ x
    dbw = (2.0 / nv) * (e @ kernel_matvec(kind, X, x, bw, Z=Xv, deriv=True)) \
        - g @ kernel_matvec(kind, X, x, bw, deriv=True)
    return float(e @ e / nv), float(dbw), float(dlam), g
