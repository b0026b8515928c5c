"""Seeded synthetic inputs shaped like the kernel-ridge-regression workloads.

This module only draws random numbers; it contains none of the solver's
arithmetic.  Both the CUDA path and the FP64 oracle consume exactly the FP32
arrays returned here (the oracle promotes them to FP64), so the two sides see
identical inputs.

The problem being solved is the regularized kernel system (K + lam*I) x = b of
kernel ridge regression (paper Sec. 2.1, Eq. "rlaopt-krr").  The paper gives no
data for this path, so every workload is synthetic:

* ``krr_rbf_small``    n=4096,  d=16,  X ~ N(0, I), RBF sigma=sqrt(d)=4,
                       y = sin(X w) + 0.1 eps, w ~ N(0, I/d), lam = 1e-4 n, r = 100.
* ``krr_laplace_mix``  n=200000, d=64, 20-cluster Gaussian mixture (centres
                       ~ N(0, 4I), points ~ centre + N(0, I), uniform labels),
                       Laplace sigma=8, lam = 1e-6 n, r = 500,
                       y = sin(||x|| / sqrt(d)) + 0.1 eps.
* ``krr_matern_large`` n=1e6, d=32, X ~ U[0,1]^d z-scored per column,
                       Matern-5/2 lengthscale 1, lam = 1e-7 n, r = 1000,
                       y = sin(X w) + 0.1 eps.
* ``krr_rbf_block``    n=1e5, d=128, X ~ N(0, I), RBF sigma=sqrt(d),
                       64 right-hand sides N(0,1) x 16 shifts lam in
                       logspace(-8, -3, 16) * n, r = 800.
* ``krr_rbf_hyper``    train n=1e5, val n=2e4, d=32, X ~ N(0, I), RBF
                       sigma0 = sqrt(d), lam0 = 1e-4 n_train, r = 500,
                       y = sin(X w) + 0.1 eps for both splits.
* ``ridge_spectral``   ridge regression (Sec. 5.1): X = U Sigma_alpha V^T,
                       Sigma_alpha = diag(i^(-alpha/2)), y = U g / ||g||.

The sketch matrix Omega is n x r with entries N(0,1)/sqrt(n), drawn with seed
1000 + seed, so that Omega^T Omega is close to the identity.
"""
from __future__ import annotations

import dataclasses
import numpy as np

RBF, LAPLACE, MATERN52 = 0, 1, 2
KERNEL_NAMES = {RBF: "rbf", LAPLACE: "laplace", MATERN52: "matern52"}


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # n x d float32, row-major
    B: np.ndarray            # n x nrhs float32 right-hand sides (targets y)
    kernel: int              # RBF / LAPLACE / MATERN52
    bandwidth: float         # sigma (RBF, Laplace) or lengthscale (Matern)
    lambdas: np.ndarray      # absolute shifts lam (float64), one per shift
    rank: int                # Nystrom rank r
    refine_every: int = 20   # true-residual replacement period
    Xval: np.ndarray | None = None
    yval: np.ndarray | None = None
    seed: int = 0

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def gaussian_sketch(n: int, r: int, seed: int) -> np.ndarray:
    """Omega in R^{n x r}, N(0,1)/sqrt(n) drawn with seed 1000+seed, in FP32."""
    rng = np.random.default_rng(1000 + seed)
    return _f32(rng.standard_normal((n, r)) / np.sqrt(n))


def krr_rbf_small(seed: int = 0, n: int = 4096, d: int = 16) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    w = rng.standard_normal(d) / np.sqrt(d)
    y = np.sin(X @ w) + 0.1 * rng.standard_normal(n)
    return Workload("krr_rbf_small", _f32(X), _f32(y[:, None]), RBF, float(np.sqrt(d)),
                    np.array([1e-4 * n]), 100, seed=seed)


def krr_laplace_mix(seed: int = 0, n: int = 200_000, d: int = 64, rank: int = 500) -> Workload:
    rng = np.random.default_rng(seed)
    centres = 2.0 * rng.standard_normal((20, d))
    labels = rng.integers(0, 20, size=n)
    X = centres[labels] + rng.standard_normal((n, d))
    y = np.sin(np.linalg.norm(X, axis=1) / np.sqrt(d)) + 0.1 * rng.standard_normal(n)
    return Workload("krr_laplace_mix", _f32(X), _f32(y[:, None]), LAPLACE, 8.0,
                    np.array([1e-6 * n]), rank, seed=seed)


def krr_matern_large(seed: int = 0, n: int = 1_000_000, d: int = 32, lengthscale: float = 1.0,
                     rank: int = 1000) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    X = (X - X.mean(axis=0)) / X.std(axis=0)
    w = rng.standard_normal(d) / np.sqrt(d)
    y = np.sin(X @ w) + 0.1 * rng.standard_normal(n)
    return Workload("krr_matern_large", _f32(X), _f32(y[:, None]), MATERN52, lengthscale,
                    np.array([1e-7 * n]), rank, refine_every=20, seed=seed)


def krr_rbf_block(seed: int = 0, n: int = 100_000, d: int = 128, nrhs: int = 64,
                  n_shifts: int = 16, rank: int = 800) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    B = rng.standard_normal((n, nrhs))
    lambdas = np.logspace(-8, -3, n_shifts) * n
    return Workload("krr_rbf_block", _f32(X), _f32(B), RBF, float(np.sqrt(d)), lambdas, rank,
                    seed=seed)


def krr_rbf_hyper(seed: int = 0, n: int = 100_000, nval: int = 20_000, d: int = 32,
                  rank: int = 500) -> Workload:
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(d) / np.sqrt(d)
    X = rng.standard_normal((n, d))
    Xv = rng.standard_normal((nval, d))
    y = np.sin(X @ w) + 0.1 * rng.standard_normal(n)
    yv = np.sin(Xv @ w) + 0.1 * rng.standard_normal(nval)
    return Workload("krr_rbf_hyper", _f32(X), _f32(y[:, None]), RBF, float(np.sqrt(d)),
                    np.array([1e-4 * n]), rank, Xval=_f32(Xv), yval=_f32(yv), seed=seed)


@dataclasses.dataclass
class RidgeWorkload:
    """Ridge regression data of the paper's ridge experiments (Sec. 5.1):
    X = U diag(i^(-alpha/2)) V^T (n x p, n >= p), y = U g / ||g||; the system is
    (X^T X + lam I) w = X^T y.  U (n x p) and V (p x p) have orthonormal
    columns (QR of Gaussian matrices; the paper uses structured orthogonal
    matrices, which only matters for speed at large n)."""
    X: np.ndarray        # n x p float32
    y: np.ndarray        # n float32
    U: np.ndarray        # n x p float64
    V: np.ndarray        # p x p float64
    g: np.ndarray        # p float64 (before normalization)
    alpha: float
    lam: float


def ridge_spectral(seed: int = 0, n: int = 4096, p: int = 1024, alpha: float = 1.0,
                   lam: float = 1e-4) -> RidgeWorkload:
    if n < p:
        raise ValueError("the ridge workloads have n >= p")
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, p)))
    V, _ = np.linalg.qr(rng.standard_normal((p, p)))
    sig = np.arange(1, p + 1, dtype=np.float64) ** (-alpha / 2.0)
    g = rng.standard_normal(p)
    X = (U * sig) @ V.T
    y = U @ (g / np.linalg.norm(g))
    return RidgeWorkload(_f32(X), _f32(y), U, V, g, float(alpha), float(lam))


def random_points(n: int, d: int, seed: int, scale: float = 1.0, shift: float = 0.0) -> np.ndarray:
    """Plain Gaussian point cloud for kernel-level parity cases."""
    rng = np.random.default_rng(seed)
    return _f32(shift + scale * rng.standard_normal((n, d)))


def random_block(n: int, m: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _f32(rng.standard_normal((n, m)))
