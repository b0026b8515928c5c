"""Parity of the kernel-operator products (fused tensor-core path in both
precision modes, and the plain FP32 path) with the FP64 oracle.

Error measure: per output, |O - O_ref| / sum_j |K_ij| |V_jc| (the scale of
the terms being summed).  Bounds: KOP_FAST forms distances from a 2-term BF16
split (about 2^-16 relative per coordinate), so the kernel exponent is off by
about 2^-15 * |x|^2 / s^2; with the test data |x|^2 / s^2 <= ~6 this gives
< 3e-4.  KOP_ACCURATE and KOP_PLAIN are FP32-level: < 4e-6."""
import numpy as np
import pytest
import torch

from oracle import kop_oracle as O
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {ops.FAST: 3e-4, ops.ACCURATE: 4e-6, ops.PLAIN: 4e-6, ops.EXACT: 1e-12}


def _rel_err(kind, Xq, Xk, V, bw, got, deriv=False):
    D2 = O.sqdist(Xq, Xk)
    f = O.dkernel_dbw_from_sqdist if deriv else O.kernel_from_sqdist
    Km = f(kind, D2, bw)
    V64 = V.astype(np.float64)
    ref = Km @ V64
    scale = np.abs(Km) @ np.abs(V64) + 1e-300
    return np.max(np.abs(got.astype(np.float64) - ref) / scale)


CASES = [  # n, d, m
    (1, 3, 1), (2, 16, 1), (127, 16, 1), (129, 32, 3), (300, 64, 1), (257, 5, 8), (640, 128, 2),
    (1000, 100, 1), (385, 64, 13),
]


@pytest.mark.parametrize("mode", [ops.FAST, ops.ACCURATE, ops.PLAIN])
@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE, ops.MATERN52])
@pytest.mark.parametrize("n,d,m", CASES)
def test_matvec_parity(n, d, m, kind, mode):
    X = W.random_points(n, d, seed=n + d, scale=1.0, shift=2.0)
    V = W.random_block(n, m, seed=7 * n + m)
    bw = float(np.sqrt(d)) * (0.8 if kind == ops.RBF else 1.5)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    got = op.matvec(torch.from_numpy(V).cuda(), mode=mode).cpu().numpy()
    op.sync()
    assert _rel_err(kind, X, X, V, bw, got) < TOL[mode]


@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE, ops.MATERN52])
@pytest.mark.parametrize("n,d,m", [(1, 3, 1), (129, 16, 2), (300, 64, 9), (257, 5, 1)])
def test_exact_fp64_operator(n, d, m, kind):
    X = W.random_points(n, d, seed=n + 3 * d, shift=2.0)
    V = np.random.default_rng(n).standard_normal((n, m))
    bw = float(np.sqrt(d))
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    for deriv in (False, True):
        got = op.matvec_f64(torch.from_numpy(V).cuda(), deriv=deriv).cpu().numpy()
        f = O.dkernel_dbw_from_sqdist if deriv else O.kernel_from_sqdist
        Km = f(kind, O.sqdist(X, X), bw)
        ref = Km @ V
        assert np.max(np.abs(got - ref) / (np.abs(Km) @ np.abs(V) + 1e-300)) < TOL[ops.EXACT]
    got32 = op.matvec(torch.from_numpy(V.astype(np.float32)).cuda(), mode=ops.EXACT).cpu().numpy()
    assert _rel_err(kind, X, X, V.astype(np.float32), bw, got32) < 1e-6


@pytest.mark.parametrize("n", [1, 200, 385, 1000])
def test_single_column_product_diagonal_is_exact(n):
    # the single-vector FAST product takes each pair of row blocks once (both
    # contributions of a tile from one evaluation): a unit vector e_j gives
    # K[:, j], whose diagonal entry is exactly 1
    X = W.random_points(n, 16, seed=n)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.LAPLACE, 4.0)
    K = O.kernel_matrix(O.LAPLACE, X, X, 4.0)
    for j in sorted({0, n // 3, n - 1}):
        e = np.zeros((n, 1), dtype=np.float32)
        e[j, 0] = 1.0
        got = op.matvec(torch.from_numpy(e).cuda(), mode=ops.FAST).cpu().numpy()[:, 0]
        assert got[j] == 1.0
        assert np.max(np.abs(got - K[:, j])) < 3e-4


@pytest.mark.parametrize("mode", [ops.FAST, ops.ACCURATE])
def test_diagonal_is_exact(mode):
    n, d = 200, 64
    X = W.random_points(n, d, seed=3)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, 8.0)
    E = np.zeros((n, 8), dtype=np.float32)
    cols = [0, 5, 127, 128, 150, 199, 64, 1]
    for c, j in enumerate(cols):
        E[j, c] = 1.0
    got = op.matvec(torch.from_numpy(E).cuda(), mode=mode).cpu().numpy()
    for c, j in enumerate(cols):
        assert got[j, c] == 1.0


@pytest.mark.parametrize("mode", [ops.FAST, ops.ACCURATE, ops.PLAIN])
@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE, ops.MATERN52])
def test_cross_and_derivative_parity(kind, mode):
    n, nz, d, m = 333, 77, 32, 2
    X = W.random_points(n, d, seed=1)
    Z = W.random_points(nz, d, seed=2, shift=0.3)
    bw = 7.0
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    Vn = W.random_block(n, m, seed=3)
    Vz = W.random_block(nz, m, seed=4)
    got = op.cross_matvec(torch.from_numpy(Z).cuda(), torch.from_numpy(Vn).cuda(), mode=mode).cpu().numpy()
    assert _rel_err(kind, Z, X, Vn, bw, got) < TOL[mode]
    got = op.cross_matvec(torch.from_numpy(Z).cuda(), torch.from_numpy(Vz).cuda(), transpose=True,
                          mode=mode).cpu().numpy()
    assert _rel_err(kind, X, Z, Vz, bw, got) < TOL[mode]
    got = op.dbw_matvec(torch.from_numpy(Vn).cuda(), mode=mode).cpu().numpy()
    assert _rel_err(kind, X, X, Vn, bw, got, deriv=True) < 2 * TOL[mode]
    op.sync()


def _sampled_rel_err(kind, X, V, bw, got, rows):
    # element-wise on sampled output rows, against the FP64 host oracle; the
    # kernels are positive, so sum_j |K_ij| |V_jc| = (K |V|)_ic
    from oracle import cmatvec
    V64 = V.astype(np.float64)
    ref = cmatvec.kernel_matvec(_KIND[kind], X, V64, bw, Z=X[rows])
    scale = cmatvec.kernel_matvec(_KIND[kind], X, np.abs(V64), bw, Z=X[rows]) + 1e-300
    return np.max(np.abs(got[rows].astype(np.float64) - ref) / scale)


_KIND = {ops.RBF: O.RBF, ops.LAPLACE: O.LAPLACE, ops.MATERN52: O.MATERN52}


# many column chunks of the tensor-core contraction (chunks of <= 256 columns:
# m = 500 and 1024 run 2 and 4 chunks on grid.y) and row blocks that take
# more than one wave of the one-CTA-per-SM grid (n = 40000: 313 row blocks)
@pytest.mark.parametrize("kind", [ops.RBF, ops.LAPLACE, ops.MATERN52])
@pytest.mark.parametrize("n,d,m,mode", [
    (3000, 64, 256, ops.FAST), (3001, 64, 500, ops.FAST), (2500, 16, 1024, ops.FAST), (20000, 32, 500, ops.FAST),
    (40000, 64, 1, ops.FAST), (40000, 64, 1, ops.ACCURATE), (40000, 64, 2, ops.PLAIN), (40001, 16, 8, ops.FAST),
    (38400, 64, 1, ops.FAST), (30001, 32, 1, ops.FAST), (12345, 128, 1, ops.FAST),
])
def test_matvec_parity_wide_blocks_and_many_waves(n, d, m, mode, kind):
    X = W.random_points(n, d, seed=n + d + m, scale=1.0, shift=1.0)
    V = W.random_block(n, m, seed=3 * n + m)
    bw = float(np.sqrt(d)) * (0.8 if kind == ops.RBF else 1.5)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), kind, bw)
    got = op.matvec(torch.from_numpy(V).cuda(), mode=mode).cpu().numpy()
    op.sync()
    rows = np.unique(np.concatenate([np.arange(0, n, max(1, n // 200)), [n - 1]]))
    assert _sampled_rel_err(kind, X, V, bw, got, rows) < TOL[mode]


@pytest.mark.parametrize("n,d,kind", [(20000, 64, ops.RBF), (30001, 128, ops.LAPLACE)])
def test_block_product_has_no_drift(n, d, kind):
    """The tensor core truncates when it adds into its FP32 accumulator, so
    one accumulator over the whole sweep of n keys drifts towards zero
    (measured -1.2e-4 relative at n = 2e4, -6e-4 at n = 1e5: enough to make
    K + lam I indefinite for small lam).  The block product (m > 8) restarts
    its accumulator every few tiles; its error against the FP64 operator must
    stay near FP32 rounding: a bias v^T (O - O64) / v^T O64 below 1e-5 and a
    relative error below 1e-5, whatever n."""
    rng = np.random.default_rng(n)
    X = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).cuda()
    op = ops.KernelOperator(X, kind, float(np.sqrt(d)))
    V = torch.from_numpy(rng.standard_normal((n, 16)).astype(np.float32)).cuda()
    O64 = op.matvec_f64(V.double())
    Of = op.matvec(V, mode=ops.FAST).double()
    Vd = V.double()
    bias = ((Vd * (Of - O64)).sum(0) / (Vd * O64).sum(0)).cpu().numpy()
    rel = ((Of - O64).norm() / O64.norm()).item()
    assert np.all(np.abs(bias) < 1e-5), bias
    assert rel < 1e-5, rel


def test_block_product_autotuner():
    """The tile autotuner of the block product (kop_set_autotune) tunes a shape
    once, caches it, and returns the same product as the fixed heuristic up
    to rounding (the candidates differ only in how the work is tiled)."""
    rng = np.random.default_rng(7)
    n, d, m = 6000, 32, 200
    X = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).cuda()
    V = torch.from_numpy(rng.standard_normal((n, m)).astype(np.float32)).cuda()
    op = ops.KernelOperator(X, ops.RBF, float(np.sqrt(d)))
    ops.set_autotune(False)
    ref = op.matvec(V, mode=ops.FAST)
    assert ops.autotune_shapes() == 0
    ops.set_autotune(True)
    got = op.matvec(V, mode=ops.FAST)
    assert ops.autotune_shapes() == 1
    again = op.matvec(V, mode=ops.FAST)
    assert ops.autotune_shapes() == 1
    assert torch.equal(got, again)  # the cached shape: the same arithmetic
    scale = (torch.exp(-torch.cdist(X, X) ** 2 / (2 * d)).abs() @ V.abs()).max().item()
    assert (got - ref).abs().max().item() <= 1e-5 * scale
