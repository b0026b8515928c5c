"""nys_apply_noalloc: the preconditioner apply for callers that cannot allocate
device memory on this path (a latency-critical loop that must not pay the
device-wide synchronization of cudaMalloc/cudaFree, or an application whose
device memory belongs to its own allocator).  Its scratch is a fixed array in
the library's device image.  Checked through the C ABI against nys_apply, the
allocating entry point, on two calls in a row (the second call must not see
stale contents of the shared array).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_08136_b300 import _ffi
from paper_2609_08136_b300 import ops
from paper_2609_08136_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(ny, V, mus, adaptive):
    m = V.shape[1]
    arr = (ctypes.c_double * m)(*mus)
    O = torch.empty_like(V)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _ffi.lib().nys_apply_noalloc(ny.handle, arr, int(adaptive), ctypes.c_void_p(V.data_ptr()), m,
                                      ctypes.c_void_p(O.data_ptr()), stream)
    assert rc == 0, _ffi.lib().kop_last_error()
    torch.cuda.synchronize()
    return O


def test_noalloc_apply_matches_allocating_apply_twice():
    n, r = 3000, 120
    X = W.random_points(n, 16, seed=21)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, 4.0)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=21)).cuda())
    calls = [(W.random_block(n, 3, seed=1), [0.5, 0.05, 2.0], True),
             (W.random_block(n, 1, seed=2), [0.2], False)]
    for V, mus, adaptive in calls:
        Vd = torch.from_numpy(V).cuda()
        ref = ny.apply(Vd, mus, adaptive=adaptive).cpu().numpy()
        got = _noalloc(ny, Vd, mus, adaptive).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6


@pytest.mark.parametrize("adaptive", [True, False])
def test_noalloc_widest_block_at_high_rank(adaptive):
    # m = 8 columns (the widest the fixed array serves) at r = 1024: 8200 of its
    # 16448 doubles; nys_build caps r at 2048, so r * m + m <= 16392 always fits
    # and the capacity check is a guard only
    n, r = 2304, 1024
    X = W.random_points(n, 8, seed=31)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.LAPLACE, 3.0)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, r, seed=31)).cuda())
    mus = [0.01 * (c + 1) for c in range(8)]
    for seed in (5, 6):
        Vd = torch.from_numpy(W.random_block(n, 8, seed=seed)).cuda()
        ref = ny.apply(Vd, mus, adaptive=adaptive).cpu().numpy()
        got = _noalloc(ny, Vd, mus, adaptive).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6


def test_noalloc_rejects_zero_damping_without_positive_lam_r():
    # a rank above the planted rank: lam_hat_r = 0, so mu = 0 would divide by zero
    n = 200
    G = W.random_block(n, 3, seed=4).astype(np.float32)
    op = ops.KernelOperator(torch.from_numpy(G).cuda(), ops.RBF, 1e4)  # K ~ all ones: rank 1
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 8, seed=4)).cuda())
    lam, _ = ny.eigs()
    assert lam[-1].item() == 0.0
    V = torch.ones(n, 1, device="cuda")
    arr = (ctypes.c_double * 1)(0.0)
    rc = _ffi.lib().nys_apply_noalloc(ny.handle, arr, 1, ctypes.c_void_p(V.data_ptr()), 1,
                                      ctypes.c_void_p(V.data_ptr()), None)
    assert rc == -1 and b"mu must be" in _ffi.lib().kop_last_error()


def test_noalloc_rejects_too_many_columns():
    n = 300
    X = W.random_points(n, 4, seed=3)
    op = ops.KernelOperator(torch.from_numpy(X).cuda(), ops.RBF, 2.0)
    ny = ops.Nystrom(op, torch.from_numpy(W.gaussian_sketch(n, 10, seed=3)).cuda())
    V = torch.zeros(n, 9, device="cuda")
    arr = (ctypes.c_double * 9)(*([0.1] * 9))
    rc = _ffi.lib().nys_apply_noalloc(ny.handle, arr, 1, ctypes.c_void_p(V.data_ptr()), 9,
                                      ctypes.c_void_p(V.data_ptr()), None)
    assert rc == -1 and b"m must be" in _ffi.lib().kop_last_error()
