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
