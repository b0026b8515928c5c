"""Thin PyTorch binding of the kop C ABI: device tensors in, device tensors out.

PyTorch supplies device memory and the current stream; every step of the
computation runs in the library's CUDA kernels.  Names follow include/kop.h.
"""
from __future__ import annotations

import ctypes
import warnings

import torch

from . import _ffi
from ._ffi import check

RBF, LAPLACE, MATERN52 = 0, 1, 2
FAST, ACCURATE, PLAIN, EXACT = 0, 1, 2, 3
KERNELS = {"rbf": RBF, "laplace": LAPLACE, "matern52": MATERN52}


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str, cols: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if t.dim() == 1:
        t = t.unsqueeze(1)
    return t.contiguous()


def _kind(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def set_autotune(enable: bool = True):
    """Turn the block product's tile autotuner on or off (kop_set_autotune;
    clears the tuned shapes)."""
    check(_ffi.lib().kop_set_autotune(int(bool(enable))), "kop_set_autotune")


def autotune_shapes() -> int:
    """Number of block-product shapes tuned so far."""
    return int(_ffi.lib().kop_autotune_shapes())


def sfu_rates(stream=None):
    """Measured SFU throughput (ops/s): {'ex2': ..., 'sqrt': ..., 'rsqrt': ...}."""
    arr = (ctypes.c_double * 3)()
    check(_ffi.lib().kop_sfu_rates(arr, _stream(stream)), "kop_sfu_rates")
    return {"ex2": arr[0], "sqrt": arr[1], "rsqrt": arr[2]}


class KernelOperator:
    """K(X, X) for points X (n x d, CUDA float32): kop_create / kop_matvec."""

    def __init__(self, X: torch.Tensor, kernel="rbf", bandwidth: float = 1.0, stream=None):
        X = _dev_f32(X, "X")
        self.n, self.d = X.shape
        self.kernel = _kind(kernel)
        self.bandwidth = float(bandwidth)
        self.device = X.device
        h = ctypes.c_void_p()
        check(_ffi.lib().kop_create(_ptr(X), self.n, self.d, self.kernel, self.bandwidth, _stream(stream),
                                    ctypes.byref(h)), "kop_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _ffi.lib().kop_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bandwidth(self, bw: float):
        check(_ffi.lib().kop_set_bandwidth(self._h, float(bw)), "kop_set_bandwidth")
        self.bandwidth = float(bw)

    def check_cache_floats(self) -> int:
        """Floats of the stored check matrix: the 128 x 128 tiles of each pair
        of row blocks once, nb * (nb // 2 + 1) * 128^2 with nb = ceil(n / 128)."""
        nb = (self.n + 127) // 128
        return nb * (nb // 2 + 1) * 128 * 128

    def set_check_cache(self, enable: bool = True, buffer: torch.Tensor | None = None):
        """Keep the kernel matrix of the solver's direct-difference checks in
        device memory (kop_set_check_cache): in `buffer` (a CUDA float32
        tensor of at least check_cache_floats() elements, which must outlive
        its use), else reserved by the library.  Raises KopError (KOP_ENOMEM)
        when the library's reservation does not fit."""
        ptr, size = None, 0
        if enable and buffer is not None:
            if buffer.dtype != torch.float32 or not buffer.is_cuda or not buffer.is_contiguous():
                raise TypeError("buffer must be a contiguous CUDA float32 tensor")
            ptr, size = _ptr(buffer), buffer.numel()
        self._check_buffer = buffer if enable else None
        check(_ffi.lib().kop_set_check_cache(self._h, int(bool(enable)), ptr, size), "kop_set_check_cache")

    def matvec(self, V: torch.Tensor, mode: int = FAST, out: torch.Tensor | None = None, stream=None):
        vec = V.dim() == 1
        V2 = _dev_f32(V, "V")
        if V2.shape[0] != self.n:
            raise ValueError("V must have n rows")
        O = out if out is not None else torch.empty_like(V2)
        check(_ffi.lib().kop_matvec(self._h, _ptr(V2), V2.shape[1], _ptr(O), int(mode), _stream(stream)),
              "kop_matvec")
        return O[:, 0] if vec and out is None else O

    def matvec_f64(self, V: torch.Tensor, deriv: bool = False, stream=None):
        """FP64 product with the exact (FP64 CUDA-core) operator."""
        vec = V.dim() == 1
        V2 = (V.unsqueeze(1) if vec else V).to(torch.float64).contiguous()
        O = torch.empty_like(V2)
        check(_ffi.lib().kop_matvec_f64(self._h, _ptr(V2), V2.shape[1], _ptr(O), int(bool(deriv)), _stream(stream)),
              "kop_matvec_f64")
        return O[:, 0] if vec else O

    def dbw_matvec(self, V: torch.Tensor, mode: int = FAST, stream=None):
        vec = V.dim() == 1
        V2 = _dev_f32(V, "V")
        O = torch.empty_like(V2)
        check(_ffi.lib().kop_dbw_matvec(self._h, _ptr(V2), V2.shape[1], _ptr(O), int(mode), _stream(stream)),
              "kop_dbw_matvec")
        return O[:, 0] if vec else O

    def grad_points(self, a: torch.Tensor, b: torch.Tensor, mode: int = ACCURATE, stream=None):
        """d(a^T K(X) b) / dX as an n x d tensor (kop_grad_points)."""
        a2 = _dev_f32(a.reshape(-1), "a")
        b2 = _dev_f32(b.reshape(-1), "b")
        if a2.shape[0] != self.n or b2.shape[0] != self.n:
            raise ValueError("a and b must have n entries")
        G = torch.empty((self.n, self.d), dtype=torch.float32, device=self.device)
        check(_ffi.lib().kop_grad_points(self._h, _ptr(a2), _ptr(b2), int(mode), _ptr(G), _stream(stream)),
              "kop_grad_points")
        return G

    def cross_matvec(self, Z: torch.Tensor, V: torch.Tensor, transpose: bool = False, deriv: bool = False,
                     mode: int = FAST, stream=None):
        """K(Z, X) V (transpose=False) or K(X, Z) V (transpose=True)."""
        vec = V.dim() == 1
        Z = _dev_f32(Z, "Z")
        V2 = _dev_f32(V, "V")
        rows = self.n if transpose else Z.shape[0]
        O = torch.empty((rows, V2.shape[1]), dtype=torch.float32, device=V2.device)
        check(_ffi.lib().kop_cross_matvec(self._h, _ptr(Z), Z.shape[0], _ptr(V2), V2.shape[1], _ptr(O),
                                          int(bool(transpose)), int(bool(deriv)), int(mode), _stream(stream)),
              "kop_cross_matvec")
        return O[:, 0] if vec else O

    def sync(self, stream=None):
        check(_ffi.lib().kop_sync(self._h, _stream(stream)), "kop_sync")


class RidgeOperator(KernelOperator):
    """A = X^T X for a data matrix X (n x p, CUDA float32): kop_create_ridge.
    Vectors have p entries; matvec, Nystrom, pcg_solve and pcg_adjoint accept it."""

    def __init__(self, X: torch.Tensor, stream=None):
        X = _dev_f32(X, "X")
        self.rows, self.n = X.shape
        self.d = None
        self.kernel = None
        self.bandwidth = None
        self.device = X.device
        h = ctypes.c_void_p()
        check(_ffi.lib().kop_create_ridge(_ptr(X), self.rows, self.n, _stream(stream), ctypes.byref(h)),
              "kop_create_ridge")
        self._h = h


class Nystrom:
    """Randomized Nystrom preconditioner of an operator: nys_build / nys_apply."""

    def __init__(self, op: KernelOperator, Omega: torch.Tensor, nu_rel: float = 0.0, mode: int = FAST,
                 stream=None):
        Om = _dev_f32(Omega, "Omega")
        if Om.shape[0] != op.n:
            raise ValueError("Omega must have n rows")
        self.op = op
        self.r = Om.shape[1]
        h = ctypes.c_void_p()
        check(_ffi.lib().nys_build(op.handle, _ptr(Om), self.r, float(nu_rel), int(mode), _stream(stream),
                                   ctypes.byref(h)), "nys_build")
        self._h = h

    @classmethod
    def adaptive(cls, op: KernelOperator, Omega: torch.Tensor, rank_init: int, rank_max: int | None = None,
                 g0: torch.Tensor | None = None, power_iters: int = 10, err_tol: float = 1e-2,
                 nu_rel: float = 0.0, mode: int = FAST, stream=None):
        """Nystrom approximation with rank adaptation (nys_build_adaptive):
        ranks rank_init, 2 rank_init, ... up to rank_max, using the first r
        columns of Omega (n x >= rank_max), until the power-iteration error
        estimate from g0 (n-vector) is <= err_tol * lam_hat_1.  The result has
        .r, .err_est and .hist = [(rank, estimate), ...]."""
        rank_max = rank_init if rank_max is None else int(rank_max)
        Om = _dev_f32(Omega, "Omega")
        if Om.shape[0] != op.n or Om.shape[1] < rank_max:
            raise ValueError("Omega must be n x (>= rank_max)")
        if g0 is None:
            raise ValueError("g0 (the power iteration's start vector) is required")
        g = _dev_f32(g0.reshape(-1, 1), "g0")
        if g.shape[0] != op.n:
            raise ValueError("g0 must have n entries")
        h = ctypes.c_void_p()
        r = ctypes.c_int32()
        err = ctypes.c_double()
        hl = 16
        hr = (ctypes.c_int32 * hl)()
        he = (ctypes.c_double * hl)()
        check(_ffi.lib().nys_build_adaptive(op.handle, _ptr(Om), Om.shape[1], int(rank_init), rank_max,
                                            int(power_iters), float(err_tol), _ptr(g), float(nu_rel), int(mode),
                                            _stream(stream), ctypes.byref(h), ctypes.byref(r), ctypes.byref(err),
                                            hr, he, hl), "nys_build_adaptive")
        self = cls.__new__(cls)
        self.op = op
        self.r = r.value
        self._h = h
        self.err_est = err.value
        hist = []
        for i in range(hl):
            if hr[i] == 0:
                break
            hist.append((int(hr[i]), float(he[i])))
        self.hist = hist
        return self

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _ffi.lib().nys_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eigs(self):
        lam = (ctypes.c_double * self.r)()
        nu = ctypes.c_double()
        r = ctypes.c_int32()
        check(_ffi.lib().nys_eigs(self._h, lam, ctypes.byref(nu), ctypes.byref(r)), "nys_eigs")
        return torch.tensor(list(lam), dtype=torch.float64), nu.value

    def factor(self, stream=None):
        U = torch.empty((self.op.n, self.r), dtype=torch.float32, device=self.op.device)
        check(_ffi.lib().nys_factor(self._h, _ptr(U), _stream(stream)), "nys_factor")
        return U

    def apply(self, V: torch.Tensor, mu, adaptive: bool = True, stream=None):
        vec = V.dim() == 1
        V2 = _dev_f32(V, "V")
        m = V2.shape[1]
        mus = [float(mu)] * m if not hasattr(mu, "__len__") else [float(x) for x in mu]
        arr = (ctypes.c_double * m)(*mus)
        O = torch.empty_like(V2)
        check(_ffi.lib().nys_apply(self._h, arr, int(bool(adaptive)), _ptr(V2), m, _ptr(O), _stream(stream)),
              "nys_apply")
        return O[:, 0] if vec else O


class NotConvergedWarning(RuntimeWarning):
    """A solve returned KOP_NOT_CONVERGED: maxit was reached and the outputs
    are the last iterate, whose certified residual is above the tolerance."""


def _warn_unconverged(rc: int, where: str):
    if rc == 1:
        warnings.warn(f"{where}: maxit reached before the tolerance (KOP_NOT_CONVERGED)", NotConvergedWarning,
                      stacklevel=3)


class SolveResult:
    def __init__(self, x, iters, res_hist, true_relres, status):
        self.x, self.iters, self.res_hist, self.true_relres, self.status = x, iters, res_hist, true_relres, status

    @property
    def converged(self):
        return self.status == 0


def pcg_solve(op: KernelOperator, B: torch.Tensor, lambdas, nys: Nystrom | None = None, mu=None,
              adaptive: bool = True, tol: float = 1e-6, maxit: int = 1000, refine_every: int = 30,
              inner_mode: int = FAST, refine_mode: int = PLAIN, check_mode: int = PLAIN, history: bool = False,
              x0: torch.Tensor | None = None, stream=None):
    """Block PCG for (K + lam_s I) x = B[:, j] over all shifts s and columns j
    (column s * nrhs + j of the result), from x0 (n x cols FP64) or 0."""
    vec = B.dim() == 1
    B2 = _dev_f32(B, "B")
    nrhs = B2.shape[1]
    lams = [float(lambdas)] if not hasattr(lambdas, "__len__") else [float(x) for x in lambdas]
    ns = len(lams)
    cols = ns * nrhs
    lam_arr = (ctypes.c_double * ns)(*lams)
    mu_arr = None
    if mu is not None:
        mus = [float(mu)] * ns if not hasattr(mu, "__len__") else [float(x) for x in mu]
        mu_arr = (ctypes.c_double * ns)(*mus)
    X = torch.empty((op.n, cols), dtype=torch.float64, device=B2.device)
    X0 = None
    if x0 is not None:
        X0 = x0.reshape(op.n, cols).to(device=B2.device, dtype=torch.float64).contiguous()
    iters = (ctypes.c_int32 * cols)()
    hist = (ctypes.c_double * ((maxit + 1) * cols))() if history else None
    tr = (ctypes.c_double * cols)()
    rc = check(_ffi.lib().pcg_solve(op.handle, nys.handle if nys is not None else None, lam_arr, ns, mu_arr,
                                    int(bool(adaptive)), _ptr(B2), nrhs, _ptr(X0) if X0 is not None else None,
                                    float(tol), int(maxit), int(refine_every),
                                    int(inner_mode), int(refine_mode), int(check_mode), _ptr(X), iters, hist, tr,
                                    _stream(stream)), "pcg_solve")
    h = None
    if history:
        import numpy as np
        h = np.array(list(hist)).reshape(maxit + 1, cols)
    x = X[:, 0] if (vec and cols == 1) else X
    return SolveResult(x, list(iters), h, list(tr), rc)


def pcg_adjoint(op: KernelOperator, x: torch.Tensor, dLdx: torch.Tensor, lam: float, nys: Nystrom | None = None,
                adaptive: bool = True, tol: float = 1e-6, maxit: int = 1000, refine_every: int = 30,
                inner_mode: int = FAST, refine_mode: int = PLAIN, check_mode: int = PLAIN, stream=None):
    """g = (K + lam I)^{-1} dL/dx, and dL/dlam = -g^T x, dL/dbw = -g^T (dK/dbw) x.
    x, dL/dx and g are FP64 device vectors."""
    x2 = x.detach().reshape(-1).to(torch.float64).contiguous()
    d2 = dLdx.detach().reshape(-1).to(torch.float64).contiguous()
    if not (x2.is_cuda and d2.is_cuda):
        raise TypeError("x and dLdx must be CUDA tensors")
    g = torch.empty_like(x2)
    it = ctypes.c_int32()
    dl = ctypes.c_double()
    db = ctypes.c_double()
    rc = check(_ffi.lib().pcg_adjoint(op.handle, nys.handle if nys is not None else None, float(lam),
                                      int(bool(adaptive)), _ptr(x2), _ptr(d2), float(tol), int(maxit),
                                      int(refine_every), int(inner_mode), int(refine_mode), int(check_mode), _ptr(g),
                                      ctypes.byref(it), ctypes.byref(dl), ctypes.byref(db), _stream(stream)),
               "pcg_adjoint")
    _warn_unconverged(rc, "pcg_adjoint")
    return g, dl.value, db.value, it.value


class _KRRSolve(torch.autograd.Function):
    """x = (K(bw) + lam I)^{-1} b (FP64 x) with an adjoint backward (pcg_adjoint)."""

    @staticmethod
    def forward(ctx, b, bw, lam, op, nys, kw):
        op.set_bandwidth(float(bw))
        res = pcg_solve(op, b.detach().to(torch.float32), [float(lam)], nys=nys, **kw)
        _warn_unconverged(res.status, "krr_solve")
        x = res.x.reshape(b.shape)
        ctx.save_for_backward(x)
        # the operator is shared and mutable: the backward pass restores the
        # bandwidth this solve used
        ctx.op, ctx.nys, ctx.kw, ctx.lam, ctx.bw = op, nys, kw, float(lam), float(bw)
        ctx.b_dtype, ctx.bw_dtype, ctx.lam_dtype = b.dtype, bw.dtype, lam.dtype
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        kw = {k: v for k, v in ctx.kw.items() if k != "history"}
        ctx.op.set_bandwidth(ctx.bw)
        g, dlam, dbw, _ = pcg_adjoint(ctx.op, x, gx, ctx.lam, nys=ctx.nys, **kw)
        return (g.reshape(x.shape).to(ctx.b_dtype), torch.tensor(dbw, dtype=ctx.bw_dtype),
                torch.tensor(dlam, dtype=ctx.lam_dtype), None, None, None)


def krr_solve(op: KernelOperator, b: torch.Tensor, bw: torch.Tensor, lam: torch.Tensor, nys: Nystrom | None = None,
              **kw):
    """Differentiable solve of (K(bw) + lam I) x = b with respect to b, bw and lam
    (bw and lam are 0-dim CPU tensors).  The paper differentiates through the
    solver (Sec. 3.2); here the backward pass is one adjoint solve."""
    return _KRRSolve.apply(b, bw, lam, op, nys, kw)


def solve_grad_points(op: KernelOperator, x: torch.Tensor, g: torch.Tensor, mode: int = ACCURATE):
    """Gradient of a loss L(x) with respect to the training points X through the
    operator, for x = (K(X) + lam I)^{-1} b and the adjoint g = (K + lam I)^{-1} dL/dx
    (pcg_adjoint): dL/dX = -d(g^T K(X) x)/dX (kop_grad_points), n x d."""
    return -op.grad_points(g.reshape(-1).float(), x.reshape(-1).float(), mode=mode)


class NysADMMLinearSolver:
    """The linear solve inside NysADMM (ADMMConfig, App. A.4) through the
    library's admm_create / admm_solve: the k-th call solves
    (A + (rho + sigma) I) x = rhs to the relative tolerance max(tol_min, k^-gamma),
    warm-started from the previous call's x, with one Nystrom preconditioner of
    A (damping rho + sigma) rebuilt every `update_freq` calls from Omega."""

    def __init__(self, op: KernelOperator, Omega: torch.Tensor, update_freq: int = 20, sigma: float = 1e-6,
                 gamma: float = 1.2, tol_min: float = 1e-8, maxit: int = 1000, nys_mode: int = FAST,
                 refine_every: int = 30, inner_mode: int = FAST, refine_mode: int = PLAIN, check_mode: int = PLAIN,
                 stream=None):
        Om = _dev_f32(Omega, "Omega")
        if Om.shape[0] != op.n:
            raise ValueError("Omega must have n rows")
        self.op = op
        self.device = Om.device
        h = ctypes.c_void_p()
        check(_ffi.lib().admm_create(op.handle, _ptr(Om), Om.shape[1], int(update_freq), float(sigma), float(gamma),
                                     float(tol_min), int(maxit), int(refine_every), int(nys_mode), int(inner_mode),
                                     int(refine_mode), int(check_mode), _stream(stream), ctypes.byref(h)),
              "admm_create")
        self._h = h
        self.k = 0
        self.builds = 0
        self.x = None
        self.last = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _ffi.lib().admm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, rhs: torch.Tensor, rho: float, stream=None) -> torch.Tensor:
        r = _dev_f32(rhs.reshape(-1), "rhs")
        x = torch.empty(self.op.n, dtype=torch.float64, device=self.device)
        it, tr, tol, rb = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        rc = check(_ffi.lib().admm_solve(self._h, _ptr(r), float(rho), _ptr(x), ctypes.byref(it), ctypes.byref(tr),
                                         ctypes.byref(tol), ctypes.byref(rb), _stream(stream)), "admm_solve")
        self.k += 1
        self.builds += int(rb.value)
        self.x = x
        self.last = SolveResult(x, [it.value], None, [tr.value], rc)
        self.last.tol = tol.value
        return x


def pcg_adjoint_val(op: KernelOperator, x: torch.Tensor, Xv: torch.Tensor, yv: torch.Tensor, lam: float,
                    nys: Nystrom | None = None, adaptive: bool = True, tol: float = 1e-6, maxit: int = 1000,
                    refine_every: int = 30, inner_mode: int = FAST, refine_mode: int = PLAIN, check_mode: int = PLAIN,
                    stream=None):
    """Validation loss L = (1/n_val) ||K(Xv, X) x - yv||^2 of a solution x of
    (K + lam I) x = y (FP64 device vector) and its derivatives, all in the
    library (pcg_adjoint_val).  Returns (loss, dL/dbw, dL/dlam, g = dL/dy, iters)."""
    x2 = x.detach().reshape(-1).to(torch.float64).contiguous()
    Xv2 = _dev_f32(Xv, "Xv")
    yv2 = _dev_f32(yv.reshape(-1), "yv")
    if not x2.is_cuda or x2.shape[0] != op.n:
        raise ValueError("x must be a CUDA vector of n entries")
    if Xv2.shape[1] != op.d or yv2.shape[0] != Xv2.shape[0]:
        raise ValueError("Xv must be n_val x d and yv must have n_val entries")
    g = torch.empty_like(x2)
    it = ctypes.c_int32()
    loss, dl, db = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = check(_ffi.lib().pcg_adjoint_val(op.handle, nys.handle if nys is not None else None, float(lam),
                                          int(bool(adaptive)), _ptr(x2), _ptr(Xv2), Xv2.shape[0], _ptr(yv2),
                                          float(tol), int(maxit), int(refine_every), int(inner_mode),
                                          int(refine_mode), int(check_mode), _ptr(g), ctypes.byref(it),
                                          ctypes.byref(loss), ctypes.byref(dl), ctypes.byref(db), _stream(stream)),
               "pcg_adjoint_val")
    _warn_unconverged(rc, "pcg_adjoint_val")
    return loss.value, db.value, dl.value, g, it.value


def krr_val_loss_and_grad(op: KernelOperator, nys: Nystrom | None, y: torch.Tensor, Xv: torch.Tensor,
                          yv: torch.Tensor, lam: float, tol: float = 1e-6, maxit: int = 1000, refine_every: int = 30,
                          inner_mode: int = FAST, refine_mode: int = PLAIN, check_mode: int = PLAIN, stream=None):
    """Validation loss L = (1/n_val) ||K(Xv, X) x - yv||^2 with x = (K + lam I)^{-1} y,
    and its derivatives with respect to the bandwidth and lam: pcg_solve, then
    pcg_adjoint_val (the loss, the adjoint solve and both derivatives in the
    library).  Returns (loss, dL/dbw, dL/dlam)."""
    kw = dict(tol=tol, maxit=maxit, refine_every=refine_every, inner_mode=inner_mode, refine_mode=refine_mode,
              check_mode=check_mode)
    res = pcg_solve(op, y, [lam], nys=nys, stream=stream, **kw)
    _warn_unconverged(res.status, "krr_val_loss_and_grad")
    loss, dbw, dlam, _, _ = pcg_adjoint_val(op, res.x, Xv, yv, lam, nys=nys, stream=stream, **kw)
    return loss, dbw, dlam
