// Randomized Nystrom preconditioner: nys_build / nys_apply / nys_eigs /
// nys_factor / nys_destroy.
//
// The approximation is the one of Frangella, Tropp & Udell (the paper's
// randomized Nystrom preconditioner, Sec. 1 and Sec. 2.3; configuration in
// App. A.5):  Y = K Omega, a shift nu, Y_nu = Y + nu Omega,
// C = chol(Omega^T Y_nu), B = Y_nu C^-1 = U S V^T, lam_hat = max(0, S^2 - nu).
// Here B is never formed: its thin SVD comes from the r x r matrix
//   B^T B = C^-T (Y_nu^T Y_nu) C^-1 = V S^2 V^T
// (Y_nu^T Y_nu = Y^T Y + nu (Omega^T Y + Y^T Omega) + nu^2 Omega^T Omega, so
// only three r x r Gram blocks are needed), then U = Y_nu C^-1 V S^-1 is one
// tall product.  All r x r work is FP64 on the device.  The O(n r^2) passes
// (Omega^T Omega, Omega^T Y, U = Y_nu W and the Cholesky-QR products) run on
// the tensor cores with FP32-accurate products (kop_tcgemm.cu); Y^T Y is
// summed error-free on the CUDA cores, because the core squares the
// condition of the sketch.  One Cholesky-QR pass afterwards restores the
// orthonormality of U lost to FP32 rounding.  The caller's FP32 test matrix
// is used as given in every step: the fast sketch's contraction carries it
// (scaled per column by a power of two) as an FP16 hi + lo pair against the
// kernel values rounded to FP16, the Gram blocks as the exact three-term
// split.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kop_dense.h"
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

// Per-column damping of the preconditioner apply.
//   d_k(c) = 1 / (lam_k + mu_c) - 1 / rho_c,   alpha_c = 1 / rho_c,
//   rho_c = lam_r + mu_c (adaptive) or mu_c.
// W (r x m) is scaled in place; an FP32 copy is written when Wf != NULL.
__global__ void nys_scale_kernel(double* __restrict__ W, int r, int m, const double* __restrict__ lam,
                                 const double* __restrict__ mu, int adaptive, float* __restrict__ Wf,
                                 double* __restrict__ alpha, float* __restrict__ alpha_f, int split_inplace) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * m) return;
  const int k = (int)(t / m), c = (int)(t - (int64_t)k * m);
  const double rho = adaptive ? lam[r - 1] + mu[c] : mu[c];
  const double w = W[t] * (1.0 / (lam[k] + mu[c]) - 1.0 / rho);
  if (split_inplace) {
    // w as the exact-to-2^-48 pair hi + lo of FP32 values, in W's own slot
    const float hi = (float)w;
    reinterpret_cast<float2*>(W)[t] = make_float2(hi, (float)(w - (double)hi));
  } else {
    W[t] = w;
  }
  if (Wf) Wf[t] = (float)w;
  if (k == 0) {
    alpha[c] = 1.0 / rho;
    if (alpha_f) alpha_f[c] = (float)(1.0 / rho);
  }
}

// Device side of nys_apply with caller-provided scratch:
//   Wd: r*m doubles, alpha: m doubles, Wf: r*m floats, alpha_f: m floats.
// Up to 8 columns the whole apply runs with FP64-accurate sums (error-free
// float-float arithmetic) on the stored FP32 U, so that P^-1 is applied as one
// fixed symmetric operator: in plain FP32 the cancellation between v / rho and
// the projected part loses a factor (lam_1 + mu) / rho of accuracy on the
// leading subspace.  Wider blocks use the tensor-core products with FP32
// accuracy (the solver tolerates the inexact apply).
int nys_apply_dev(const nys_s* ny, const double* mu_dev, int adaptive, const float* V, int m, float* O, double* Wd,
                  double* alpha, float* Wf, float* alpha_f, cudaStream_t st) {
  const int r = ny->r;
  const int64_t n = ny->n;
  const int64_t tot = (int64_t)r * m;
  if (m <= 8) {
    int rc = utv_ff(ny->U, r, n, r, V, m, Wd, st);
    if (rc) return rc;
    nys_scale_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Wd, r, m, ny->lam_dev, mu_dev, adaptive, nullptr,
                                                                    alpha, nullptr, 1);
    KOP_LAUNCHED();
    return uw_ff(ny->U, r, n, r, reinterpret_cast<const float2*>(Wd), V, m, alpha, O, st);
  }
  // wider blocks: W = U^T V and O = alpha (.) V + U W' on the tensor cores
  // (FP32-accurate products), from BF16 splits of U kept with the factor
  nys_s* nym = const_cast<nys_s*>(ny);
  if (!nym->Ut) {
    KOP_CUDA_TRY(cudaMalloc(&nym->Ut, sizeof(__nv_bfloat16) * (size_t)tsplit_elems(n, r)));
    cudaError_t e = cudaMalloc(&nym->Ur, sizeof(__nv_bfloat16) * (size_t)rsplit_elems(n, r));
    if (e != cudaSuccess) {
      cudaFree(nym->Ut);
      nym->Ut = nullptr;
      nym->Ur = nullptr;
      return cuda_fail(e, "nys_apply: cudaMalloc");
    }
    int rc = tsplit(ny->U, nullptr, 0.0f, r, n, r, nym->Ut, st);
    if (rc == KOP_OK) rc = rsplit(ny->U, nullptr, 0.0f, r, n, r, nym->Ur, st);
    if (rc) {
      cudaFree(nym->Ut);
      cudaFree(nym->Ur);
      nym->Ut = nym->Ur = nullptr;
      return rc;
    }
  }
  DevBuf vb;
  vb.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&vb.p, sizeof(__nv_bfloat16) * (size_t)tsplit_elems(n, m), st));
  __nv_bfloat16* Vt = (__nv_bfloat16*)vb.p;
  int* status = ny->op->status;
  int rc = tsplit(V, nullptr, 0.0f, m, n, m, Vt, st);
  if (rc == KOP_OK) rc = gram_tc(ny->Ut, Vt, n, r, m, false, Wd, m, status, st);
  if (rc) return rc;
  nys_scale_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Wd, r, m, ny->lam_dev, mu_dev, adaptive, Wf, alpha,
                                                                  alpha_f, 0);
  KOP_LAUNCHED();
  return tall_tc(ny->Ur, n, r, Wf, m, m, V, m, alpha_f, O, m, status, st);
}

static int read_info(const int* dev, int* host, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  return KOP_OK;
}

}  // namespace kop

using namespace kop;

extern "C" int nys_build(kop_t op, const float* Omega, int32_t r, double nu_rel, int32_t mode, void* stream,
                         nys_t* out) {
  if (!out) return fail(KOP_EINVAL, "nys_build: out is NULL");
  *out = nullptr;
  if (!op || !Omega) return fail(KOP_EINVAL, "nys_build: NULL argument");
  const int64_t n = op_dim(op);
  if (r < 1 || r > 2048 || r > n) return fail(KOP_EINVAL, "nys_build: r must be in [1, min(n, 2048)]");
  if (mode < KOP_FAST || mode > KOP_EXACT) return fail(KOP_EINVAL, "nys_build: bad mode");
  if (!std::isfinite(nu_rel)) return fail(KOP_EINVAL, "nys_build: nu_rel must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  if (!(nu_rel > 0.0)) nu_rel = mode == KOP_FAST ? std::ldexp(1.0, -16) : std::ldexp(1.0, -21);

  const size_t rr = (size_t)r * r;
  const int64_t n_pad = op_dim_pad(op);
  // workspace
  DevBuf wsY, wsR, wsU;
  wsY.st = wsR.st = wsU.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&wsY.p, sizeof(float) * (size_t)n * r, st));
  const size_t nd = 9 * rr + 4 * (size_t)r + 16 + sym_eig_work_doubles(r);
  KOP_CUDA_TRY(cudaMallocAsync(&wsR.p, sizeof(double) * nd + sizeof(float) * rr + sizeof(int) * (r + 8), st));
  KOP_CUDA_TRY(cudaMallocAsync(&wsU.p, sizeof(float) * (size_t)n_pad * r, st));
  float* Y = (float*)wsY.p;
  float* U2 = (float*)wsU.p;
  double* Goo = (double*)wsR.p;
  double* Goy = Goo + rr;
  double* Gyy = Goy + rr;
  double* M = Gyy + rr;   // becomes L
  double* G2 = M + rr;
  double* Z = G2 + rr;
  double* H = Z + rr;
  double* E = H + rr;
  double* Wm = E + rr;
  double* w = Wm + rr;
  double* lam = w + r;
  double* scal = lam + r;  // 16
  double* jw = scal + 16;
  float* Wf = (float*)(jw + sym_eig_work_doubles(r));
  int* perm = (int*)(Wf + rr);
  int* info = perm + r;

  int rc;
  // 1. sketch Y = K Omega (fused operator, m = r)
  rc = op_apply(op, mode, Omega, r, r, Y, r, st, /*sketch=*/true);
  if (rc) return rc;
  // 2. Gram blocks: Omega^T Omega and Omega^T Y on the tensor cores from BF16
  // splits of the two matrices (two scratch buffers, reused below)
  DevBuf wsS1, wsS2;
  wsS1.st = wsS2.st = st;
  const size_t split_elems = (size_t)std::max(tsplit_elems(n, r), rsplit_elems(n, r));
  KOP_CUDA_TRY(cudaMallocAsync(&wsS1.p, sizeof(__nv_bfloat16) * split_elems, st));
  KOP_CUDA_TRY(cudaMallocAsync(&wsS2.p, sizeof(__nv_bfloat16) * split_elems, st));
  __nv_bfloat16* S1 = (__nv_bfloat16*)wsS1.p;
  __nv_bfloat16* S2 = (__nv_bfloat16*)wsS2.p;
  if ((rc = tsplit(Omega, nullptr, 0.0f, r, n, r, S1, st))) return rc;
  if ((rc = tsplit(Y, nullptr, 0.0f, r, n, r, S2, st))) return rc;
  if ((rc = gram_tc(S1, S1, n, r, r, true, Goo, r, op->status, st))) return rc;
  if ((rc = gram_tc(S1, S2, n, r, r, false, Goy, r, op->status, st))) return rc;
  // Y^T Y error-free: the core C^-T (Y_nu^T Y_nu) C^-1 squares the condition
  // of the sketch, and FP32 sums make its smallest eigenvalues negative once
  // the spectrum spans ~1e5
  if ((rc = gram_sym(Y, r, n, r, Gyy, r, st))) return rc;
  // 3. ||Y||_2 by power iteration on Y^T Y
  if ((rc = power_max_eig(Gyy, r, 60, scal, st))) return rc;
  double ymax2 = 0.0;
  KOP_CUDA_TRY(cudaMemcpyAsync(&ymax2, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  {
    const int s = kop_sync(op, stream);
    if (s != KOP_OK) return s;
  }
  if (!std::isfinite(ymax2) || !(ymax2 > 0.0)) return fail(KOP_ENOTPD, "nys_build: sketch is zero or not finite");
  double nu = nu_rel * std::sqrt(ymax2);
  // 4. C = chol(sym(Omega^T Y_nu)); grow nu on a failed pivot
  int attempt = 0, hinfo = 1;
  for (; attempt < 4; ++attempt) {
    if ((rc = combine(Goo, Goy, Gyy, r, nu, 0, M, st))) return rc;
    if ((rc = cholesky(M, r, info, st))) return rc;
    if ((rc = read_info(info, &hinfo, st))) return rc;
    if (hinfo == 0) break;
    nu *= 10.0;
  }
  if (hinfo != 0) return fail(KOP_ENOTPD, "nys_build: Cholesky of Omega^T Y_nu failed after growing the shift");
  // 5. Y_nu^T Y_nu
  if ((rc = combine(Goo, Goy, Gyy, r, nu, 1, G2, st))) return rc;
  // 6. H = L^-1 G2 L^-T  (C = L^T)
  if ((rc = trsm(M, r, G2, r, r, 0, st))) return rc;          // G2 <- L^-1 G2
  if ((rc = transpose(G2, r, Z, 0, st))) return rc;           // Z = (L^-1 G2)^T
  if ((rc = trsm(M, r, Z, r, r, 0, st))) return rc;           // Z <- L^-1 Z
  if ((rc = transpose(Z, r, H, 1, st))) return rc;            // H = sym(Z)
  // 7. H = E diag(w) E^T
  KOP_CUDA_TRY(cudaMemsetAsync(op->status, 0, sizeof(int), st));
  if ((rc = sym_eig(H, r, jw, op->status, w, E, st))) return rc;
  // 8. descending order, lam_hat, Wm = E_sorted diag(w)^-1/2
  if ((rc = sort_desc(w, r, perm, st))) return rc;
  if ((rc = nys_finish(w, E, perm, r, nu, lam, Wm, st))) return rc;
  // 9. W = C^-1 Wm = L^-T Wm
  if ((rc = trsm(M, r, Wm, r, r, 1, st))) return rc;
  if ((rc = d2f(Wm, Wf, (int64_t)rr, st))) return rc;
  // 10. U = (Y + nu Omega) W   (rows beyond n stay zero)
  nys_s* ny = new nys_s();
  ny->op = op;
  ny->r = r;
  ny->n = n;
  ny->nu = nu;
  cudaError_t e = cudaMalloc(&ny->U, sizeof(float) * (size_t)n_pad * r);
  if (e == cudaSuccess) e = cudaMalloc(&ny->lam_dev, sizeof(double) * r);
  if (e != cudaSuccess) {
    if (ny->U) cudaFree(ny->U);
    delete ny;
    return cuda_fail(e, "nys_build: cudaMalloc");
  }
  ny->lam_host = new double[r];
  auto drop = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFree(ny->U);
    cudaFree(ny->lam_dev);
    delete[] ny->lam_host;
    delete ny;
    return code;
  };
  KOP_CUDA_TRY(cudaMemsetAsync(U2, 0, sizeof(float) * (size_t)n_pad * r, st));
  if ((rc = rsplit(Y, Omega, (float)nu, r, n, r, S2, st))) return drop(rc);
  if ((rc = tall_tc(S2, n, r, Wf, r, r, nullptr, 0, nullptr, U2, r, op->status, st))) return drop(rc);
  // 11. Cholesky-QR: U <- U2 Lu^-T with Lu Lu^T = U2^T U2
  if ((rc = tsplit(U2, nullptr, 0.0f, r, n, r, S1, st))) return drop(rc);
  if ((rc = gram_tc(S1, S1, n, r, r, true, Goo, r, op->status, st))) return drop(rc);
  if ((rc = cholesky(Goo, r, info, st))) return drop(rc);
  if ((rc = read_info(info, &hinfo, st))) return drop(rc);
  if (hinfo != 0) return drop(fail(KOP_ENOTPD, "nys_build: U lost rank (Cholesky-QR failed)"));
  if ((rc = eye(Z, r, st))) return drop(rc);
  if ((rc = trsm(Goo, r, Z, r, r, 1, st))) return drop(rc);   // Z = Lu^-T
  if ((rc = d2f(Z, Wf, (int64_t)rr, st))) return drop(rc);
  if (cudaMemsetAsync(ny->U, 0, sizeof(float) * (size_t)n_pad * r, st) != cudaSuccess) return drop(KOP_ECUDA);
  if ((rc = rsplit(U2, nullptr, 0.0f, r, n, r, S2, st))) return drop(rc);
  if ((rc = tall_tc(S2, n, r, Wf, r, r, nullptr, 0, nullptr, ny->U, r, op->status, st))) return drop(rc);
  if (cudaMemcpyAsync(ny->lam_dev, lam, sizeof(double) * r, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ny->lam_host, lam, sizeof(double) * r, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return drop(KOP_ECUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess) return drop(cuda_fail(cudaGetLastError(), "nys_build"));
  {
    const int s = kop_sync(op, stream);
    if (s != KOP_OK) return drop(s);
  }
  *out = ny;
  return KOP_OK;
}

extern "C" int nys_destroy(nys_t ny) {
  if (!ny) return KOP_OK;
  cudaDeviceSynchronize();
  cudaFree(ny->U);
  if (ny->Ut) cudaFree(ny->Ut);
  if (ny->Ur) cudaFree(ny->Ur);
  cudaFree(ny->lam_dev);
  delete[] ny->lam_host;
  delete ny;
  return KOP_OK;
}

extern "C" int nys_eigs(nys_t ny, double* lam_hat, double* nu, int32_t* r) {
  if (!ny) return fail(KOP_EINVAL, "nys_eigs: NULL handle");
  if (lam_hat)
    for (int k = 0; k < ny->r; ++k) lam_hat[k] = ny->lam_host[k];
  if (nu) *nu = ny->nu;
  if (r) *r = ny->r;
  return KOP_OK;
}

extern "C" int nys_factor(nys_t ny, float* U_out, void* stream) {
  if (!ny || !U_out) return fail(KOP_EINVAL, "nys_factor: NULL argument");
  KOP_CUDA_TRY(cudaMemcpyAsync(U_out, ny->U, sizeof(float) * (size_t)ny->n * ny->r, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return KOP_OK;
}

extern "C" int nys_apply(nys_t ny, const double* mu, int32_t adaptive, const float* V, int32_t m, float* O,
                         void* stream) {
  if (!ny || !mu || !V || !O) return fail(KOP_EINVAL, "nys_apply: NULL argument");
  if (m < 1) return fail(KOP_EINVAL, "nys_apply: m must be >= 1");
  // mu = 0 needs lam_hat_r > 0 (adaptive): otherwise 1 / (lam_k + mu) divides by zero
  const bool zero_ok = adaptive && ny->lam_host[ny->r - 1] > 0.0;
  for (int c = 0; c < m; ++c)
    if (!(mu[c] >= 0.0) || !std::isfinite(mu[c]) || (!zero_ok && !(mu[c] > 0.0)))
      return fail(KOP_EINVAL, "nys_apply: mu must be finite and > 0 (mu = 0 only when adaptive with lam_hat_r > 0)");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t r = ny->r;
  DevBuf ws;
  ws.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(double) * (r * m + 2 * m) + sizeof(float) * (r * m + m), st));
  double* Wd = (double*)ws.p;
  double* mu_dev = Wd + r * m;
  double* alpha = mu_dev + m;
  float* Wf = (float*)(alpha + m);
  float* alpha_f = Wf + r * m;
  KOP_CUDA_TRY(cudaMemcpyAsync(mu_dev, mu, sizeof(double) * m, cudaMemcpyHostToDevice, st));
  const int rc = nys_apply_dev(ny, mu_dev, adaptive, V, m, O, Wd, alpha, Wf, alpha_f, st);
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  return rc;
}
