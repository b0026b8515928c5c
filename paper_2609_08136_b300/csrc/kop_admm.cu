// The linear solve inside NysADMM (ADMMConfig, App. A.4; NysADMM is cited in
// Sec. 2.3 and Sec. 4.3): the k-th call solves
//     (A + (rho_k + sigma) I) x_k = rhs_k
// warm-started from x_{k-1}, to the relative tolerance max(tol_min, k^-gamma),
// with one randomized Nystrom preconditioner of A damped by rho_k + sigma and
// rebuilt every `update_freq` calls from the same test matrix.  The paper
// lists sigma, gamma and preconditioner_update_freq without formulas; the
// schedule here is this library's reading of them.  Everything else (the
// solve, the preconditioner, the certification of the stop) is pcg_solve's.
#include <cmath>

#include "kop_device.cuh"
#include "kop_internal.h"

struct admm_s {
  kop_s* op = nullptr;
  float* Omega = nullptr;  // device copy, n x r
  int r = 0, update_freq = 0, maxit = 0, refine_every = 0;
  int nys_mode = KOP_FAST, inner_mode = KOP_FAST, refine_mode = KOP_PLAIN, check_mode = KOP_PLAIN;
  double sigma = 0.0, gamma = 1.0, tol_min = 0.0;
  int64_t k = 0;       // calls so far
  int32_t builds = 0;  // Nystrom builds so far
  nys_s* ny = nullptr;
  double* x = nullptr;  // device, n FP64: the previous solution
};

using namespace kop;

static bool admm_mode_ok(int m) { return m >= KOP_FAST && m <= KOP_EXACT; }

extern "C" int admm_create(kop_t op, const float* Omega, int32_t r, int32_t update_freq, double sigma, double gamma,
                           double tol_min, int32_t maxit, int32_t refine_every, int32_t nys_mode, int32_t inner_mode,
                           int32_t refine_mode, int32_t check_mode, void* stream, admm_t* out) {
  if (!out) return fail(KOP_EINVAL, "admm_create: out is NULL");
  *out = nullptr;
  if (!op || !Omega) return fail(KOP_EINVAL, "admm_create: NULL argument");
  const int64_t n = op_dim(op);
  if (r < 1 || r > 2048 || r > n) return fail(KOP_EINVAL, "admm_create: r must be in [1, min(n, 2048)]");
  if (update_freq < 0 || maxit < 1 || refine_every < 0)
    return fail(KOP_EINVAL, "admm_create: need update_freq >= 0, maxit >= 1, refine_every >= 0");
  if (!(sigma >= 0.0) || !std::isfinite(sigma) || !(gamma >= 0.0) || !std::isfinite(gamma) || !(tol_min > 0.0) ||
      !(tol_min < 1.0))
    return fail(KOP_EINVAL, "admm_create: need sigma >= 0, gamma >= 0 finite, 0 < tol_min < 1");
  if (!admm_mode_ok(nys_mode) || !admm_mode_ok(inner_mode) || !admm_mode_ok(refine_mode) || !admm_mode_ok(check_mode))
    return fail(KOP_EINVAL, "admm_create: bad mode");
  cudaStream_t st = (cudaStream_t)stream;
  admm_s* a = new admm_s();
  a->op = op;
  a->r = r;
  a->update_freq = update_freq;
  a->sigma = sigma;
  a->gamma = gamma;
  a->tol_min = tol_min;
  a->maxit = maxit;
  a->refine_every = refine_every;
  a->nys_mode = nys_mode;
  a->inner_mode = inner_mode;
  a->refine_mode = refine_mode;
  a->check_mode = check_mode;
  cudaError_t e = cudaMalloc(&a->Omega, sizeof(float) * (size_t)n * r);
  if (e == cudaSuccess) e = cudaMalloc(&a->x, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a->Omega, Omega, sizeof(float) * (size_t)n * r, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(a->Omega);
    cudaFree(a->x);
    delete a;
    return cuda_fail(e, "admm_create");
  }
  *out = a;
  return KOP_OK;
}

extern "C" int admm_destroy(admm_t a) {
  if (!a) return KOP_OK;
  nys_destroy(a->ny);
  cudaDeviceSynchronize();
  cudaFree(a->Omega);
  cudaFree(a->x);
  delete a;
  return KOP_OK;
}

extern "C" int admm_solve(admm_t a, const float* rhs, double rho, double* x_out, int32_t* iters, double* true_relres,
                          double* tol_used, int32_t* rebuilt, void* stream) {
  if (!a || !rhs || !x_out) return fail(KOP_EINVAL, "admm_solve: NULL argument");
  if (!(rho >= 0.0) || !std::isfinite(rho) || !(rho + a->sigma > 0.0))
    return fail(KOP_EINVAL, "admm_solve: need rho >= 0 finite and rho + sigma > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = op_dim(a->op);
  const int64_t k = a->k + 1;
  int rc = KOP_OK;
  const bool rebuild = !a->ny || (a->update_freq > 0 && (k - 1) % a->update_freq == 0);
  if (rebuild) {
    nys_destroy(a->ny);
    a->ny = nullptr;
    if ((rc = nys_build(a->op, a->Omega, a->r, 0.0, a->nys_mode, stream, &a->ny))) return rc;
    ++a->builds;
  }
  const double shift = rho + a->sigma;
  double tol = std::pow((double)k, -a->gamma);
  if (tol < a->tol_min) tol = a->tol_min;
  int32_t it = 0;
  double tr = 0.0;
  rc = pcg_solve(a->op, a->ny, &shift, 1, nullptr, 1, rhs, 1, a->k > 0 ? a->x : nullptr, tol, a->maxit,
                 a->refine_every, a->inner_mode, a->refine_mode, a->check_mode, x_out, &it, nullptr, &tr, stream);
  if (rc < 0) return rc;
  KOP_CUDA_TRY(cudaMemcpyAsync(a->x, x_out, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  a->k = k;
  if (iters) *iters = it;
  if (true_relres) *true_relres = tr;
  if (tol_used) *tol_used = tol;
  if (rebuilt) *rebuilt = rebuild ? 1 : 0;
  return rc;
}
