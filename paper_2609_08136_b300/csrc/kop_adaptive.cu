// Nystrom approximation with rank adaptation: nys_build_adaptive.
//
// The NystromConfig table (App. A.5) gives the controls: rank_init,
// rank_max, num_power_iters (error estimation) and error_tolerance.  The
// scheme is Frangella, Tropp & Udell's adaptive one: start at rank_init, and
// while the estimated error of the rank-r approximation is too large, double r
// (capped at rank_max).  The rank-r approximation uses the first r columns of
// one n x rank_max test matrix, so each larger sketch extends the smaller one.
// Its error ||K - U diag(lam_hat) U^T||_2 is estimated by power iteration on
// the positive semidefinite error matrix E: from v = g0 / ||g0||,
//   w = K v - U (lam_hat * (U^T v)),  est = ||w||,  v = w / est,
// num_power_iters times; r is accepted when est <= error_tolerance * lam_hat_1.
// K v is the fused operator product (m = 1, in the build's mode); the U
// products are the float-float kernels of the preconditioner apply.
#include <cmath>
#include <string>

#include "kop_dense.h"
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

// Dst (n x r, contiguous) = the first r columns of Src (n x ld).
__global__ void gather_cols_kernel(const float* __restrict__ src, int64_t n, int ld, int r, float* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * r) return;
  const int64_t i = t / r;
  const int c = (int)(t - i * r);
  dst[t] = src[i * ld + c];
}

// W[k] = lam[k] * W[k], stored in place as the pair hi + lo of FP32 values
// (the operand form of uw_ff).
__global__ void lam_scale_split_kernel(double* __restrict__ W, const double* __restrict__ lam, int r) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r) return;
  const double w = W[k] * lam[k];
  const float hi = (float)w;
  reinterpret_cast<float2*>(W)[k] = make_float2(hi, (float)(w - (double)hi));
}

// acc += sum_i x_i^2 in FP64.
__global__ void __launch_bounds__(256) norm2_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ acc) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(acc, t);
  }
}

// y = x * scale (FP64 factor).
__global__ void scale_kernel(const float* __restrict__ x, int64_t n, double scale, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)((double)x[i] * scale);
}

// ||x||_2 of a device vector (synchronizes the stream).
static int device_norm(const float* x, int64_t n, double* acc, double* out, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double), st));
  int blocks = 2 * num_sms();
  if ((int64_t)blocks * 256 > n) blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  norm2_kernel<<<blocks, 256, 0, st>>>(x, n, acc);
  KOP_LAUNCHED();
  double h = 0.0;
  KOP_CUDA_TRY(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  *out = std::sqrt(h);
  return KOP_OK;
}

// Power-iteration estimate of ||K - U diag(lam_hat) U^T||_2 (see the file
// comment).  Scratch: v, kv, o (n floats each), wd (r doubles), dev (2 doubles).
static int error_estimate(nys_s* ny, int mode, const float* g0, int iters, float* v, float* kv, float* o, double* wd,
                          double* dev, double* est_out, cudaStream_t st) {
  kop_s* op = ny->op;
  const int64_t n = ny->n;
  const int r = ny->r;
  const unsigned nb = (unsigned)((n + 255) / 256);
  double* acc = dev;
  double* alpha = dev + 1;  // -1: uw_ff returns -K v + U W = -E v
  const double minus_one = -1.0;
  KOP_CUDA_TRY(cudaMemcpyAsync(alpha, &minus_one, sizeof(double), cudaMemcpyHostToDevice, st));
  double nrm = 0.0;
  int rc = device_norm(g0, n, acc, &nrm, st);
  if (rc) return rc;
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return fail(KOP_EINVAL, "nys_build_adaptive: g0 is zero or not finite");
  scale_kernel<<<nb, 256, 0, st>>>(g0, n, 1.0 / nrm, v);
  KOP_LAUNCHED();
  double est = 0.0;
  for (int it = 0; it < iters; ++it) {
    if ((rc = op_apply(op, mode, v, 1, 1, kv, 1, st))) return rc;
    if ((rc = utv_ff(ny->U, r, n, r, v, 1, wd, st))) return rc;
    lam_scale_split_kernel<<<(unsigned)((r + 127) / 128), 128, 0, st>>>(wd, ny->lam_dev, r);
    KOP_LAUNCHED();
    if ((rc = uw_ff(ny->U, r, n, r, reinterpret_cast<const float2*>(wd), kv, 1, alpha, o, st))) return rc;
    if ((rc = device_norm(o, n, acc, &est, st))) return rc;
    if (!std::isfinite(est)) return fail(KOP_ECUDA, "nys_build_adaptive: error estimate is not finite");
    if (est == 0.0) break;
    scale_kernel<<<nb, 256, 0, st>>>(o, n, 1.0 / est, v);
    KOP_LAUNCHED();
  }
  *est_out = est;
  return kop_sync(op, st);
}

}  // namespace kop

using namespace kop;

extern "C" int nys_build_adaptive(kop_t op, const float* Omega, int32_t ld_omega, int32_t rank_init,
                                  int32_t rank_max, int32_t power_iters, double err_tol, const float* g0,
                                  double nu_rel, int32_t mode, void* stream, nys_t* out, int32_t* rank_out,
                                  double* err_out, int32_t* hist_rank, double* hist_err, int32_t hist_len) {
  if (!out) return fail(KOP_EINVAL, "nys_build_adaptive: out is NULL");
  *out = nullptr;
  if (!op || !Omega || !g0) return fail(KOP_EINVAL, "nys_build_adaptive: NULL argument");
  const int64_t n = op_dim(op);
  if (rank_init < 1 || rank_max < rank_init || rank_max > 2048 || rank_max > n)
    return fail(KOP_EINVAL, "nys_build_adaptive: need 1 <= rank_init <= rank_max <= min(n, 2048)");
  if (ld_omega < rank_max) return fail(KOP_EINVAL, "nys_build_adaptive: ld_omega < rank_max");
  if (power_iters < 1 || power_iters > 1000) return fail(KOP_EINVAL, "nys_build_adaptive: power_iters must be in [1, 1000]");
  if (!(err_tol >= 0.0) || !std::isfinite(err_tol)) return fail(KOP_EINVAL, "nys_build_adaptive: bad error tolerance");
  if (hist_len < 0 || (hist_len > 0 && (!hist_rank || !hist_err)))
    return fail(KOP_EINVAL, "nys_build_adaptive: bad history arrays");
  cudaStream_t st = (cudaStream_t)stream;
  // scratch: the gathered test matrix (n x rank_max floats at most), three n-vectors,
  // rank_max doubles and two more
  // (each array starts on a 256-byte boundary)
  const size_t nv = ((size_t)n + 63) / 64 * 64;
  const size_t fl = ((size_t)n * rank_max + 63) / 64 * 64 + 3 * nv;
  DevBuf ws;
  ws.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(float) * fl + sizeof(double) * ((size_t)rank_max + 2), st));
  float* Om = (float*)ws.p;
  float* v = Om + ((size_t)n * rank_max + 63) / 64 * 64;
  float* kv = v + nv;
  float* o = kv + nv;
  double* wd = (double*)(o + nv);
  double* dev = wd + rank_max;

  int r = rank_init, builds = 0;
  for (;;) {
    const int64_t tot = n * (int64_t)r;
    gather_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Omega, n, ld_omega, r, Om);
    KOP_LAUNCHED();
    nys_t ny = nullptr;
    int rc = nys_build(op, Om, r, nu_rel, mode, stream, &ny);
    if (rc) return rc;
    double est = 0.0;
    rc = error_estimate(ny, mode, g0, power_iters, v, kv, o, wd, dev, &est, st);
    if (rc) {
      nys_destroy(ny);
      return rc;
    }
    if (builds < hist_len) {
      hist_rank[builds] = r;
      hist_err[builds] = est;
    }
    ++builds;
    if (est <= err_tol * ny->lam_host[0] || r >= rank_max) {
      *out = ny;
      if (rank_out) *rank_out = r;
      if (err_out) *err_out = est;
      return KOP_OK;
    }
    nys_destroy(ny);
    r = 2 * r < rank_max ? 2 * r : rank_max;
  }
}
