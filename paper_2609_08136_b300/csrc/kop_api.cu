// C ABI of the kernel operator (kop_*): argument checks, handle lifetime and
// dispatch to the fused / plain operator kernels.
#include <cmath>
#include <string>

#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

int op_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, int mode,
              const float* V, int m, int ldv, float* O, int ldo, int* status, cudaStream_t st, bool sketch) {
  if (kf >= KF_GRBF && (mode == KOP_PLAIN || mode == KOP_PLAIN_CHECK))
    return fail(KOP_EINVAL, "point-gradient products run in the FAST, ACCURATE or EXACT mode");
  if (mode == KOP_PLAIN) return plain_matvec(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, st);
  if (mode == KOP_PLAIN_CHECK) return plain_matvec(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, st, true);
  if (mode == KOP_EXACT) return exact_matvec_f32(Q, Ks, kf, kc.bw, V, m, ldv, O, ldo, st);
  return fused_matvec(Q, Ks, self, kf, kc, mode == KOP_ACCURATE ? 3 : 2, V, m, ldv, O, ldo, status, st,
                      sketch);
}

int op_apply(kop_s* op, int mode, const float* V, int m, int ldv, float* O, int ldo, cudaStream_t st,
             bool sketch) {
  if (op->ridge) return ridge_apply(op, mode, V, m, ldv, O, ldo, st);
  const KConst kc = kernel_constants(op->kernel, op->bw);
  return op_matvec(op->pts, op->pts, true, op->kernel, kc, mode, V, m, ldv, O, ldo, op->status, st, sketch);
}

int op_apply_f64(kop_s* op, const double* V, int m, int ldv, double* O, int ldo, cudaStream_t st) {
  if (op->ridge) return ridge_apply_f64(op, V, m, ldv, O, ldo, st);
  return exact_matvec(op->pts, op->pts, op->kernel, op->bw, V, m, ldv, O, ldo, st);
}

static bool bad_mode(int mode) { return mode < KOP_FAST || mode > KOP_EXACT; }

// Entry points that exist only for kernel operators.
static int need_kernel(const kop_s* op, const char* where) {
  return op->ridge ? fail(KOP_EINVAL, std::string(where) + ": not defined for a ridge (X^T X) operator") : KOP_OK;
}

}  // namespace kop

using namespace kop;

extern "C" int kop_create(const float* X, int64_t n, int32_t d, int32_t kernel, double bandwidth, void* stream,
                          kop_t* out) {
  if (!out) return fail(KOP_EINVAL, "kop_create: out is NULL");
  *out = nullptr;
  if (!X) return fail(KOP_EINVAL, "kop_create: X is NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(KOP_EINVAL, "kop_create: n must be in [1, 2^31)");
  if (d < 1 || d > 128) return fail(KOP_EINVAL, "kop_create: d must be in [1, 128]");
  if (kernel < KOP_RBF || kernel > KOP_MATERN52) return fail(KOP_EINVAL, "kop_create: unknown kernel");
  if (!(bandwidth > 0.0) || !std::isfinite(bandwidth)) return fail(KOP_EINVAL, "kop_create: bandwidth must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  kop_s* op = new kop_s();
  op->kernel = kernel;
  op->bw = bandwidth;
  int rc = KOP_OK;
  cudaError_t e = cudaMalloc(&op->mean, sizeof(double) * 128 + 256);
  if (e != cudaSuccess) {
    delete op;
    return cuda_fail(e, "kop_create: cudaMalloc");
  }
  op->status = (int*)((char*)op->mean + sizeof(double) * 128);
  e = cudaMemsetAsync(op->status, 0, sizeof(int), st);
  if (e == cudaSuccess) rc = pointset_alloc(op->pts, n, d, st);
  else rc = cuda_fail(e, "kop_create: memset");
  if (rc == KOP_OK) rc = column_mean(X, n, d, op->mean, st);
  if (rc == KOP_OK) rc = pointset_fill(op->pts, X, op->mean, st);
  if (rc == KOP_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "kop_create: synchronize");
  }
  if (rc != KOP_OK) {
    pointset_free(op->pts, st);
    cudaStreamSynchronize(st);
    cudaFree(op->mean);
    delete op;
    return rc;
  }
  *out = op;
  return KOP_OK;
}

extern "C" int kop_destroy(kop_t op) {
  if (!op) return KOP_OK;
  cudaDeviceSynchronize();
  if (op->ridge) {
    cudaFree(op->rX);
    cudaFree(op->status);
    delete op;
    return KOP_OK;
  }
  pointset_free(op->pts, 0);
  if (op->kc_owned) cudaFree(op->kc);
  if (op->kc_scratch) cudaFree(op->kc_scratch);
  cudaFree(op->mean);
  cudaDeviceSynchronize();
  delete op;
  return KOP_OK;
}

extern "C" int kop_set_bandwidth(kop_t op, double bandwidth) {
  if (!op) return fail(KOP_EINVAL, "kop_set_bandwidth: NULL handle");
  if (int rc = need_kernel(op, "kop_set_bandwidth")) return rc;
  if (!(bandwidth > 0.0) || !std::isfinite(bandwidth)) return fail(KOP_EINVAL, "kop_set_bandwidth: bandwidth must be > 0");
  op->bw = bandwidth;
  return KOP_OK;
}

static int check_cache_release(kop_s* op) {
  if (op->kc && op->kc_owned) {
    KOP_CUDA_TRY(cudaDeviceSynchronize());
    KOP_CUDA_TRY(cudaFree(op->kc));
  }
  op->kc = nullptr;
  if (op->kc_scratch) {
    KOP_CUDA_TRY(cudaDeviceSynchronize());
    KOP_CUDA_TRY(cudaFree(op->kc_scratch));
  }
  op->kc_scratch = nullptr;
  op->kc_scratch_floats = 0;
  op->kc_owned = 0;
  return KOP_OK;
}

extern "C" int kop_set_check_cache(kop_t op, int32_t enable, float* buffer, int64_t buffer_floats) {
  if (!op) return fail(KOP_EINVAL, "kop_set_check_cache: NULL handle");
  if (int rc = need_kernel(op, "kop_set_check_cache")) return rc;
  if (!enable) return check_cache_release(op);
  if (!buffer) {
    if (op->kc_owned) return KOP_OK;
    if (int rc = check_cache_release(op)) return rc;
    return check_cache_reserve(op);
  }
  if (buffer_floats < check_cache_floats(op->pts.n))
    return fail(KOP_EINVAL, "kop_set_check_cache: buffer smaller than nb * (floor(nb / 2) + 1) * 128^2 floats");
  if (reinterpret_cast<uintptr_t>(buffer) % 16 != 0)
    return fail(KOP_EINVAL, "kop_set_check_cache: buffer not 16-byte aligned");
  if (int rc = check_cache_release(op)) return rc;
  op->kc = buffer;
  op->kc_owned = 0;
  return KOP_OK;
}

extern "C" int kop_matvec(kop_t op, const float* V, int32_t m, float* O, int32_t mode, void* stream) {
  if (!op || !V || !O) return fail(KOP_EINVAL, "kop_matvec: NULL argument");
  if (m < 1) return fail(KOP_EINVAL, "kop_matvec: m must be >= 1");
  if (bad_mode(mode)) return fail(KOP_EINVAL, "kop_matvec: unknown mode");
  return op_apply(op, mode, V, m, m, O, m, (cudaStream_t)stream);
}

extern "C" int kop_matvec_f64(kop_t op, const double* V, int32_t m, double* O, int32_t deriv, void* stream) {
  if (!op || !V || !O) return fail(KOP_EINVAL, "kop_matvec_f64: NULL argument");
  if (m < 1) return fail(KOP_EINVAL, "kop_matvec_f64: m must be >= 1");
  if (!deriv) return op_apply_f64(op, V, m, m, O, m, (cudaStream_t)stream);
  if (int rc = need_kernel(op, "kop_matvec_f64")) return rc;
  return exact_matvec(op->pts, op->pts, op->kernel + (deriv ? 3 : 0), op->bw, V, m, m, O, m, (cudaStream_t)stream);
}

extern "C" int kop_dbw_matvec(kop_t op, const float* V, int32_t m, float* O, int32_t mode, void* stream) {
  if (!op || !V || !O) return fail(KOP_EINVAL, "kop_dbw_matvec: NULL argument");
  if (m < 1) return fail(KOP_EINVAL, "kop_dbw_matvec: m must be >= 1");
  if (bad_mode(mode)) return fail(KOP_EINVAL, "kop_dbw_matvec: unknown mode");
  if (int rc = need_kernel(op, "kop_dbw_matvec")) return rc;
  const KConst kc = kernel_constants(op->kernel + 3, op->bw);
  return op_matvec(op->pts, op->pts, true, op->kernel + 3, kc, mode, V, m, m, O, m, op->status,
                   (cudaStream_t)stream);
}

extern "C" int kop_cross_matvec(kop_t op, const float* Z, int64_t nz, const float* V, int32_t m, float* O,
                                int32_t transpose, int32_t deriv, int32_t mode, void* stream) {
  if (!op || !Z || !V || !O) return fail(KOP_EINVAL, "kop_cross_matvec: NULL argument");
  if (nz < 1 || nz >= (int64_t(1) << 31)) return fail(KOP_EINVAL, "kop_cross_matvec: nz must be in [1, 2^31)");
  if (m < 1) return fail(KOP_EINVAL, "kop_cross_matvec: m must be >= 1");
  if (bad_mode(mode)) return fail(KOP_EINVAL, "kop_cross_matvec: unknown mode");
  if (int rc = need_kernel(op, "kop_cross_matvec")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PointSet zs;
  int rc = pointset_alloc(zs, nz, op->pts.d, st);
  if (rc != KOP_OK) return rc;
  rc = pointset_fill(zs, Z, op->mean, st);
  const int kf = op->kernel + (deriv ? 3 : 0);
  const KConst kc = kernel_constants(kf, op->bw);
  if (rc == KOP_OK) {
    if (!transpose)
      rc = op_matvec(zs, op->pts, false, kf, kc, mode, V, m, m, O, m, op->status, st);
    else
      rc = op_matvec(op->pts, zs, false, kf, kc, mode, V, m, m, O, m, op->status, st);
  }
  pointset_free(zs, st);
  return rc;
}

extern "C" int kop_sync(kop_t op, void* stream) {
  if (!op) return fail(KOP_EINVAL, "kop_sync: NULL handle");
  cudaStream_t st = (cudaStream_t)stream;
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  int h = 0;
  KOP_CUDA_TRY(cudaMemcpy(&h, op->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != KOP_DEV_OK) {
    KOP_CUDA_TRY(cudaMemset(op->status, 0, sizeof(int)));
    if (h == KOP_DEV_TIMEOUT) return fail(KOP_ETIMEOUT, "a bounded device wait timed out");
    return fail(KOP_ECUDA, "device status " + std::to_string(h));
  }
  return KOP_OK;
}
