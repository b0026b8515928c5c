// nys_apply_noalloc: the preconditioner apply without any device allocation.
//
// nys_apply takes its scratch (the r x m projection U^T V, the per-column
// damping) from the stream-ordered allocator on every call.  Some callers must
// not allocate on this path: a latency-critical loop that cannot afford the
// device-wide synchronization cudaMalloc/cudaFree imply, or an application
// whose device memory is owned entirely by its own allocator.  This variant
// keeps its scratch in a fixed array in the library's device image instead.
//
// Properties of that array, for users of this entry point:
//  - it holds 16448 doubles (128.5 KB) on every GPU that
//    loads the library, until the process exits; r * m + m doubles of it are
//    used, which any Nystrom rank (r <= 2048) with m <= 8 columns fits;
//  - every call uses the same array and it keeps the last call's contents;
//    the accumulators are cleared on the stream at the start of each call;
//  - calls whose GPU work overlaps (different streams, or host threads
//    without ordering between them) race on the array;
//  - the first call on a device looks up the array's device address (with
//    that device current) and caches it; make that first call before any
//    stream capture.
#include <cmath>
#include <mutex>
#include <string>

#include "kop_dense.h"
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

// r * m projection coefficients (r <= 2048, m <= 8) plus m damping factors.
constexpr int kNoallocMaxCols = 8;
constexpr size_t kNoallocScratchDoubles = 2048 * kNoallocMaxCols + 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

struct NoallocMu {
  double mu[kNoallocMaxCols];
};

// w = W[k][c] (1 / (lam_k + mu_c) - 1 / rho_c), stored in W's own slot as the
// FP32 pair hi + lo (exact to 2^-48) that the float-float product U w reads;
// alpha[c] = 1 / rho_c.
__global__ void noalloc_scale_kernel(double* __restrict__ W, int r, int m, const double* __restrict__ lam,
                                     NoallocMu mu, int adaptive, double* __restrict__ alpha) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= r * m) return;
  const int k = t / m, c = t - k * m;
  const double rho = adaptive ? lam[r - 1] + mu.mu[c] : mu.mu[c];
  const double w = W[t] * (1.0 / (lam[k] + mu.mu[c]) - 1.0 / rho);
  const float hi = (float)w;
  reinterpret_cast<float2*>(W)[t] = make_float2(hi, (float)(w - (double)hi));
  if (k == 0) alpha[c] = 1.0 / rho;
}

// Device address of the scratch array, looked up once per device.
static int noalloc_scratch(double** out) {
  static std::mutex mu;
  static double* ptrs[64] = {nullptr};
  int dev = 0;
  KOP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KOP_ECUDA, "nys_apply_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "nys_apply_noalloc: cudaGetSymbolAddress");
    ptrs[dev] = (double*)p;
  }
  *out = ptrs[dev];
  return KOP_OK;
}

}  // namespace kop

using namespace kop;

extern "C" int nys_apply_noalloc(nys_t ny, const double* mu, int32_t adaptive, const float* V, int32_t m, float* O,
                                 void* stream) {
  if (!ny || !mu || !V || !O) return fail(KOP_EINVAL, "nys_apply_noalloc: NULL argument");
  if (m < 1 || m > kNoallocMaxCols) return fail(KOP_EINVAL, "nys_apply_noalloc: m must be in [1, 8]");
  const size_t need = (size_t)ny->r * m + m;
  if (need > kNoallocScratchDoubles)
    return fail(KOP_EINVAL, "nys_apply_noalloc: r * m + m = " + std::to_string(need) +
                                " exceeds the fixed scratch of " + std::to_string(kNoallocScratchDoubles) + " doubles");
  NoallocMu mus;
  for (int c = 0; c < kNoallocMaxCols; ++c) mus.mu[c] = 0.0;
  // mu = 0 needs lam_hat_r > 0 (adaptive): otherwise 1 / (lam_k + mu) divides by zero
  const bool zero_ok = adaptive && ny->lam_host[ny->r - 1] > 0.0;
  for (int c = 0; c < m; ++c) {
    if (!(mu[c] >= 0.0) || !std::isfinite(mu[c]) || (!zero_ok && !(mu[c] > 0.0)))
      return fail(KOP_EINVAL,
                  "nys_apply_noalloc: mu must be finite and > 0 (mu = 0 only when adaptive with lam_hat_r > 0)");
    mus.mu[c] = mu[c];
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int r = ny->r;
  double* W = scratch;                 // r x m
  double* alpha = scratch + (size_t)r * m;  // m
  // the same float-float projections as nys_apply (error-free FP32 pairs)
  rc = utv_ff(ny->U, r, ny->n, r, V, m, W, st);  // clears W, then W = U^T V
  if (rc) return rc;
  noalloc_scale_kernel<<<(r * m + 255) / 256, 256, 0, st>>>(W, r, m, ny->lam_dev, mus, adaptive ? 1 : 0, alpha);
  KOP_LAUNCHED();
  return uw_ff(ny->U, r, ny->n, r, reinterpret_cast<const float2*>(W), V, m, alpha, O, st);
}
