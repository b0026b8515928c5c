// Diagnostics: measured SFU (special-function unit) throughput.
//
// The m = 1 kernel product is bound by the SFU, not by the tensor cores or
// HBM: every kernel entry needs one exp2 (RBF) or one square root and one
// exp2 (Laplace, Matern).  The roofline of that product therefore needs the
// SFU rates of the GPU it runs on, which this measures: independent chains of
// ex2.approx, sqrt.approx and rsqrt.approx, many per thread, on every SM.
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

template <int OP>
__global__ void __launch_bounds__(512) sfu_probe_kernel(float* out, int iters) {
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if constexpr (OP == 0) v[i] = ex2_approx(v[i]) * -0.5f;
      else if constexpr (OP == 1) v[i] = sqrt_approx(v[i]) + 0.25f;
      else v[i] = rsqrt_approx(v[i]) + 0.25f;
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += v[i];
  if (s == 12345.0f) out[0] = s;  // keeps the chains live; practically never taken
}

}  // namespace kop

using namespace kop;

extern "C" int kop_sfu_rates(double* rates, void* stream) {
  if (!rates) return fail(KOP_EINVAL, "kop_sfu_rates: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  float* out = nullptr;
  KOP_CUDA_TRY(cudaMallocAsync((void**)&out, sizeof(float), st));
  const int iters = 2048, threads = 512, blocks = 4 * num_sms();
  cudaEvent_t e0, e1;
  KOP_CUDA_TRY(cudaEventCreate(&e0));
  KOP_CUDA_TRY(cudaEventCreate(&e1));
  int rc = KOP_OK;
  for (int op = 0; op < 3 && rc == KOP_OK; ++op) {
    float best = 0.0f;
    for (int rep = 0; rep < 4; ++rep) {  // the first pass warms up; the fastest of the others counts
      float ms = 0.0f;
      cudaEventRecord(e0, st);
      if (op == 0) sfu_probe_kernel<0><<<blocks, threads, 0, st>>>(out, iters);
      else if (op == 1) sfu_probe_kernel<1><<<blocks, threads, 0, st>>>(out, iters);
      else sfu_probe_kernel<2><<<blocks, threads, 0, st>>>(out, iters);
      note_launch();
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "kop_sfu_rates");
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1 || (rep > 1 && ms < best)) best = ms;
    }
    rates[op] = (double)blocks * threads * iters * 16 / (best * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  return rc;
}

extern "C" int kop_set_autotune(int32_t enable) {
  kop::set_mma_autotune(enable);
  return KOP_OK;
}

extern "C" int32_t kop_autotune_shapes(void) { return kop::mma_tuned_shapes(); }
