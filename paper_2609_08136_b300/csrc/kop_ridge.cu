// Normal operator A = X^T X of a data matrix X (n x p): the operator of ridge
// regression, (X^T X + lam I) w = X^T y (the paper's ridge experiments,
// Sec. 5.1, solve it by NysPCG).  A is never formed: A V = X^T (X V), two
// passes over X per product, HBM-bound for the PCG's few columns.
//
//   T = X V   one warp per row of X; lanes stride the p columns
//   O = X^T T CTAs take row blocks of X; each thread owns columns and sums its
//             rows, then adds its partial sums to FP64 accumulators atomically
// Three arithmetics: FP32 (fast), error-free float-float (exact FP32
// products by FMA, TwoSum sums, T carried as a hi + lo pair: the accurate,
// plain and check modes) and FP64 (the exact mode, FP64 vectors).
// Columns are processed 8 at a time.
#include <cmath>
#include <type_traits>

#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

constexpr int KR_MV = 8;

// TwoSum accumulate (s, e) += b.
KOP_DEV void ff_acc(float& s, float& e, float b) {
  const float t = s + b;
  const float bb = t - s;
  e += (s - (t - bb)) + (b - bb);
  s = t;
}

// T (n x mc, two arrays hi/lo for ACC = 1; FP64 for ACC = 2) = X V[:, c0:c0+mc]
template <int ACC, typename VT, typename TT>
__global__ void __launch_bounds__(256) ridge_xv_kernel(const float* __restrict__ X, int64_t n, int p,
                                                       const VT* __restrict__ V, int ldv, int c0, int mc,
                                                       TT* __restrict__ T, TT* __restrict__ Tlo) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* xr = X + row * p;
  if constexpr (ACC == 0) {
    float s[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = 0.0f;
    for (int k = lane; k < p; k += 32) {
      const float x = xr[k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) s[c] = fmaf(x, (float)V[(int64_t)k * ldv + c0 + c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) {
      float v = s[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && c < mc) T[row * mc + c] = v;
    }
  } else if constexpr (ACC == 1) {
    float s[KR_MV], e[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = e[c] = 0.0f;
    for (int k = lane; k < p; k += 32) {
      const float x = xr[k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) {
          const float v = (float)V[(int64_t)k * ldv + c0 + c];
          const float pr = x * v;
          e[c] += fmaf(x, v, -pr);
          ff_acc(s[c], e[c], pr);
        }
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) {
      // the pair sum across lanes in FP64 (a float-float value fits a double)
      double v = (double)s[c] + (double)e[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && c < mc) {
        const float hi = (float)v;
        T[row * mc + c] = hi;
        Tlo[row * mc + c] = (float)(v - (double)hi);
      }
    }
  } else {
    double s[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = 0.0;
    for (int k = lane; k < p; k += 32) {
      const double x = xr[k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) s[c] = fma(x, (double)V[(int64_t)k * ldv + c0 + c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) {
      double v = s[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && c < mc) T[row * mc + c] = (TT)v;
    }
  }
}

// Acc (p x mc, FP64, zeroed) += X^T T over the rows [r0, r1) of this CTA.
template <int ACC, typename TT>
__global__ void __launch_bounds__(256) ridge_xt_kernel(const float* __restrict__ X, int64_t n, int p,
                                                       const TT* __restrict__ T, const TT* __restrict__ Tlo, int mc,
                                                       int64_t rows_per_block, double* __restrict__ Acc) {
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p) return;
  if constexpr (ACC == 0) {
    float s[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = 0.0f;
    for (int64_t i = r0; i < r1; ++i) {
      const float x = X[i * p + k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) s[c] = fmaf(x, (float)T[i * mc + c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c)
      if (c < mc) atomicAdd(&Acc[(int64_t)k * mc + c], (double)s[c]);
  } else if constexpr (ACC == 1) {
    float s[KR_MV], e[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = e[c] = 0.0f;
    for (int64_t i = r0; i < r1; ++i) {
      const float x = X[i * p + k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) {
          const float th = (float)T[i * mc + c], tl = (float)Tlo[i * mc + c];
          const float pr = x * th;
          e[c] += fmaf(x, th, -pr) + x * tl;
          ff_acc(s[c], e[c], pr);
        }
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c)
      if (c < mc) atomicAdd(&Acc[(int64_t)k * mc + c], (double)s[c] + (double)e[c]);
  } else {
    double s[KR_MV];
#pragma unroll
    for (int c = 0; c < KR_MV; ++c) s[c] = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
      const double x = X[i * p + k];
#pragma unroll
      for (int c = 0; c < KR_MV; ++c)
        if (c < mc) s[c] = fma(x, (double)T[i * mc + c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < KR_MV; ++c)
      if (c < mc) atomicAdd(&Acc[(int64_t)k * mc + c], s[c]);
  }
}

// O[:, c0:c0+mc] (ld ldo) = Acc (p x mc)
template <typename OT>
__global__ void ridge_store_kernel(const double* __restrict__ Acc, int p, int mc, OT* __restrict__ O, int ldo,
                                   int c0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)p * mc) return;
  const int64_t k = t / mc;
  const int c = (int)(t - k * mc);
  O[k * ldo + c0 + c] = (OT)Acc[t];
}

template <int ACC, typename VT, typename OT>
static int ridge_apply_t(const kop_s* op, const VT* V, int m, int ldv, OT* O, int ldo, cudaStream_t st) {
  const int64_t n = op->rn;
  const int p = op->rp;
  using TT = typename std::conditional<ACC == 2, double, float>::type;
  DevBuf ws;
  ws.st = st;
  const size_t tbytes = sizeof(TT) * (size_t)n * KR_MV;
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, 2 * tbytes + sizeof(double) * (size_t)p * KR_MV, st));
  TT* T = (TT*)ws.p;
  TT* Tlo = (TT*)((char*)ws.p + tbytes);
  double* Acc = (double*)((char*)ws.p + 2 * tbytes);
  // row blocks of X^T T: about four CTAs per SM over the columns' blocks
  const int cblocks = (p + 255) / 256;
  int64_t rblocks = (4 * (int64_t)num_sms() + cblocks - 1) / cblocks;
  int64_t rpb = (n + rblocks - 1) / rblocks;
  if (rpb < 64) rpb = 64;
  rblocks = (n + rpb - 1) / rpb;
  for (int c0 = 0; c0 < m; c0 += KR_MV) {
    const int mc = m - c0 < KR_MV ? m - c0 : KR_MV;
    ridge_xv_kernel<ACC, VT, TT><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(op->rX, n, p, V, ldv, c0, mc, T,
                                                                                 Tlo);
    KOP_LAUNCHED();
    KOP_CUDA_TRY(cudaMemsetAsync(Acc, 0, sizeof(double) * (size_t)p * mc, st));
    ridge_xt_kernel<ACC, TT><<<dim3((unsigned)cblocks, (unsigned)rblocks), 256, 0, st>>>(op->rX, n, p, T, Tlo, mc,
                                                                                        rpb, Acc);
    KOP_LAUNCHED();
    ridge_store_kernel<OT><<<(unsigned)(((int64_t)p * mc + 255) / 256), 256, 0, st>>>(Acc, p, mc, O, ldo, c0);
    KOP_LAUNCHED();
  }
  return KOP_OK;
}

int ridge_apply(const kop_s* op, int mode, const float* V, int m, int ldv, float* O, int ldo, cudaStream_t st) {
  if (mode == KOP_FAST) return ridge_apply_t<0, float, float>(op, V, m, ldv, O, ldo, st);
  return ridge_apply_t<1, float, float>(op, V, m, ldv, O, ldo, st);
}

int ridge_apply_f64(const kop_s* op, const double* V, int m, int ldv, double* O, int ldo, cudaStream_t st) {
  return ridge_apply_t<2, double, double>(op, V, m, ldv, O, ldo, st);
}

}  // namespace kop

using namespace kop;

extern "C" int kop_create_ridge(const float* X, int64_t n, int32_t p, void* stream, kop_t* out) {
  if (!out) return fail(KOP_EINVAL, "kop_create_ridge: out is NULL");
  *out = nullptr;
  if (!X) return fail(KOP_EINVAL, "kop_create_ridge: X is NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(KOP_EINVAL, "kop_create_ridge: n must be in [1, 2^31)");
  if (p < 1 || p > 65536) return fail(KOP_EINVAL, "kop_create_ridge: p must be in [1, 65536]");
  cudaStream_t st = (cudaStream_t)stream;
  kop_s* op = new kop_s();
  op->ridge = 1;
  op->rn = n;
  op->rp = p;
  cudaError_t e = cudaMalloc(&op->status, 256);
  if (e == cudaSuccess) e = cudaMalloc(&op->rX, sizeof(float) * (size_t)n * p);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(op->rX, X, sizeof(float) * (size_t)n * p, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(op->rX);
    cudaFree(op->status);
    delete op;
    return cuda_fail(e, "kop_create_ridge");
  }
  *out = op;
  return KOP_OK;
}
