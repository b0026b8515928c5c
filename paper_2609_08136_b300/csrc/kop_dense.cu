// Dense helpers of the Nystrom construction and the preconditioner apply:
// tall-skinny products over the n rows (FP32 data, FP64 accumulation) and
// the small r x r factorizations in FP64 (Cholesky, triangular solves, the
// symmetric eigen-decomposition by parallel cyclic Jacobi, sorting).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "kop_device.cuh"
#include "kop_dense.h"
#include "kop_internal.h"

namespace kop {

// ------------------------------------------------------------------ Gram
// C (p x p, FP64, row-major, ldc) = A^T A over rows [0, n) of A (n x p, lda),
// error-free: CTA tile 64 x 64 of C (tiles on and above the diagonal only;
// an off-diagonal tile is added to both halves), 256 threads with 4 x 4
// outputs each; rows are staged in shared memory 32 at a time, every product
// is taken exactly (p + e = a b, e by FMA) and summed error-free over 128 rows
// (TwoSum into a float-float pair), and those partials in FP64 (FP64 is slow
// on this part, so it runs once per 128 rows); CTAs along y split the rows
// and add their partial tiles atomically.  C is accurate to about FP64
// rounding.  The Nystrom core needs that for Y^T Y, whose small
// eigen-directions (down to ~1e-5 of the largest, squared condition) FP32
// sums would swamp; the other Gram blocks run on the tensor cores
// (kop_tcgemm.cu).
constexpr int GT = 64, GK = 32, GFLUSH = 4;  // FP64 flush every GFLUSH * GK rows

__global__ void __launch_bounds__(256) gram_sym_kernel(const float* __restrict__ A, int lda, int64_t n, int p,
                                                       int tp, double* __restrict__ C, int ldc,
                                                       int64_t rows_per_split) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Bs[GK][GT + 4];
  int ti = 0, idx = blockIdx.x;
  while (idx >= tp - ti) {
    idx -= tp - ti;
    ++ti;
  }
  const int tj = ti + idx;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int p0 = ti * GT, q0 = tj * GT;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r1 = r0 + rows_per_split < n ? r0 + rows_per_split : n;
  double acc[4][4];
  float part[4][4], perr[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = 0.0;
      part[i][j] = perr[i][j] = 0.0f;
    }
  int chunk = 0;
  for (int64_t k0 = r0; k0 < r1; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e / GT, c = e - kk * GT;
      const int64_t row = k0 + kk;
      As[kk][c] = (row < r1 && p0 + c < p) ? A[row * lda + p0 + c] : 0.0f;
      Bs[kk][c] = (row < r1 && q0 + c < p) ? A[row * lda + q0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float pr = a[i] * b[j];
          const float pe = fmaf(a[i], b[j], -pr);
          const float t = part[i][j] + pr;
          const float bb = t - part[i][j];
          perr[i][j] += ((part[i][j] - (t - bb)) + (pr - bb)) + pe;
          part[i][j] = t;
        }
    }
    if (++chunk == GFLUSH || k0 + GK >= r1) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] += (double)part[i][j] + (double)perr[i][j];
          part[i][j] = perr[i][j] = 0.0f;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pi = p0 + ty * 4 + i;
    if (pi >= p) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int qj = q0 + tx * 4 + j;
      if (qj >= p) continue;
      atomicAdd(&C[(int64_t)pi * ldc + qj], acc[i][j]);
      if (ti != tj) atomicAdd(&C[(int64_t)qj * ldc + pi], acc[i][j]);
    }
  }
}

int gram_sym(const float* A, int lda, int64_t n, int p, double* C, int ldc, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)p * ldc, st));
  if (n <= 0) return KOP_OK;
  const int tp = (p + GT - 1) / GT;
  const int tiles = tp * (tp + 1) / 2;
  int64_t splits = (2 * num_sms() + tiles - 1) / tiles;
  const int64_t max_splits = (n + 255) / 256;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  int64_t rps = (n + splits - 1) / splits;
  rps = ((rps + GK - 1) / GK) * GK;
  splits = (n + rps - 1) / rps;
  gram_sym_kernel<<<dim3((unsigned)tiles, (unsigned)splits), 256, 0, st>>>(A, lda, n, p, tp, C, ldc, rps);
  KOP_LAUNCHED();
  return KOP_OK;
}

// ------------------------------------------------------------------ single vector
// w (p, FP64, pre-zeroed) += U^T v over rows; U n x p (ldu), v n (stride ldv).
__global__ void __launch_bounds__(256) utv_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                  const float* __restrict__ v, int ldv, int64_t rows_per_block,
                                                  double* __restrict__ w) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    float s = 0.0f, e = 0.0f;
    for (int64_t i = r0; i < r1; i += 16) {
      float part = 0.0f;
      const int64_t iend = i + 16 < r1 ? i + 16 : r1;
      for (int64_t ii = i; ii < iend; ++ii) part = fmaf(U[ii * ldu + k], v[ii * ldv], part);
      two_sum_acc(s, e, part);
    }
    atomicAdd(&w[k], (double)s + (double)e);
  }
}

// o[i] = alpha[0] * v[i] + sum_k U[i][k] w[k]; one warp per row.
__global__ void __launch_bounds__(256) uw_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                 const float* __restrict__ w, const float* __restrict__ v, int ldv,
                                                 const float* __restrict__ alpha, float* __restrict__ o, int ldo) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float s = 0.0f;
  for (int k = lane; k < p; k += 32) s = fmaf(U[row * ldu + k], w[k], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) o[row * ldo] = fmaf(alpha[0], v[row * ldv], s);
}

int utv(const float* U, int ldu, int64_t n, int p, const float* v, int ldv, double* w, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(double) * p, st));
  int64_t blocks = 4 * num_sms();
  int64_t rpb = (n + blocks - 1) / blocks;
  if (rpb < 64) rpb = 64;
  blocks = (n + rpb - 1) / rpb;
  utv_kernel<<<(unsigned)blocks, 256, 0, st>>>(U, ldu, n, p, v, ldv, rpb, w);
  KOP_LAUNCHED();
  return KOP_OK;
}

int uw(const float* U, int ldu, int64_t n, int p, const float* w, const float* v, int ldv, const float* alpha,
       float* o, int ldo, cudaStream_t st) {
  const int64_t threads = n * 32;
  uw_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(U, ldu, n, p, w, v, ldv, alpha, o, ldo);
  KOP_LAUNCHED();
  return KOP_OK;
}

// ------------------------------------------------------------------ FP64 projections
// W (p x m, FP64, pre-zeroed) += U^T V for m <= 8 columns, products and sums in
// FP64.  Thread k owns column k of U; the rows of V are read as broadcasts.
__global__ void __launch_bounds__(256) utv64_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                    const float* __restrict__ V, int m, int64_t rows_per_block,
                                                    double* __restrict__ W) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
      const double u = (double)U[i * ldu + k];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < m) acc[c] = fma(u, (double)V[i * m + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < m) atomicAdd(&W[(int64_t)k * m + c], acc[c]);
  }
}

// O[i][c] = (float)(alpha[c] V[i][c] + sum_k U[i][k] W[k][c]) in FP64; one warp per row.
__global__ void __launch_bounds__(256) uw64_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                   const double* __restrict__ W, const float* __restrict__ V, int m,
                                                   const double* __restrict__ alpha, float* __restrict__ O) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) s[c] = 0.0;
  for (int k = lane; k < p; k += 32) {
    const double u = (double)U[row * ldu + k];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < m) s[c] = fma(u, W[(int64_t)k * m + c], s[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c >= m) break;
    double x = s[c];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) O[row * m + c] = (float)fma(alpha[c], (double)V[row * m + c], x);
  }
}

// Float-float variants of the two projections: products are split exactly
// (TwoProduct) and summed error-free (TwoSum) in FP32 pairs, which keeps the
// accuracy of FP64 accumulation (the inputs are FP32) at FP32 throughput;
// B300's CUDA-core FP64 rate is far below its FP32 rate.
KOP_DEV void ff_add_prod(float& s, float& e, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float t = s + p;
  const float bb = t - s;
  e += ((s - (t - bb)) + (p - bb)) + pe;
  s = t;
}

// W[k][c] += sum_i U[i][k] V[i][c] (m <= MB columns).  A CTA of 256 threads
// takes a block of rows and 512 columns (grid.y over the column chunks); each
// thread owns the columns k = k0 + tid + 256 j, j < 2, and sweeps its rows RU
// at a time with every load of the RU rows issued before the first update, so
// that enough of U is in flight to run at the HBM rate.  The block's sums go
// to W with FP64 atomics.
template <int MB>
__global__ void __launch_bounds__(256) utv_ff_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                     const float* __restrict__ V, int m, int64_t rows_per_block,
                                                     double* __restrict__ W) {
  constexpr int J = 2, RU = MB <= 2 ? 8 : 4;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  int k[J];
  bool act[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    k[j] = (int)blockIdx.y * 512 + (int)threadIdx.x + 256 * j;
    act[j] = k[j] < p;
  }
  float s[J][MB], e[J][MB];
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int c = 0; c < MB; ++c) s[j][c] = e[j][c] = 0.0f;
  int64_t i = r0;
  for (; i + RU <= r1; i += RU) {
    float u[RU][J], v[RU][MB];
#pragma unroll
    for (int q = 0; q < RU; ++q) {
#pragma unroll
      for (int j = 0; j < J; ++j) u[q][j] = act[j] ? U[(i + q) * ldu + k[j]] : 0.0f;
#pragma unroll
      for (int c = 0; c < MB; ++c) v[q][c] = c < m ? __ldg(V + (i + q) * m + c) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < RU; ++q)
#pragma unroll
      for (int j = 0; j < J; ++j)
#pragma unroll
        for (int c = 0; c < MB; ++c) ff_add_prod(s[j][c], e[j][c], u[q][j], v[q][c]);
  }
  for (; i < r1; ++i) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float u = act[j] ? U[i * ldu + k[j]] : 0.0f;
#pragma unroll
      for (int c = 0; c < MB; ++c) ff_add_prod(s[j][c], e[j][c], u, c < m ? __ldg(V + i * m + c) : 0.0f);
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int c = 0; c < MB; ++c)
      if (act[j] && c < m) atomicAdd(&W[(int64_t)k[j] * m + c], (double)s[j][c] + (double)e[j][c]);
}

// O[i][c] = alpha[c] V[i][c] + sum_k U[i][k] W[k][c]; W is given as pairs
// hi + lo of FP32 values (FP64 arithmetic is slow on this GPU, so the split is
// made once per W, not once per row), one warp per row.  General form, any p
// and m <= 8.
__global__ void __launch_bounds__(256) uw_ff_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                    const float2* __restrict__ W, const float* __restrict__ V, int m,
                                                    const double* __restrict__ alpha, float* __restrict__ O) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float s[8], e[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) s[c] = e[c] = 0.0f;
  for (int k = lane; k < p; k += 32) {
    const float u = U[row * ldu + k];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < m) {
        const float2 w = W[(int64_t)k * m + c];
        ff_add_prod(s[c], e[c], u, w.x);
        e[c] = fmaf(u, w.y, e[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c >= m) break;
    double x = (double)s[c] + (double)e[c];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) O[row * m + c] = (float)fma(alpha[c], (double)V[row * m + c], x);
  }
}

// (s, e) += (s2, e2) for float-float values (TwoSum on the leading parts).
KOP_DEV void ff_add_pair(float& s, float& e, float s2, float e2) {
  const float t = s + s2;
  const float bb = t - s;
  e += ((s - (t - bb)) + (s2 - bb)) + e2;
  s = t;
}

// The same product for p <= 512 and m <= MB <= 2, the shape of the PCG's
// apply: persistent warps, each holding its 16 W pairs per column in
// registers (lane owns k = lane + 32 t), take two rows per step with all 32
// loads of U issued first; the cross-lane sum and the alpha V term are
// float-float too, so no FP64 arithmetic runs per row.
template <int MB>
__global__ void __launch_bounds__(256) uw_ff_reg_kernel(const float* __restrict__ U, int ldu, int64_t n, int p,
                                                        const float2* __restrict__ W, const float* __restrict__ V,
                                                        int m, const double* __restrict__ alpha,
                                                        float* __restrict__ O) {
  constexpr int T = 16, RR = 2;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float2 w[T][MB];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int k = lane + 32 * t;
#pragma unroll
    for (int c = 0; c < MB; ++c) w[t][c] = (k < p && c < m) ? W[(int64_t)k * m + c] : make_float2(0.0f, 0.0f);
  }
  float ah[MB], al[MB];
#pragma unroll
  for (int c = 0; c < MB; ++c) {
    const double a = c < m ? alpha[c] : 0.0;
    ah[c] = (float)a;
    al[c] = (float)(a - (double)ah[c]);
  }
  for (int64_t row0 = warp * RR; row0 < n; row0 += nwarps * RR) {
    float u[RR][T];
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      const int64_t row = row0 + q;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int k = lane + 32 * t;
        u[q][t] = (row < n && k < p) ? U[row * ldu + k] : 0.0f;
      }
    }
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      const int64_t row = row0 + q;
#pragma unroll
      for (int c = 0; c < MB; ++c) {
        float s = 0.0f, e = 0.0f;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          ff_add_prod(s, e, u[q][t], w[t][c].x);
          e = fmaf(u[q][t], w[t][c].y, e);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
          const float e2 = __shfl_xor_sync(0xffffffffu, e, off);
          ff_add_pair(s, e, s2, e2);
        }
        if (lane == c && c < m && row < n) {
          const float v = V[row * m + c];
          const float pr = ah[c] * v;
          const float pe = fmaf(ah[c], v, -pr) + al[c] * v;
          ff_add_pair(s, e, pr, pe);
          O[row * m + c] = s + e;
        }
      }
    }
  }
}

// Resident 256-thread CTAs per SM of a kernel (queried once per instance).
template <typename Kern>
static int ctas_per_sm(Kern kern) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, 0) != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

template <int MB>
static void utv_ff_launch(const float* U, int ldu, int64_t n, int p, const float* V, int m, double* W,
                          cudaStream_t st) {
  static const int occ = ctas_per_sm(utv_ff_kernel<MB>);
  const int chunks = (p + 511) / 512;
  int64_t rblocks = ((int64_t)occ * num_sms() + chunks - 1) / chunks;
  int64_t rpb = (n + rblocks - 1) / rblocks;
  if (rpb < 16) rpb = 16;
  rblocks = (n + rpb - 1) / rpb;
  utv_ff_kernel<MB><<<dim3((unsigned)rblocks, (unsigned)chunks), 256, 0, st>>>(U, ldu, n, p, V, m, rpb, W);
}

int utv_ff(const float* U, int ldu, int64_t n, int p, const float* V, int m, double* W, cudaStream_t st) {
  if (m < 1 || m > 8) return fail(KOP_EINVAL, "utv_ff: m must be in [1, 8]");
  KOP_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)p * m, st));
  if (m == 1) utv_ff_launch<1>(U, ldu, n, p, V, m, W, st);
  else if (m == 2) utv_ff_launch<2>(U, ldu, n, p, V, m, W, st);
  else if (m <= 4) utv_ff_launch<4>(U, ldu, n, p, V, m, W, st);
  else utv_ff_launch<8>(U, ldu, n, p, V, m, W, st);
  KOP_LAUNCHED();
  return KOP_OK;
}

template <int MB>
static void uw_ff_reg_launch(const float* U, int ldu, int64_t n, int p, const float2* W, const float* V, int m,
                             const double* alpha, float* O, cudaStream_t st) {
  static const int occ = ctas_per_sm(uw_ff_reg_kernel<MB>);
  // one wave of persistent CTAs, but no more warps than row pairs
  int64_t blocks = (int64_t)occ * num_sms();
  const int64_t need = (n + 15) / 16;  // 8 warps x 2 rows per CTA
  if (blocks > need) blocks = need;
  uw_ff_reg_kernel<MB><<<(unsigned)blocks, 256, 0, st>>>(U, ldu, n, p, W, V, m, alpha, O);
}

int uw_ff(const float* U, int ldu, int64_t n, int p, const float2* W, const float* V, int m, const double* alpha,
          float* O, cudaStream_t st) {
  if (m < 1 || m > 8) return fail(KOP_EINVAL, "uw_ff: m must be in [1, 8]");
  if (p <= 512 && m == 1) {
    uw_ff_reg_launch<1>(U, ldu, n, p, W, V, m, alpha, O, st);
  } else if (p <= 512 && m == 2) {
    uw_ff_reg_launch<2>(U, ldu, n, p, W, V, m, alpha, O, st);
  } else {
    const int64_t threads = n * 32;
    uw_ff_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(U, ldu, n, p, W, V, m, alpha, O);
  }
  KOP_LAUNCHED();
  return KOP_OK;
}

int utv64(const float* U, int ldu, int64_t n, int p, const float* V, int m, double* W, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)p * m, st));
  int64_t blocks = 4 * num_sms();
  int64_t rpb = (n + blocks - 1) / blocks;
  if (rpb < 64) rpb = 64;
  blocks = (n + rpb - 1) / rpb;
  utv64_kernel<<<(unsigned)blocks, 256, 0, st>>>(U, ldu, n, p, V, m, rpb, W);
  KOP_LAUNCHED();
  return KOP_OK;
}

int uw64(const float* U, int ldu, int64_t n, int p, const double* W, const float* V, int m, const double* alpha,
         float* O, cudaStream_t st) {
  const int64_t threads = n * 32;
  uw64_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(U, ldu, n, p, W, V, m, alpha, O);
  KOP_LAUNCHED();
  return KOP_OK;
}

// ------------------------------------------------------------------ r x r FP64
// Element-wise combinations of the r x r Gram blocks.
//   mode 0: M = (Goy + Goy^T)/2 + nu Goo
//   mode 1: M = Gyy + nu (Goy + Goy^T) + nu^2 Goo
__global__ void combine_kernel(const double* __restrict__ Goo, const double* __restrict__ Goy,
                               const double* __restrict__ Gyy, int r, double nu, int mode, double* __restrict__ M) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)r * r) return;
  const int i = (int)(idx / r), j = (int)(idx - (int64_t)i * r);
  const double s = Goy[(int64_t)i * r + j] + Goy[(int64_t)j * r + i];
  if (mode == 0)
    M[idx] = 0.5 * s + nu * Goo[idx];
  else
    M[idx] = Gyy[idx] + nu * s + nu * nu * Goo[idx];
}

int combine(const double* Goo, const double* Goy, const double* Gyy, int r, double nu, int mode, double* M,
            cudaStream_t st) {
  const int64_t tot = (int64_t)r * r;
  combine_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Goo, Goy, Gyy, r, nu, mode, M);
  KOP_LAUNCHED();
  return KOP_OK;
}

// In-place lower Cholesky A = L L^T (row-major r x r; the strict upper part is
// zeroed), blocked by CH_NB columns: per block column k0, (1) one CTA factors
// the CH_NB x CH_NB diagonal block in shared memory, (2) the rows below solve
// x L_kk^T = a (one thread per row), (3) the trailing lower triangle takes the
// rank-CH_NB update on 32 x 32 tiles.  info[0] = 0 on success, k + 1 if pivot
// k is not positive (or not finite); the later kernels then return at once.
constexpr int CH_NB = 64;

__global__ void __launch_bounds__(1024) chol_diag_kernel(double* A, int r, int k0, int nb, int* info) {
  __shared__ double D[CH_NB][CH_NB + 1];
  __shared__ int bad;
  if (*(volatile int*)info) return;  // uniform: every thread reads the same word
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    D[i][j] = A[(int64_t)(k0 + i) * r + k0 + j];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const double akk = D[k][k];
      if (!(akk > 0.0) || !isfinite(akk)) bad = k0 + k + 1;
      else D[k][k] = sqrt(akk);
    }
    __syncthreads();
    if (bad) break;
    for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) D[i][k] /= D[k][k];
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
      const int i = t / nb, j = t - i * nb;
      if (j > k && j <= i) D[i][j] -= D[i][k] * D[j][k];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    if (j <= i) A[(int64_t)(k0 + i) * r + k0 + j] = D[i][j];
  }
  if (threadIdx.x == 0 && bad) *info = bad;
}

__global__ void __launch_bounds__(128) chol_panel_kernel(double* A, int r, int k0, int nb, const int* info) {
  __shared__ double L[CH_NB][CH_NB + 1];
  if (*(volatile const int*)info) return;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    L[i][j] = j <= i ? A[(int64_t)(k0 + i) * r + k0 + j] : 0.0;
  }
  __syncthreads();
  const int row = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= r) return;
  double* a = A + (int64_t)row * r + k0;
  double x[CH_NB];
#pragma unroll
  for (int j = 0; j < CH_NB; ++j)
    if (j < nb) x[j] = a[j];
#pragma unroll
  for (int j = 0; j < CH_NB; ++j) {
    if (j < nb) {
      double s = x[j];
#pragma unroll
      for (int t = 0; t < j; ++t) s -= L[j][t] * x[t];
      x[j] = s / L[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < CH_NB; ++j)
    if (j < nb) a[j] = x[j];
}

// trailing update of the lower triangle rows / columns [k1, r), k1 = k0 + nb:
// A[i][j] -= sum_t A[i][k0 + t] A[j][k0 + t]; one CTA per 32 x 32 tile with
// ti >= tj, 256 threads with 4 outputs each
__global__ void __launch_bounds__(256) chol_update_kernel(double* A, int r, int k0, int nb, int tiles,
                                                          const int* info) {
  __shared__ double Pi[32][CH_NB + 1];
  __shared__ double Pj[32][CH_NB + 1];
  if (*(volatile const int*)info) return;
  int ti = 0, idx = blockIdx.x;
  while (idx > ti) {  // tile (ti, tj), tj <= ti, row-major over the lower triangle
    idx -= ti + 1;
    ++ti;
  }
  const int tj = idx;
  const int k1 = k0 + nb;
  const int i0 = k1 + 32 * ti, j0 = k1 + 32 * tj;
  for (int t = threadIdx.x; t < 32 * nb; t += blockDim.x) {
    const int rr = t / nb, c = t - rr * nb;
    Pi[rr][c] = i0 + rr < r ? A[(int64_t)(i0 + rr) * r + k0 + c] : 0.0;
    Pj[rr][c] = j0 + rr < r ? A[(int64_t)(j0 + rr) * r + k0 + c] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;  // rows ty, cols tx + 8 q
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < nb; ++c) {
    const double ai = Pi[ty][c];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(ai, Pj[tx + 8 * q][c], acc[q]);
  }
  const int i = i0 + ty;
  if (i >= r) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + tx + 8 * q;
    if (j < r && j <= i) A[(int64_t)i * r + j] -= acc[q];
  }
}

__global__ void zero_upper_kernel(double* A, int r) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * r) return;
  const int i = (int)(t / r), j = (int)(t - (int64_t)i * r);
  if (j > i) A[t] = 0.0;
}

int cholesky(double* A, int r, int* info, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
  for (int k0 = 0; k0 < r; k0 += CH_NB) {
    const int nb = r - k0 < CH_NB ? r - k0 : CH_NB;
    chol_diag_kernel<<<1, 1024, 0, st>>>(A, r, k0, nb, info);
    KOP_LAUNCHED();
    const int rest = r - k0 - nb;
    if (rest <= 0) break;
    chol_panel_kernel<<<(unsigned)((rest + 127) / 128), 128, 0, st>>>(A, r, k0, nb, info);
    KOP_LAUNCHED();
    const int tr = (rest + 31) / 32;
    const int tiles = tr * (tr + 1) / 2;
    chol_update_kernel<<<(unsigned)tiles, 256, 0, st>>>(A, r, k0, nb, tiles, info);
    KOP_LAUNCHED();
  }
  const int64_t tot = (int64_t)r * r;
  zero_upper_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, r);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Triangular solves with r x r L (lower, row-major) and q right-hand sides
// stored as COLUMNS of B (r x q, row-major, ldb); the solution overwrites B.
//   trans = 0: L X = B   (forward)
//   trans = 1: L^T X = B (backward)
// One warp per right-hand side column.
__global__ void __launch_bounds__(256) trsm_kernel(const double* __restrict__ L, int r, double* B, int ldb, int q,
                                                   int trans) {
  const int col = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= q) return;
  if (!trans) {
    for (int i = 0; i < r; ++i) {
      double s = 0.0;
      for (int k = lane; k < i; k += 32) s += L[(int64_t)i * r + k] * B[(int64_t)k * ldb + col];
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) B[(int64_t)i * ldb + col] = (B[(int64_t)i * ldb + col] - s) / L[(int64_t)i * r + i];
      __syncwarp();
    }
  } else {
    for (int i = r - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k < r; k += 32) s += L[(int64_t)k * r + i] * B[(int64_t)k * ldb + col];
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) B[(int64_t)i * ldb + col] = (B[(int64_t)i * ldb + col] - s) / L[(int64_t)i * r + i];
      __syncwarp();
    }
  }
}

int trsm(const double* L, int r, double* B, int ldb, int q, int trans, cudaStream_t st) {
  const int64_t threads = (int64_t)q * 32;
  trsm_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(L, r, B, ldb, q, trans);
  KOP_LAUNCHED();
  return KOP_OK;
}

// B = A^T (r x r) and optionally symmetrize: S = (A + A^T) / 2.
__global__ void transpose_kernel(const double* __restrict__ A, int r, double* __restrict__ B, int sym) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * r) return;
  const int i = (int)(t / r), j = (int)(t - (int64_t)i * r);
  B[t] = sym ? 0.5 * (A[t] + A[(int64_t)j * r + i]) : A[(int64_t)j * r + i];
}

int transpose(const double* A, int r, double* B, int sym, cudaStream_t st) {
  const int64_t tot = (int64_t)r * r;
  transpose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, r, B, sym);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Largest eigenvalue of a symmetric psd r x r matrix by power iteration (one
// CTA, FP64).  Thread i forms w_i = sum_k G[k][i] v_k (G is symmetric, so the
// reads along i are coalesced); G is staged in shared memory when it fits.
// out[0] = the Rayleigh quotient after `iters` steps, or once it changes by
// less than 1e-10 of itself between steps.
__global__ void __launch_bounds__(1024) power_kernel(const double* __restrict__ G, int r, int iters, int cached,
                                                     double* out) {
  extern __shared__ double pv[];  // v (r), w (r), [G (r x r)]
  double* v = pv;
  double* w = pv + r;
  const double* M = G;
  if (cached) {
    double* Gs = pv + 2 * r;
    for (int64_t t = threadIdx.x; t < (int64_t)r * r; t += blockDim.x) Gs[t] = G[t];
    M = Gs;
  }
  __shared__ double red[3][32];
  __shared__ double tot[3];
  for (int i = threadIdx.x; i < r; i += blockDim.x) v[i] = 1.0 + 0.01 * (double)(i % 7);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < r; ++k) s = fma(M[(int64_t)k * r + i], v[k], s);
      w[i] = s;
    }
    __syncthreads();
    // lam = v.w / v.v ; v = w / |w|
    double vals[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      vals[0] += v[i] * w[i];
      vals[1] += v[i] * v[i];
      vals[2] += w[i] * w[i];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      for (int off = 16; off > 0; off >>= 1) vals[c] += __shfl_xor_sync(0xffffffffu, vals[c], off);
      if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = vals[c];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double y = threadIdx.x < (blockDim.x >> 5) ? red[c][threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
        if (threadIdx.x == 0) tot[c] = y;
      }
    }
    __syncthreads();
    const double prev = lam;
    lam = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
    const double inv = tot[2] > 0.0 ? 1.0 / sqrt(tot[2]) : 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) v[i] = w[i] * inv;
    __syncthreads();
    if (it > 0 && fabs(lam - prev) <= 1e-10 * fabs(lam)) break;  // uniform: every thread reads tot
  }
  if (threadIdx.x == 0) out[0] = lam;
}

int power_max_eig(const double* G, int r, int iters, double* out, cudaStream_t st) {
  // dynamic shared memory: at most the per-CTA limit less the kernel's
  // static reduction arrays
  const size_t dyn_limit = smem_limit_bytes() - 1024;
  const size_t base = sizeof(double) * 2 * r;
  const bool cached = base + sizeof(double) * (size_t)r * r <= dyn_limit;
  const size_t smem = cached ? base + sizeof(double) * (size_t)r * r : base;
  static bool attr = false;
  if (!attr) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(power_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_limit));
    attr = true;
  }
  power_kernel<<<1, 1024, smem, st>>>(G, r, iters, cached ? 1 : 0, out);
  KOP_LAUNCHED();
  return KOP_OK;
}

// ------------------------------------------------------------------ Jacobi
// Symmetric eigen-decomposition A = V diag(w) V^T by cyclic Jacobi with the
// round-robin (tournament) ordering, so that all re/2 rotations of one step
// touch disjoint index pairs and are applied at once:
//   B = J^T A J,   V <- V J,
// where column i of J has a_i at row i and b_i at row partner(i).  For a pair
// (p, q) the rotation zeroing A_pq is the one of Golub & Van Loan
// (symmetric Schur decomposition): tau = (A_qq - A_pp) / (2 A_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c;
// column p of J is (c at p, -s at q), column q is (s at p, c at q).
// The matrix is padded to an even size re with a zero row/column that is
// never rotated.  One cooperative launch; steps are separated by a bounded
// grid barrier.  Sweeps stop when the off-diagonal Frobenius norm falls below
// tol times the norm of the diagonal, or after max_sweeps.
struct JacobiArgs {
  double* A;  // re x re, current
  double* B;  // re x re, next
  double* V;  // re x re
  double* V2;
  int re;
  int max_sweeps;
  double tol;
  double* offsum;  // per sweep: [2 * s] = off^2, [2 * s + 1] = diag^2
  unsigned int* bar_count;
  unsigned int* bar_gen;
  int* status;
  int* sweeps_done;
};

KOP_DEV int rr_partner_pos(int pos, int re) { return re - 1 - pos; }

// Index sitting at position `pos` of the tournament table in step s:
// position 0 holds index 0; positions 1..re-1 hold (pos - 1 + s) mod (re - 1) + 1.
KOP_DEV int rr_index(int pos, int s, int re) { return pos == 0 ? 0 : ((pos - 1 + s) % (re - 1)) + 1; }

KOP_DEV bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int nblocks, int* status) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = gen;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (*vgen == g) {
        if (globaltimer_ns() - t0 > KOP_WAIT_LIMIT_NS) {
          ok = 0;
          atomicExch(status, KOP_DEV_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Block shape: every CTA recomputes the step's rotations (FP64 square roots
// and divisions, slow on this part), so large matrices run one CTA of 512
// threads per SM; small ones two of 256 (measured: r = 500 223 vs 240 ms per
// build, r = 100 7.1 vs 7.8 ms).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) jacobi_kernel(JacobiArgs a) {
  extern __shared__ double js[];
  double* ca = js;            // re: a_i
  double* cb = js + a.re;     // re: b_i
  int* partner = (int*)(js + 2 * a.re);
  __shared__ double red[2][THREADS / 32];
  const int re = a.re;
  const unsigned int nblocks = gridDim.x;
  const int64_t tot = (int64_t)re * re;
  double* A = a.A;
  double* B = a.B;
  double* V = a.V;
  double* V2 = a.V2;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    for (int step = 0; step < re - 1; ++step) {
      // every CTA computes all rotations of this step from the current A
      for (int pos = threadIdx.x; pos < re / 2; pos += blockDim.x) {
        int p = rr_index(pos, step, re), q = rr_index(rr_partner_pos(pos, re), step, re);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const double app = __ldcg(&A[(int64_t)p * re + p]);
        const double aqq = __ldcg(&A[(int64_t)q * re + q]);
        const double apq = __ldcg(&A[(int64_t)p * re + q]);
        double c = 1.0, s = 0.0;
        if (apq != 0.0 && fabs(apq) > 1e-300) {
          const double tau = (aqq - app) / (2.0 * apq);
          double t;
          if (fabs(tau) > 1e150)
            t = 0.5 / tau;
          else
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        ca[p] = c;
        cb[p] = -s;
        partner[p] = q;
        ca[q] = c;
        cb[q] = s;
        partner[q] = p;
      }
      __syncthreads();
      const bool last = step == re - 2;
      double off = 0.0, dia = 0.0;
      for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)nblocks * blockDim.x) {
        const int i = (int)(t / re), j = (int)(t - (int64_t)i * re);
        const int pi = partner[i], pj = partner[j];
        const double ai = ca[i], bi = cb[i], aj = ca[j], bj = cb[j];
        double v = ai * aj * __ldcg(&A[t]) + ai * bj * __ldcg(&A[(int64_t)i * re + pj]) +
                   bi * aj * __ldcg(&A[(int64_t)pi * re + j]) + bi * bj * __ldcg(&A[(int64_t)pi * re + pj]);
        if (j == pi) v = 0.0;  // the rotated pair's off-diagonal entry is zero by construction
        B[t] = v;
        V2[t] = aj * __ldcg(&V[t]) + bj * __ldcg(&V[(int64_t)i * re + pj]);
        if (last) {
          if (i == j)
            dia += v * v;
          else
            off += v * v;
        }
      }
      if (last) {
        for (int o = 16; o > 0; o >>= 1) {
          off += __shfl_xor_sync(0xffffffffu, off, o);
          dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((threadIdx.x & 31) == 0) {
          red[0][threadIdx.x >> 5] = off;
          red[1][threadIdx.x >> 5] = dia;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double so = 0.0, sd = 0.0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            so += red[0][w];
            sd += red[1][w];
          }
          atomicAdd(&a.offsum[2 * sweep], so);
          atomicAdd(&a.offsum[2 * sweep + 1], sd);
        }
      }
      double* tA = A;
      A = B;
      B = tA;
      double* tV = V;
      V = V2;
      V2 = tV;
      if (!grid_barrier(a.bar_count, a.bar_gen, nblocks, a.status)) return;
    }
    const double so = __ldcg(&a.offsum[2 * sweep]), sd = __ldcg(&a.offsum[2 * sweep + 1]);
    if (so <= a.tol * a.tol * sd) {
      ++sweep;
      break;
    }
  }
  // results must end in a.A / a.V: copy if the last step left them in the other buffers
  if (A != a.A) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)nblocks * blockDim.x) {
      a.A[t] = __ldcg(&A[t]);
      a.V[t] = __ldcg(&V[t]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sweeps_done = sweep;
}

// Copy r x r into the padded re x re buffer, identity into V.
__global__ void jacobi_init_kernel(const double* __restrict__ H, int r, int re, double* A, double* V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)re * re) return;
  const int i = (int)(t / re), j = (int)(t - (int64_t)i * re);
  A[t] = (i < r && j < r) ? H[(int64_t)i * r + j] : 0.0;
  V[t] = i == j ? 1.0 : 0.0;
}

int sym_eig(const double* H, int r, double* work, int* status, double* evals_out, double* evecs_out,
            cudaStream_t st) {
  // work layout: A, B, V, V2 (re^2 each) + offsum (2 * 64) + barrier words + sweeps
  const int re = r + (r & 1);
  const size_t rr = (size_t)re * re;
  double* A = work;
  double* B = A + rr;
  double* V = B + rr;
  double* V2 = V + rr;
  double* offsum = V2 + rr;
  unsigned int* bar = (unsigned int*)(offsum + 128);
  int* sweeps = (int*)(bar + 2);
  KOP_CUDA_TRY(cudaMemsetAsync(offsum, 0, sizeof(double) * 128 + 16, st));
  jacobi_init_kernel<<<(unsigned)((rr + 255) / 256), 256, 0, st>>>(H, r, re, A, V);
  KOP_LAUNCHED();
  JacobiArgs a;
  a.A = A;
  a.B = B;
  a.V = V;
  a.V2 = V2;
  a.re = re;
  a.max_sweeps = 40;
  a.tol = 1e-13;
  a.offsum = offsum;
  a.bar_count = bar;
  a.bar_gen = bar + 1;
  a.status = status;
  a.sweeps_done = sweeps;
  const size_t smem = sizeof(double) * 2 * re + sizeof(int) * re;
  const bool big = re >= 256;
  const void* fn = big ? (const void*)jacobi_kernel<512> : (const void*)jacobi_kernel<256>;
  const int threads = big ? 512 : 256, per_sm_max = big ? 1 : 2;
  if (smem > 48 * 1024) KOP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  KOP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  if (per_sm < 1) return fail(KOP_ECUDA, "jacobi: kernel does not fit on an SM");
  int blocks = num_sms() * (per_sm < per_sm_max ? per_sm : per_sm_max);
  const int64_t want = (int64_t)((rr + threads - 1) / threads);
  if (want < blocks) blocks = (int)want;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  KOP_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, smem, st));
  note_launch();
  // unpad: eigenvalues = diag(A)[0..r), eigenvectors = V[0..r, 0..r)
  extract_eig(A, V, r, re, evals_out, evecs_out, st);
  return KOP_OK;
}

__global__ void extract_kernel(const double* __restrict__ A, const double* __restrict__ V, int r, int re,
                               double* __restrict__ w, double* __restrict__ E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < r) w[t] = A[t * re + t];
  if (t < (int64_t)r * r) {
    const int i = (int)(t / r), j = (int)(t - (int64_t)i * r);
    E[t] = V[(int64_t)i * re + j];
  }
}

void extract_eig(const double* A, const double* V, int r, int re, double* w, double* E, cudaStream_t st) {
  const int64_t tot = (int64_t)r * r;
  extract_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, V, r, re, w, E);
  note_launch();
}

// Descending order: perm[k] = index of the k-th largest eigenvalue (ties by index).
__global__ void sort_desc_kernel(const double* __restrict__ w, int r, int* __restrict__ perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) {
    const double wi = w[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const double wj = w[j];
      rank += (wj > wi) || (wj == wi && j < i);
    }
    perm[rank] = i;
  }
}

int sort_desc(const double* w, int r, int* perm, cudaStream_t st) {
  sort_desc_kernel<<<(r + 255) / 256, 256, 0, st>>>(w, r, perm);
  KOP_LAUNCHED();
  return KOP_OK;
}

// After sorting: lam[k] = max(0, w[perm[k]] - nu); Wm[:, k] = E[:, perm[k]] / sqrt(w[perm[k]]).
__global__ void nys_finish_kernel(const double* __restrict__ w, const double* __restrict__ E, const int* __restrict__ perm,
                                  int r, double nu, double* __restrict__ lam, double* __restrict__ Wm) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * r) return;
  const int i = (int)(t / r), k = (int)(t - (int64_t)i * r);
  const int src = perm[k];
  const double wk = w[src];
  const double sig = sqrt(wk > 1e-300 ? wk : 1e-300);
  Wm[t] = E[(int64_t)i * r + src] / sig;
  if (i == 0) lam[k] = wk - nu > 0.0 ? wk - nu : 0.0;
}

int nys_finish(const double* w, const double* E, const int* perm, int r, double nu, double* lam, double* Wm,
               cudaStream_t st) {
  const int64_t tot = (int64_t)r * r;
  nys_finish_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(w, E, perm, r, nu, lam, Wm);
  KOP_LAUNCHED();
  return KOP_OK;
}

__global__ void d2f_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

int d2f(const double* a, float* b, int64_t n, cudaStream_t st) {
  d2f_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Identity into an r x r FP64 matrix.
__global__ void eye_kernel(double* M, int r) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)r * r) M[t] = (t / r == t % r) ? 1.0 : 0.0;
}

int eye(double* M, int r, cudaStream_t st) {
  const int64_t tot = (int64_t)r * r;
  eye_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, r);
  KOP_LAUNCHED();
  return KOP_OK;
}

}  // namespace kop
