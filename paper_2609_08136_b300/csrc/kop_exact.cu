// FP64 CUDA-core kernel operator (KOP_EXACT): O = K(Q, X) V with FP64
// vectors, direct differences of the original FP32 points in FP64, the kernel
// function in FP64 and FP64 accumulation.
//
// This is the true-residual operator of the solver's iterative refinement:
// the paper checks the relative residual in float64 (App. B.2), and on badly
// conditioned systems FP32 rounding of the kernel values alone leaves a
// residual floor near 1e-6.  B300's FP64 rate makes this about two orders of
// magnitude slower than the fused product, so it is used for the periodic
// true residual, not for the inner iterations.  One thread per query row;
// tiles of 32 points and their V rows are staged in shared memory.  When the
// query rows alone cannot fill the GPU (the solver's sampled FP64 residual
// rows), the keys are split over the grid's second dimension and the partial
// sums are added with FP64 atomics.
#include <cmath>

#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

constexpr int K4_ROWS = 128;
constexpr int K4_KEYS = 32;

template <int KF>
KOP_DEV double exact_kernel_value(double d2, double bw) {
  if constexpr (KF == KF_RBF) {
    return exp(-d2 / (2.0 * bw * bw));
  } else if constexpr (KF == KF_LAPLACE) {
    return exp(-sqrt(d2) / bw);
  } else if constexpr (KF == KF_MATERN) {
    const double a = 2.23606797749978969640 * sqrt(d2) / bw;
    return (1.0 + a + a * a / 3.0) * exp(-a);
  } else if constexpr (KF == KF_DRBF) {
    return exp(-d2 / (2.0 * bw * bw)) * d2 / (bw * bw * bw);
  } else if constexpr (KF == KF_DLAPLACE) {
    const double r = sqrt(d2);
    return exp(-r / bw) * r / (bw * bw);
  } else if constexpr (KF == KF_GRBF) {
    return exp(-d2 / (2.0 * bw * bw)) / (bw * bw);
  } else if constexpr (KF == KF_GLAPLACE) {
    const double r = sqrt(d2);
    return r > 0.0 ? exp(-r / bw) / (bw * r) : 0.0;
  } else if constexpr (KF == KF_GMATERN) {
    const double a = 2.23606797749978969640 * sqrt(d2) / bw;
    return (5.0 / (3.0 * bw * bw)) * (1.0 + a) * exp(-a);
  } else {
    const double a = 2.23606797749978969640 * sqrt(d2) / bw;
    return exp(-a) * (a * a / 3.0) * (1.0 + a) / bw;
  }
}

template <int KF, int MV>
__global__ void __launch_bounds__(K4_ROWS) k4_exact_kernel(const float* __restrict__ Q, const float* __restrict__ Xk,
                                                           int d, const double* __restrict__ V, int ldv,
                                                           double* __restrict__ O, int ldo, int nq, int nk, int m,
                                                           double bw, int kchunk) {
  extern __shared__ double sd[];
  double* Qs = sd;                          // d x (K4_ROWS + 1), transposed
  double* Xs = Qs + d * (K4_ROWS + 1);      // K4_KEYS x d
  double* Vs = Xs + K4_KEYS * d;            // K4_KEYS x MV
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * K4_ROWS;
  for (int idx = tid; idx < K4_ROWS * d; idx += K4_ROWS) {
    const int r = idx / d, k = idx - r * d;
    Qs[k * (K4_ROWS + 1) + r] = (row0 + r < nq) ? (double)Q[(int64_t)(row0 + r) * d + k] : 0.0;
  }
  double acc[MV];
#pragma unroll
  for (int c = 0; c < MV; ++c) acc[c] = 0.0;
  // keys [kb, ke) of this CTA: all of them, or one chunk of a split grid
  const int kb = blockIdx.y * kchunk;
  const int ke = (nk - kb) < kchunk ? nk : kb + kchunk;
  for (int j0 = kb; j0 < ke; j0 += K4_KEYS) {
    __syncthreads();
    for (int idx = tid; idx < K4_KEYS * d; idx += K4_ROWS) {
      const int jj = idx / d;
      Xs[idx] = (j0 + jj < ke) ? (double)Xk[(int64_t)j0 * d + idx] : 0.0;
    }
    for (int idx = tid; idx < K4_KEYS * MV; idx += K4_ROWS) {
      const int jj = idx / MV, c = idx - jj * MV;
      Vs[idx] = (j0 + jj < ke && c < m) ? V[(int64_t)(j0 + jj) * ldv + c] : 0.0;
    }
    __syncthreads();
    const int jn = ke - j0 < K4_KEYS ? ke - j0 : K4_KEYS;
    for (int jj = 0; jj < jn; ++jj) {
      double d2 = 0.0;
      for (int k = 0; k < d; ++k) {
        const double t = Qs[k * (K4_ROWS + 1) + tid] - Xs[jj * d + k];
        d2 = fma(t, t, d2);
      }
      const double kv = exact_kernel_value<KF>(d2, bw);
#pragma unroll
      for (int c = 0; c < MV; ++c) acc[c] = fma(kv, Vs[jj * MV + c], acc[c]);
    }
  }
  const int gi = row0 + tid;
  if (gi < nq) {
#pragma unroll
    for (int c = 0; c < MV; ++c)
      if (c < m) {
        if (gridDim.y > 1)
          atomicAdd(O + (int64_t)gi * ldo + c, acc[c]);
        else
          O[(int64_t)gi * ldo + c] = acc[c];
      }
  }
}

// Key chunk of a split grid for nq query rows: about four CTAs per SM in
// all, chunks of whole 32-key tiles; nk (no split) when the row blocks alone
// fill the GPU.  A split grid accumulates into O, which must be zero.
static int exact_key_chunk(int64_t nq, int64_t nk) {
  const int64_t rb = (nq + K4_ROWS - 1) / K4_ROWS;
  const int64_t want = 4 * (int64_t)num_sms();
  if (rb >= want / 2 || nk <= 4 * K4_KEYS) return (int)nk;
  int64_t splits = (want + rb - 1) / rb;
  int64_t chunk = (nk + splits - 1) / splits;
  chunk = (chunk + K4_KEYS - 1) / K4_KEYS * K4_KEYS;
  return (int)chunk;
}

template <int KF, int MV>
static int launch_exact_t(const PointSet& Q, const PointSet& Ks, const double* V, int m, int ldv, double* O, int ldo,
                          double bw, cudaStream_t st) {
  auto kern = k4_exact_kernel<KF, MV>;
  const int d = Q.d;
  const size_t smem = sizeof(double) * ((size_t)d * (K4_ROWS + 1) + (size_t)K4_KEYS * d + K4_KEYS * MV);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  const int kchunk = exact_key_chunk(Q.n, Ks.n);
  dim3 grid((unsigned)((Q.n + K4_ROWS - 1) / K4_ROWS), (unsigned)((Ks.n + kchunk - 1) / kchunk));
  if (grid.y > 1) {
    // split keys: the CTAs add into O (column block of m <= MV columns)
    KOP_CUDA_TRY(cudaMemset2DAsync(O, sizeof(double) * ldo, 0, sizeof(double) * m, Q.n, st));
  }
  kern<<<grid, K4_ROWS, smem, st>>>(Q.xorig, Ks.xorig, d, V, ldv, O, ldo, (int)Q.n, (int)Ks.n, m, bw, kchunk);
  KOP_LAUNCHED();
  return KOP_OK;
}

template <int KF>
static int launch_exact_kf(const PointSet& Q, const PointSet& Ks, const double* V, int m, int ldv, double* O, int ldo,
                           double bw, cudaStream_t st) {
  for (int c0 = 0; c0 < m; c0 += 8) {
    const int mc = (m - c0) < 8 ? (m - c0) : 8;
    int rc;
    if (mc == 1)
      rc = launch_exact_t<KF, 1>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    else if (mc <= 2)
      rc = launch_exact_t<KF, 2>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    else
      rc = launch_exact_t<KF, 8>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    if (rc) return rc;
  }
  return KOP_OK;
}

int exact_matvec(const PointSet& Q, const PointSet& Ks, int kf, double bw, const double* V, int m, int ldv, double* O,
                 int ldo, cudaStream_t st) {
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  switch (kf) {
    case KF_RBF: return launch_exact_kf<KF_RBF>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_LAPLACE: return launch_exact_kf<KF_LAPLACE>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_MATERN: return launch_exact_kf<KF_MATERN>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_DRBF: return launch_exact_kf<KF_DRBF>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_DLAPLACE: return launch_exact_kf<KF_DLAPLACE>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_GRBF: return launch_exact_kf<KF_GRBF>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_GLAPLACE: return launch_exact_kf<KF_GLAPLACE>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_GMATERN: return launch_exact_kf<KF_GMATERN>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    default: return launch_exact_kf<KF_DMATERN>(Q, Ks, V, m, ldv, O, ldo, bw, st);
  }
}

// The same product for few query rows with the distances in error-free FP32
// arithmetic instead of FP64 (the solver's certification of a stop: the FP64
// residual of sampled rows).  The difference of two FP32 coordinates is kept
// exactly as a pair (TwoDiff), its square as a pair (TwoProduct), and the
// squares are summed with TwoSum into a hi / lo pair, so D2 = hi + lo carries
// about 2^-44 relative error; the kernel value and the contraction are FP64
// as in k4_exact_kernel.  B300 runs FP32 about 64 times faster than FP64, and
// the distance is most of the work.
KOP_DEV double ef_sqdist(const float* __restrict__ q, int qstride, const float* __restrict__ x, int d) {
  float hi = 0.0f, lo = 0.0f;
  for (int k = 0; k < d; ++k) {
    const float a = q[k * qstride], b = x[k];
    const float t = a - b;  // TwoDiff: t + te = a - b exactly
    const float bb = t - a;
    const float te = (a - (t - bb)) - (b + bb);
    const float p = t * t;  // TwoProduct: p + pe = t^2 exactly
    const float pe = fmaf(t, t, -p);
    const float c = fmaf(2.0f * t, te, te * te);  // 2 t te + te^2 (tiny)
    const float sum = hi + p;                      // TwoSum: sum + se = hi + p exactly
    const float bp = sum - hi;
    const float se = (hi - (sum - bp)) + (p - bp);
    hi = sum;
    lo += (se + pe) + c;
  }
  return (double)hi + (double)lo;
}

template <int KF, int MV>
__global__ void __launch_bounds__(K4_ROWS) k4_cert_kernel(const float* __restrict__ Q, const float* __restrict__ Xk,
                                                          int d, const double* __restrict__ V, int ldv,
                                                          double* __restrict__ O, int ldo, int nq, int nk, int m,
                                                          double bw, int kchunk) {
  extern __shared__ double sd[];
  double* Vs = sd;                              // K4_KEYS x MV
  float* Qs = (float*)(Vs + K4_KEYS * MV);      // d x (K4_ROWS + 1), transposed
  float* Xs = Qs + d * (K4_ROWS + 1);           // K4_KEYS x d
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * K4_ROWS;
  for (int idx = tid; idx < K4_ROWS * d; idx += K4_ROWS) {
    const int r = idx / d, k = idx - r * d;
    Qs[k * (K4_ROWS + 1) + r] = (row0 + r < nq) ? Q[(int64_t)(row0 + r) * d + k] : 0.0f;
  }
  double acc[MV];
#pragma unroll
  for (int c = 0; c < MV; ++c) acc[c] = 0.0;
  const int kb = blockIdx.y * kchunk;
  const int ke = (nk - kb) < kchunk ? nk : kb + kchunk;
  for (int j0 = kb; j0 < ke; j0 += K4_KEYS) {
    __syncthreads();
    for (int idx = tid; idx < K4_KEYS * d; idx += K4_ROWS) {
      const int jj = idx / d;
      Xs[idx] = (j0 + jj < ke) ? Xk[(int64_t)j0 * d + idx] : 0.0f;
    }
    for (int idx = tid; idx < K4_KEYS * MV; idx += K4_ROWS) {
      const int jj = idx / MV, c = idx - jj * MV;
      Vs[idx] = (j0 + jj < ke && c < m) ? V[(int64_t)(j0 + jj) * ldv + c] : 0.0;
    }
    __syncthreads();
    const int jn = ke - j0 < K4_KEYS ? ke - j0 : K4_KEYS;
    for (int jj = 0; jj < jn; ++jj) {
      const double d2 = ef_sqdist(Qs + tid, K4_ROWS + 1, Xs + jj * d, d);
      const double kv = exact_kernel_value<KF>(d2, bw);
#pragma unroll
      for (int c = 0; c < MV; ++c) acc[c] = fma(kv, Vs[jj * MV + c], acc[c]);
    }
  }
  const int gi = row0 + tid;
  if (gi < nq) {
#pragma unroll
    for (int c = 0; c < MV; ++c)
      if (c < m) {
        if (gridDim.y > 1)
          atomicAdd(O + (int64_t)gi * ldo + c, acc[c]);
        else
          O[(int64_t)gi * ldo + c] = acc[c];
      }
  }
}

template <int KF, int MV>
static int launch_cert_t(const PointSet& Q, const PointSet& Ks, const double* V, int m, int ldv, double* O, int ldo,
                         double bw, cudaStream_t st) {
  auto kern = k4_cert_kernel<KF, MV>;
  const int d = Q.d;
  const size_t smem = sizeof(double) * K4_KEYS * MV + sizeof(float) * ((size_t)d * (K4_ROWS + 1) + (size_t)K4_KEYS * d);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  const int kchunk = exact_key_chunk(Q.n, Ks.n);
  dim3 grid((unsigned)((Q.n + K4_ROWS - 1) / K4_ROWS), (unsigned)((Ks.n + kchunk - 1) / kchunk));
  if (grid.y > 1) KOP_CUDA_TRY(cudaMemset2DAsync(O, sizeof(double) * ldo, 0, sizeof(double) * m, Q.n, st));
  kern<<<grid, K4_ROWS, smem, st>>>(Q.xorig, Ks.xorig, d, V, ldv, O, ldo, (int)Q.n, (int)Ks.n, m, bw, kchunk);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Column groups of up to 32: the error-free distance (most of the FP32 work)
// is formed once per group.
template <int KF>
static int launch_cert_kf(const PointSet& Q, const PointSet& Ks, const double* V, int m, int ldv, double* O, int ldo,
                          double bw, cudaStream_t st) {
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int mc = (m - c0) < 32 ? (m - c0) : 32;
    int rc;
    if (mc == 1)
      rc = launch_cert_t<KF, 1>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    else if (mc <= 2)
      rc = launch_cert_t<KF, 2>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    else if (mc <= 8)
      rc = launch_cert_t<KF, 8>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    else
      rc = launch_cert_t<KF, 32>(Q, Ks, V + c0, mc, ldv, O + c0, ldo, bw, st);
    if (rc) return rc;
  }
  return KOP_OK;
}

int cert_matvec(const PointSet& Q, const PointSet& Ks, int kf, double bw, const double* V, int m, int ldv, double* O,
                int ldo, cudaStream_t st) {
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  switch (kf) {
    case KF_RBF: return launch_cert_kf<KF_RBF>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    case KF_LAPLACE: return launch_cert_kf<KF_LAPLACE>(Q, Ks, V, m, ldv, O, ldo, bw, st);
    default: return launch_cert_kf<KF_MATERN>(Q, Ks, V, m, ldv, O, ldo, bw, st);
  }
}

__global__ void f2d_kernel(const float* __restrict__ a, int ld, int m, int64_t n, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  const int64_t i = t / m;
  const int c = (int)(t - i * m);
  b[t] = (double)a[i * ld + c];
}

__global__ void d2f_out_kernel(const double* __restrict__ a, int m, int64_t n, float* __restrict__ b, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  const int64_t i = t / m;
  const int c = (int)(t - i * m);
  b[i * ld + c] = (float)a[t];
}

// FP32 in / FP32 out wrapper (the FP64 product is rounded once at the end).
int exact_matvec_f32(const PointSet& Q, const PointSet& Ks, int kf, double bw, const float* V, int m, int ldv,
                     float* O, int ldo, cudaStream_t st) {
  double* buf = nullptr;
  const size_t nv = (size_t)Ks.n * m, no = (size_t)Q.n * m;
  KOP_CUDA_TRY(cudaMallocAsync((void**)&buf, sizeof(double) * (nv + no), st));
  f2d_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(V, ldv, m, Ks.n, buf);
  KOP_LAUNCHED();
  int rc = exact_matvec(Q, Ks, kf, bw, buf, m, m, buf + nv, m, st);
  if (rc == KOP_OK) {
    d2f_out_kernel<<<(unsigned)((no + 255) / 256), 256, 0, st>>>(buf + nv, m, Q.n, O, ldo);
    KOP_LAUNCHED();
  }
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace kop
