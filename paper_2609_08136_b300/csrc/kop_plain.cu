// Plain FP32 CUDA-core kernel operator: the speed baseline of the fused path
// (same contract, no tensor cores).  Distances by direct differences of the
// centred FP32 points, k by expf/sqrtf, contraction by FP32 FMAs with a
// compensated running sum per output.  One thread per query row; key tiles of
// 32 points and their V rows are staged in shared memory and read as
// broadcasts.  The differences and squares run on packed pairs of features
// (two-lane FP32 instructions, each lane rounded as a scalar FP32 operation):
// even and odd features accumulate separately and are added at the end.  With COMP the contraction is error-free per entry (TwoProduct
// + TwoSum): the solver's acceptance check uses that form, because direct
// differences keep the kernel argument accurate where the norm identity of the
// tensor-core path loses digits (points far from the common centre).
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

constexpr int K2_ROWS = 128;
constexpr int K2_KEYS = 32;

// Two-lane FP32 arithmetic on a packed pair (lo, hi).
KOP_DEV uint64_t pk2(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
KOP_DEV float2 unpk2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
KOP_DEV uint64_t sub_f32x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
KOP_DEV uint64_t fma_f32x2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct PlainConst {
  float e0, e1, c2;
};

template <int KF>
KOP_DEV float plain_kernel_value(float d2, const PlainConst& p) {
  if constexpr (KF == KF_RBF) {
    return expf(d2 * p.e0);
  } else if constexpr (KF == KF_LAPLACE) {
    return expf(sqrtf(d2) * p.e0);
  } else if constexpr (KF == KF_MATERN) {
    const float a = sqrtf(d2) * p.e1;
    return (1.0f + a + a * a * (1.0f / 3.0f)) * expf(-a);
  } else if constexpr (KF == KF_DRBF) {
    return expf(d2 * p.e0) * d2 * p.c2;
  } else if constexpr (KF == KF_DLAPLACE) {
    const float r = sqrtf(d2);
    return expf(r * p.e0) * r * p.c2;
  } else {
    const float a = sqrtf(d2) * p.e1;
    return expf(-a) * (a * a * (1.0f / 3.0f)) * (1.0f + a) * p.c2;
  }
}

template <int KF, int MV, bool COMP>
__global__ void __launch_bounds__(K2_ROWS) k2_plain_kernel(const float* __restrict__ Q, const float* __restrict__ Xk,
                                                           const float* __restrict__ V, float* __restrict__ O, int nq,
                                                           int nk, int dp, int m, int ldv, int ldo, PlainConst pc) {
  extern __shared__ float sm[];
  float* Qs = sm;                              // dp x (K2_ROWS + 1), transposed
  float* Xs = Qs + dp * (K2_ROWS + 1);         // K2_KEYS x dp
  float* Vs = Xs + K2_KEYS * dp;               // K2_KEYS x MV
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * K2_ROWS;
  const int col0 = blockIdx.y * MV;
  const int mc = (m - col0) < MV ? (m - col0) : MV;
  for (int idx = tid; idx < K2_ROWS * dp; idx += K2_ROWS) {
    const int r = idx / dp, k = idx - r * dp;
    Qs[k * (K2_ROWS + 1) + r] = Q[(int64_t)(row0 + r) * dp + k];
  }
  float acc_s[MV], acc_e[MV];
#pragma unroll
  for (int c = 0; c < MV; ++c) acc_s[c] = acc_e[c] = 0.0f;
  for (int j0 = 0; j0 < nk; j0 += K2_KEYS) {
    __syncthreads();
    for (int idx = tid; idx < K2_KEYS * dp; idx += K2_ROWS) Xs[idx] = Xk[(int64_t)j0 * dp + idx];
    for (int idx = tid; idx < K2_KEYS * MV; idx += K2_ROWS) {
      const int jj = idx / MV, c = idx - jj * MV, j = j0 + jj;
      Vs[idx] = (j < nk && c < mc) ? V[(int64_t)j * ldv + col0 + c] : 0.0f;
    }
    __syncthreads();
    uint64_t d2p[K2_KEYS];  // (sum over even features, sum over odd features)
#pragma unroll
    for (int jj = 0; jj < K2_KEYS; ++jj) d2p[jj] = 0ull;
    for (int k0 = 0; k0 < dp; k0 += 16) {
      uint64_t q2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        q2[i] = pk2(Qs[(k0 + 2 * i) * (K2_ROWS + 1) + tid], Qs[(k0 + 2 * i + 1) * (K2_ROWS + 1) + tid]);
#pragma unroll
      for (int jj = 0; jj < K2_KEYS; ++jj) {
        const float4* xr = reinterpret_cast<const float4*>(Xs + jj * dp + k0);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 x4 = xr[k4];
          uint64_t t = sub_f32x2(q2[2 * k4], pk2(x4.x, x4.y));
          d2p[jj] = fma_f32x2(t, t, d2p[jj]);
          t = sub_f32x2(q2[2 * k4 + 1], pk2(x4.z, x4.w));
          d2p[jj] = fma_f32x2(t, t, d2p[jj]);
        }
      }
    }
    float d2[K2_KEYS];
#pragma unroll
    for (int jj = 0; jj < K2_KEYS; ++jj) {
      const float2 h = unpk2(d2p[jj]);
      d2[jj] = h.x + h.y;
    }
    float part[MV], perr[MV];
#pragma unroll
    for (int c = 0; c < MV; ++c) part[c] = perr[c] = 0.0f;
#pragma unroll
    for (int jj = 0; jj < K2_KEYS; ++jj) {
      const float kv = plain_kernel_value<KF>(d2[jj], pc);
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        const float v = Vs[jj * MV + c];
        if constexpr (COMP) {
          const float p = kv * v;
          const float pe = fmaf(kv, v, -p);
          const float t = part[c] + p;
          const float bb = t - part[c];
          perr[c] += ((part[c] - (t - bb)) + (p - bb)) + pe;
          part[c] = t;
        } else {
          part[c] = fmaf(kv, v, part[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < MV; ++c) {
      two_sum_acc(acc_s[c], acc_e[c], part[c]);
      acc_e[c] += perr[c];
    }
  }
  const int gi = row0 + tid;
  if (gi < nq) {
#pragma unroll
    for (int c = 0; c < MV; ++c)
      if (c < mc) O[(int64_t)gi * ldo + col0 + c] = acc_s[c] + acc_e[c];
  }
}

static PlainConst plain_constants(int kf, double bw) {
  PlainConst p{0.f, 0.f, 0.f};
  switch (kf) {
    case KF_RBF:
    case KF_DRBF:
      p.e0 = (float)(-1.0 / (2.0 * bw * bw));
      p.c2 = (float)(1.0 / (bw * bw * bw));
      break;
    case KF_LAPLACE:
    case KF_DLAPLACE:
      p.e0 = (float)(-1.0 / bw);
      p.c2 = (float)(1.0 / (bw * bw));
      break;
    default:
      p.e1 = (float)(2.23606797749979 / bw);
      p.c2 = (float)(1.0 / bw);
      break;
  }
  return p;
}

template <int KF, int MV, bool COMP>
static int launch_plain_t(const PointSet& Q, const PointSet& Ks, const float* V, int m, int ldv, float* O, int ldo,
                          const PlainConst& pc, cudaStream_t st) {
  auto kern = k2_plain_kernel<KF, MV, COMP>;
  const int dp = Q.dp;
  const size_t smem = sizeof(float) * ((size_t)dp * (K2_ROWS + 1) + (size_t)K2_KEYS * dp + K2_KEYS * MV);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  dim3 grid((unsigned)((Q.n + K2_ROWS - 1) / K2_ROWS), (unsigned)((m + MV - 1) / MV));
  kern<<<grid, K2_ROWS, smem, st>>>(Q.xc, Ks.xc, V, O, (int)Q.n, (int)Ks.n, dp, m, ldv, ldo, pc);
  KOP_LAUNCHED();
  return KOP_OK;
}

template <int KF, bool COMP>
static int launch_plain_kf(const PointSet& Q, const PointSet& Ks, const float* V, int m, int ldv, float* O, int ldo,
                           const PlainConst& pc, cudaStream_t st) {
  if (m == 1) return launch_plain_t<KF, 1, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
  if (m == 2) return launch_plain_t<KF, 2, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
  if (m <= 4) return launch_plain_t<KF, 4, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
  return launch_plain_t<KF, 8, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
}

template <bool COMP>
static int plain_dispatch(int kf, const PointSet& Q, const PointSet& Ks, const float* V, int m, int ldv, float* O,
                          int ldo, const PlainConst& pc, cudaStream_t st) {
  switch (kf) {
    case KF_RBF: return launch_plain_kf<KF_RBF, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
    case KF_LAPLACE: return launch_plain_kf<KF_LAPLACE, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
    case KF_MATERN: return launch_plain_kf<KF_MATERN, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
    case KF_DRBF: return launch_plain_kf<KF_DRBF, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
    case KF_DLAPLACE: return launch_plain_kf<KF_DLAPLACE, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
    default: return launch_plain_kf<KF_DMATERN, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st);
  }
}

int plain_matvec(const PointSet& Q, const PointSet& Ks, bool /*self*/, int kf, const KConst& kc, const float* V,
                 int m, int ldv, float* O, int ldo, cudaStream_t st, bool compensated) {
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  const PlainConst pc = plain_constants(kf, kc.bw);
  return compensated ? plain_dispatch<true>(kf, Q, Ks, V, m, ldv, O, ldo, pc, st)
                     : plain_dispatch<false>(kf, Q, Ks, V, m, ldv, O, ldo, pc, st);
}

}  // namespace kop
