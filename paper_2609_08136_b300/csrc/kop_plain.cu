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

// Kst != NULL: the column block 0 also stores every kernel value it computes,
// Kst[i * ldk + j] for the rows i < nq and all keys of its tiles (0 for the
// padding keys j >= nk); ldk a multiple of 4.  BUILD: only store, for the keys
// j >= the block's first row (the upper block triangle of a symmetric K; the
// rest is mirrored afterwards), with no contraction and no output.
template <int KF, int MV, bool COMP, bool BUILD = false>
__global__ void __launch_bounds__(K2_ROWS) k2_plain_kernel(const float* __restrict__ Q, const float* __restrict__ Xk,
                                                           const float* __restrict__ V, float* __restrict__ O, int nq,
                                                           int nk, int dp, int m, int ldv, int ldo, PlainConst pc,
                                                           float* __restrict__ Kst, int64_t ldk) {
  extern __shared__ float sm[];
  float* Qs = sm;                              // dp x (K2_ROWS + 1), transposed
  float* Xs = Qs + dp * (K2_ROWS + 1);         // K2_KEYS x dp
  float* Vs = Xs + K2_KEYS * dp;               // K2_KEYS x MV
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * K2_ROWS;
  const int col0 = blockIdx.y * MV;
  const int mc = (m - col0) < MV ? (m - col0) : MV;
  const int gi = row0 + tid;
  float* const krow = (Kst != nullptr && blockIdx.y == 0 && gi < nq) ? Kst + (int64_t)gi * ldk : nullptr;
  for (int idx = tid; idx < K2_ROWS * dp; idx += K2_ROWS) {
    const int r = idx / dp, k = idx - r * dp;
    Qs[k * (K2_ROWS + 1) + r] = Q[(int64_t)(row0 + r) * dp + k];
  }
  float acc_s[MV], acc_e[MV];
#pragma unroll
  for (int c = 0; c < MV; ++c) acc_s[c] = acc_e[c] = 0.0f;
  for (int j0 = BUILD ? row0 : 0; j0 < nk; j0 += K2_KEYS) {
    __syncthreads();
    for (int idx = tid; idx < K2_KEYS * dp; idx += K2_ROWS) Xs[idx] = Xk[(int64_t)j0 * dp + idx];
    if constexpr (!BUILD) {
      for (int idx = tid; idx < K2_KEYS * MV; idx += K2_ROWS) {
        const int jj = idx / MV, c = idx - jj * MV, j = j0 + jj;
        Vs[idx] = (j < nk && c < mc) ? V[(int64_t)j * ldv + col0 + c] : 0.0f;
      }
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
    // kernel values in place of the distances
#pragma unroll
    for (int jj = 0; jj < K2_KEYS; ++jj) d2[jj] = plain_kernel_value<KF>(d2[jj], pc);
    if (krow != nullptr) {
#pragma unroll
      for (int j4 = 0; j4 < K2_KEYS; j4 += 4) {
        const int j = j0 + j4;
        *reinterpret_cast<float4*>(krow + j) =
            make_float4(j + 0 < nk ? d2[j4 + 0] : 0.0f, j + 1 < nk ? d2[j4 + 1] : 0.0f,
                        j + 2 < nk ? d2[j4 + 2] : 0.0f, j + 3 < nk ? d2[j4 + 3] : 0.0f);
      }
    }
    if constexpr (BUILD) continue;
#pragma unroll
    for (int jj = 0; jj < K2_KEYS; ++jj) {
      const float kv = d2[jj];
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
  if (!BUILD && gi < nq) {
#pragma unroll
    for (int c = 0; c < MV; ++c)
      if (c < mc) O[(int64_t)gi * ldo + col0 + c] = acc_s[c] + acc_e[c];
  }
}

// The lower block triangle of the stored symmetric K from the upper one:
// Kc[i][j] = Kc[j][i] for the keys j below the first row of i's 128-row block
// (32 x 32 tiles through shared memory; rows i < n, keys j < n).
__global__ void __launch_bounds__(256) kcache_mirror_kernel(float* __restrict__ Kc, int64_t ldk, int n) {
  __shared__ float tile[32][33];
  const int ti = blockIdx.y * 32, tj = blockIdx.x * 32;  // destination rows ti.., keys tj..
  if (tj >= (ti / K2_ROWS) * K2_ROWS) return;         // on or above the block diagonal: computed
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int src_row = tj + r, src_col = ti + tx;  // Kc[tj + r][ti + tx]
    tile[r][tx] = (src_row < n && src_col < n) ? Kc[(int64_t)src_row * ldk + src_col] : 0.0f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int row = ti + r, col = tj + tx;
    if (row < n && col < n) Kc[(int64_t)row * ldk + col] = tile[tx][r];
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
                          const PlainConst& pc, cudaStream_t st, float* Kst, int64_t ldk) {
  auto kern = k2_plain_kernel<KF, MV, COMP>;
  const int dp = Q.dp;
  const size_t smem = sizeof(float) * ((size_t)dp * (K2_ROWS + 1) + (size_t)K2_KEYS * dp + K2_KEYS * MV);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  dim3 grid((unsigned)((Q.n + K2_ROWS - 1) / K2_ROWS), (unsigned)((m + MV - 1) / MV));
  kern<<<grid, K2_ROWS, smem, st>>>(Q.xc, Ks.xc, V, O, (int)Q.n, (int)Ks.n, dp, m, ldv, ldo, pc, Kst, ldk);
  KOP_LAUNCHED();
  return KOP_OK;
}

template <int KF, bool COMP>
static int launch_plain_kf(const PointSet& Q, const PointSet& Ks, const float* V, int m, int ldv, float* O, int ldo,
                           const PlainConst& pc, cudaStream_t st, float* Kst, int64_t ldk) {
  if (m == 1) return launch_plain_t<KF, 1, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
  if (m == 2) return launch_plain_t<KF, 2, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
  if (m <= 4) return launch_plain_t<KF, 4, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
  return launch_plain_t<KF, 8, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
}

template <bool COMP>
static int plain_dispatch(int kf, const PointSet& Q, const PointSet& Ks, const float* V, int m, int ldv, float* O,
                          int ldo, const PlainConst& pc, cudaStream_t st, float* Kst = nullptr, int64_t ldk = 0) {
  switch (kf) {
    case KF_RBF: return launch_plain_kf<KF_RBF, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
    case KF_LAPLACE: return launch_plain_kf<KF_LAPLACE, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
    case KF_MATERN: return launch_plain_kf<KF_MATERN, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
    case KF_DRBF: return launch_plain_kf<KF_DRBF, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
    case KF_DLAPLACE: return launch_plain_kf<KF_DLAPLACE, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
    default: return launch_plain_kf<KF_DMATERN, COMP>(Q, Ks, V, m, ldv, O, ldo, pc, st, Kst, ldk);
  }
}

int plain_matvec(const PointSet& Q, const PointSet& Ks, bool /*self*/, int kf, const KConst& kc, const float* V,
                 int m, int ldv, float* O, int ldo, cudaStream_t st, bool compensated) {
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  const PlainConst pc = plain_constants(kf, kc.bw);
  return compensated ? plain_dispatch<true>(kf, Q, Ks, V, m, ldv, O, ldo, pc, st)
                     : plain_dispatch<false>(kf, Q, Ks, V, m, ldv, O, ldo, pc, st);
}

// ---------------------------------------------------------------------------
// The check operator with the kernel matrix kept in HBM.  K(X, X) in FP32 is
// n^2 * 4 bytes (160 GB at n = 200000, which a B300 holds).  The first check
// product of a solve computes it by direct differences as above and stores
// it; later check products of the same solve stream the stored matrix with
// the same error-free contraction instead of recomputing the distances.

// O[i][c0 + c] = sum_{j < nk} Kc[i][j] V[j][c0 + c], TwoProduct + TwoSum per
// entry as in the direct kernel.  A warp takes RW rows (8; 4 for 8 columns);
// lane l reads the float4 of keys j = jb + 4 l of each row and the V rows of
// those 4 keys once for the RW rows.  Keys j >= nk (the tail of a row up to
// ldk) count as 0.
template <int MV>
__global__ void __launch_bounds__(256) kcache_gemv_kernel(const float* __restrict__ Kc, int64_t ldk, int nq, int nk,
                                                          const float* __restrict__ V, int m, int ldv,
                                                          float* __restrict__ O, int ldo) {
  constexpr int RW = MV <= 4 ? 8 : 4;
  const int lane = threadIdx.x & 31;
  const int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RW;
  if (i0 >= nq) return;  // warp-uniform
  const int nr = nq - i0 < RW ? (int)(nq - i0) : RW;
  const int c0 = blockIdx.y * MV;
  const int mc = m - c0 < MV ? m - c0 : MV;
  float s[RW][MV], e[RW][MV];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < MV; ++c) s[r][c] = e[r][c] = 0.0f;
  for (int jb = 0; jb < nk; jb += 128) {
    const int j = jb + 4 * lane;
    float v[4][MV];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < MV; ++c) v[q][c] = (j + q < nk && c < mc) ? __ldg(V + (int64_t)(j + q) * ldv + c0 + c) : 0.0f;
    float4 k[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r)
      k[r] = r < nr ? *reinterpret_cast<const float4*>(Kc + (i0 + r) * ldk + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (jb + 128 > nk) {  // the last block of keys: entries past nk are not data
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        if (j + 0 >= nk) k[r].x = 0.0f;
        if (j + 1 >= nk) k[r].y = 0.0f;
        if (j + 2 >= nk) k[r].z = 0.0f;
        if (j + 3 >= nk) k[r].w = 0.0f;
      }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const float kr[4] = {k[r].x, k[r].y, k[r].z, k[r].w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < MV; ++c) {
          const float p = kr[q] * v[q][c];
          const float pe = fmaf(kr[q], v[q][c], -p);
          const float t = s[r][c] + p;
          const float bb = t - s[r][c];
          e[r][c] += ((s[r][c] - (t - bb)) + (p - bb)) + pe;
          s[r][c] = t;
        }
    }
  }
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < MV; ++c) {
      float a = s[r][c], b = e[r][c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float a2 = __shfl_xor_sync(0xffffffffu, a, off);
        const float b2 = __shfl_xor_sync(0xffffffffu, b, off);
        const float t = a + a2;
        const float bb = t - a;
        b += ((a - (t - bb)) + (a2 - bb)) + b2;
        a = t;
      }
      if (lane == 0 && r < nr && c < mc) O[(i0 + r) * ldo + c0 + c] = a + b;
    }
}

template <int MV>
static void kcache_launch(const float* Kc, int64_t ldk, int nq, int nk, const float* V, int m, int ldv, float* O,
                          int ldo, cudaStream_t st) {
  constexpr int rows_per_cta = 8 * (MV <= 4 ? 8 : 4);
  const dim3 grid((unsigned)((nq + rows_per_cta - 1) / rows_per_cta), (unsigned)((m + MV - 1) / MV));
  kcache_gemv_kernel<MV><<<grid, 256, 0, st>>>(Kc, ldk, nq, nk, V, m, ldv, O, ldo);
}

int check_cache_reserve(kop_s* op) {
  if (op->kc) return KOP_OK;
  const int64_t n = op->pts.n;
  const int64_t ld = check_cache_ld(n);
  const size_t bytes = sizeof(float) * (size_t)n * (size_t)ld;
  size_t fr = 0, tot = 0;
  KOP_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  // keep 4 GB for the solver's own buffers and the caller's
  if (fr < bytes + (size_t(4) << 30)) return fail(KOP_ENOMEM, "kop_set_check_cache: not enough free device memory");
  const cudaError_t e = cudaMalloc(&op->kc, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    op->kc = nullptr;
    return fail(KOP_ENOMEM, "kop_set_check_cache: cudaMalloc failed");
  }
  op->kc_ld = ld;
  op->kc_owned = 1;
  return KOP_OK;
}

template <int KF>
static int launch_build_t(const PointSet& P, const PlainConst& pc, float* Kc, int64_t ldk, cudaStream_t st) {
  auto kern = k2_plain_kernel<KF, 1, true, true>;
  const int dp = P.dp;
  const size_t smem = sizeof(float) * ((size_t)dp * (K2_ROWS + 1) + (size_t)K2_KEYS * dp + K2_KEYS * 1);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  dim3 grid((unsigned)((P.n + K2_ROWS - 1) / K2_ROWS), 1);
  kern<<<grid, K2_ROWS, smem, st>>>(P.xc, P.xc, nullptr, nullptr, (int)P.n, (int)P.n, dp, 1, 1, 1, pc, Kc, ldk);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Store the direct-difference K(X, X) in op->kc: the upper block triangle
// (each pair of row blocks once), then its mirror image.
static int check_cache_build(kop_s* op, cudaStream_t st) {
  const PlainConst pc = plain_constants(op->kernel, op->bw);
  int rc;
  switch (op->kernel) {
    case KF_RBF: rc = launch_build_t<KF_RBF>(op->pts, pc, op->kc, op->kc_ld, st); break;
    case KF_LAPLACE: rc = launch_build_t<KF_LAPLACE>(op->pts, pc, op->kc, op->kc_ld, st); break;
    default: rc = launch_build_t<KF_MATERN>(op->pts, pc, op->kc, op->kc_ld, st); break;
  }
  if (rc) return rc;
  const int n = (int)op->pts.n;
  const unsigned t = (unsigned)((n + 31) / 32);
  kcache_mirror_kernel<<<dim3(t, t), 256, 0, st>>>(op->kc, op->kc_ld, n);
  KOP_LAUNCHED();
  return KOP_OK;
}

int check_matvec_cached(kop_s* op, bool build, const float* V, int m, int ldv, float* O, int ldo, cudaStream_t st) {
  const int n = (int)op->pts.n;
  if (build) {
    const int rc = check_cache_build(op, st);
    if (rc) return rc;
  }
  if (m == 1) kcache_launch<1>(op->kc, op->kc_ld, n, n, V, m, ldv, O, ldo, st);
  else if (m == 2) kcache_launch<2>(op->kc, op->kc_ld, n, n, V, m, ldv, O, ldo, st);
  else if (m <= 4) kcache_launch<4>(op->kc, op->kc_ld, n, n, V, m, ldv, O, ldo, st);
  else kcache_launch<8>(op->kc, op->kc_ld, n, n, V, m, ldv, O, ldo, st);
  KOP_LAUNCHED();
  return KOP_OK;
}

}  // namespace kop
