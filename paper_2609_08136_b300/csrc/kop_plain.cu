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

// BUILD: no contraction and no output; the kernel values of the key blocks
// of the row block's band (sym_band_count: each pair of blocks of the
// symmetric K once) are stored into the tile-packed Kst (see
// check_cache_floats; 0 for the padding keys j >= nk).
template <int KF, int MV, bool COMP, bool BUILD = false>
__global__ void __launch_bounds__(K2_ROWS) k2_plain_kernel(const float* __restrict__ Q, const float* __restrict__ Xk,
                                                           const float* __restrict__ V, float* __restrict__ O, int nq,
                                                           int nk, int dp, int m, int ldv, int ldo, PlainConst pc,
                                                           float* __restrict__ Kst) {
  extern __shared__ float sm[];
  float* Qs = sm;                              // dp x (K2_ROWS + 1), transposed
  float* Xs = Qs + dp * (K2_ROWS + 1);         // K2_KEYS x dp
  float* Vs = Xs + K2_KEYS * dp;               // K2_KEYS x MV
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * K2_ROWS;
  const int col0 = blockIdx.y * MV;
  const int mc = (m - col0) < MV ? (m - col0) : MV;
  const int gi = row0 + tid;
  const int hb = (nk + K2_ROWS - 1) / K2_ROWS / 2;  // band positions per row block - 1
  for (int idx = tid; idx < K2_ROWS * dp; idx += K2_ROWS) {
    const int r = idx / dp, k = idx - r * dp;
    Qs[k * (K2_ROWS + 1) + r] = Q[(int64_t)(row0 + r) * dp + k];
  }
  float acc_s[MV], acc_e[MV];
#pragma unroll
  for (int c = 0; c < MV; ++c) acc_s[c] = acc_e[c] = 0.0f;
  const int nb = (nk + K2_ROWS - 1) / K2_ROWS;
  const int ntl = BUILD ? sym_band_count(blockIdx.x, nb) * (K2_ROWS / K2_KEYS) : (nk + K2_KEYS - 1) / K2_KEYS;
  for (int tl = 0; tl < ntl; ++tl) {
    int j0 = tl * K2_KEYS;
    if constexpr (BUILD) {
      // sub-tile tl % 4 of band block I + tl / 4 (mod nb); keys past nk (but
      // below the padded count) are stored as 0
      const int J = (int)blockIdx.x + tl / (K2_ROWS / K2_KEYS);
      j0 = (J < nb ? J : J - nb) * K2_ROWS + (tl % (K2_ROWS / K2_KEYS)) * K2_KEYS;
    }
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
    if constexpr (BUILD) {
      // row tid of tile (I, t = tl / 4), columns (tl % 4) * 32 ..
      if (gi < nq) {
        float* kd = Kst + (((int64_t)blockIdx.x * (hb + 1) + tl / (K2_ROWS / K2_KEYS)) * K2_ROWS + tid) * K2_ROWS +
                    (tl % (K2_ROWS / K2_KEYS)) * K2_KEYS;
#pragma unroll
        for (int j4 = 0; j4 < K2_KEYS; j4 += 4) {
          const int j = j0 + j4;
          *reinterpret_cast<float4*>(kd + j4) =
              make_float4(j + 0 < nk ? d2[j4 + 0] : 0.0f, j + 1 < nk ? d2[j4 + 1] : 0.0f,
                          j + 2 < nk ? d2[j4 + 2] : 0.0f, j + 3 < nk ? d2[j4 + 3] : 0.0f);
        }
      }
    } else {
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
  }
  if (!BUILD && gi < nq) {
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
  kern<<<grid, K2_ROWS, smem, st>>>(Q.xc, Ks.xc, V, O, (int)Q.n, (int)Ks.n, dp, m, ldv, ldo, pc, nullptr);
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

// ---------------------------------------------------------------------------
// The check operator with the kernel matrix kept in HBM.  K(X, X) in FP32
// costs n^2 * 4 bytes in full; the stored form keeps each pair of row blocks
// once (about n^2 * 2 bytes: 80 GB at n = 200000).  The first check product
// of a solve computes the band tiles by direct differences as above and
// stores them; every check product of the solve then reads each stored tile
// once and uses it for both of its contributions.

int check_cache_reserve(kop_s* op) {
  if (op->kc) return KOP_OK;
  const int64_t n = op->pts.n;
  const size_t bytes = sizeof(float) * (size_t)check_cache_floats(n);
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
  op->kc_owned = 1;
  return KOP_OK;
}

template <int KF>
static int launch_build_t(const PointSet& P, const PlainConst& pc, float* Kc, cudaStream_t st) {
  auto kern = k2_plain_kernel<KF, 1, true, true>;
  const int dp = P.dp;
  const size_t smem = sizeof(float) * ((size_t)dp * (K2_ROWS + 1) + (size_t)K2_KEYS * dp + K2_KEYS * 1);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  dim3 grid((unsigned)((P.n + K2_ROWS - 1) / K2_ROWS), 1);
  kern<<<grid, K2_ROWS, smem, st>>>(P.xc, P.xc, nullptr, nullptr, (int)P.n, (int)P.n, dp, 1, 1, 1, pc, Kc);
  KOP_LAUNCHED();
  return KOP_OK;
}

// Store the direct-difference K(X, X) in op->kc for each pair of row blocks
// once (the band of each block).
static int check_cache_build(kop_s* op, cudaStream_t st) {
  const PlainConst pc = plain_constants(op->kernel, op->bw);
  switch (op->kernel) {
    case KF_RBF: return launch_build_t<KF_RBF>(op->pts, pc, op->kc, st);
    case KF_LAPLACE: return launch_build_t<KF_LAPLACE>(op->pts, pc, op->kc, st);
    default: return launch_build_t<KF_MATERN>(op->pts, pc, op->kc, st);
  }
}

// The symmetric product with the stored matrix, for the solver's checks: the
// vectors come in exact hi / lo FP32 pairs (x = hi + lo, columns c and cols + c
// of V2) and the result of each column is returned as an unevaluated
// (sum, error) pair in the same two columns of T (the residual adds them in
// FP64).  Per entry: TwoProduct K hi + TwoSum into the running sum, and the
// product with lo (2^-24 of the rest) into the error term.
//
// The CTA of row block I reads each tile K[I][J] of its band once (128 x 128
// floats, double-buffered through shared memory with asynchronous copies) and
// uses it twice: row part T_I += K_IJ x_J (accumulated over the band) and,
// for J != I, column part C[J][t - 1] = K_IJ^T x_I, stored as (sum, error)
// pairs for a second kernel that adds the column parts in a fixed order.
// Four threads per row / column take a quarter of the tile each, with two
// independent accumulators, combined in a fixed order.  Rows and keys past n
// count as 0.
constexpr int KS2_LD = 132;       // padded row pitch of a tile in shared memory (floats)
constexpr int KS2_THREADS = 512;  // 4 threads per row / column

// (s, e) += k (hi + lo), error-free up to the (negligible) rounding of k lo.
KOP_DEV void ef_acc_pair(float& s, float& e, float k, float hi, float lo) {
  const float p = k * hi;
  const float pe = fmaf(k, hi, -p);
  const float t = s + p;
  const float bb = t - s;
  const float err = (s - (t - bb)) + (p - bb);
  s = t;
  e = fmaf(k, lo, e + (err + pe));
}

// COMPUTE: no stored matrix.  The CTA computes each band tile K[I][J] into
// shared memory by direct differences, with the arithmetic of the build (so
// both forms give the same values), from the centred points Xc (n_pad x dp):
// thread (r, q) forms row r against keys q * 32 .. + 31.  One buffer, no
// prefetch (the distances dominate).  Shared memory: tile, then the two
// vector tiles and the reduction area, then (COMPUTE) X_I transposed
// (dp x 129) and X_J (128 x dp).
template <int NC, int KF = KF_RBF, bool COMPUTE = false>
__global__ void __launch_bounds__(KS2_THREADS, 1)
    kcache_symv_kernel(const float* __restrict__ Kc, int n, int nb, int h, const float* __restrict__ V2, int cols,
                       int c0, float* __restrict__ T, float* __restrict__ C, const float* __restrict__ Xc, int dp,
                       PlainConst pc) {
  extern __shared__ __align__(16) float ksm[];
  constexpr int NBUF = COMPUTE ? 1 : 2;
  float* tile[2] = {ksm, ksm + (NBUF - 1) * 128 * KS2_LD};
  float2* xj[2] = {reinterpret_cast<float2*>(ksm + NBUF * 128 * KS2_LD),
                   reinterpret_cast<float2*>(ksm + NBUF * 128 * KS2_LD) + (NBUF - 1) * 128 * NC};
  float2* xi = reinterpret_cast<float2*>(ksm + NBUF * 128 * KS2_LD) + NBUF * 128 * NC;
  float* red = reinterpret_cast<float*>(xi + 128 * NC);  // quarters 1..3: 3 x 128 x NC x (s, e)
  float* Qs = red + 3 * 128 * NC * 2;                   // COMPUTE: dp x (128 + 1)
  float* Xs = Qs + (COMPUTE ? dp * 129 : 0);            // COMPUTE: 128 x dp (16-byte aligned: dp % 16 == 0)
  const int tid = threadIdx.x;
  const int I = blockIdx.x;
  const int cnt = sym_band_count(I, nb);
  const int r = tid & 127, q = tid >> 7;
  const int ld = 2 * cols;
  auto xpair = [&](int row, int c) -> float2 {
    return (row < n && c0 + c < cols)
               ? make_float2(V2[(int64_t)row * ld + c0 + c], V2[(int64_t)row * ld + cols + c0 + c])
               : make_float2(0.0f, 0.0f);
  };
  for (int idx = tid; idx < 128 * NC; idx += KS2_THREADS) xi[idx] = xpair(I * 128 + idx / NC, idx % NC);
  if constexpr (COMPUTE) {
    for (int idx = tid; idx < 128 * dp; idx += KS2_THREADS) {
      const int rr = idx / dp, k = idx - rr * dp;
      Qs[k * 129 + rr] = Xc[(int64_t)(I * 128 + rr) * dp + k];
    }
  }
  // COMPUTE: block J's points and vector tile, then the kernel values
  auto compute = [&](int t) {
    const int J = I + t < nb ? I + t : I + t - nb;
    for (int idx = tid; idx < 128 * dp / 4; idx += KS2_THREADS)
      reinterpret_cast<float4*>(Xs)[idx] = reinterpret_cast<const float4*>(Xc + (int64_t)J * 128 * dp)[idx];
    for (int idx = tid; idx < 128 * NC; idx += KS2_THREADS) xj[0][idx] = xpair(J * 128 + idx / NC, idx % NC);
    __syncthreads();
    uint64_t d2p[32];  // (sum over even features, sum over odd features)
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) d2p[jj] = 0ull;
    for (int k0 = 0; k0 < dp; k0 += 16) {
      uint64_t q2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) q2[i] = pk2(Qs[(k0 + 2 * i) * 129 + r], Qs[(k0 + 2 * i + 1) * 129 + r]);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float4* xr = reinterpret_cast<const float4*>(Xs + (q * 32 + jj) * dp + k0);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 x4 = xr[k4];
          uint64_t d = sub_f32x2(q2[2 * k4], pk2(x4.x, x4.y));
          d2p[jj] = fma_f32x2(d, d, d2p[jj]);
          d = sub_f32x2(q2[2 * k4 + 1], pk2(x4.z, x4.w));
          d2p[jj] = fma_f32x2(d, d, d2p[jj]);
        }
      }
    }
    const bool row_in = I * 128 + r < n;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const float2 hh = unpk2(d2p[jj]);
      const float kv = plain_kernel_value<KF>(hh.x + hh.y, pc);
      tile[0][r * KS2_LD + q * 32 + jj] = (row_in && J * 128 + q * 32 + jj < n) ? kv : 0.0f;
    }
  };
  auto load = [&](int t, int buf) {
    const int J = I + t < nb ? I + t : I + t - nb;
    float* Tl = tile[buf];
    for (int idx = tid; idx < 128 * 32; idx += KS2_THREADS) {  // 128 rows x 32 float4
      const int rr = idx >> 5, qq = idx & 31, i = I * 128 + rr;
      const float* src = Kc + (((int64_t)I * (h + 1) + t) * 128 + rr) * 128 + 4 * qq;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Tl + rr * KS2_LD + 4 * qq);
      const int bytes = i < n ? 16 : 0;  // rows past n: zero fill
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
    }
    for (int idx = tid; idx < 128 * NC; idx += KS2_THREADS) xj[buf][idx] = xpair(J * 128 + idx / NC, idx % NC);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // this thread's quarter folded, then quarters 1..3 added by quarter 0 in a
  // fixed order
  auto combine = [&](float (&as)[2][NC], float (&ae)[2][NC], float (&os)[NC], float (&oe)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      os[c] = as[0][c];
      oe[c] = ae[0][c] + ae[1][c];
      two_sum_acc(os[c], oe[c], as[1][c]);
    }
    if (q > 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float* rd = red + (((q - 1) * 128 + r) * NC + c) * 2;
        rd[0] = os[c];
        rd[1] = oe[c];
      }
    }
    __syncthreads();
    if (q == 0) {
#pragma unroll
      for (int qq = 0; qq < 3; ++qq)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float* rd = red + ((qq * 128 + r) * NC + c) * 2;
          two_sum_acc(os[c], oe[c], rd[0]);
          oe[c] += rd[1];
        }
    }
  };
  float rs[2][NC], re[2][NC];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) rs[a][c] = re[a][c] = 0.0f;
  if constexpr (!COMPUTE) load(0, 0);
  for (int t = 0; t < cnt; ++t) {
    const int buf = COMPUTE ? 0 : (t & 1);
    const int J = I + t < nb ? I + t : I + t - nb;
    if constexpr (COMPUTE) {
      compute(t);
    } else if (t + 1 < cnt) {
      load(t + 1, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* Tl = tile[buf];
    const float2* X = xj[buf];
    // row part: row r, columns q * 32 .. + 31 in a rotated order (no bank
    // conflicts), two accumulators; keys past n are 0
    const int jlim = n - J * 128;
#pragma unroll 8
    for (int cc = 0; cc < 32; ++cc) {
      const int c = q * 32 + ((cc + r) & 31);
      const float kv = c < jlim ? Tl[r * KS2_LD + c] : 0.0f;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const float2 x = X[c * NC + k];
        ef_acc_pair(rs[cc & 1][k], re[cc & 1][k], kv, x.x, x.y);
      }
    }
    if (t > 0) {
      // column part: column r, rows q * 32 .. + 31 (rows past n were zero-filled)
      float cs[2][NC], ce[2][NC];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < NC; ++k) cs[a][k] = ce[a][k] = 0.0f;
#pragma unroll 8
      for (int rr = 0; rr < 32; ++rr) {
        const int row = q * 32 + rr;
        const float kv = Tl[row * KS2_LD + r];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float2 x = xi[row * NC + k];
          ef_acc_pair(cs[rr & 1][k], ce[rr & 1][k], kv, x.x, x.y);
        }
      }
      float os[NC], oe[NC];
      combine(cs, ce, os, oe);
      if (q == 0) {
        float2* dst = reinterpret_cast<float2*>(C) + (((int64_t)J * h + (t - 1)) * 128 + r) * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) dst[k] = make_float2(os[k], oe[k]);
      }
    }
    __syncthreads();  // the buffers are reloaded by the next iteration's prefetch
  }
  float os[NC], oe[NC];
  combine(rs, re, os, oe);
  const int i = I * 128 + r;
  if (q == 0 && i < n) {
#pragma unroll
    for (int k = 0; k < NC; ++k)
      if (c0 + k < cols) {
        T[(int64_t)i * ld + c0 + k] = os[k];
        T[(int64_t)i * ld + cols + c0 + k] = oe[k];
      }
  }
}

// (T[i][c0 + k], T[i][cols + c0 + k]) += the column parts of row block
// J = i / 128, in the order of t, as (sum, error) pairs.
template <int NC>
__global__ void kcache_combine_kernel(float* __restrict__ T, int cols, int c0, const float* __restrict__ C, int n,
                                      int nb, int h) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * NC) return;
  const int i = (int)(g / NC), k = (int)(g - (int64_t)i * NC);
  if (c0 + k >= cols) return;
  const int J = i >> 7, jj = i & 127;
  const int64_t ld = 2 * (int64_t)cols;
  float s = T[i * ld + c0 + k], e = T[i * ld + cols + c0 + k];
  const float2* C2 = reinterpret_cast<const float2*>(C);
  for (int t = 1; t <= h; ++t) {
    const int I = J - t >= 0 ? J - t : J - t + nb;
    if (t < sym_band_count(I, nb)) {
      const float2 p = C2[(((int64_t)J * h + (t - 1)) * 128 + jj) * NC + k];
      two_sum_acc(s, e, p.x);
      e += p.y;
    }
  }
  T[i * ld + c0 + k] = s;
  T[i * ld + cols + c0 + k] = e;
}

static size_t symv_smem(int nc, bool compute, int dp) {
  const int nbuf = compute ? 1 : 2;
  size_t b = sizeof(float) * (nbuf * 128 * KS2_LD) + sizeof(float2) * (nbuf + 1) * 128 * nc +
             sizeof(float) * 3 * 128 * nc * 2;
  if (compute) b += sizeof(float) * ((size_t)dp * 129 + (size_t)128 * dp) + 16;
  return b;
}

template <int NC, int KF, bool COMPUTE>
static int symv_launch_t(kop_s* op, const float* V2, int cols, int c0, float* T, cudaStream_t st) {
  auto kern = kcache_symv_kernel<NC, KF, COMPUTE>;
  const int dp = op->pts.dp;
  const size_t smem = symv_smem(NC, COMPUTE, dp);
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  const int n = (int)op->pts.n;
  const int nb = (n + 127) / 128, h = nb / 2;
  const PlainConst pc = plain_constants(op->kernel, op->bw);
  kern<<<(unsigned)nb, KS2_THREADS, smem, st>>>(op->kc, n, nb, h, V2, cols, c0, T, op->kc_scratch, op->pts.xc, dp,
                                                pc);
  KOP_LAUNCHED();
  if (h > 0) {
    const int64_t tot = (int64_t)n * NC;
    kcache_combine_kernel<NC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(T, cols, c0, op->kc_scratch, n, nb, h);
    KOP_LAUNCHED();
  }
  return KOP_OK;
}

template <int NC>
static int symv_launch(kop_s* op, bool compute, const float* V2, int cols, int c0, float* T, cudaStream_t st) {
  if (!compute) return symv_launch_t<NC, KF_RBF, false>(op, V2, cols, c0, T, st);
  switch (op->kernel) {
    case KF_RBF: return symv_launch_t<NC, KF_RBF, true>(op, V2, cols, c0, T, st);
    case KF_LAPLACE: return symv_launch_t<NC, KF_LAPLACE, true>(op, V2, cols, c0, T, st);
    default: return symv_launch_t<NC, KF_MATERN, true>(op, V2, cols, c0, T, st);
  }
}

// Column-part scratch for the symmetric check products: nb x h x 128 pairs
// per column group.  false when it does not fit next to the caller's data.
static int sym_scratch(kop_s* op, int cols, cudaStream_t st, bool* fits) {
  const int n = (int)op->pts.n;
  const int nb = (n + 127) / 128, h = nb / 2;
  const int nc = cols <= 1 ? 1 : (cols <= 2 ? 2 : 4);
  const size_t need = (size_t)nb * h * 128 * nc * 2;  // (sum, error) pairs
  *fits = true;
  if (need > op->kc_scratch_floats) {
    if (op->kc_scratch) cudaFreeAsync(op->kc_scratch, st);
    op->kc_scratch = nullptr;
    op->kc_scratch_floats = 0;
    size_t fr = 0, tot = 0;
    KOP_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    if (fr < sizeof(float) * need + (size_t(4) << 30)) {
      *fits = false;
      return KOP_OK;
    }
    KOP_CUDA_TRY(cudaMallocAsync((void**)&op->kc_scratch, sizeof(float) * (need > 0 ? need : 1), st));
    op->kc_scratch_floats = need;
  }
  return KOP_OK;
}

static int sym_products(kop_s* op, bool compute, const float* V2, int cols, float* T, cudaStream_t st) {
  const int nc = cols <= 1 ? 1 : (cols <= 2 ? 2 : 4);
  for (int c0 = 0; c0 < cols; c0 += nc) {
    int rc;
    if (nc == 1) rc = symv_launch<1>(op, compute, V2, cols, c0, T, st);
    else if (nc == 2) rc = symv_launch<2>(op, compute, V2, cols, c0, T, st);
    else rc = symv_launch<4>(op, compute, V2, cols, c0, T, st);
    if (rc) return rc;
  }
  return KOP_OK;
}

int check_matvec_cached(kop_s* op, bool build, const float* V2, int cols, float* T, cudaStream_t st) {
  if (build) {
    const int rc = check_cache_build(op, st);
    if (rc) return rc;
  }
  bool fits = true;
  if (int rc = sym_scratch(op, cols, st, &fits)) return rc;
  if (!fits) return fail(KOP_ENOMEM, "check product: no device memory for the column parts");
  return sym_products(op, false, V2, cols, T, st);
}

int check_matvec_computed(kop_s* op, const float* V2, int cols, float* T, cudaStream_t st, bool* done) {
  *done = false;
  if (symv_smem(cols <= 1 ? 1 : (cols <= 2 ? 2 : 4), true, op->pts.dp) > smem_limit_bytes()) return KOP_OK;
  bool fits = true;
  if (int rc = sym_scratch(op, cols, st, &fits)) return rc;
  if (!fits) return KOP_OK;
  *done = true;
  return sym_products(op, true, V2, cols, T, st);
}

}  // namespace kop
