// Fused kernel-operator product O = f(K(Q, X)) V on the tensor cores.
//
// This is the matrix-free operator of the paper (Sec. 4.3: the linear
// operator is applied without ever being formed; Sec. 2.1: K_ij = k(x_i, x_j)
// and each CG iteration costs one O(n^2) product).  Per 128-row block of Q a
// CTA streams tiles of X:
//   S   = Q_I X_J^T      tcgen05.mma, BF16 split operands, FP32 in TMEM
//   D2  = |q_i|^2 + |x_j|^2 - 2 S_ij   (clamped at 0, exactly 0 on the
//                                        diagonal of a symmetric product)
//   K   = k(D2)          in registers (ex2 / sqrt on the SFU)
//   O  += K V_J          FP32 FMAs in registers (this file: m <= 8 columns)
// K never reaches global memory.  Warp roles: warp 0 loads tiles (TMA for the
// split operands, plain loads for norms and V), warp 1 issues the MMAs,
// warp 2 owns the TMEM allocation, warps 4..11 (two warpgroups, one half of
// the tile columns each) run the epilogue.  The S accumulator is double
// buffered in TMEM so that the MMAs of tile t+1 overlap the epilogue of t.
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

constexpr int K1_THREADS = 384;
constexpr int K1_NST = 2;  // smem pipeline stages (2 CTAs fit per SM for d <= 64)

template <int KF>
KOP_DEV float kernel_value(float d2, float c0, float c1, float c2) {
  if constexpr (KF == KF_RBF) {
    return ex2_approx(d2 * c0);
  } else if constexpr (KF == KF_LAPLACE) {
    return ex2_approx(sqrt_approx(d2) * c0);
  } else if constexpr (KF == KF_MATERN) {
    float a = sqrt_approx(d2) * c1;
    return fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f) * ex2_approx(a * c0);
  } else if constexpr (KF == KF_DRBF) {
    return ex2_approx(d2 * c0) * d2 * c2;
  } else if constexpr (KF == KF_DLAPLACE) {
    float r = sqrt_approx(d2);
    return ex2_approx(r * c0) * r * c2;
  } else {
    float a = sqrt_approx(d2) * c1;
    return ex2_approx(a * c0) * (a * a * (1.0f / 3.0f)) * (1.0f + a) * c2;
  }
}

struct FusedArgs {
  const float* qnorm;  // padded to the Q block grid
  const float* knorm;  // padded to the X tile grid
  const float* V;
  float* O;
  int nq, nk, m, ldv, ldo;
  int dp, row_bytes, swz, self;
  float c0, c1, c2;
  int* status;
};

// Shared-memory layout of the FMA-epilogue kernel (offsets from a 1024-byte
// aligned base).
struct K1Layout {
  uint32_t q_split, x_split, qs, xs, kn, vs, qn, bars, holder, abort_word, red, total;
  __host__ __device__ K1Layout(int nsplit, int dp, int bn, int mv) {
    q_split = 128u * dp * 2;
    x_split = (uint32_t)bn * dp * 2;
    qs = 0;
    xs = qs + nsplit * q_split;
    kn = xs + K1_NST * nsplit * x_split;
    vs = kn + K1_NST * bn * 4;
    qn = vs + K1_NST * bn * mv * 4;
    bars = qn + 128 * 4;
    holder = bars + (2 * K1_NST + 6) * 8;
    abort_word = holder + 4;
    red = abort_word + 12;
    total = red + 128 * mv * 2 * 4;
  }
};

// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast.
KOP_DEV bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// Time-bounded wait that ignores the abort word (used only to let in-flight
// asynchronous work land before the CTA exits).
KOP_DEV void drain_wait(uint64_t* bar, uint32_t parity) {
  uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > KOP_WAIT_LIMIT_NS) break;
  }
}

// (A split, B split) of the i-th partial product.  Small terms come first so
// that the large hi*hi product is added last, to an accumulator that still
// holds only small values.
//   2 splits (hi, mid):       hi*mid, mid*hi, hi*hi
//   3 splits (hi, mid, lo):   mid*mid, hi*lo, lo*hi, hi*mid, mid*hi, hi*hi
template <int NSPLIT>
KOP_DEV constexpr int n_terms() { return NSPLIT == 2 ? 3 : 6; }
template <int NSPLIT>
KOP_DEV constexpr int term_a(int t) {
  return NSPLIT == 2 ? (t == 1 ? 1 : 0) : (t == 0 ? 1 : t == 2 ? 2 : t == 4 ? 1 : 0);
}
template <int NSPLIT>
KOP_DEV constexpr int term_b(int t) {
  return NSPLIT == 2 ? (t == 0 ? 1 : 0) : (t == 0 ? 1 : t == 1 ? 2 : t == 3 ? 1 : 0);
}

template <int KF, int NSPLIT, int MV, int BN>
__global__ void __launch_bounds__(K1_THREADS, 1)
    k1_fma_kernel(const __grid_constant__ CUtensorMap tq0, const __grid_constant__ CUtensorMap tq1,
                  const __grid_constant__ CUtensorMap tq2, const __grid_constant__ CUtensorMap tk0,
                  const __grid_constant__ CUtensorMap tk1, const __grid_constant__ CUtensorMap tk2,
                  const FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const K1Layout L(NSPLIT, a.dp, BN, MV);
  uint8_t* qs = smem + L.qs;
  uint8_t* xs = smem + L.xs;
  float* kn = (float*)(smem + L.kn);
  float* vs = (float*)(smem + L.vs);
  float* qn = (float*)(smem + L.qn);
  uint64_t* bars = (uint64_t*)(smem + L.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + K1_NST;
  uint64_t* tfull = bars + 2 * K1_NST;
  uint64_t* tempty = tfull + 2;
  uint64_t* qbar = tempty + 2;
  uint64_t* drain = qbar + 1;
  uint32_t* holder = (uint32_t*)(smem + L.holder);
  volatile int* abort_word = (volatile int*)(smem + L.abort_word);
  float* red = (float*)(smem + L.red);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * 128;
  const int ntiles = (a.nk + BN - 1) / BN;
  const int rb = a.row_bytes;
  const int nsub = (a.dp * 2) / rb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < K1_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + 256);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(qbar, 1);
    mbar_init(drain, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(holder, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    const CUtensorMap* mq[3] = {&tq0, &tq1, &tq2};
    const CUtensorMap* mk[3] = {&tk0, &tk1, &tk2};
    for (int i = lane; i < 128; i += 32) qn[i] = a.qnorm[row0 + i];
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_expect_tx(qbar, NSPLIT * L.q_split);
      for (int sp = 0; sp < NSPLIT; ++sp)
        for (int ks = 0; ks < nsub; ++ks)
          for (int rr = 0; rr < 128 / BN; ++rr)
            tma_load_2d(qs + sp * L.q_split + ks * (128 * rb) + rr * (BN * rb), mq[sp], qbar, ks * 64,
                        row0 + rr * BN);
    }
    int t = 0;
    for (; t < ntiles; ++t) {
      const int s = t % K1_NST;
      const uint32_t ph = (t / K1_NST) & 1;
      if (!warp_wait(&empty[s], ph ^ 1, abort_word, a.status)) break;
      const int j0 = t * BN;
      for (int i = lane; i < BN; i += 32) kn[s * BN + i] = a.knorm[j0 + i];
      for (int i = lane; i < BN * MV; i += 32) {
        const int jj = i / MV, c = i - jj * MV, j = j0 + jj;
        vs[s * BN * MV + i] = (j < a.nk && c < a.m) ? a.V[(int64_t)j * a.ldv + c] : 0.0f;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], NSPLIT * L.x_split);
        for (int sp = 0; sp < NSPLIT; ++sp)
          for (int ks = 0; ks < nsub; ++ks)
            tma_load_2d(xs + (s * NSPLIT + sp) * L.x_split + ks * (BN * rb), mk[sp], &full[s], ks * 64, j0);
      }
      __syncwarp();
    }
    if (t < ntiles && lane == 0) {
      // aborted: let the loads already issued land before the CTA exits
      for (int u = (t - K1_NST > 0 ? t - K1_NST : 0); u < t; ++u) drain_wait(&full[u % K1_NST], (u / K1_NST) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_bf16_f32(128, BN);
    const uint32_t sbo = 8u * rb;
    const int steps_per_sub = rb / 32;
    bool ok = warp_wait(qbar, 0, abort_word, a.status);
    for (int t = 0; ok && t < ntiles; ++t) {
      const int s = t % K1_NST;
      const uint32_t ph = (t / K1_NST) & 1;
      const int b = t & 1;
      const uint32_t bph = (t >> 1) & 1;
      if (!warp_wait(&full[s], ph, abort_word, a.status)) break;
      if (!warp_wait(&tempty[b], bph ^ 1, abort_word, a.status)) break;
      tc_fence_after();
      if (lane == 0) {
        const uint32_t d = tmem + b * BN;
        uint32_t acc = 0;
#pragma unroll
        for (int term = 0; term < n_terms<NSPLIT>(); ++term) {
          const uint32_t abase = smem_u32(qs + term_a<NSPLIT>(term) * L.q_split);
          const uint32_t bbase = smem_u32(xs + (s * NSPLIT + term_b<NSPLIT>(term)) * L.x_split);
          for (int kc = 0; kc < a.dp / 16; ++kc) {
            const int ks = kc / steps_per_sub, w = kc - ks * steps_per_sub;
            const uint64_t ad = sdesc(abase + ks * (128 * rb) + w * 32, sbo, a.swz);
            const uint64_t bd = sdesc(bbase + ks * (BN * rb) + w * 32, sbo, a.swz);
            tc_mma_ss(d, ad, bd, idesc, acc);
            acc = 1;
          }
        }
        tc_commit(&tfull[b]);
        tc_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (lane == 0) {
      tc_commit(drain);
      drain_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int ep = warp - 4, wg = ep >> 2, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gi = row0 + row;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    constexpr int HALF = BN / 2;
    constexpr int NCH = HALF / 32;
    float acc_s[MV], acc_e[MV];
#pragma unroll
    for (int c = 0; c < MV; ++c) acc_s[c] = acc_e[c] = 0.0f;
    bool ok = warp_wait(qbar, 0, abort_word, a.status);
    const float qni = qn[row];
    for (int t = 0; ok && t < ntiles; ++t) {
      const int s = t % K1_NST;
      const uint32_t ph = (t / K1_NST) & 1;
      const int b = t & 1;
      const uint32_t bph = (t >> 1) & 1;
      if (!warp_wait(&tfull[b], bph, abort_word, a.status)) break;
      tc_fence_after();
      uint32_t r[NCH][32];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        tmem_ld32(lane_addr + b * BN + wg * HALF + ch * 32, r[ch]);
        tmem_ld_wait(r[ch]);
      }
      tc_fence_before();
      mbar_arrive(&tempty[b]);
      if (!warp_wait(&full[s], ph, abort_word, a.status)) break;
      const float* knS = kn + s * BN + wg * HALF;
      const float* vS = vs + (s * BN + wg * HALF) * MV;
      const int jbase = t * BN + wg * HALF;
      float part[MV];
#pragma unroll
      for (int c = 0; c < MV; ++c) part[c] = 0.0f;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int jl = ch * 32 + jj;
          const float sij = __uint_as_float(r[ch][jj]);
          float d2 = fmaxf(fmaf(-2.0f, sij, qni + knS[jl]), 0.0f);
          if (a.self && jbase + jl == gi) d2 = 0.0f;
          const float kv = kernel_value<KF>(d2, a.c0, a.c1, a.c2);
#pragma unroll
          for (int c = 0; c < MV; ++c) part[c] = fmaf(kv, vS[jl * MV + c], part[c]);
        }
      }
      mbar_arrive(&empty[s]);
#pragma unroll
      for (int c = 0; c < MV; ++c) two_sum_acc(acc_s[c], acc_e[c], part[c]);
    }
    if (wg == 1) {
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        red[(row * MV + c) * 2] = acc_s[c];
        red[(row * MV + c) * 2 + 1] = acc_e[c];
      }
    }
    named_bar_sync(1, 256);
    if (wg == 0 && gi < a.nq && !*abort_word) {
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        if (c < a.m) {
          const float hi = acc_s[c] + red[(row * MV + c) * 2];
          const float lo = acc_e[c] + red[(row * MV + c) * 2 + 1];
          a.O[(int64_t)gi * a.ldo + c] = hi + lo;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ---------------------------------------------------------------- host side
static int swizzle_code(int row_bytes) { return row_bytes == 128 ? 2 : (row_bytes == 64 ? 4 : 6); }

template <int KF, int NSPLIT, int MV, int BN>
static int launch_fma_t(const PointSet& Q, const PointSet& Ks, const FusedArgs& a, cudaStream_t st) {
  auto kern = k1_fma_kernel<KF, NSPLIT, MV, BN>;
  const K1Layout L(NSPLIT, a.dp, BN, MV);
  const size_t smem = L.total + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  const int bi = BN == 128 ? 0 : 1;
  dim3 grid((unsigned)((a.nq + 127) / 128));
  kern<<<grid, K1_THREADS, smem, st>>>(Q.tm[0][bi], Q.tm[1][bi], Q.tm[2][bi], Ks.tm[0][bi], Ks.tm[1][bi],
                                       Ks.tm[2][bi], a);
  KOP_LAUNCHED();
  return KOP_OK;
}

template <int KF, int NSPLIT, int BN>
static int launch_fma_mv(int mv, const PointSet& Q, const PointSet& Ks, const FusedArgs& a, cudaStream_t st) {
  if (mv == 1) return launch_fma_t<KF, NSPLIT, 1, BN>(Q, Ks, a, st);
  if (mv == 4) return launch_fma_t<KF, NSPLIT, 4, BN>(Q, Ks, a, st);
  return launch_fma_t<KF, NSPLIT, 8, BN>(Q, Ks, a, st);
}

template <int KF>
static int launch_fma_kf(int nsplit, int bn, int mv, const PointSet& Q, const PointSet& Ks, const FusedArgs& a,
                         cudaStream_t st) {
  if (nsplit == 2)
    return bn == 128 ? launch_fma_mv<KF, 2, 128>(mv, Q, Ks, a, st) : launch_fma_mv<KF, 2, 64>(mv, Q, Ks, a, st);
  return bn == 128 ? launch_fma_mv<KF, 3, 128>(mv, Q, Ks, a, st) : launch_fma_mv<KF, 3, 64>(mv, Q, Ks, a, st);
}

size_t fma_smem_bytes(int nsplit, int dp, int bn, int mv) { return K1Layout(nsplit, dp, bn, mv).total + 1024; }

int fused_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, int nsplit,
                 const float* V, int m, int ldv, float* O, int ldo, int* status, cudaStream_t st) {
  if (Q.dp != Ks.dp) return fail(KOP_EINVAL, "fused_matvec: point sets of different widths");
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  if (m > 8 && nsplit == 2) return fused_matvec_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st);
  const int dp = Q.dp;
  int bn = 128;
  if (fma_smem_bytes(nsplit, dp, 128, 8) > smem_limit_bytes()) bn = 64;
  if (fma_smem_bytes(nsplit, dp, bn, 8) > smem_limit_bytes())
    return fail(KOP_EINVAL, "fused_matvec: feature width too large for the fused kernel");
  FusedArgs a;
  a.qnorm = Q.norms;
  a.knorm = Ks.norms;
  a.nq = (int)Q.n;
  a.nk = (int)Ks.n;
  a.ldv = ldv;
  a.ldo = ldo;
  a.dp = dp;
  a.row_bytes = dp >= 64 ? 128 : dp * 2;
  a.swz = swizzle_code(a.row_bytes);
  a.self = self ? 1 : 0;
  a.c0 = kc.c0;
  a.c1 = kc.c1;
  a.c2 = kc.c2;
  a.status = status;
  for (int c0 = 0; c0 < m; c0 += 8) {
    const int mc = (m - c0) < 8 ? (m - c0) : 8;
    const int mv = mc == 1 ? 1 : (mc <= 4 ? 4 : 8);
    a.V = V + c0;
    a.O = O + c0;
    a.m = mc;
    int rc;
    switch (kf) {
      case KF_RBF: rc = launch_fma_kf<KF_RBF>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_LAPLACE: rc = launch_fma_kf<KF_LAPLACE>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_MATERN: rc = launch_fma_kf<KF_MATERN>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_DRBF: rc = launch_fma_kf<KF_DRBF>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_DLAPLACE: rc = launch_fma_kf<KF_DLAPLACE>(nsplit, bn, mv, Q, Ks, a, st); break;
      default: rc = launch_fma_kf<KF_DMATERN>(nsplit, bn, mv, Q, Ks, a, st); break;
    }
    if (rc != KOP_OK) return rc;
  }
  return KOP_OK;
}

}  // namespace kop
