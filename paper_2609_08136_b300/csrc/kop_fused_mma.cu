// Fused kernel-operator product for blocks of many vectors (m > 8): the
// contraction O += K_IJ V_J runs on the tensor cores as well.
//
// Same product as kop_fused.cu (the paper's matrix-free operator, Sec. 4.3;
// the sketch Y = K Omega of the Nystrom preconditioner is this product with
// m = r), but after the epilogue has turned the distance tile S into kernel
// values K_IJ in registers, it writes them back into the same TMEM columns as
// a BF16 hi/lo pair (K = hi + lo to about 2^-16), and one thread issues
//   O += K_lo V_hi + K_hi V_lo + K_hi V_hi
// with A read from TMEM and V^T (split into BF16 hi/lo by a prep kernel) read
// from shared memory.  O (128 rows x MC columns, FP32) stays in TMEM for the
// whole sweep over X and is written once at the end.  Tiles of 64 points.
#include "kop_device.cuh"
#include "kop_epilogue.cuh"
#include "kop_internal.h"

namespace kop {

constexpr int K3_THREADS = 384;
constexpr int K3_NST = 2;
constexpr int K3_BN = 64;

struct MmaArgs {
  const float* qnorm;
  const float* knorm;
  float* O;
  int nq, nk, m, ldo;
  int dp, row_bytes, swz, self, mc, tcols;
  float m2c, c2;
  int* status;
};

struct K3Layout {
  uint32_t q_split, x_split, v_split, qs, xs, vs, kn, bars, holder, abort_word, total;
  __host__ __device__ K3Layout(int dp, int mc) {
    q_split = 128u * dp * 2;
    x_split = (uint32_t)K3_BN * dp * 2;
    v_split = (uint32_t)mc * K3_BN * 2;
    qs = 0;
    xs = qs + 2 * q_split;
    vs = xs + K3_NST * 2 * x_split;
    kn = vs + K3_NST * 2 * v_split;
    bars = kn + K3_NST * K3_BN * 4;
    holder = bars + (3 * K3_NST + 8) * 8;
    abort_word = holder + 4;
    total = abort_word + 12;
  }
};

KOP_DEV bool warp_wait3(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

KOP_DEV void drain_wait3(uint64_t* bar, uint32_t parity) {
  uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > KOP_WAIT_LIMIT_NS) break;
  }
}

KOP_DEV uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);  // .x = lo_elem in the low half
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int KF>
__global__ void __launch_bounds__(K3_THREADS, 1)
    k1_mma_kernel(const __grid_constant__ CUtensorMap tq0, const __grid_constant__ CUtensorMap tq1,
                  const __grid_constant__ CUtensorMap tk0, const __grid_constant__ CUtensorMap tk1,
                  const __grid_constant__ CUtensorMap tv0, const __grid_constant__ CUtensorMap tv1,
                  const MmaArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const K3Layout L(a.dp, a.mc);
  uint8_t* qs = smem + L.qs;
  uint8_t* xs = smem + L.xs;
  uint8_t* vs = smem + L.vs;
  float* kn = (float*)(smem + L.kn);
  uint64_t* bars = (uint64_t*)(smem + L.bars);
  uint64_t* full = bars;                 // K3_NST
  uint64_t* empty = bars + K3_NST;       // K3_NST
  uint64_t* sfull = bars + 2 * K3_NST;   // 2
  uint64_t* pfull = sfull + 2;           // 2
  uint64_t* sfree = pfull + 2;           // 2
  uint64_t* qbar = sfree + 2;
  uint64_t* ofull = qbar + 1;
  uint64_t* drain = ofull + 1;
  uint32_t* holder = (uint32_t*)(smem + L.holder);
  volatile int* abort_word = (volatile int*)(smem + L.abort_word);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * 128;
  const int m0 = blockIdx.y * a.mc;
  const int ntiles = (a.nk + K3_BN - 1) / K3_BN;
  const int rb = a.row_bytes;
  const int nsub = (a.dp * 2) / rb;
  const uint32_t OCOL = 2 * K3_BN;  // O accumulator columns start after the two S buffers

  if (threadIdx.x == 0) {
    for (int s = 0; s < K3_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + 256);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&pfull[b], 256);
      mbar_init(&sfree[b], 1);
    }
    mbar_init(qbar, 1);
    mbar_init(ofull, 1);
    mbar_init(drain, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(holder, a.tcols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    const CUtensorMap* mq[2] = {&tq0, &tq1};
    const CUtensorMap* mk[2] = {&tk0, &tk1};
    const CUtensorMap* mvv[2] = {&tv0, &tv1};
    if (lane == 0) {
      mbar_arrive_expect_tx(qbar, 2 * L.q_split);
      for (int sp = 0; sp < 2; ++sp)
        for (int ks = 0; ks < nsub; ++ks)
          for (int rr = 0; rr < 128 / K3_BN; ++rr)
            tma_load_2d(qs + sp * L.q_split + ks * (128 * rb) + rr * (K3_BN * rb), mq[sp], qbar, ks * 64,
                        row0 + rr * K3_BN);
    }
    int t = 0;
    for (; t < ntiles; ++t) {
      const int s = t % K3_NST;
      const uint32_t ph = (t / K3_NST) & 1;
      if (!warp_wait3(&empty[s], ph ^ 1, abort_word, a.status)) break;
      const int j0 = t * K3_BN;
      for (int i = lane; i < K3_BN; i += 32) kn[s * K3_BN + i] = a.knorm[j0 + i];
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], 2 * L.x_split + 2 * L.v_split);
        for (int sp = 0; sp < 2; ++sp) {
          for (int ks = 0; ks < nsub; ++ks)
            tma_load_2d(xs + (s * 2 + sp) * L.x_split + ks * (K3_BN * rb), mk[sp], &full[s], ks * 64, j0);
          tma_load_2d(vs + (s * 2 + sp) * L.v_split, mvv[sp], &full[s], j0, m0);
        }
      }
      __syncwarp();
    }
    if (t < ntiles && lane == 0) {
      for (int u = (t - K3_NST > 0 ? t - K3_NST : 0); u < t; ++u) drain_wait3(&full[u % K3_NST], (u / K3_NST) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc_s = idesc_bf16_f32(128, K3_BN);
    const uint32_t idesc_o = idesc_bf16_f32(128, a.mc);
    const uint32_t sbo = 8u * rb;
    const int steps_per_sub = rb / 32;
    bool ok = warp_wait3(qbar, 0, abort_word, a.status);
    uint32_t oacc = 0;
    for (int t = 0; ok && t <= ntiles; ++t) {
      if (t < ntiles) {
        const int s = t % K3_NST;
        const uint32_t ph = (t / K3_NST) & 1;
        const int b = t & 1;
        const uint32_t bph = (t >> 1) & 1;
        if (!warp_wait3(&full[s], ph, abort_word, a.status)) break;
        if (!warp_wait3(&sfree[b], bph ^ 1, abort_word, a.status)) break;
        tc_fence_after();
        if (lane == 0) {
          const uint32_t d = tmem + b * K3_BN;
          uint32_t acc = 0;
#pragma unroll
          for (int term = 0; term < 3; ++term) {
            const int ta = term == 1 ? 1 : 0, tb = term == 0 ? 1 : 0;  // hi*mid, mid*hi, hi*hi
            const uint32_t abase = smem_u32(qs + ta * L.q_split);
            const uint32_t bbase = smem_u32(xs + (s * 2 + tb) * L.x_split);
            for (int kc = 0; kc < a.dp / 16; ++kc) {
              const int ks = kc / steps_per_sub, w = kc - ks * steps_per_sub;
              tc_mma_ss(d, sdesc(abase + ks * (128 * rb) + w * 32, sbo, a.swz),
                        sdesc(bbase + ks * (K3_BN * rb) + w * 32, sbo, a.swz), idesc_s, acc);
              acc = 1;
            }
          }
          tc_commit(&sfull[b]);
        }
        __syncwarp();
      }
      if (t >= 1) {
        const int u = t - 1;
        const int s = u % K3_NST;
        const int b = u & 1;
        const uint32_t bph = (u >> 1) & 1;
        if (!warp_wait3(&pfull[b], bph, abort_word, a.status)) break;
        tc_fence_after();
        if (lane == 0) {
          const uint32_t pbase = tmem + b * K3_BN;
#pragma unroll
          for (int term = 0; term < 3; ++term) {
            // (P split, V split): lo*hi, hi*lo, hi*hi; P hi at +0, lo at +16 within each 32-column chunk
            const uint32_t poff = term == 0 ? 16u : 0u;
            const int vsp = term == 1 ? 1 : 0;
            const uint32_t vbase = smem_u32(vs + (s * 2 + vsp) * L.v_split);
#pragma unroll
            for (int kk = 0; kk < K3_BN / 16; ++kk) {
              const uint32_t acol = pbase + 32u * (kk >> 1) + 8u * (kk & 1) + poff;
              tc_mma_ts(tmem + OCOL, acol, sdesc(vbase + kk * 32, 1024u, 2u), idesc_o, oacc);
              oacc = 1;
            }
          }
          tc_commit(&sfree[b]);
          tc_commit(&empty[s]);
        }
        __syncwarp();
      }
    }
    if (lane == 0) {
      tc_commit(ofull);
      tc_commit(drain);
      drain_wait3(drain, 0);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int ep = warp - 4, wg = ep >> 2, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gi = row0 + row;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    bool ok = warp_wait3(qbar, 0, abort_word, a.status);
    const float qni = a.qnorm[gi];
    for (int t = 0; ok && t < ntiles; ++t) {
      const int s = t % K3_NST;
      const uint32_t ph = (t / K3_NST) & 1;
      const int b = t & 1;
      const uint32_t bph = (t >> 1) & 1;
      if (!warp_wait3(&sfull[b], bph, abort_word, a.status)) { ok = false; break; }
      tc_fence_after();
      uint32_t r[32];
      const uint32_t col = b * K3_BN + wg * 32;
      tmem_ld32(lane_addr + col, r);
      tmem_ld_wait(r);
      if (!warp_wait3(&full[s], ph, abort_word, a.status)) { ok = false; break; }
      const float* knS = kn + s * K3_BN + wg * 32;
      const int jbase = t * K3_BN + wg * 32;
      float kv[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        float u = fmaf(__uint_as_float(r[jj]), a.m2c, qni + knS[jj]);
        if (a.self && jbase + jj == gi) u = 0.0f;
        kv[jj] = (jbase + jj < a.nk) ? kval_u<KF>(u, a.c2) : 0.0f;
      }
      mbar_arrive(&empty[s]);
      uint32_t ph16[16], pl16[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float k0 = kv[2 * e], k1 = kv[2 * e + 1];
        const __nv_bfloat16 h0 = __float2bfloat16_rn(k0), h1 = __float2bfloat16_rn(k1);
        ph16[e] = pack_bf16x2(__bfloat162float(h0), __bfloat162float(h1));
        pl16[e] = pack_bf16x2(k0 - __bfloat162float(h0), k1 - __bfloat162float(h1));
      }
      tmem_st16(lane_addr + col, ph16);
      tmem_st16(lane_addr + col + 16, pl16);
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&pfull[b]);
    }
    // write out O: each warpgroup half of the MC columns, 32 at a time
    if (ok && warp_wait3(ofull, 0, abort_word, a.status)) {
      tc_fence_after();
      const int half = a.mc / 2;
      for (int c0 = wg * half; c0 < (wg + 1) * half; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(lane_addr + OCOL + c0, r);
        tmem_ld_wait(r);
        if (gi < a.nq && !*abort_word) {
          float* orow = a.O + (int64_t)gi * a.ldo + m0 + c0;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (m0 + c0 + c < a.m) orow[c] = __uint_as_float(r[c]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tcols);
  }
}

// V (nk x m, ld ldv, FP32) -> V^T split into BF16 hi and lo, each m_pad x nk_pad
// (row c holds column c of V), zero padded.
__global__ void vsplit_kernel(const float* __restrict__ V, int nk, int m, int ldv, int nk_pad, int m_pad,
                              __nv_bfloat16* __restrict__ vh, __nv_bfloat16* __restrict__ vl) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (j < nk && c < m) ? V[(int64_t)j * ldv + c] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, j = j0 + threadIdx.x;
    if (c < m_pad && j < nk_pad) {
      const float v = tile[threadIdx.x][r];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      vh[(int64_t)c * nk_pad + j] = h;
      vl[(int64_t)c * nk_pad + j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

size_t mma_smem_bytes(int dp, int mc) { return K3Layout(dp, mc).total + 1024; }

// Column chunk per CTA: a multiple of 64 (each epilogue warpgroup writes out
// half of it, 32 columns at a time), at most 256 (MMA N limit), the widest
// whose pipeline fits in shared memory, then narrowed to balance the chunks.
int mma_chunk(int dp, int m) {
  const int mpad = ((m + 63) / 64) * 64;
  int mc = mpad < 256 ? mpad : 256;
  while (mc > 64 && mma_smem_bytes(dp, mc) > smem_limit_bytes()) mc -= 64;
  if (mma_smem_bytes(dp, mc) > smem_limit_bytes()) return 0;
  const int nch = (mpad + mc - 1) / mc;
  const int w = ((mpad / nch + 63) / 64) * 64;
  return w < mc ? w : mc;
}

template <int KF>
static int launch_mma_t(const PointSet& Q, const PointSet& Ks, const CUtensorMap* tv, const MmaArgs& a,
                        cudaStream_t st) {
  auto kern = k1_mma_kernel<KF>;
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    attr_set = true;
  }
  dim3 grid((unsigned)((a.nq + 127) / 128), (unsigned)((a.m + a.mc - 1) / a.mc));
  kern<<<grid, K3_THREADS, mma_smem_bytes(a.dp, a.mc), st>>>(Q.tm[0][1], Q.tm[1][1], Ks.tm[0][1], Ks.tm[1][1],
                                                              tv[0], tv[1], a);
  KOP_LAUNCHED();
  return KOP_OK;
}

int fused_matvec_mma(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, const float* V,
                     int m, int ldv, float* O, int ldo, int* status, cudaStream_t st) {
  const int mc = mma_chunk(Q.dp, m);
  if (mc == 0) return fail(KOP_EINVAL, "fused_matvec_mma: feature width too large");
  {
    int sc = ensure_scaled_norms(const_cast<PointSet&>(Q), kc.scale, st);
    if (sc == KOP_OK && &Q != &Ks) sc = ensure_scaled_norms(const_cast<PointSet&>(Ks), kc.scale, st);
    if (sc) return sc;
  }
  const int nch = (m + mc - 1) / mc;
  const int m_pad = nch * mc;
  const int64_t nk_pad = Ks.n_pad;
  __nv_bfloat16* vsplit = nullptr;
  KOP_CUDA_TRY(cudaMallocAsync((void**)&vsplit, (size_t)2 * m_pad * nk_pad * 2, st));
  __nv_bfloat16* vh = vsplit;
  __nv_bfloat16* vl = vsplit + (size_t)m_pad * nk_pad;
  dim3 vb(32, 8), vg((unsigned)(nk_pad / 32), (unsigned)((m_pad + 31) / 32));
  vsplit_kernel<<<vg, vb, 0, st>>>(V, (int)Ks.n, m, ldv, (int)nk_pad, m_pad, vh, vl);
  cudaError_t e = cudaGetLastError();
  int rc = e == cudaSuccess ? KOP_OK : cuda_fail(e, "vsplit_kernel");
  CUtensorMap tv[2];
  if (rc == KOP_OK) rc = encode_tmap_bf16(&tv[0], vh, m_pad, (int)nk_pad, 64, mc);
  if (rc == KOP_OK) rc = encode_tmap_bf16(&tv[1], vl, m_pad, (int)nk_pad, 64, mc);
  if (rc == KOP_OK) {
    MmaArgs a;
    a.qnorm = Q.snorm;
    a.knorm = Ks.snorm;
    a.O = O;
    a.nq = (int)Q.n;
    a.nk = (int)Ks.n;
    a.m = m;
    a.ldo = ldo;
    a.dp = Q.dp;
    a.row_bytes = Q.dp >= 64 ? 128 : Q.dp * 2;
    a.swz = a.row_bytes == 128 ? 2 : (a.row_bytes == 64 ? 4 : 6);
    a.self = self ? 1 : 0;
    a.mc = mc;
    a.tcols = (2 * K3_BN + mc) <= 256 ? 256 : 512;
    a.m2c = -2.0f * kc.scale;
    a.c2 = kc.c2;
    a.status = status;
    switch (kf) {
      case KF_RBF: rc = launch_mma_t<KF_RBF>(Q, Ks, tv, a, st); break;
      case KF_LAPLACE: rc = launch_mma_t<KF_LAPLACE>(Q, Ks, tv, a, st); break;
      case KF_MATERN: rc = launch_mma_t<KF_MATERN>(Q, Ks, tv, a, st); break;
      case KF_DRBF: rc = launch_mma_t<KF_DRBF>(Q, Ks, tv, a, st); break;
      case KF_DLAPLACE: rc = launch_mma_t<KF_DLAPLACE>(Q, Ks, tv, a, st); break;
      default: rc = launch_mma_t<KF_DMATERN>(Q, Ks, tv, a, st); break;
    }
  }
  cudaFreeAsync(vsplit, st);
  return rc;
}

}  // namespace kop
