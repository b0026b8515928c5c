// Fused kernel-operator product O = k(Q, X) V on the tensor cores, for blocks
// of up to 8 vectors (the PCG iterations: m = 1 per right-hand side).
//
// This is the matrix-free operator of the paper (Sec. 4.3: the linear
// operator is applied without being formed; Sec. 2.1: K_ij = k(x_i, x_j), and
// every CG iteration costs one O(n^2) product).  Per 128-row block of Q a CTA
// streams tiles of 128 (or 64) points of X:
//   S  = Q_I X_J^T       tcgen05.mma on BF16 split operands, FP32 in TMEM
//   u  = s|q_i|^2 + s|x_j|^2 - 2 s S_ij     (s folds the bandwidth; see
//                                             kop_epilogue.cuh)
//   K  = k(u)            in registers (SFU ex2 / sqrt)
//   O += K V_J           FP32 FMAs, compensated running sum per output
// K never reaches global memory.  Warp roles: warp 0 issues all loads
// asynchronously (tensor-map TMA for the split operands, bulk copies for the
// scaled norms and V), warp 1 issues the MMAs, warp 2 owns TMEM, and NWG
// epilogue warpgroups (warps 4..) turn distances into kernel values and
// contract them with V, each warpgroup 64 columns of a tile: a tile of BN
// points is taken by a group of BN / 64 warpgroups, and the groups take
// alternate tiles.  One CTA per SM holds all of TMEM as 512 / BN S buffers
// (at most four), so the MMAs run ahead of the epilogue.  Two rings
// feed the pipeline: X tiles (warp 0), released as soon as their distance
// MMAs complete, and the tiles' scaled norms and V rows (warp 3), released by
// the epilogue.
#include "kop_device.cuh"
#include "kop_epilogue.cuh"
#include "kop_internal.h"
#include "kop_sdist.cuh"

namespace kop {

constexpr int K1_MAXST = 4;
// S buffers in TMEM for a tile width: as many as fit in 512 columns, at most four.
__host__ __device__ constexpr int k1_nsb(int bn) { return 512 / bn < 4 ? 512 / bn : 4; }
constexpr int K1_NKV = 4;  // slots of the norm / V ring

struct FusedArgs {
  const float* qnorm;  // scaled row norms of Q, padded to the 128-row grid
  const float* knorm;  // scaled row norms of X, padded
  const float* V;      // nk x MV floats (row stride MV), 16-byte aligned
  float* O;
  int nq, nk, m, ldo;
  int dp, row_bytes, swz, self, nst;
  int v_padded;        // V has nk_pad rows (else the last tile copies only nk - j0 rows)
  int nk_pad;          // rows of the padded X norms (a multiple of 128)
  float m2c, c2;       // -2 s, derivative factor
  int* status;
};

// Shared-memory layout (offsets from a 1024-byte aligned base).
struct K1Layout {
  uint32_t q_split, x_split, qs, xs, kn, vs, bars, holder, abort_word, red, total;
  __host__ __device__ K1Layout(int nsplit, int dp, int bn, int mv, int nst, int nwg) {
    q_split = 128u * dp * 2;
    x_split = (uint32_t)bn * dp * 2;
    qs = 0;
    xs = qs + nsplit * q_split;
    kn = xs + nst * nsplit * x_split;
    vs = kn + K1_NKV * bn * 4;
    bars = vs + K1_NKV * bn * mv * 4;
    holder = bars + (2 * K1_MAXST + 2 * K1_NKV + 2 * 4 + 2) * 8;
    abort_word = holder + 4;
    red = abort_word + 12;
    total = red + (nwg - 1) * 128 * mv * 2 * 4;
  }
};

// Warp-uniform bounded wait: every lane polls once (no divergent branch when
// the phase is already complete), then lane 0 polls and broadcasts.
KOP_DEV bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
// The same with back-off, for the producer and MMA warps.
KOP_DEV bool warp_wait_bg(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_backoff(bar, parity, abort_word, status);
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

// Epilogue over one 32-column chunk.  MASK: check the diagonal and the ragged
// tail per entry (only the tiles that need it take this path).  COMP: exact
// products and error-free sums per entry (TwoProduct + TwoSum into part /
// perr), used by the accurate mode so that the true residual is not limited by
// the rounding of FP32 partial sums.
template <int KF, int MV, bool MASK, bool COMP>
KOP_DEV void chunk_fma(const uint32_t (&r)[32], float qn, const float* __restrict__ kn, const float* __restrict__ v,
                       float m2c, float c2, int jbase, int gi, int nk, bool self, float (&part)[MV],
                       float (&perr)[MV]) {
  // stage 1: scaled squared distances (in place over the loaded S values)
  float kv[32];
#pragma unroll
  for (int j4 = 0; j4 < 32; j4 += 4) {
    const float4 k4 = *reinterpret_cast<const float4*>(kn + j4);
    kv[j4 + 0] = fmaf(__uint_as_float(r[j4 + 0]), m2c, qn + k4.x);
    kv[j4 + 1] = fmaf(__uint_as_float(r[j4 + 1]), m2c, qn + k4.y);
    kv[j4 + 2] = fmaf(__uint_as_float(r[j4 + 2]), m2c, qn + k4.z);
    kv[j4 + 3] = fmaf(__uint_as_float(r[j4 + 3]), m2c, qn + k4.w);
  }
  if constexpr (MASK) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      if (self && jbase + jj == gi) kv[jj] = 0.0f;
  }
  // stage 2: kernel values (independent SFU chains)
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) kv[jj] = kval_u<KF>(kv[jj], c2);
  if constexpr (MASK) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      if (jbase + jj >= nk) kv[jj] = 0.0f;
  }
  // stage 3: contraction with V
  if constexpr (MV == 1 && !COMP) {
    float p4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j4 = 0; j4 < 32; j4 += 4) {
      float4 v4 = *reinterpret_cast<const float4*>(v + j4);
      if constexpr (MASK) {
        if (jbase + j4 + 0 >= nk) v4.x = 0.0f;
        if (jbase + j4 + 1 >= nk) v4.y = 0.0f;
        if (jbase + j4 + 2 >= nk) v4.z = 0.0f;
        if (jbase + j4 + 3 >= nk) v4.w = 0.0f;
      }
      p4[0] = fmaf(kv[j4 + 0], v4.x, p4[0]);
      p4[1] = fmaf(kv[j4 + 1], v4.y, p4[1]);
      p4[2] = fmaf(kv[j4 + 2], v4.z, p4[2]);
      p4[3] = fmaf(kv[j4 + 3], v4.w, p4[3]);
    }
    part[0] += (p4[0] + p4[1]) + (p4[2] + p4[3]);
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      float vv[MV];
#pragma unroll
      for (int c4 = 0; c4 < MV; c4 += 4) {
        if constexpr (MV == 1) {
          vv[0] = v[jj];
        } else {
          const float4 v4 = *reinterpret_cast<const float4*>(v + jj * MV + c4);
          vv[c4] = v4.x;
          vv[c4 + 1] = v4.y;
          vv[c4 + 2] = v4.z;
          vv[c4 + 3] = v4.w;
        }
      }
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        float vc = vv[c];
        if constexpr (MASK) {
          if (jbase + jj >= nk) vc = 0.0f;
        }
        if constexpr (COMP) {
          const float p = kv[jj] * vc;
          const float pe = fmaf(kv[jj], vc, -p);
          const float t = part[c] + p;
          const float bb = t - part[c];
          perr[c] += ((part[c] - (t - bb)) + (p - bb)) + pe;
          part[c] = t;
        } else {
          part[c] = fmaf(kv[jj], vc, part[c]);
        }
      }
    }
  }
}

template <int KF, int NSPLIT, int MV, int BN, int NWG>
__global__ void __launch_bounds__(128 + 128 * NWG, 1)
    k1_fma_kernel(const __grid_constant__ CUtensorMap tq0, const __grid_constant__ CUtensorMap tq1,
                  const __grid_constant__ CUtensorMap tq2, const __grid_constant__ CUtensorMap tk0,
                  const __grid_constant__ CUtensorMap tk1, const __grid_constant__ CUtensorMap tk2,
                  const FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nst = a.nst;
  constexpr int NSB = k1_nsb(BN);
  constexpr int WPG = BN / 64;    // warpgroups per tile
  constexpr int G = NWG / WPG;    // tile groups
  static_assert(BN % 64 == 0 && NWG % WPG == 0 && G >= 1, "bad epilogue split");
  const K1Layout L(NSPLIT, a.dp, BN, MV, nst, NWG);
  uint8_t* qs = smem + L.qs;
  uint8_t* xs = smem + L.xs;
  float* kn = (float*)(smem + L.kn);
  float* vs = (float*)(smem + L.vs);
  uint64_t* bars = (uint64_t*)(smem + L.bars);
  uint64_t* full = bars;                     // X ring
  uint64_t* empty = bars + K1_MAXST;
  uint64_t* kvfull = bars + 2 * K1_MAXST;    // norm / V ring
  uint64_t* kvempty = kvfull + K1_NKV;
  uint64_t* tfull = kvempty + K1_NKV;
  uint64_t* tempty = tfull + NSB;
  uint64_t* qbar = tempty + NSB;
  uint64_t* drain = qbar + 1;
  uint32_t* holder = (uint32_t*)(smem + L.holder);
  volatile int* abort_word = (volatile int*)(smem + L.abort_word);
  float* red = (float*)(smem + L.red);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * 128;
  const int ntiles = (a.nk + BN - 1) / BN;
  // Each row block starts its sweep at its own tile, so that the CTAs resident
  // at one time read different tiles of X instead of all hitting the same L2
  // lines; tile_of maps the sweep index t to the tile it processes.
  const int toff = (int)(((int64_t)blockIdx.x * ntiles) / gridDim.x);
  auto tile_of = [&](int t) { return t + toff < ntiles ? t + toff : t + toff - ntiles; };
  const int rb = a.row_bytes;
  const int nsub = (a.dp * 2) / rb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < K1_NKV; ++s) {
      mbar_init(&kvfull[s], 1);
      mbar_init(&kvempty[s], 128 * WPG);
    }
    for (int b = 0; b < NSB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128 * WPG);
    }
    mbar_init(qbar, 1);
    mbar_init(drain, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(holder, NSB * BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ------------------------------------------------------------ X producer
    const CUtensorMap* mq[3] = {&tq0, &tq1, &tq2};
    const CUtensorMap* mk[3] = {&tk0, &tk1, &tk2};
    if (lane == 0) {
      mbar_arrive_expect_tx(qbar, NSPLIT * L.q_split);
      for (int sp = 0; sp < NSPLIT; ++sp)
        for (int ks = 0; ks < nsub; ++ks)
          tma_load_2d(qs + sp * L.q_split + ks * (128 * rb), mq[sp], qbar, ks * 64, row0);
    }
    int t = 0, s = 0;
    uint32_t ph = 0;
    for (; t < ntiles; ++t) {
      if (!warp_wait_bg(&empty[s], ph ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        const int j0 = tile_of(t) * BN;
        mbar_arrive_expect_tx(&full[s], NSPLIT * L.x_split);
        for (int sp = 0; sp < NSPLIT; ++sp)
          for (int ks = 0; ks < nsub; ++ks)
            tma_load_2d(xs + (s * NSPLIT + sp) * L.x_split + ks * (BN * rb), mk[sp], &full[s], ks * 64, j0);
      }
      __syncwarp();
      if (++s == nst) { s = 0; ph ^= 1u; }
    }
    if (t < ntiles && lane == 0) {
      // aborted: let the loads already issued land before the CTA exits
      for (int u = (t - nst > 0 ? t - nst : 0); u < t; ++u) drain_wait(&full[u % nst], (u / nst) & 1);
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------ norm / V producer
    int t = 0, s = 0;
    uint32_t ph = 0;
    for (; t < ntiles; ++t) {
      if (!warp_wait_bg(&kvempty[s], ph ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        const int j0 = tile_of(t) * BN;
        // a wide last tile may run past the padded rows: copy only what exists
        // (the rest of the slot is masked by the epilogue)
        const int rows_k = a.nk_pad - j0 < BN ? a.nk_pad - j0 : BN;
        const int lim_v = a.v_padded ? a.nk_pad : a.nk;
        const int rows_v = lim_v - j0 < BN ? lim_v - j0 : BN;
        const uint32_t vbytes = (uint32_t)rows_v * MV * 4;
        mbar_arrive_expect_tx(&kvfull[s], (uint32_t)rows_k * 4 + vbytes);
        bulk_load(kn + s * BN, a.knorm + j0, (uint32_t)rows_k * 4, &kvfull[s]);
        bulk_load(vs + s * BN * MV, a.V + (int64_t)j0 * MV, vbytes, &kvfull[s]);
      }
      __syncwarp();
      if (++s == K1_NKV) { s = 0; ph ^= 1u; }
    }
    if (t < ntiles && lane == 0)
      for (int u = (t - K1_NKV > 0 ? t - K1_NKV : 0); u < t; ++u) drain_wait(&kvfull[u % K1_NKV], (u / K1_NKV) & 1);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // The loop adds constant offsets to descriptors prepared here (one MMA
    // must issue faster than the tensor pipe runs it); ring slot and phase are
    // counters.
    const uint32_t idesc = idesc_bf16_f32(128, BN);
    const uint32_t sbo = 8u * rb;
    const int nks = a.dp / 16;  // K steps of 16 over the padded feature width
    const uint64_t dq0 = sdesc(smem_u32(qs), sbo, a.swz);
    const uint64_t dx0 = sdesc(smem_u32(xs), sbo, a.swz);
    const uint32_t q_split16 = L.q_split >> 4, x_split16 = L.x_split >> 4;
    const uint32_t q_sub16 = (128u * rb) >> 4, x_sub16 = ((uint32_t)BN * rb) >> 4;
    bool ok = warp_wait(qbar, 0, abort_word, a.status);
    int s = 0;
    uint32_t ph = 0;
    for (int t = 0; ok && t < ntiles; ++t) {
      const int b = t % NSB;
      const uint32_t bph = (t / NSB) & 1;
      if (!warp_wait(&full[s], ph, abort_word, a.status)) break;
      if (!warp_wait(&tempty[b], bph ^ 1, abort_word, a.status)) break;
      tc_fence_after();
      {
        const uint32_t d = tmem + b * BN;
        const uint64_t xb = dx0 + (uint64_t)(s * NSPLIT) * x_split16;
        switch (nks) {
          case 1: issue_s_tile<NSPLIT, 1, true>(d, dq0, xb, q_split16, x_split16, q_sub16, x_sub16, idesc); break;
          case 2: issue_s_tile<NSPLIT, 2, true>(d, dq0, xb, q_split16, x_split16, q_sub16, x_sub16, idesc); break;
          case 4: issue_s_tile<NSPLIT, 4, true>(d, dq0, xb, q_split16, x_split16, q_sub16, x_sub16, idesc); break;
          default: issue_s_tile<NSPLIT, 8, true>(d, dq0, xb, q_split16, x_split16, q_sub16, x_sub16, idesc); break;
        }
        if (lane == 0) {
          tc_commit(&tfull[b]);
          tc_commit(&empty[s]);
        }
      }
      __syncwarp();
      if (++s == nst) { s = 0; ph ^= 1u; }
    }
    if (lane == 0) {
      tc_commit(drain);
      drain_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int wgi = (warp - 4) >> 2, grp = wgi / WPG, wg = wgi - grp * WPG, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gi = row0 + row;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    constexpr int NCH = 2;  // 32-column chunks per warpgroup
    const float qn = a.qnorm[gi];
    const bool self = a.self != 0;
    float acc_s[MV], acc_e[MV];
#pragma unroll
    for (int c = 0; c < MV; ++c) acc_s[c] = acc_e[c] = 0.0f;
    for (int t = grp; t < ntiles; t += G) {
      const int b = t % NSB;
      const uint32_t bph = (t / NSB) & 1;
      const int s = t % K1_NKV;
      const uint32_t ph = (t / K1_NKV) & 1;
      if (!warp_wait(&tfull[b], bph, abort_word, a.status)) break;
      tc_fence_after();
      if (!warp_wait(&kvfull[s], ph, abort_word, a.status)) break;
      const int j0 = tile_of(t) * BN;
      const bool mask = (self && j0 < row0 + 128 && j0 + BN > row0) || (j0 + BN > a.nk);
      constexpr bool COMP = NSPLIT == 3;
      float part[MV], perr[MV];
#pragma unroll
      for (int c = 0; c < MV; ++c) part[c] = perr[c] = 0.0f;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        const int col = wg * 64 + ch * 32;
        uint32_t r[32];
        tmem_ld32(lane_addr + b * BN + col, r);
        tmem_ld_wait(r);
        const float* knS = kn + s * BN + col;
        const float* vS = vs + (s * BN + col) * MV;
        if (mask)
          chunk_fma<KF, MV, true, COMP>(r, qn, knS, vS, a.m2c, a.c2, j0 + col, gi, a.nk, self, part, perr);
        else
          chunk_fma<KF, MV, false, COMP>(r, qn, knS, vS, a.m2c, a.c2, j0 + col, gi, a.nk, self, part, perr);
      }
      tc_fence_before();
      mbar_arrive(&tempty[b]);
      mbar_arrive(&kvempty[s]);
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        two_sum_acc(acc_s[c], acc_e[c], part[c]);
        acc_e[c] += perr[c];
      }
    }
    // combine the NWG partial sums of each row: all warpgroups but the first
    // leave theirs in shared memory
    const int contrib = wgi;
    if (contrib > 0) {
      float* rd = red + (size_t)(contrib - 1) * 128 * MV * 2;
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        rd[(row * MV + c) * 2] = acc_s[c];
        rd[(row * MV + c) * 2 + 1] = acc_e[c];
      }
    }
    named_bar_sync(1, 128 * NWG);
    if (contrib == 0 && gi < a.nq && !*abort_word) {
#pragma unroll
      for (int c = 0; c < MV; ++c) {
        if (c < a.m) {
          float hi = acc_s[c], lo = acc_e[c];
          for (int k = 0; k < NWG - 1; ++k) {
            const float* rd = red + (size_t)k * 128 * MV * 2;
            two_sum_acc(hi, lo, rd[(row * MV + c) * 2]);
            lo += rd[(row * MV + c) * 2 + 1];
          }
          a.O[(int64_t)gi * a.ldo + c] = hi + lo;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, NSB * BN);
  }
}

// V (n x m, ld ldv) -> padded n_pad x mv block (zero rows / columns).
__global__ void vpad_kernel(const float* __restrict__ V, int64_t n, int m, int ldv, int64_t n_pad, int mv,
                            float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pad * mv) return;
  const int64_t i = t / mv;
  const int c = (int)(t - i * mv);
  out[t] = (i < n && c < m) ? V[i * ldv + c] : 0.0f;
}

// ---------------------------------------------------------------- host side
static int swizzle_code(int row_bytes) { return row_bytes == 128 ? 2 : (row_bytes == 64 ? 4 : 6); }

// Epilogue warpgroups: four where the epilogue's registers allow 640 threads,
// else two.
constexpr int fma_wgs(int nsplit, int mv) { return (nsplit == 2 && mv <= 4) ? 4 : 2; }

size_t fma_smem_bytes(int nsplit, int dp, int bn, int mv, int nst) {
  return K1Layout(nsplit, dp, bn, mv, nst, fma_wgs(nsplit, mv)).total + 1024;
}

template <int KF, int NSPLIT, int MV, int BN>
static int launch_fma_t(const PointSet& Q, const PointSet& Ks, const FusedArgs& a, cudaStream_t st) {
  constexpr int NWG = fma_wgs(NSPLIT, MV);
  if constexpr (BN / 64 > NWG) {
    return fail(KOP_EINVAL, "fused_matvec: tile too wide for the epilogue");
  } else {
    auto kern = k1_fma_kernel<KF, NSPLIT, MV, BN, NWG>;
    size_t smem = fma_smem_bytes(NSPLIT, a.dp, BN, MV, a.nst);
    // one CTA per SM: it allocates all of TMEM
    const size_t one_per_sm = smem_limit_bytes() / 2 + 4096;
    if (smem < one_per_sm) smem = one_per_sm;
    static bool attr_set = false;
    if (!attr_set) {
      KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
      KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      attr_set = true;
    }
    // Q in boxes of 128 rows, X in boxes of BN rows
    const int bi = BN == 128 ? 0 : 1;
    dim3 grid((unsigned)((a.nq + 127) / 128));
    kern<<<grid, 128 + 128 * NWG, smem, st>>>(Q.tm[0][0], Q.tm[1][0], Q.tm[2][0], Ks.tm[0][bi], Ks.tm[1][bi],
                                              Ks.tm[2][bi], a);
    KOP_LAUNCHED();
    return KOP_OK;
  }
}

template <int KF, int NSPLIT, int BN>
static int launch_fma_mv(int mv, const PointSet& Q, const PointSet& Ks, const FusedArgs& a, cudaStream_t st) {
  if (mv == 1) return launch_fma_t<KF, NSPLIT, 1, BN>(Q, Ks, a, st);
  if (mv == 4) return launch_fma_t<KF, NSPLIT, 4, BN>(Q, Ks, a, st);
  return launch_fma_t<KF, NSPLIT, 8, BN>(Q, Ks, a, st);
}

template <int KF, int NSPLIT>
static int launch_fma_bn(int bn, int mv, const PointSet& Q, const PointSet& Ks, const FusedArgs& a,
                         cudaStream_t st) {
  if (bn == 128) return launch_fma_mv<KF, NSPLIT, 128>(mv, Q, Ks, a, st);
  return launch_fma_mv<KF, NSPLIT, 64>(mv, Q, Ks, a, st);
}

template <int KF>
static int launch_fma_kf(int nsplit, int bn, int mv, const PointSet& Q, const PointSet& Ks, const FusedArgs& a,
                         cudaStream_t st) {
  if (nsplit == 2) return launch_fma_bn<KF, 2>(bn, mv, Q, Ks, a, st);
  return launch_fma_bn<KF, 3>(bn, mv, Q, Ks, a, st);
}

int fused_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, int nsplit,
                 const float* V, int m, int ldv, float* O, int ldo, int* status, cudaStream_t st, bool sketch) {
  if (Q.dp != Ks.dp) return fail(KOP_EINVAL, "fused_matvec: point sets of different widths");
  if (Q.n == 0 || Ks.n == 0 || m == 0) return KOP_OK;
  if (m > 8 && nsplit == 2)
    return fused_matvec_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st, sketch);
  const int dp = Q.dp;
  const size_t lim = smem_limit_bytes();
  // tile width: 128 points where a 2-stage X ring fits, else 64.  (256-point
  // tiles leave two S buffers, and measured slower: with the epilogue busy on
  // the special-function units the distance MMAs of the next tile arrive late.)
  auto width_for = [&](int mv) { return fma_smem_bytes(nsplit, dp, 128, mv, 2) <= lim ? 128 : 64; };
  if (fma_smem_bytes(nsplit, dp, 64, 8, 2) > lim)
    return fail(KOP_EINVAL, "fused_matvec: feature width too large for the fused kernel");
  // X ring depth: the deepest that fits (one CTA per SM)
  auto stages_for = [&](int bn, int mv) {
    int nst = 2;
    while (nst < K1_MAXST && fma_smem_bytes(nsplit, dp, bn, mv, nst + 1) <= lim) ++nst;
    return nst;
  };
  int rc = ensure_scaled_norms(const_cast<PointSet&>(Q), kc.scale, st);
  if (rc == KOP_OK && &Q != &Ks) rc = ensure_scaled_norms(const_cast<PointSet&>(Ks), kc.scale, st);
  if (rc) return rc;
  if (self && &Q == &Ks && m == 1 && nsplit == 2) {
    // one vector with the point set itself: each pair of row blocks once
    if (ldv == 1 && ((uintptr_t)V % 16 == 0) && (Ks.n % 4 == 0))
      return fused_matvec_sym(const_cast<PointSet&>(Q), kf, kc, V, 0, O, status, st);
    float* vp = nullptr;
    KOP_CUDA_TRY(cudaMallocAsync((void**)&vp, sizeof(float) * Ks.n_pad, st));
    vpad_kernel<<<(unsigned)((Ks.n_pad + 255) / 256), 256, 0, st>>>(V, Ks.n, 1, ldv, Ks.n_pad, 1, vp);
    KOP_LAUNCHED();
    rc = fused_matvec_sym(const_cast<PointSet&>(Q), kf, kc, vp, 1, O, status, st);
    cudaFreeAsync(vp, st);
    return rc;
  }
  FusedArgs a;
  a.qnorm = Q.snorm;
  a.knorm = Ks.snorm;
  a.nq = (int)Q.n;
  a.nk = (int)Ks.n;
  a.nk_pad = (int)Ks.n_pad;
  a.ldo = ldo;
  a.dp = dp;
  a.row_bytes = dp >= 64 ? 128 : dp * 2;
  a.swz = swizzle_code(a.row_bytes);
  a.self = self ? 1 : 0;
  a.m2c = -2.0f * kc.scale;
  a.c2 = kc.c2;
  a.status = status;
  float* vpad = nullptr;
  for (int c0 = 0; c0 < m && rc == KOP_OK; c0 += 8) {
    const int mc = (m - c0) < 8 ? (m - c0) : 8;
    const int mv = mc == 1 ? 1 : (mc <= 4 ? 4 : 8);
    const int bn = width_for(mv);
    a.nst = stages_for(bn, mv);
    // V is read with bulk copies: used in place when its rows are exactly mv
    // floats and 16-byte aligned, else staged in a padded copy
    const bool direct = (mc == mv) && (ldv == mv) && (c0 == 0) && ((uintptr_t)V % 16 == 0) &&
                        (((int64_t)Ks.n * mv * 4) % 16 == 0);
    if (direct) {
      a.V = V;
      a.v_padded = 0;
    } else {
      if (!vpad) {
        cudaError_t e = cudaMallocAsync((void**)&vpad, sizeof(float) * Ks.n_pad * 8, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused_matvec: V staging");
      }
      const int64_t tot = Ks.n_pad * mv;
      vpad_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(V + c0, Ks.n, mc, ldv, Ks.n_pad, mv, vpad);
      KOP_LAUNCHED();
      a.V = vpad;
      a.v_padded = 1;
    }
    a.O = O + c0;
    a.m = mc;
    switch (kf) {
      case KF_RBF: rc = launch_fma_kf<KF_RBF>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_LAPLACE: rc = launch_fma_kf<KF_LAPLACE>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_MATERN: rc = launch_fma_kf<KF_MATERN>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_DRBF: rc = launch_fma_kf<KF_DRBF>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_DLAPLACE: rc = launch_fma_kf<KF_DLAPLACE>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_GRBF: rc = launch_fma_kf<KF_GRBF>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_GLAPLACE: rc = launch_fma_kf<KF_GLAPLACE>(nsplit, bn, mv, Q, Ks, a, st); break;
      case KF_GMATERN: rc = launch_fma_kf<KF_GMATERN>(nsplit, bn, mv, Q, Ks, a, st); break;
      default: rc = launch_fma_kf<KF_DMATERN>(nsplit, bn, mv, Q, Ks, a, st); break;
    }
  }
  if (vpad) cudaFreeAsync(vpad, st);
  return rc;
}

}  // namespace kop
