// Fused kernel-operator product O = K(X, X) v for one vector, using the
// symmetry of K: the PCG product of every iteration (the paper's O(n^2)
// matrix-free operator, Sec. 4.3; K_ij = k(x_i, x_j) = K_ji, Sec. 2.1).
//
// The row blocks of 128 points form nb tiles.  Each unordered pair of blocks
// {I, J} is evaluated once: CTA I takes the tiles J = I + t (mod nb),
// t = 0 .. cnt_I - 1, with cnt_I = floor(nb / 2) + 1 (when nb is even the
// blocks I >= nb / 2 take one tile fewer, so that the pairs at distance nb / 2
// are not taken twice).  For a tile the MMA computes the distances in the
// transposed orientation, D = X_J Q_I^T (TMEM lane = key j of J, column =
// query i of I), so that each epilogue thread owns one key j and 32 query
// columns i, and both contributions of the entry K_ij are thread-local sums:
//   row part     acc_i += K_ij v_j   (the query rows I; 32 registers kept
//                                      over the whole sweep)
//   column part  col_j += K_ij v_i   (the key rows J; one value per tile)
// The four epilogue warpgroups take 32 query columns each; per tile a
// combining warp adds their column parts in a fixed order and stores them to
// a scratch slot C[J][t - 1] (128 floats).  After the sweep the 128 key-slot partials of
// every query row are summed (error-free sums) and written to O, and a second
// kernel adds the column parts of every row block in a fixed order.  The
// diagonal tile (t = 0) contributes its row part only.  The result is
// deterministic.  Compared with the plain fused product the kernel values
// (one sqrt and one ex2 per Laplace entry on the special-function unit, which
// bounds the single-vector product) and the distance MMAs are halved.
#include "kop_device.cuh"
#include "kop_epilogue.cuh"
#include "kop_internal.h"
#include "kop_sdist.cuh"

namespace kop {

constexpr int KS_MAXST = 4;  // X ring depth at most
constexpr int KS_NSB = 4;    // S buffers of 128 TMEM columns
constexpr int KS_NKV = 4;    // norm / v ring slots
static_assert(KS_NKV == KS_NSB, "a key slot is released together with its S buffer");
constexpr int KS_NWG = 4;    // epilogue warpgroups
constexpr int KS_WCOLS = 128 / KS_NWG;  // query columns per warpgroup
constexpr int KS_NCX = 4;    // slots of the column-part ring
constexpr int KS_THREADS = 128 + 128 * KS_NWG;
// arrivals per phase on the barriers the epilogue releases: one per warp
// (lane 0, after the warp's reads or writes)
constexpr int KS_ARRIVALS = 4 * KS_NWG;

struct SymArgs {
  const float* snorm;  // scaled row norms, n_pad
  const float* V;      // the vector: n floats (or n_pad when v_padded), 16-byte aligned
  float* O;            // n: the result
  float* C;            // column parts: nb x h x 128
  int n, n_pad, nb, h;
  int dp, row_bytes, swz, nst;
  int v_padded;
  float m2c, c2;
  int* status;
};

// The final reduction of the row parts reuses the Q and X operand area:
// KS_NWG x 128 key slots x (KS_WCOLS + 1) floats.
__host__ __device__ constexpr uint32_t ks_red_bytes() { return (uint32_t)KS_NWG * 128 * (KS_WCOLS + 1) * 4; }

struct KSLayout {
  uint32_t q_split, x_split, qs, xs, kn, vk, qn, vq, colx, bars, holder, abort_word, total;
  __host__ __device__ KSLayout(int nsplit, int dp, int nst) {
    q_split = 128u * dp * 2;
    x_split = 128u * dp * 2;
    qs = 0;
    xs = qs + nsplit * q_split;
    kn = xs + nst * nsplit * x_split;
    if (kn < ks_red_bytes()) kn = ks_red_bytes();  // the reduction area stays clear of the rest
    vk = kn + KS_NKV * 128 * 4;
    qn = vk + KS_NKV * 128 * 4;
    vq = qn + 128 * 4;
    colx = vq + 128 * 4;                  // [KS_NCX][KS_NWG][128] column parts
    bars = colx + KS_NCX * KS_NWG * 128 * 4;
    holder = bars + (2 * KS_MAXST + KS_NKV + 2 * KS_NSB + 2 * KS_NCX + 2) * 8;
    abort_word = holder + 4;
    total = abort_word + 4;
  }
};

// Warp-uniform bounded wait of the epilogue warps; the common case (the phase
// has completed) costs one try_wait and one vote; a warp that has run ahead
// of the others backs off instead of taking issue slots from them.
KOP_DEV bool ks_wait(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_backoff(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
// The MMA warp's wait: it is on the critical path, so it never sleeps.
KOP_DEV bool ks_wait_spin(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
KOP_DEV bool ks_wait_bg(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_backoff(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
KOP_DEV void ks_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > KOP_WAIT_LIMIT_NS) break;
  }
}

template <int KF, int NSPLIT>
__global__ void __launch_bounds__(KS_THREADS, 1)
    k1_sym_kernel(const __grid_constant__ CUtensorMap tp0, const __grid_constant__ CUtensorMap tp1,
                  const __grid_constant__ CUtensorMap tp2, const SymArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nst = a.nst;
  const KSLayout L(NSPLIT, a.dp, nst);
  uint8_t* qs = smem + L.qs;
  uint8_t* xs = smem + L.xs;
  float* kn = (float*)(smem + L.kn);
  float* vk = (float*)(smem + L.vk);
  float* qn = (float*)(smem + L.qn);
  float* vq = (float*)(smem + L.vq);
  float* colx = (float*)(smem + L.colx);
  uint64_t* bars = (uint64_t*)(smem + L.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + KS_MAXST;
  // a key slot is released with its S buffer (same ring position): the
  // norm / v producer waits on tempty
  uint64_t* kvfull = bars + 2 * KS_MAXST;
  uint64_t* tfull = kvfull + KS_NKV;
  uint64_t* tempty = tfull + KS_NSB;
  uint64_t* cxfull = tempty + KS_NSB;   // column parts written (all epilogue threads)
  uint64_t* cxempty = cxfull + KS_NCX;  // column parts read (the combining warp)
  uint64_t* qbar = cxempty + KS_NCX;
  uint64_t* drain = qbar + 1;
  uint32_t* holder = (uint32_t*)(smem + L.holder);
  volatile int* abort_word = (volatile int*)(smem + L.abort_word);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x;
  const int row0 = I * 128;
  const int cnt = sym_band_count(I, a.nb);
  const int rb = a.row_bytes;
  const int nsub = (a.dp * 2) / rb;
  const CUtensorMap* maps[3] = {&tp0, &tp1, &tp2};

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < KS_NKV; ++s) mbar_init(&kvfull[s], 1);
    for (int b = 0; b < KS_NSB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], KS_ARRIVALS);
    }
    for (int c = 0; c < KS_NCX; ++c) {
      mbar_init(&cxfull[c], KS_ARRIVALS);
      mbar_init(&cxempty[c], 1);
    }
    mbar_init(qbar, 1);
    mbar_init(drain, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(holder, KS_NSB * 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ------------------------------------------------------------ operand loads
    if (lane == 0) {
      mbar_arrive_expect_tx(qbar, NSPLIT * L.q_split);
      for (int sp = 0; sp < NSPLIT; ++sp)
        for (int ks = 0; ks < nsub; ++ks)
          tma_load_2d(qs + sp * L.q_split + ks * (128 * rb), maps[sp], qbar, ks * 64, row0);
    }
    int t = 0, s = 0;
    uint32_t ph = 0;
    for (; t < cnt; ++t) {
      if (!ks_wait_bg(&empty[s], ph ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        const int J = I + t < a.nb ? I + t : I + t - a.nb;
        mbar_arrive_expect_tx(&full[s], NSPLIT * L.x_split);
        for (int sp = 0; sp < NSPLIT; ++sp)
          for (int ks = 0; ks < nsub; ++ks)
            tma_load_2d(xs + (s * NSPLIT + sp) * L.x_split + ks * (128 * rb), maps[sp], &full[s], ks * 64, J * 128);
      }
      __syncwarp();
      if (++s == nst) { s = 0; ph ^= 1u; }
    }
    if (t < cnt && lane == 0)
      for (int u = (t - nst > 0 ? t - nst : 0); u < t; ++u) ks_drain(&full[u % nst], (u / nst) & 1);
  } else if (warp == 3) {
    // ------------------------------------------------------------ key norms and v
    int t = 0, s = 0;
    uint32_t ph = 0;
    for (; t < cnt; ++t) {
      if (!ks_wait_bg(&tempty[s], ph ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        const int J = I + t < a.nb ? I + t : I + t - a.nb;
        const int j0 = J * 128;
        const int lim_v = a.v_padded ? a.n_pad : a.n;
        const int rows_v = lim_v - j0 < 128 ? lim_v - j0 : 128;
        mbar_arrive_expect_tx(&kvfull[s], 128u * 4 + (uint32_t)rows_v * 4);
        bulk_load(kn + s * 128, a.snorm + j0, 128u * 4, &kvfull[s]);
        bulk_load(vk + s * 128, a.V + j0, (uint32_t)rows_v * 4, &kvfull[s]);
      }
      __syncwarp();
      if (++s == KS_NKV) { s = 0; ph ^= 1u; }
    }
    if (t < cnt && lane == 0)
      for (int u = (t - KS_NKV > 0 ? t - KS_NKV : 0); u < t; ++u) ks_drain(&kvfull[u % KS_NKV], (u / KS_NKV) & 1);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    // D = X_J Q_I^T: the key tile is the A operand (TMEM lanes = keys)
    const uint32_t idesc = idesc_bf16_f32(128, 128);
    const uint32_t sbo = 8u * rb;
    const int nks = a.dp / 16;
    const uint64_t dq0 = sdesc(smem_u32(qs), sbo, a.swz);
    const uint64_t dx0 = sdesc(smem_u32(xs), sbo, a.swz);
    const uint32_t split16 = L.q_split >> 4, sub16 = (128u * rb) >> 4;
    bool ok = ks_wait_spin(qbar, 0, abort_word, a.status);
    int s = 0;
    uint32_t ph = 0;
    for (int t = 0; ok && t < cnt; ++t) {
      const int b = t % KS_NSB;
      const uint32_t bph = (t / KS_NSB) & 1;
      if (!ks_wait_spin(&full[s], ph, abort_word, a.status)) break;
      if (!ks_wait_spin(&tempty[b], bph ^ 1, abort_word, a.status)) break;
      tc_fence_after();
      const uint32_t d = tmem + b * 128;
      const uint64_t xb = dx0 + (uint64_t)(s * NSPLIT) * split16;
      switch (nks) {
        case 1: issue_s_tile<NSPLIT, 1, true>(d, xb, dq0, split16, split16, sub16, sub16, idesc); break;
        case 2: issue_s_tile<NSPLIT, 2, true>(d, xb, dq0, split16, split16, sub16, sub16, idesc); break;
        case 4: issue_s_tile<NSPLIT, 4, true>(d, xb, dq0, split16, split16, sub16, sub16, idesc); break;
        default: issue_s_tile<NSPLIT, 8, true>(d, xb, dq0, split16, split16, sub16, sub16, idesc); break;
      }
      if (lane == 0) {
        tc_commit(&tfull[b]);
        tc_commit(&empty[s]);
      }
      __syncwarp();
      if (++s == nst) { s = 0; ph ^= 1u; }
    }
    if (lane == 0) {
      tc_commit(drain);
      ks_drain(drain, 0);
    }
    __syncwarp();
  } else if (warp == 2) {
    // ------------------------------------------------------------ column parts
    // tile t >= 1: the four warpgroups' parts of each key, added in a fixed
    // order, to the scratch slot of (J, t)
    for (int t = 1; t < cnt; ++t) {
      const int c = (t - 1) % KS_NCX;
      const uint32_t ph = ((t - 1) / KS_NCX) & 1;
      if (!ks_wait_bg(&cxfull[c], ph, abort_word, a.status)) break;
      const int J = I + t < a.nb ? I + t : I + t - a.nb;
      const float* cx = colx + c * KS_NWG * 128;
      float* dst = a.C + ((int64_t)J * a.h + (t - 1)) * 128;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = q * 32 + lane;
        float sum = cx[k];
#pragma unroll
        for (int w = 1; w < KS_NWG; ++w) sum += cx[w * 128 + k];
        dst[k] = sum;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cxempty[c]);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int e = threadIdx.x - 128;  // 0 .. 128 * KS_NWG - 1
    const int wgi = e >> 7;           // query columns wgi * KS_WCOLS .. + KS_WCOLS - 1
    const int quarter = warp & 3;     // TMEM lanes (keys) quarter * 32 .. + 31
    const int kj = quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wgi * KS_WCOLS);
    // the block's own scaled norms and v (zero past n)
    if (e < 128) {
      qn[e] = a.snorm[row0 + e];
      vq[e] = row0 + e < a.n ? a.V[row0 + e] : 0.0f;
    }
    named_bar_sync(1, 128 * KS_NWG);
    // row sums of the warpgroup's query columns, two columns per packed lane pair
    float2 acc[KS_WCOLS / 2];
#pragma unroll
    for (int c = 0; c < KS_WCOLS / 2; ++c) acc[c] = make_float2(0.0f, 0.0f);
    bool live = true;
    for (int t = 0; t < cnt; ++t) {
      const int b = t % KS_NSB;
      const uint32_t bph = (t / KS_NSB) & 1;
      const int s = t % KS_NKV;
      const uint32_t ph = (t / KS_NKV) & 1;
      const int J = I + t < a.nb ? I + t : I + t - a.nb;
      float col = 0.0f;
      if (live) live = ks_wait(&tfull[b], bph, abort_word, a.status);
      if (live) live = ks_wait(&kvfull[s], ph, abort_word, a.status);
      if (live) {
        tc_fence_after();
        const float knj = kn[s * 128 + kj];
        const float vj = J * 128 + kj < a.n ? vk[s * 128 + kj] : 0.0f;
        const float2 kn2 = make_float2(knj, knj), m2 = make_float2(a.m2c, a.m2c), vj2 = make_float2(vj, vj);
        float2 p2a = make_float2(0.0f, 0.0f), p2b = make_float2(0.0f, 0.0f);
        // chunks of 32 query columns
#pragma unroll
        for (int ch = 0; ch < KS_WCOLS / 32; ++ch) {
          uint32_t r[32];
          tmem_ld32(lane_addr + b * 128 + ch * 32, r);
          tmem_ld_wait(r);
          if (ch == KS_WCOLS / 32 - 1) {
            // the S buffer and the key slot are read: release them
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
          }
          const int cb = wgi * KS_WCOLS + ch * 32;
          float2 kv[16];
#pragma unroll
          for (int c4 = 0; c4 < 32; c4 += 4) {
            const float4 q4 = *reinterpret_cast<const float4*>(qn + cb + c4);
            kv[c4 / 2] = fma2(make_float2(__uint_as_float(r[c4 + 0]), __uint_as_float(r[c4 + 1])), m2,
                              add2(make_float2(q4.x, q4.y), kn2));
            kv[c4 / 2 + 1] = fma2(make_float2(__uint_as_float(r[c4 + 2]), __uint_as_float(r[c4 + 3])), m2,
                                  add2(make_float2(q4.z, q4.w), kn2));
          }
          if (t == 0 && cb <= kj && kj < cb + 32) {  // the diagonal: D2 = 0 exactly
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
              if (cb + c == kj) kv[c / 2].x = 0.0f;
              if (cb + c + 1 == kj) kv[c / 2].y = 0.0f;
            }
          }
#pragma unroll
          for (int c = 0; c < 16; ++c) kv[c] = kval_u2<KF>(kv[c], a.c2);
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[ch * 16 + c] = fma2(kv[c], vj2, acc[ch * 16 + c]);
          if (t > 0) {
#pragma unroll
            for (int c4 = 0; c4 < 32; c4 += 4) {
              const float4 v4 = *reinterpret_cast<const float4*>(vq + cb + c4);
              p2a = fma2(kv[c4 / 2], make_float2(v4.x, v4.y), p2a);
              p2b = fma2(kv[c4 / 2 + 1], make_float2(v4.z, v4.w), p2b);
            }
          }
        }
        col = (p2a.x + p2a.y) + (p2b.x + p2b.y);
      }
      if (t > 0 && live) {
        // this warpgroup's column part of key kj, for the combining warp
        const int c = (t - 1) % KS_NCX;
        const uint32_t cph = ((t - 1) / KS_NCX) & 1;
        live = ks_wait(&cxempty[c], cph ^ 1, abort_word, a.status);
        if (live) {
          colx[(c * KS_NWG + wgi) * 128 + kj] = col;
          __syncwarp();
          if (lane == 0) mbar_arrive(&cxfull[c]);
        }
      }
    }
    // row parts: the 128 key-slot partials of each query row, summed in a
    // fixed order with error-free sums (the operand area is free: every MMA
    // has completed)
    named_bar_sync(1, 128 * KS_NWG);
    float* red = (float*)smem;
#pragma unroll
    for (int c = 0; c < KS_WCOLS / 2; ++c) {
      red[(wgi * 128 + kj) * (KS_WCOLS + 1) + 2 * c] = acc[c].x;
      red[(wgi * 128 + kj) * (KS_WCOLS + 1) + 2 * c + 1] = acc[c].y;
    }
    named_bar_sync(1, 128 * KS_NWG);
    if (quarter < KS_WCOLS / 32) {
      const int c = quarter * 32 + lane;
      const int i = row0 + wgi * KS_WCOLS + c;
      float hi = 0.0f, lo = 0.0f;
      for (int k = 0; k < 128; ++k) two_sum_acc(hi, lo, red[(wgi * 128 + k) * (KS_WCOLS + 1) + c]);
      if (i < a.n && !*abort_word) a.O[i] = hi + lo;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, KS_NSB * 128);
  }
}

// O[j] += the column parts of row block J, C[J][t - 1] for the tiles t that
// CTA I = J - t (mod nb) took, in the order of t, with error-free sums.
__global__ void sym_combine_kernel(float* __restrict__ O, const float* __restrict__ C, int n, int nb, int h) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int J = j >> 7, jj = j & 127;
  float s = O[j], e = 0.0f;
  for (int t = 1; t <= h; ++t) {
    const int I = J - t >= 0 ? J - t : J - t + nb;
    if (t < sym_band_count(I, nb)) two_sum_acc(s, e, C[((int64_t)J * h + (t - 1)) * 128 + jj]);
  }
  O[j] = s + e;
}

// ---------------------------------------------------------------- host side
size_t sym_smem_bytes(int nsplit, int dp, int nst) { return KSLayout(nsplit, dp, nst).total + 1024; }

template <int KF, int NSPLIT>
static int launch_sym_t(const PointSet& P, const SymArgs& a, cudaStream_t st) {
  auto kern = k1_sym_kernel<KF, NSPLIT>;
  static bool attr_set = false;
  if (!attr_set) {
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit_bytes()));
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr_set = true;
  }
  size_t smem = sym_smem_bytes(NSPLIT, a.dp, a.nst);
  // one CTA per SM: it allocates all of TMEM
  const size_t one_per_sm = smem_limit_bytes() / 2 + 4096;
  if (smem < one_per_sm) smem = one_per_sm;
  kern<<<(unsigned)a.nb, KS_THREADS, smem, st>>>(P.tm[0][0], P.tm[1][0], P.tm[2][0], a);
  KOP_LAUNCHED();
  if (a.h > 0) {
    sym_combine_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a.O, a.C, a.n, a.nb, a.h);
    KOP_LAUNCHED();
  }
  return KOP_OK;
}

// O (n) = K(P, P) v (v: n floats, or n_pad when v_padded), 2-term split.
int fused_matvec_sym(PointSet& P, int kf, const KConst& kc, const float* v, int v_padded, float* O, int* status,
                     cudaStream_t st) {
  const int dp = P.dp;
  const size_t lim = smem_limit_bytes();
  int nst = 2;
  while (nst < KS_MAXST && sym_smem_bytes(2, dp, nst + 1) <= lim) ++nst;
  if (sym_smem_bytes(2, dp, nst) > lim) return fail(KOP_EINVAL, "fused_matvec_sym: feature width too large");
  SymArgs a;
  a.n = (int)P.n;
  a.n_pad = (int)P.n_pad;
  a.nb = (int)(P.n_pad / 128);
  a.h = a.nb / 2;
  a.snorm = P.snorm;
  a.V = v;
  a.v_padded = v_padded;
  a.O = O;
  a.dp = dp;
  a.row_bytes = dp >= 64 ? 128 : dp * 2;
  a.swz = a.row_bytes == 128 ? 2 : (a.row_bytes == 64 ? 4 : 6);
  a.nst = nst;
  a.m2c = -2.0f * kc.scale;
  a.c2 = kc.c2;
  a.status = status;
  const size_t cfl = (size_t)a.nb * a.h * 128;
  if (cfl > P.sym_scratch_floats) {
    if (P.sym_scratch) cudaFreeAsync(P.sym_scratch, st);
    P.sym_scratch = nullptr;
    P.sym_scratch_floats = 0;
    KOP_CUDA_TRY(cudaMallocAsync((void**)&P.sym_scratch, sizeof(float) * cfl, st));
    P.sym_scratch_floats = cfl;
  }
  a.C = P.sym_scratch;
  switch (kf) {
    case KF_RBF: return launch_sym_t<KF_RBF, 2>(P, a, st);
    case KF_LAPLACE: return launch_sym_t<KF_LAPLACE, 2>(P, a, st);
    case KF_MATERN: return launch_sym_t<KF_MATERN, 2>(P, a, st);
    case KF_DRBF: return launch_sym_t<KF_DRBF, 2>(P, a, st);
    case KF_DLAPLACE: return launch_sym_t<KF_DLAPLACE, 2>(P, a, st);
    case KF_GRBF: return launch_sym_t<KF_GRBF, 2>(P, a, st);
    case KF_GLAPLACE: return launch_sym_t<KF_GLAPLACE, 2>(P, a, st);
    case KF_GMATERN: return launch_sym_t<KF_GMATERN, 2>(P, a, st);
    default: return launch_sym_t<KF_DMATERN, 2>(P, a, st);
  }
}

}  // namespace kop
