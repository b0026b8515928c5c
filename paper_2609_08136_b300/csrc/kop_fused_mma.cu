// Fused kernel-operator product for blocks of many vectors (m > 8): the
// contraction O += K_IJ V_J runs on the tensor cores as well.
//
// Same product as kop_fused.cu (the paper's matrix-free operator, Sec. 4.3;
// the sketch Y = K Omega of the Nystrom preconditioner is this product with
// m = r), but after the epilogue has turned the distance tile S into kernel
// values K_IJ in registers, it writes them back into the same TMEM columns as
// a 16-bit hi/lo pair, and one thread issues
//   O += K_lo V_hi + K_hi V_lo + K_hi V_hi
// with A read from TMEM and V^T (split into hi/lo by a prep kernel) read
// from shared memory.  O (128 rows x MC columns, FP32) stays in TMEM for the
// whole sweep over X (restarted every few tiles into a running sum, see
// K3_DRAIN) and is written once at the end.  Tiles of 64 points.  Kernel
// values (in [0, 1]) and V (scaled per column by a power of two) travel as
// FP16 hi / lo pairs, 22 significant bits; derivative kernels as BF16 pairs.
// S has four TMEM buffers and the MMA warp issues PV(t) before S(t+3), so the
// tensor pipe works on one tile's contraction while two pairs of epilogue
// warpgroups (even and odd tiles) turn the next tiles' distances into kernel
// values.  Two producer warps keep three rings filled: X tiles (released as
// soon as their distance MMAs finish), the X tiles' norms (read by the
// epilogue) and V tiles (released by the contraction).
#include <cuda_fp16.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kop_device.cuh"
#include "kop_epilogue.cuh"
#include "kop_internal.h"
#include "kop_sdist.cuh"

namespace kop {

constexpr int K3_THREADS = 640;  // 4 control warps + 4 epilogue warpgroups
constexpr int K3_MAXX = 4;       // X-tile ring (freed when the distance MMAs finish)
constexpr int K3_MAXV = 4;       // V-tile ring (freed when the contraction finishes)
constexpr int K3_BN = 64;
constexpr int K3_NSB = 4;  // S buffers in TMEM (even: a buffer always serves the same warpgroup pair)
// Ring of the scaled norms of the X tiles, loaded with the X tiles and read by
// the epilogue.  It has no "empty" barrier: the norms of tile t + K3_NKS are
// loaded after the distance MMAs of tile t + K3_NKS - nx completed, which were
// issued after the contraction of tile t + K3_NKS - nx - lookahead >= t, which
// waited for the epilogue of tile t; so K3_NKS >= K3_MAXX + K3_NSB - 1.
constexpr int K3_NKS = 8;
// The tensor core truncates when it adds to an FP32 accumulator, so a long
// chain of MMAs into O drifts towards zero (about 2^-24 of |O| per MMA, 12
// MMAs per tile: measured -6e-4 relative at n = 1e5, enough to make
// K + lam I indefinite for lam = 1e-3 there).  For the solver's products O is
// therefore restarted every K3_DRAIN tiles and its partials summed, rounding
// to nearest, into a running sum in TMEM (128-column chunks; measured bias
// -7e-7).  The Nystrom sketch keeps one accumulator and 256-column chunks:
// its drift rescales the sketch by the same relative amount, which the
// randomized preconditioner does not notice, and the narrower chunks would
// double its distance and kernel-value work; it also drops the kernel
// values' lo half (see MmaArgs::klo).
constexpr int K3_DRAIN = 4;
static_assert(K3_NKS >= K3_MAXX + K3_NSB - 1, "norm ring too shallow");

struct MmaArgs {
  const float* qnorm;
  const float* knorm;
  float* O;
  int nq, nk, m, ldo;
  int dp, row_bytes, swz, self, mc, tcols, nx, nv, vsplits;
  int m_pad;  // rows of one blocked V^T tile (all column chunks)
  float m2c, c2;
  int* status;
  // contraction in FP16 hi / lo pairs (kernel values in [0, 1]) with V scaled
  // per column by an exact power of two; inv_scale[c] undoes it on output
  int f16;
  const float* inv_scale;
  // O is restarted every `drain` tiles (0: never) and its partial added to a
  // running sum in TMEM (columns OCOL + mc .., so mc <= 128)
  int drain;
  // klo = 0: the kernel values' lo half is dropped (the sketch: K rounded to
  // FP16 times V exactly), two contraction MMAs instead of three
  int klo;
};

struct K3Layout {
  uint32_t q_split, x_split, v_split, qs, xs, vs, kn, bars, holder, abort_word, total;
  __host__ __device__ K3Layout(int dp, int mc, int nx, int nv, int vsplits) {
    q_split = 128u * dp * 2;
    x_split = (uint32_t)K3_BN * dp * 2;
    v_split = (uint32_t)mc * K3_BN * 2;
    qs = 0;
    xs = qs + 2 * q_split;
    vs = xs + nx * 2 * x_split;
    kn = vs + nv * vsplits * v_split;
    bars = kn + K3_NKS * K3_BN * 4;
    holder = bars + (2 * K3_MAXX + 2 * K3_MAXV + K3_NKS + 3 * K3_NSB + 6) * 8;
    abort_word = holder + 4;
    total = abort_word + 12;
  }
};

KOP_DEV bool warp_wait3(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  // fast path without a divergent branch: every lane polls once
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
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

template <int KF>
__global__ void __launch_bounds__(K3_THREADS, 1)
    k1_mma_kernel(const __grid_constant__ CUtensorMap tq0, const __grid_constant__ CUtensorMap tq1,
                  const __grid_constant__ CUtensorMap tk0, const __grid_constant__ CUtensorMap tk1,
                  const __grid_constant__ CUtensorMap tv0, const __grid_constant__ CUtensorMap tv1,
                  const MmaArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nx = a.nx, nv = a.nv;
  const int nvs = a.vsplits;
  const K3Layout L(a.dp, a.mc, nx, nv, nvs);
  uint8_t* qs = smem + L.qs;
  uint8_t* xs = smem + L.xs;
  uint8_t* vs = smem + L.vs;
  float* kn = (float*)(smem + L.kn);
  uint64_t* bars = (uint64_t*)(smem + L.bars);
  uint64_t* xfull = bars;                    // nx
  uint64_t* xempty = bars + K3_MAXX;         // nx
  uint64_t* vfull = bars + 2 * K3_MAXX;      // nv
  uint64_t* vempty = vfull + K3_MAXV;        // nv
  uint64_t* nfull = vempty + K3_MAXV;        // K3_NKS
  uint64_t* sfull = nfull + K3_NKS;          // K3_NSB
  uint64_t* pfull = sfull + K3_NSB;          // K3_NSB
  uint64_t* sfree = pfull + K3_NSB;          // K3_NSB
  uint64_t* qbar = sfree + K3_NSB;
  uint64_t* ofull = qbar + 1;
  uint64_t* drain = ofull + 1;
  uint64_t* opart = drain + 1;  // O holds the partial of the last K3_DRAIN tiles
  uint64_t* odone = opart + 1;  // the epilogue has added it to the output
  uint32_t* holder = (uint32_t*)(smem + L.holder);
  volatile int* abort_word = (volatile int*)(smem + L.abort_word);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * 128;
  const int m0 = blockIdx.y * a.mc;
  const int ntiles = (a.nk + K3_BN - 1) / K3_BN;
  // Each row block starts its sweep at its own tile, so that the CTAs resident
  // at one time read different X and V tiles instead of all hitting the same
  // L2 lines; tile_of maps the sweep index t to the tile it processes.
  const int toff = (int)(((int64_t)blockIdx.x * ntiles) / gridDim.x);
  auto tile_of = [&](int t) { return t + toff < ntiles ? t + toff : t + toff - ntiles; };
  const int rb = a.row_bytes;
  const int nsub = (a.dp * 2) / rb;
  const uint32_t OCOL = 256;  // O accumulator columns start after the S buffers

  if (threadIdx.x == 0) {
    for (int s = 0; s < nx; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&xempty[s], 1);
    }
    for (int s = 0; s < nv; ++s) {
      mbar_init(&vfull[s], 1);
      mbar_init(&vempty[s], 1);
    }
    for (int s = 0; s < K3_NKS; ++s) mbar_init(&nfull[s], 1);
    for (int b = 0; b < K3_NSB; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&pfull[b], 256);
      mbar_init(&sfree[b], 1);
    }
    mbar_init(qbar, 1);
    mbar_init(ofull, 1);
    mbar_init(drain, 1);
    mbar_init(opart, 1);
    mbar_init(odone, 16);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(holder, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ------------------------------------------------------------ X producer
    // Q once, then X(t) into the X ring and the scaled norms of tile t into the norm ring
    const CUtensorMap* mq[2] = {&tq0, &tq1};
    const CUtensorMap* mk[2] = {&tk0, &tk1};
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
      const int s = t % nx;
      if (!warp_wait3(&xempty[s], ((t / nx) & 1) ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        const int j0 = tile_of(t) * K3_BN;
        mbar_arrive_expect_tx(&xfull[s], 2 * L.x_split);
        for (int sp = 0; sp < 2; ++sp)
          for (int ks = 0; ks < nsub; ++ks)
            tma_load_2d(xs + (s * 2 + sp) * L.x_split + ks * (K3_BN * rb), mk[sp], &xfull[s], ks * 64, j0);
        const int ns = t % K3_NKS;
        mbar_arrive_expect_tx(&nfull[ns], K3_BN * 4);
        bulk_load(kn + ns * K3_BN, a.knorm + j0, K3_BN * 4, &nfull[ns]);
      }
      __syncwarp();
    }
    if (t < ntiles && lane == 0) {
      for (int u = (t - nx > 0 ? t - nx : 0); u < t; ++u) drain_wait3(&xfull[u % nx], (u / nx) & 1);
      for (int u = (t - K3_NKS > 0 ? t - K3_NKS : 0); u < t; ++u) drain_wait3(&nfull[u % K3_NKS], (u / K3_NKS) & 1);
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------ V producer
    const CUtensorMap* mvv[2] = {&tv0, &tv1};
    int t = 0;
    for (; t < ntiles; ++t) {
      const int s = t % nv;
      if (!warp_wait3(&vempty[s], ((t / nv) & 1) ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        mbar_arrive_expect_tx(&vfull[s], nvs * L.v_split);
        for (int sp = 0; sp < nvs; ++sp)
          tma_load_2d(vs + (s * nvs + sp) * L.v_split, mvv[sp], &vfull[s], 0, tile_of(t) * a.m_pad + m0);
      }
      __syncwarp();
    }
    if (t < ntiles && lane == 0)
      for (int u = (t - nv > 0 ? t - nv : 0); u < t; ++u) drain_wait3(&vfull[u % nv], (u / nv) & 1);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // order: S(0) .. S(L-1), then for each u: PV(u), S(u + L), with the
    // lookahead L = min(S buffers - 1, X stages).  One MMA must issue in far
    // less time than the tensor pipe takes for it (about 32 cycles for a
    // 128 x 64 x 16 distance step), so the loop only adds constant offsets to
    // descriptors prepared here, and ring slots and phases are counters.
    const uint32_t idesc_s = idesc_bf16_f32(128, K3_BN);
    const uint32_t idesc_o = a.f16 ? idesc_f16_f32(128, a.mc) : idesc_bf16_f32(128, a.mc);
    const uint32_t sbo = 8u * rb;
    const int nks = a.dp / 16;  // K steps of 16 over the padded feature width
    const uint64_t dq_hi = sdesc(smem_u32(qs), sbo, a.swz);
    const uint64_t dx0 = sdesc(smem_u32(xs), sbo, a.swz);
    const uint64_t dv0 = sdesc(smem_u32(vs), 1024u, 2u);
    const uint32_t q_sub16 = (128u * rb) >> 4, x_sub16 = ((uint32_t)K3_BN * rb) >> 4;
    const uint32_t q_split16 = L.q_split >> 4, x_split16 = L.x_split >> 4, v_split16 = L.v_split >> 4;
    bool ok = warp_wait3(qbar, 0, abort_word, a.status);
    uint32_t oacc = 0;
    int sx = 0, sv = 0;            // ring slots of the next S / PV tile
    uint32_t phx = 0, phv = 0;     // their phases
    int ts = 0;                    // next S tile
    const int look = (K3_NSB - 1) < nx ? (K3_NSB - 1) : nx;
    for (int step = 0; ok; ++step) {
      // step < look: S(step); afterwards PV(step - look), then S(step)
      const int u = step - look;
      if (u >= ntiles) break;
      if (u >= 0) {
        const int b = u & (K3_NSB - 1);
        if (!warp_wait3(&vfull[sv], phv, abort_word, a.status)) { ok = false; break; }
        if (!warp_wait3(&pfull[b], (u / K3_NSB) & 1, abort_word, a.status)) { ok = false; break; }
        if (a.drain && u > 0 && u % a.drain == 0) {
          // the epilogue has drained O: the next partial starts from zero
          if (!warp_wait3(odone, ((u / a.drain) - 1) & 1, abort_word, a.status)) { ok = false; break; }
          oacc = 0;
        }
        tc_fence_after();
        {
          // (P split, V split): lo*hi, hi*hi [, hi*lo]; P hi at +0, lo at +16 of each 32-column chunk
          const uint32_t pb = tmem + b * K3_BN;
          const uint64_t vd = dv0 + (uint64_t)(sv * nvs) * v_split16;
          if (a.klo) {
#pragma unroll
            for (int kk = 0; kk < K3_BN / 16; ++kk) {
              tc_mma_ts_elect(tmem + OCOL, pb + 32u * (kk >> 1) + 8u * (kk & 1) + 16u, vd + 2 * kk, idesc_o, oacc);
              oacc = 1;
            }
          }
#pragma unroll
          for (int kk = 0; kk < K3_BN / 16; ++kk) {
            tc_mma_ts_elect(tmem + OCOL, pb + 32u * (kk >> 1) + 8u * (kk & 1), vd + 2 * kk, idesc_o, oacc);
            oacc = 1;
          }
          if (nvs == 2) {
#pragma unroll
            for (int kk = 0; kk < K3_BN / 16; ++kk)
              tc_mma_ts_elect(tmem + OCOL, pb + 32u * (kk >> 1) + 8u * (kk & 1), vd + v_split16 + 2 * kk, idesc_o, 1u);
          }
          tc_commit_elect(&sfree[b]);
          tc_commit_elect(&vempty[sv]);
          if (a.drain && (u + 1) % a.drain == 0 && u + 1 < ntiles) tc_commit_elect(opart);
        }
        __syncwarp();
        if (++sv == nv) { sv = 0; phv ^= 1u; }
      }
      if (ts < ntiles) {
        const int b = ts & (K3_NSB - 1);
        if (!warp_wait3(&xfull[sx], phx, abort_word, a.status)) { ok = false; break; }
        if (!warp_wait3(&sfree[b], ((ts / K3_NSB) & 1) ^ 1, abort_word, a.status)) { ok = false; break; }
        tc_fence_after();
        {
          // hi(Q) mid(X) + mid(Q) hi(X) + hi(Q) hi(X)
          const uint32_t d = tmem + b * K3_BN;
          const uint64_t xb = dx0 + (uint64_t)(2 * sx) * x_split16;
          switch (nks) {
            case 1: issue_s_tile<2, 1, false>(d, dq_hi, xb, q_split16, x_split16, q_sub16, x_sub16, idesc_s); break;
            case 2: issue_s_tile<2, 2, false>(d, dq_hi, xb, q_split16, x_split16, q_sub16, x_sub16, idesc_s); break;
            case 4: issue_s_tile<2, 4, false>(d, dq_hi, xb, q_split16, x_split16, q_sub16, x_sub16, idesc_s); break;
            default: issue_s_tile<2, 8, false>(d, dq_hi, xb, q_split16, x_split16, q_sub16, x_sub16, idesc_s); break;
          }
          tc_commit_elect(&sfull[b]);
          tc_commit_elect(&xempty[sx]);
        }
        __syncwarp();
        if (++sx == nx) { sx = 0; phx ^= 1u; }
        ++ts;
      }
    }
    tc_commit_elect(ofull);
    tc_commit_elect(drain);
    if (lane == 0) drain_wait3(drain, 0);
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    // warpgroup pair `pair` takes the tiles t with t % 2 == pair; within a
    // pair, warpgroup `wg` takes 32 of the 64 columns of the tile
    const int ep = warp - 4, pair = ep >> 3, wg = (ep >> 2) & 1, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gi = row0 + row;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    bool ok = true;
    const float qni = a.qnorm[gi];
    // O is drained every a.drain tiles into a running sum in TMEM (rounding to
    // nearest); the final write outputs O + sum.  Warpgroup q = ep / 4 takes
    // columns [q mc / 4, (q + 1) mc / 4) of its rows in every drain and in
    // the final write.
    const int q4 = ep >> 2, mq = a.mc / 4;
    const uint32_t OSUM = OCOL + (uint32_t)a.mc;
    int ndrained = 0;
    // O (+ the running sum, once there is one) to the output
    auto flush = [&]() {
      for (int c0 = q4 * mq; c0 < (q4 + 1) * mq; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(lane_addr + OCOL + c0, r);
        if (ndrained > 0) {
          uint32_t sm[16];
          tmem_ld16(lane_addr + OSUM + c0, sm);
          tmem_ld_wait16(sm);
          tmem_ld_wait16(r);
#pragma unroll
          for (int c = 0; c < 16; ++c) r[c] = __float_as_uint(__uint_as_float(r[c]) + __uint_as_float(sm[c]));
        } else {
          tmem_ld_wait16(r);
        }
        if (gi < a.nq && !*abort_word) {
          float* orow = a.O + (int64_t)gi * a.ldo + m0 + c0;
          const float* isc = a.inv_scale + m0 + c0;
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (m0 + c0 + c < a.m) orow[c] = a.f16 ? __uint_as_float(r[c]) * isc[c] : __uint_as_float(r[c]);
        }
      }
    };
    // one drain: the running sum takes O
    auto drain_once = [&]() {
      for (int c0 = q4 * mq; c0 < (q4 + 1) * mq; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(lane_addr + OCOL + c0, r);
        if (ndrained > 0) {
          uint32_t sm[16];
          tmem_ld16(lane_addr + OSUM + c0, sm);
          tmem_ld_wait16(sm);
          tmem_ld_wait16(r);
#pragma unroll
          for (int c = 0; c < 16; ++c) r[c] = __float_as_uint(__uint_as_float(r[c]) + __uint_as_float(sm[c]));
        } else {
          tmem_ld_wait16(r);
        }
        tmem_st16(lane_addr + OSUM + c0, r);
      }
      tmem_st_wait();
    };
    auto drain_to = [&](int k) -> bool {  // drains 1 .. k
      while (ndrained < k) {
        if (!warp_wait3(opart, ndrained & 1, abort_word, a.status)) return false;
        tc_fence_after();
        drain_once();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(odone);
        ++ndrained;
      }
      return true;
    };
    for (int t = pair; ok && t < ntiles; t += 2) {
      const int b = t % K3_NSB;
      if (a.drain && !drain_to(t / a.drain)) { ok = false; break; }
      const uint32_t bph = (t / K3_NSB) & 1;
      if (!warp_wait3(&sfull[b], bph, abort_word, a.status)) { ok = false; break; }
      tc_fence_after();
      uint32_t r[32];
      const uint32_t col = b * K3_BN + wg * 32;
      tmem_ld32(lane_addr + col, r);
      tmem_ld_wait(r);
      const int nsl = t % K3_NKS;
      if (!warp_wait3(&nfull[nsl], (t / K3_NKS) & 1, abort_word, a.status)) { ok = false; break; }
      const int jt0 = tile_of(t) * K3_BN;
      const int jbase = jt0 + wg * 32;
      const float* knG = kn + nsl * K3_BN + wg * 32;
      const bool mask = (a.self && jt0 < row0 + 128 && jt0 + K3_BN > row0) || (jt0 + K3_BN > a.nk);
      float kv[32];
#pragma unroll
      for (int j4 = 0; j4 < 32; j4 += 4) {
        const float4 k4 = *reinterpret_cast<const float4*>(knG + j4);
        kv[j4 + 0] = fmaf(__uint_as_float(r[j4 + 0]), a.m2c, qni + k4.x);
        kv[j4 + 1] = fmaf(__uint_as_float(r[j4 + 1]), a.m2c, qni + k4.y);
        kv[j4 + 2] = fmaf(__uint_as_float(r[j4 + 2]), a.m2c, qni + k4.z);
        kv[j4 + 3] = fmaf(__uint_as_float(r[j4 + 3]), a.m2c, qni + k4.w);
      }
      if (mask) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
          if (a.self && jbase + jj == gi) kv[jj] = 0.0f;
      }
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) kv[jj] = kval_u<KF>(kv[jj], a.c2);
      if (mask) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
          if (jbase + jj >= a.nk) kv[jj] = 0.0f;
      }
      // K = hi + lo in BF16 (or FP16), packed two per 32-bit TMEM column
      uint32_t ph16[16], pl16[16];
      if (a.f16) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const __half2 h = __floats2half2_rn(kv[2 * e], kv[2 * e + 1]);
          const __half2 l = __floats2half2_rn(kv[2 * e] - __low2float(h), kv[2 * e + 1] - __high2float(h));
          ph16[e] = *reinterpret_cast<const uint32_t*>(&h);
          pl16[e] = *reinterpret_cast<const uint32_t*>(&l);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(kv[2 * e], kv[2 * e + 1]);
          const __nv_bfloat162 l =
              __floats2bfloat162_rn(kv[2 * e] - __low2float(h), kv[2 * e + 1] - __high2float(h));
          ph16[e] = *reinterpret_cast<const uint32_t*>(&h);
          pl16[e] = *reinterpret_cast<const uint32_t*>(&l);
        }
      }
      tmem_st16(lane_addr + col, ph16);
      if (a.klo) tmem_st16(lane_addr + col + 16, pl16);
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&pfull[b]);
    }
    // the drains this warp has not reached, then the last partial
    if (ok && a.drain) ok = drain_to((ntiles - 1) / a.drain);
    if (ok && warp_wait3(ofull, 0, abort_word, a.status)) {
      tc_fence_after();
      flush();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// V (nk x m, ld ldv, FP32) -> V^T split into BF16 hi and lo, zero padded to
// m_pad x nk_pad and blocked by tiles of 64 points: the 64-point tile jt of
// column c is the 128-byte row jt * m_pad + c, so that the box one CTA loads
// for a tile (mc columns) is one contiguous run of memory.  (Rows of a plain
// V^T lie nk_pad * 2 bytes apart, and boxes of such strided rows load slowly.)
// F16: the FP16 pair of V[j][c] * scale[c] (scale an exact power of two).
template <bool F16>
__global__ void vsplit_kernel(const float* __restrict__ V, int nk, int m, int ldv, int nk_pad, int m_pad,
                              const float* __restrict__ scale, uint16_t* __restrict__ vh, uint16_t* __restrict__ vl) {
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
      const int64_t o = ((int64_t)(j / K3_BN) * m_pad + c) * K3_BN + (j % K3_BN);
      if constexpr (F16) {
        const float v = tile[threadIdx.x][r] * (c < m ? scale[c] : 1.0f);
        const __half h = __float2half_rn(v);
        const __half l = __float2half_rn(v - __half2float(h));
        vh[o] = __half_as_ushort(h);
        vl[o] = __half_as_ushort(l);
      } else {
        const float v = tile[threadIdx.x][r];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        vh[o] = __bfloat16_as_ushort(h);
        vl[o] = __bfloat16_as_ushort(l);
      }
    }
  }
}

// Largest |V[j][c]| of each column (as the bits of a non-negative float,
// which order like integers), over a grid of row blocks.
__global__ void colmax_kernel(const float* __restrict__ V, int nk, int m, int ldv, int* __restrict__ cmax) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float mx = 0.0f;
  if (c < m)
    for (int j = blockIdx.y * 8 + threadIdx.y; j < nk; j += gridDim.y * 8) mx = fmaxf(mx, fabsf(V[(int64_t)j * ldv + c]));
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && c < m) {
    for (int y = 1; y < 8; ++y) mx = fmaxf(mx, red[y][threadIdx.x]);
    atomicMax(cmax + c, __float_as_int(mx));
  }
}

// scale[c] = 2^s with max|V[:, c]| * 2^s <= 2^14 (FP16 holds it with room for
// the hi + lo pair); inv_scale[c] = 2^-s; 1 for an all-zero column.
__global__ void colscale_kernel(const int* __restrict__ cmax, int m, float* __restrict__ scale,
                                float* __restrict__ inv_scale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  const float mx = __int_as_float(cmax[c]);
  int sh = 0;
  if (mx > 0.0f && isfinite(mx)) {
    int k;
    frexpf(mx, &k);  // mx < 2^k
    sh = 14 - k;
    sh = sh > 100 ? 100 : (sh < -100 ? -100 : sh);
  }
  scale[c] = ldexpf(1.0f, sh);
  inv_scale[c] = ldexpf(1.0f, -sh);
}

size_t mma_smem_bytes(int dp, int mc, int nx, int nv, int vsplits) {
  return K3Layout(dp, mc, nx, nv, vsplits).total + 1024;
}

// Column chunk per CTA: a multiple of 64 (each epilogue warpgroup writes out
// half of it, 32 columns at a time), at most 256 (MMA N limit), the widest
// whose pipeline fits in shared memory, then narrowed to balance the chunks.
int mma_chunk(int dp, int m, int vsplits, int mc_max) {
  const int mpad = ((m + 63) / 64) * 64;
  int mc = mpad < mc_max ? mpad : mc_max;
  while (mc > 64 && mma_smem_bytes(dp, mc, 2, 2, vsplits) > smem_limit_bytes()) mc -= 64;
  if (mma_smem_bytes(dp, mc, 2, 2, vsplits) > smem_limit_bytes()) return 0;
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
    KOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr_set = true;
  }
  dim3 grid((unsigned)((a.nq + 127) / 128), (unsigned)((a.m + a.mc - 1) / a.mc));
  kern<<<grid, K3_THREADS, mma_smem_bytes(a.dp, a.mc, a.nx, a.nv, a.vsplits), st>>>(Q.tm[0][1], Q.tm[1][1], Ks.tm[0][1], Ks.tm[1][1],
                                                              tv[0], tv[1], a);
  KOP_LAUNCHED();
  return KOP_OK;
}

// One block product with a given column chunk mc and X / V ring depths.
static int run_mma(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, const float* V, int m,
                   int ldv, float* O, int ldo, int* status, cudaStream_t st, bool sketch, int mc, int nx, int nv) {
  const int vsplits = 2;
  // kernel values lie in [0, 1]: the contraction carries them (and V, scaled
  // per column) as FP16 pairs, 22 significant bits instead of BF16's 16
  const bool f16 = kf == KF_RBF || kf == KF_LAPLACE || kf == KF_MATERN;
  const int nch = (m + mc - 1) / mc;
  const int m_pad = nch * mc;
  const int64_t nk_pad = Ks.n_pad;
  uint16_t* vsplit = nullptr;
  // V^T pairs, then (FP16) the column maxima and the two scale arrays
  const size_t vbytes = (size_t)2 * m_pad * nk_pad * 2;
  KOP_CUDA_TRY(cudaMallocAsync((void**)&vsplit, vbytes + (size_t)3 * 4 * m_pad, st));
  uint16_t* vh = vsplit;
  uint16_t* vl = vsplit + (size_t)m_pad * nk_pad;
  int* cmax = (int*)((uint8_t*)vsplit + vbytes);
  float* vscale = (float*)(cmax + m_pad);
  float* vinv = vscale + m_pad;
  dim3 vb(32, 8), vg((unsigned)(nk_pad / 32), (unsigned)((m_pad + 31) / 32));
  int rc = KOP_OK;
  if (f16) {
    cudaError_t e0 = cudaMemsetAsync(cmax, 0, sizeof(int) * m_pad, st);
    if (e0 != cudaSuccess) rc = cuda_fail(e0, "cudaMemsetAsync");
    if (rc == KOP_OK) {
      int gy = (int)((Ks.n + 8 * 64 - 1) / (8 * 64));
      if (gy > 4 * num_sms()) gy = 4 * num_sms();
      if (gy < 1) gy = 1;
      colmax_kernel<<<dim3((unsigned)((m + 31) / 32), (unsigned)gy), dim3(32, 8), 0, st>>>(V, (int)Ks.n, m, ldv, cmax);
      note_launch();
      colscale_kernel<<<(unsigned)((m_pad + 127) / 128), 128, 0, st>>>(cmax, m, vscale, vinv);
      note_launch();
      vsplit_kernel<true><<<vg, vb, 0, st>>>(V, (int)Ks.n, m, ldv, (int)nk_pad, m_pad, vscale, vh, vl);
      note_launch();
    }
  } else {
    vsplit_kernel<false><<<vg, vb, 0, st>>>(V, (int)Ks.n, m, ldv, (int)nk_pad, m_pad, nullptr, vh, vl);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (rc == KOP_OK && e != cudaSuccess) rc = cuda_fail(e, "vsplit_kernel");
  CUtensorMap tv[2];
  const int64_t vrows = (nk_pad / K3_BN) * m_pad;  // blocked V^T: 64 values per row
  if (rc == KOP_OK) rc = encode_tmap_bf16(&tv[0], vh, vrows, K3_BN, K3_BN, mc);
  if (rc == KOP_OK) rc = encode_tmap_bf16(&tv[1], vl, vrows, K3_BN, K3_BN, mc);
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
    a.tcols = 512;
    a.vsplits = vsplits;
    a.m_pad = m_pad;
    a.nx = nx;
    a.nv = nv;
    a.m2c = -2.0f * kc.scale;
    a.c2 = kc.c2;
    a.status = status;
    a.f16 = f16 ? 1 : 0;
    a.inv_scale = vinv;
    a.drain = sketch ? 0 : K3_DRAIN;
    // the sketch takes the kernel values rounded to FP16 (hi only) against V
    // carried exactly (hi + lo): it is then the sketch of a kernel matrix
    // perturbed by about 2^-12 per entry, which a preconditioner does not
    // notice (measured: the same PCG iterations on the Laplace mixture and
    // the Matern n = 1e6 workloads) for a third less contraction work
    a.klo = sketch ? 0 : 1;
    switch (kf) {
      case KF_RBF: rc = launch_mma_t<KF_RBF>(Q, Ks, tv, a, st); break;
      case KF_LAPLACE: rc = launch_mma_t<KF_LAPLACE>(Q, Ks, tv, a, st); break;
      case KF_MATERN: rc = launch_mma_t<KF_MATERN>(Q, Ks, tv, a, st); break;
      case KF_DRBF: rc = launch_mma_t<KF_DRBF>(Q, Ks, tv, a, st); break;
      case KF_DLAPLACE: rc = launch_mma_t<KF_DLAPLACE>(Q, Ks, tv, a, st); break;
      case KF_GRBF: rc = launch_mma_t<KF_GRBF>(Q, Ks, tv, a, st); break;
      case KF_GLAPLACE: rc = launch_mma_t<KF_GLAPLACE>(Q, Ks, tv, a, st); break;
      case KF_GMATERN: rc = launch_mma_t<KF_GMATERN>(Q, Ks, tv, a, st); break;
      default: rc = launch_mma_t<KF_DMATERN>(Q, Ks, tv, a, st); break;
    }
  }
  cudaFreeAsync(vsplit, st);
  return rc;
}

// ------------------------------------------------------------------ autotuner
// Tile shape of the block product: the column chunk mc (a multiple of 64; at
// most 128 for the solver's products, whose running sum takes TMEM columns,
// 256 for the sketch) and the X / V ring depths.  The first product of a
// shape (kernel, log2 n, feature width, columns, form) times every candidate
// that fits in shared memory once with CUDA events on the caller's stream and
// keeps the fastest; later products of that shape reuse it.  The choice does
// not change the result beyond rounding (all candidates compute the same
// product); the heuristic (widest chunk, deepest rings) serves while the
// tuner is off (kop_set_autotune) or the stream is being captured.
struct MmaShape {
  int kf, lgn, dp, mpad, sketch;
  bool operator<(const MmaShape& o) const {
    return std::tie(kf, lgn, dp, mpad, sketch) < std::tie(o.kf, o.lgn, o.dp, o.mpad, o.sketch);
  }
};
struct MmaTile {
  int mc, nx, nv;
};
static std::mutex g_tune_mu;
static std::map<MmaShape, MmaTile> g_tune;
static std::atomic<int> g_autotune{1};

static MmaTile heuristic_tile(int dp, int m, bool sketch) {
  const int vsplits = 2;
  MmaTile t;
  t.mc = mma_chunk(dp, m, vsplits, sketch ? 256 : 128);
  const size_t lim = smem_limit_bytes();
  // deepest rings that fit, the X ring first (it sets the MMA lookahead)
  t.nx = K3_MAXX;
  while (t.nx > 2 && mma_smem_bytes(dp, t.mc, t.nx, 2, vsplits) > lim) --t.nx;
  t.nv = K3_MAXV;
  while (t.nv > 2 && mma_smem_bytes(dp, t.mc, t.nx, t.nv, vsplits) > lim) --t.nv;
  return t;
}

int fused_matvec_mma(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, const float* V,
                     int m, int ldv, float* O, int ldo, int* status, cudaStream_t st, bool sketch) {
  const MmaTile h = heuristic_tile(Q.dp, m, sketch);
  if (h.mc == 0) return fail(KOP_EINVAL, "fused_matvec_mma: feature width too large");
  {
    int sc = ensure_scaled_norms(const_cast<PointSet&>(Q), kc.scale, st);
    if (sc == KOP_OK && &Q != &Ks) sc = ensure_scaled_norms(const_cast<PointSet&>(Ks), kc.scale, st);
    if (sc) return sc;
  }
  int lgn = 0;
  while ((int64_t(1) << (lgn + 1)) <= Ks.n) ++lgn;
  const MmaShape key{kf, lgn, Q.dp, (m + 63) / 64 * 64, sketch ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end())
      return run_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st, sketch, it->second.mc, it->second.nx,
                     it->second.nv);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  KOP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (!g_autotune.load() || cap != cudaStreamCaptureStatusNone)
    return run_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st, sketch, h.mc, h.nx, h.nv);
  // candidates: the heuristic's chunk width and the next narrower one (a
  // narrower chunk repeats the distance and kernel-value work per chunk:
  // measured 64-column chunks 3.5x slower at m = 500), with X rings of depth
  // 2 .. 4 and the deepest V ring that fits
  std::vector<MmaTile> cand;
  const size_t lim = smem_limit_bytes();
  for (int mc = h.mc > 64 ? h.mc - 64 : h.mc; mc <= h.mc; mc += 64)
    for (int nx = 2; nx <= K3_MAXX; ++nx) {
      if (mma_smem_bytes(Q.dp, mc, nx, 2, 2) > lim) continue;
      int nv = K3_MAXV;
      while (nv > 2 && mma_smem_bytes(Q.dp, mc, nx, nv, 2) > lim) --nv;
      cand.push_back(MmaTile{mc, nx, nv});
    }
  if (cand.empty()) cand.push_back(h);
  cudaEvent_t e0, e1;
  KOP_CUDA_TRY(cudaEventCreate(&e0));
  KOP_CUDA_TRY(cudaEventCreate(&e1));
  MmaTile best = h;
  float best_ms = 0.0f;
  int rc = KOP_OK;
  for (size_t i = 0; i < cand.size() && rc == KOP_OK; ++i) {
    const MmaTile& c = cand[i];
    cudaEventRecord(e0, st);
    rc = run_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st, sketch, c.mc, c.nx, c.nv);
    cudaEventRecord(e1, st);
    if (rc == KOP_OK && cudaEventSynchronize(e1) == cudaSuccess) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (i == 0 || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  // the output of the chosen shape (so that every product of this shape,
  // the first included, comes from the same arithmetic)
  return run_mma(Q, Ks, self, kf, kc, V, m, ldv, O, ldo, status, st, sketch, best.mc, best.nx, best.nv);
}

void set_mma_autotune(int enable) {
  g_autotune.store(enable ? 1 : 0);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

int mma_tuned_shapes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

}  // namespace kop
