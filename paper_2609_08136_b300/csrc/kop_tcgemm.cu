// Tensor-core tall-skinny products of the Nystrom construction and of the
// preconditioner apply on blocks of columns (Sec. 2.3: the n r^2 matrix-matrix
// products that build the preconditioner are its dominant cost):
//   Gram:  C (p x q, FP64) = A^T B  over the n rows of A (n x p) and B (n x q)
//   tall:  O (n x q, FP32) = A W (+ alpha (.) V),  A n x p, W p x q.
// Both run on tcgen05 with every FP32 operand split exactly into three BF16
// terms (x = hi + mid + lo) and the six partial products whose size is above
// 2^-24 of the leading one (mid*mid, hi*lo, lo*hi, hi*mid, mid*hi, hi*hi).
//
// Accuracy.  The tensor core sums each MMA's products into its FP32
// accumulator with a truncating alignment, so a long chain of MMAs into one
// accumulator loses about one unit in the last place per MMA, all in the same
// direction.  Each 64-deep step therefore starts two fresh accumulators, one
// for hi*hi (four MMAs) and one for the five smaller terms (at most 2^-7 of
// it), and the epilogue warps add the step's partial to an FP32 register
// (round to nearest).  A Gram CTA sums at most TG_MAX_STEPS steps (4096 rows)
// this way and adds its tile to C in FP64.  So each output carries a few
// 2^-24 of every 64-term partial plus the rounding of a short FP32 sum, as a
// plain FP32 product would, and the loop does no FP64 arithmetic (FP64 is
// slow on this part).
//
// Operands reach shared memory by TMA in 128-byte swizzled K-major rows:
//  - the Gram contracts over the n rows, so both operands are stored
//    transposed and blocked by 64 rows ("t-split"): row (kt, c) of a split
//    holds A[64 kt .. 64 kt + 63][c];
//  - the tall product contracts over p, so A is split in place ("r-split",
//    n_pad x kp, kp = p rounded up to 64) and W transposed (q_pad x kp).
// One CTA takes a 128 x 128 output tile (and, for the Gram, a range of the
// rows).  Two smem stages and two TMEM step buffers (hi*hi and corrections,
// 256 columns each) alternate, so the MMAs of step i + 1 run while the
// epilogue drains step i.  The Gram adds its tile into C atomically in FP64;
// symmetric products (A = B) evaluate only the tiles on and above the diagonal
// and add each off-diagonal tile to both halves.
#include <algorithm>

#include "kop_dense.h"
#include "kop_device.cuh"
#include "kop_internal.h"
#include "kop_sdist.cuh"

namespace kop {

constexpr int TG_THREADS = 320;  // producer, MMA, 8 epilogue warps
constexpr uint32_t TG_SPLIT_BYTES = 128u * 64u * 2u;            // one split of a 128 x 64 operand tile
constexpr uint32_t TG_STAGE_BYTES = 6u * TG_SPLIT_BYTES;        // A and B, three splits each
constexpr uint32_t TG_BAR_OFF = 2u * TG_STAGE_BYTES;            // after two stages
constexpr size_t TG_SMEM = 1024 + TG_BAR_OFF + 256;
constexpr int TG_MAX_STEPS = 64;  // 64-row steps summed in FP32 by one Gram CTA

KOP_DEV bool tg_wait(uint64_t* bar, uint32_t parity, volatile int* abort_word, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_backoff(bar, parity, abort_word, status);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

KOP_DEV void tg_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > KOP_WAIT_LIMIT_NS) break;
  }
}

// The 6 x 4 MMAs of one 64-deep step, K = 16 at a time: the five small split
// pairs into dsmall, hi*hi into dbig, each starting from zero.  da / db:
// descriptors of the hi split of the stage's A and B tiles; mid and lo follow
// at TG_SPLIT_BYTES.
KOP_DEV void tg_issue_step(uint32_t dbig, uint32_t dsmall, uint64_t da, uint64_t db, uint32_t idesc) {
  constexpr uint32_t sp16 = TG_SPLIT_BYTES >> 4;
#pragma unroll
  for (int term = 0; term < 6; ++term) {
    const uint32_t d = term == 5 ? dbig : dsmall;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t ad = da + term_a<3>(term) * sp16 + 2 * kk;
      const uint64_t bd = db + term_b<3>(term) * sp16 + 2 * kk;
      tc_mma_ss_elect(d, ad, bd, idesc, ((term == 0 || term == 5) && kk == 0) ? 0u : 1u);
    }
  }
}

struct TcArgs {
  int nsteps_total;   // 64-deep steps of the contraction
  int steps_per_cta;  // Gram: steps per CTA along grid.y; tall: all
  int rows_a, rows_b; // rows of one split in the operand maps
  // Gram
  double* C;
  int ldc, p, q;
  int tq;             // 128-column tiles of C along q
  int sym;            // A == B: tiles ti <= tj only, mirrored
  int lda_t, ldb_t;   // ld of the t-splits (p, q rounded up to 128)
  // tall
  float* O;
  int ldo;
  int64_t n;
  int qo;             // columns of O
  const float* V;
  int ldv;
  const float* alpha_col;
  int* status;
};

// GRAM = true: C += A^T B; false: O = A W (+ alpha V).
template <bool GRAM>
__global__ void __launch_bounds__(TG_THREADS, 1)
    tc6_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + TG_BAR_OFF);
  uint64_t* full = bars;        // 2
  uint64_t* empty = bars + 2;   // 2
  uint64_t* afull = bars + 4;   // 2
  uint64_t* aempty = bars + 6;  // 2
  uint32_t* holder = (uint32_t*)(bars + 8);
  volatile int* abort_word = (volatile int*)(holder + 1);

  int ti = 0, tj = 0, k0 = 0, nsteps = a.nsteps_total;
  int64_t row0 = 0;
  if constexpr (GRAM) {
    // output tile (ti, tj): row-major over the tiles, or the upper triangle
    if (a.sym) {
      int idx = blockIdx.x;
      while (idx >= a.tq - ti) {
        idx -= a.tq - ti;
        ++ti;
      }
      tj = ti + idx;
    } else {
      ti = blockIdx.x / a.tq;
      tj = blockIdx.x - ti * a.tq;
    }
    k0 = blockIdx.y * a.steps_per_cta;
    const int k1 = min(a.nsteps_total, k0 + a.steps_per_cta);
    nsteps = k1 > k0 ? k1 - k0 : 0;
  } else {
    tj = blockIdx.x;
    row0 = (int64_t)blockIdx.y * 128;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 8);
    }
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(holder, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    int i = 0;
    for (; i < nsteps; ++i) {
      const int s = i & 1;
      if (!tg_wait(&empty[s], ((i >> 1) & 1) ^ 1, abort_word, a.status)) break;
      if (lane == 0) {
        uint8_t* st = smem + s * TG_STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], TG_STAGE_BYTES);
        for (int sp = 0; sp < 3; ++sp) {
          if constexpr (GRAM) {
            const int kt = k0 + i;
            tma_load_2d(st + sp * TG_SPLIT_BYTES, &ta, &full[s], 0, sp * a.rows_a + kt * a.lda_t + ti * 128);
            tma_load_2d(st + (3 + sp) * TG_SPLIT_BYTES, &tb, &full[s], 0, sp * a.rows_b + kt * a.ldb_t + tj * 128);
          } else {
            tma_load_2d(st + sp * TG_SPLIT_BYTES, &ta, &full[s], i * 64, sp * a.rows_a + (int)row0);
            tma_load_2d(st + (3 + sp) * TG_SPLIT_BYTES, &tb, &full[s], i * 64, sp * a.rows_b + tj * 128);
          }
        }
      }
      __syncwarp();
    }
    // nothing may be in flight when the CTA exits
    if (lane == 0)
      for (int u = (i - 2 > 0 ? i - 2 : 0); u < i; ++u) tg_drain(&full[u & 1], (u >> 1) & 1);
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    const uint32_t idesc = idesc_bf16_f32(128, 128);
    const uint64_t d0 = sdesc(smem_u32(smem), 1024u, 2u);
    constexpr uint32_t stage16 = TG_STAGE_BYTES >> 4, sp16 = TG_SPLIT_BYTES >> 4;
    for (int i = 0; i < nsteps; ++i) {
      const int s = i & 1;
      if (!tg_wait(&aempty[s], ((i >> 1) & 1) ^ 1, abort_word, a.status)) break;
      if (!tg_wait(&full[s], (i >> 1) & 1, abort_word, a.status)) break;
      tc_fence_after();
      const uint64_t da = d0 + (uint64_t)s * stage16;
      const uint32_t dbig = tmem + (uint32_t)s * 256u;
      tg_issue_step(dbig, dbig + 128u, da, da + 3 * sp16, idesc);
      tc_commit_elect(&empty[s]);
      tc_commit_elect(&afull[s]);
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------------- drain
    // warp w reads TMEM lanes 32 (w % 4) ..; the two warps of a lane quarter
    // take 64 columns each
    const int ep = warp - 2, quarter = warp & 3, half = ep >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)half * 64u;
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int i = 0; i < nsteps; ++i) {
      const int b = i & 1;
      if (!tg_wait(&afull[b], (i >> 1) & 1, abort_word, a.status)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t rb[16], rs[16];
        tmem_ld16(lane_addr + (uint32_t)b * 256u + 16u * h, rb);
        tmem_ld16(lane_addr + (uint32_t)b * 256u + 128u + 16u * h, rs);
        tmem_ld_wait16(rb);
        tmem_ld_wait16(rs);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          acc[16 * h + j] += __uint_as_float(rb[j]) + __uint_as_float(rs[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[b]);
    }
    if (ok && nsteps > 0 && !*abort_word) {
      if constexpr (GRAM) {
        const int row = ti * 128 + quarter * 32 + lane;
        const int col0 = tj * 128 + half * 64;
        if (row < a.p) {
#pragma unroll
          for (int j = 0; j < 64; ++j)
            if (col0 + j < a.q) atomicAdd(&a.C[(int64_t)row * a.ldc + col0 + j], (double)acc[j]);
          if (a.sym && ti != tj) {
#pragma unroll
            for (int j = 0; j < 64; ++j)
              if (col0 + j < a.q) atomicAdd(&a.C[(int64_t)(col0 + j) * a.ldc + row], (double)acc[j]);
          }
        }
      } else {
        const int64_t row = row0 + quarter * 32 + lane;
        const int c0 = tj * 128 + half * 64;
        if (row < a.n) {
          float* orow = a.O + row * a.ldo;
          const float* vrow = a.V ? a.V + row * a.ldv : nullptr;
#pragma unroll
          for (int j = 0; j < 64; ++j) {
            const int c = c0 + j;
            if (c < a.qo) {
              float v = acc[j];
              if (vrow) v = fmaf(a.alpha_col[c], vrow[c], v);
              orow[c] = v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ splits
KOP_DEV void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// t-split of (A + beta A2) (n x p, lda): split s, entry (i, c) at
// ((s nkt + i / 64) ld + c) 64 + i % 64; zero for i >= n or c >= p.
// Block (32, 8) transposes a 64-row x 32-column tile through shared memory;
// each thread writes two consecutive rows of one column as a BF16 pair.
__global__ void tsplit_kernel(const float* __restrict__ A, const float* __restrict__ A2, float beta, int lda,
                              int64_t n, int p, int ld, int64_t nkt, __nv_bfloat16* __restrict__ T) {
  __shared__ float tile[64][33];
  const int64_t kt = blockIdx.x;
  const int c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 64; r += 8) {
    const int64_t i = kt * 64 + r;
    const int c = c0 + threadIdx.x;
    float v = 0.0f;
    if (i < n && c < p) {
      v = A[i * lda + c];
      if (A2) v = fmaf(beta, A2[i * lda + c], v);
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  const int64_t split = nkt * ld * 64;
  for (int cc = threadIdx.y; cc < 32; cc += 8) {
    const int c = c0 + cc;
    if (c >= ld) continue;
    const int r = 2 * threadIdx.x;
    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
    split3(tile[r][cc], h0, m0, l0);
    split3(tile[r + 1][cc], h1, m1, l1);
    const int64_t o = (kt * ld + c) * 64 + r;
    *reinterpret_cast<__nv_bfloat162*>(T + o) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(T + split + o) = __halves2bfloat162(m0, m1);
    *reinterpret_cast<__nv_bfloat162*>(T + 2 * split + o) = __halves2bfloat162(l0, l1);
  }
}

// r-split of (A + beta A2) (n x p, lda) into three n_pad x kp arrays.
__global__ void rsplit_kernel(const float* __restrict__ A, const float* __restrict__ A2, float beta, int lda,
                              int64_t n, int64_t n_pad, int p, int kp, __nv_bfloat16* __restrict__ R) {
  const int64_t pairs = n_pad * (kp / 2);
  const int64_t split = n_pad * kp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < pairs; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / (kp / 2);
    const int c = 2 * (int)(t - i * (kp / 2));
    float v0 = 0.0f, v1 = 0.0f;
    if (i < n) {
      if (c < p) v0 = A2 ? fmaf(beta, A2[i * lda + c], A[i * lda + c]) : A[i * lda + c];
      if (c + 1 < p) v1 = A2 ? fmaf(beta, A2[i * lda + c + 1], A[i * lda + c + 1]) : A[i * lda + c + 1];
    }
    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
    split3(v0, h0, m0, l0);
    split3(v1, h1, m1, l1);
    const int64_t o = i * kp + c;
    *reinterpret_cast<__nv_bfloat162*>(R + o) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(R + split + o) = __halves2bfloat162(m0, m1);
    *reinterpret_cast<__nv_bfloat162*>(R + 2 * split + o) = __halves2bfloat162(l0, l1);
  }
}

// W (p x q, ldw) transposed and split: three q_pad x kp arrays, entry (c, k).
__global__ void wsplit_kernel(const float* __restrict__ W, int ldw, int p, int q, int q_pad, int kp,
                              __nv_bfloat16* __restrict__ R) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int k = k0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < p && c < q) ? W[(int64_t)k * ldw + c] : 0.0f;
  }
  __syncthreads();
  const int64_t split = (int64_t)q_pad * kp;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, k = k0 + threadIdx.x;
    if (c < q_pad && k < kp) {
      __nv_bfloat16 h, m, l;
      split3(tile[threadIdx.x][r], h, m, l);
      const int64_t o = (int64_t)c * kp + k;
      R[o] = h;
      R[split + o] = m;
      R[2 * split + o] = l;
    }
  }
}

// ------------------------------------------------------------------ host
int64_t tsplit_elems(int64_t n, int p) { return 3 * ((n + 63) / 64) * (int64_t)(((p + 127) / 128) * 128) * 64; }
int64_t rsplit_elems(int64_t n, int p) { return 3 * ((n + 127) / 128 * 128) * (int64_t)(((p + 63) / 64) * 64); }

int tsplit(const float* A, const float* A2, float beta, int lda, int64_t n, int p, __nv_bfloat16* T,
           cudaStream_t st) {
  const int ld = ((p + 127) / 128) * 128;
  const int64_t nkt = (n + 63) / 64;
  dim3 grid((unsigned)nkt, (unsigned)(ld / 32));
  tsplit_kernel<<<grid, dim3(32, 8), 0, st>>>(A, A2, beta, lda, n, p, ld, nkt, T);
  KOP_LAUNCHED();
  return KOP_OK;
}

int rsplit(const float* A, const float* A2, float beta, int lda, int64_t n, int p, __nv_bfloat16* R,
           cudaStream_t st) {
  const int64_t n_pad = (n + 127) / 128 * 128;
  const int kp = ((p + 63) / 64) * 64;
  const int64_t pairs = n_pad * (kp / 2);
  const int64_t blocks = std::min<int64_t>((pairs + 255) / 256, (int64_t)num_sms() * 16);
  rsplit_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, A2, beta, lda, n, n_pad, p, kp, R);
  KOP_LAUNCHED();
  return KOP_OK;
}

static int tg_attr(const void* fn) {
  KOP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
  return KOP_OK;
}

static TcArgs tc_args(int* status) {
  TcArgs a{};
  a.status = status;
  return a;
}

int gram_tc(const __nv_bfloat16* At, const __nv_bfloat16* Bt, int64_t n, int p, int q, bool sym, double* C, int ldc,
            int* status, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)p * ldc, st));
  if (n <= 0) return KOP_OK;
  static bool attr = false;
  if (!attr) {
    if (int rc = tg_attr((const void*)tc6_kernel<true>)) return rc;
    attr = true;
  }
  const int lda_t = ((p + 127) / 128) * 128, ldb_t = ((q + 127) / 128) * 128;
  const int64_t nkt = (n + 63) / 64;
  const int64_t rows_a = nkt * lda_t, rows_b = nkt * ldb_t;
  if (3 * rows_a > INT32_MAX || 3 * rows_b > INT32_MAX) return fail(KOP_EINVAL, "gram_tc: operand too large");
  CUtensorMap ta, tb;
  if (int rc = encode_tmap_bf16(&ta, At, 3 * rows_a, 64, 64, 128)) return rc;
  if (int rc = encode_tmap_bf16(&tb, Bt, 3 * rows_b, 64, 64, 128)) return rc;
  TcArgs a = tc_args(status);
  a.C = C;
  a.ldc = ldc;
  a.p = p;
  a.q = q;
  a.nsteps_total = (int)nkt;
  a.tq = ldb_t / 128;
  a.sym = sym ? 1 : 0;
  a.rows_a = (int)rows_a;
  a.rows_b = (int)rows_b;
  a.lda_t = lda_t;
  a.ldb_t = ldb_t;
  const int tp = lda_t / 128;
  const int tiles = sym ? tp * (tp + 1) / 2 : tp * a.tq;
  // split the rows so that the grid fills the SMs (one CTA each) at least
  // once, with at most TG_MAX_STEPS steps per CTA
  int64_t splits64 = std::max<int64_t>(std::max(1, num_sms() / tiles), (nkt + TG_MAX_STEPS - 1) / TG_MAX_STEPS);
  int splits = (int)std::min<int64_t>(splits64, nkt);
  a.steps_per_cta = (int)((nkt + splits - 1) / splits);
  splits = (int)((nkt + a.steps_per_cta - 1) / a.steps_per_cta);
  tc6_kernel<true><<<dim3((unsigned)tiles, (unsigned)splits), TG_THREADS, TG_SMEM, st>>>(ta, tb, a);
  KOP_LAUNCHED();
  return KOP_OK;
}

int tall_tc(const __nv_bfloat16* Ar, int64_t n, int p, const float* W, int ldw, int q, const float* V, int ldv,
            const float* alpha_col, float* O, int ldo, int* status, cudaStream_t st) {
  if (n <= 0 || q <= 0) return KOP_OK;
  static bool attr = false;
  if (!attr) {
    if (int rc = tg_attr((const void*)tc6_kernel<false>)) return rc;
    attr = true;
  }
  const int64_t n_pad = (n + 127) / 128 * 128;
  const int kp = ((p + 63) / 64) * 64;
  const int q_pad = ((q + 127) / 128) * 128;
  if (3 * n_pad > INT32_MAX) return fail(KOP_EINVAL, "tall_tc: operand too large");
  DevBuf wb;
  wb.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&wb.p, sizeof(__nv_bfloat16) * 3 * (size_t)q_pad * kp, st));
  __nv_bfloat16* Ws = (__nv_bfloat16*)wb.p;
  wsplit_kernel<<<dim3((unsigned)(kp / 32), (unsigned)(q_pad / 32)), dim3(32, 8), 0, st>>>(W, ldw, p, q, q_pad, kp,
                                                                                            Ws);
  KOP_LAUNCHED();
  CUtensorMap ta, tw;
  if (int rc = encode_tmap_bf16(&ta, Ar, 3 * n_pad, kp, 64, 128)) return rc;
  if (int rc = encode_tmap_bf16(&tw, Ws, 3 * (int64_t)q_pad, kp, 64, 128)) return rc;
  TcArgs a = tc_args(status);
  a.O = O;
  a.ldo = ldo;
  a.n = n;
  a.qo = q;
  a.nsteps_total = kp / 64;
  a.steps_per_cta = a.nsteps_total;
  a.rows_a = (int)n_pad;
  a.rows_b = q_pad;
  a.V = V;
  a.ldv = ldv;
  a.alpha_col = alpha_col;
  tc6_kernel<false><<<dim3((unsigned)(q_pad / 128), (unsigned)(n_pad / 128)), TG_THREADS, TG_SMEM, st>>>(ta, tw, a);
  KOP_LAUNCHED();
  return KOP_OK;
}

}  // namespace kop
