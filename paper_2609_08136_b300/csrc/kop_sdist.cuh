// Issue of the distance MMAs S = Q_I X_J^T shared by the fused operator kernels.
#pragma once
#include "kop_device.cuh"

namespace kop {

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

// All MMAs of one distance tile, issued by lane 0 of the MMA warp (LANE0)
// or by the whole converged warp through elect.sync; which is faster depends
// on the kernel around it and is measured (lane 0 for the single-column
// product, elect.sync for the block product).  NKS = padded width / 16 K steps; the operands are 128-byte (or
// narrower) swizzled rows, so K step kc sits at row kc / KSPB of the split and
// 32-byte column kc % KSPB.  dq0 / xb are the descriptors of the first split
// of Q and of this X stage; *_split16 / *_sub16 are the byte strides between
// splits and between 128-byte row groups, in descriptor units (16 bytes).
// Every offset is a compile-time multiple of those strides.  Terms run in the
// order above over the whole K range, so the small products sum first.
template <int NSPLIT, int NKS, bool LANE0>
KOP_DEV void issue_s_tile(uint32_t d, uint64_t dq0, uint64_t xb, uint32_t q_split16, uint32_t x_split16,
                          uint32_t q_sub16, uint32_t x_sub16, uint32_t idesc) {
  constexpr int KSPB = NKS < 4 ? NKS : 4;
#pragma unroll
  for (int term = 0; term < n_terms<NSPLIT>(); ++term) {
#pragma unroll
    for (int kc = 0; kc < NKS; ++kc) {
      const uint32_t qo = (kc / KSPB) * q_sub16 + 2 * (kc % KSPB);
      const uint32_t xo = (kc / KSPB) * x_sub16 + 2 * (kc % KSPB);
      const uint64_t ad = dq0 + term_a<NSPLIT>(term) * q_split16 + qo;
      const uint64_t bd = xb + term_b<NSPLIT>(term) * x_split16 + xo;
      if constexpr (LANE0) {
        if ((threadIdx.x & 31) == 0) tc_mma_ss(d, ad, bd, idesc, (kc | term) ? 1u : 0u);
      } else {
        tc_mma_ss_elect(d, ad, bd, idesc, (kc | term) ? 1u : 0u);
      }
    }
  }
}

}  // namespace kop
