// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kop.h"

namespace kop {

// Kernel-function ids used by the device epilogues.  0..2 are k itself
// (enum kop_kernel), 3..5 its derivative with respect to the bandwidth.
// Kernel kinds of the products: k, dk/d(bandwidth) (3..5) and the radial
// derivative h(r) = -k'(r) / r of the point gradient (6..8).
enum {
  KF_RBF = 0, KF_LAPLACE = 1, KF_MATERN = 2,
  KF_DRBF = 3, KF_DLAPLACE = 4, KF_DMATERN = 5,
  KF_GRBF = 6, KF_GLAPLACE = 7, KF_GMATERN = 8
};

// Constants of the fused epilogue (kop_epilogue.cuh): the kernel sees
// u = scale * D2 and, for derivatives, multiplies by c2.
struct KConst {
  float scale, c2;
  double bw;  // bandwidth itself (plain path)
};
KConst kernel_constants(int kind, double bw);

// A prepared point set: centred FP32 copy, FP32 row norms and the BF16
// hi/mid/lo split, rows padded to a multiple of 128 and columns to dp.
struct PointSet {
  int64_t n = 0, n_pad = 0;
  int d = 0, dp = 0;
  float* xc = nullptr;     // n_pad x dp
  float* norms = nullptr;  // n_pad
  __nv_bfloat16* sp[3] = {nullptr, nullptr, nullptr};
  CUtensorMap tm[3][2];  // [split][0: 128-row boxes, 1: 64-row boxes]
  void* block = nullptr;
  float* xorig = nullptr;  // the caller's points, n x d FP32 (exact operator)
  float* snorm = nullptr;  // scale * norms (n_pad), built on demand
  float snorm_scale = 0.0f;
  // column parts of the symmetric single-vector product (built on demand)
  float* sym_scratch = nullptr;
  size_t sym_scratch_floats = 0;
};
// Make ps.snorm = scale * ps.norms (no-op if already built for this scale).
int ensure_scaled_norms(PointSet& ps, float scale, cudaStream_t st);

int padded_dim(int d);
int pointset_alloc(PointSet& ps, int64_t n, int d, cudaStream_t st);
void pointset_free(PointSet& ps, cudaStream_t st);
// Centre X with `mean` (device, d doubles), write xc, norms and the split.
int pointset_fill(PointSet& ps, const float* X, const double* mean, cudaStream_t st);
// Column mean of X (n x d) in FP64 into mean (device, d).
int column_mean(const float* X, int64_t n, int d, double* mean, cudaStream_t st);

// Fused operator: O (nq x m, ld ldo) = f(K(Q, Kset)) V (nk x m, ld ldv).
// nsplit: 2 (KOP_FAST) or 3 (KOP_ACCURATE).  self: Q and Kset are the same
// points, so the diagonal distance is set to exactly 0.
int fused_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, int nsplit,
                 const float* V, int m, int ldv, float* O, int ldo, int* status, cudaStream_t st,
                 bool sketch = false);
// Single-vector product of a point set with itself using the symmetry of K
// (2-term split): v holds n floats (n_pad when v_padded), 16-byte aligned.
int fused_matvec_sym(PointSet& P, int kf, const KConst& kc, const float* v, int v_padded, float* O, int* status,
                     cudaStream_t st);
// Tensor-core contraction variant for m > 8 (2-term split only).
// sketch: the Nystrom sketch, which tolerates a contraction that drifts by
// ~1e-5 relative (wider column chunks); other products keep it near FP32.
int fused_matvec_mma(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, const float* V,
                     int m, int ldv, float* O, int ldo, int* status, cudaStream_t st, bool sketch = false);
// Autotuner of the block product's tile shape (kop_fused_mma.cu): on / off
// (clears the cache), and the number of shapes tuned so far.
void set_mma_autotune(int enable);
int mma_tuned_shapes();
// Plain FP32 CUDA-core operator (same contract, no tensor cores); with
// `compensated` the contraction is error-free per entry (acceptance checks).
int plain_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, const float* V,
                 int m, int ldv, float* O, int ldo, cudaStream_t st, bool compensated = false);
// Internal mode id of the compensated plain operator (not part of the ABI).
constexpr int KOP_PLAIN_CHECK = 100;

// FP64 CUDA-core operator (KOP_EXACT): FP64 V and O, and an FP32 wrapper.
int exact_matvec(const PointSet& Q, const PointSet& Ks, int kf, double bw, const double* V, int m, int ldv, double* O,
                 int ldo, cudaStream_t st);
int exact_matvec_f32(const PointSet& Q, const PointSet& Ks, int kf, double bw, const float* V, int m, int ldv,
                     float* O, int ldo, cudaStream_t st);
// The same FP64 product (kernels k only) with error-free FP32 distances:
// for few query rows (the certification of the solver's stops).
int cert_matvec(const PointSet& Q, const PointSet& Ks, int kf, double bw, const double* V, int m, int ldv, double* O,
                int ldo, cudaStream_t st);
// Any mode.
int op_matvec(const PointSet& Q, const PointSet& Ks, bool self, int kf, const KConst& kc, int mode,
              const float* V, int m, int ldv, float* O, int ldo, int* status, cudaStream_t st,
              bool sketch = false);

int num_sms();
inline size_t smem_limit_bytes() { return 227u * 1024u; }
int encode_tmap_bf16(CUtensorMap* map, const void* base, int64_t rows, int cols, int box_cols, int box_rows);

// Error reporting: set the thread-local message and return the code.
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
// Count one kernel launch and report a launch error.
void note_launch();
#define KOP_LAUNCHED()                      \
  do {                                      \
    ::kop::note_launch();                   \
    KOP_CUDA_TRY(cudaGetLastError());       \
  } while (0)
#define KOP_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::kop::cuda_fail(_e, #expr); \
  } while (0)

}  // namespace kop

namespace kop {
// Device part of nys_apply (scratch from the caller; see kop_nystrom.cu).
int nys_apply_dev(const nys_s* ny, const double* mu_dev, int adaptive, const float* V, int m, float* O, double* Wd,
                  double* alpha, float* Wf, float* alpha_f, cudaStream_t st);
}  // namespace kop

struct kop_s {
  kop::PointSet pts;
  int kernel = 0;
  double bw = 1.0;
  double* mean = nullptr;  // device, d
  int* status = nullptr;   // device status word
  // the normal operator X^T X of a data matrix (ridge regression) instead of a
  // kernel matrix, when ridge != 0
  int ridge = 0;
  float* rX = nullptr;  // device n x p copy of X
  int64_t rn = 0;       // rows of X
  int rp = 0;           // columns of X: the operator's dimension
  // the stored direct-difference kernel matrix of the solver's checks
  // (kop_set_check_cache): the 128 x 128 tiles of each row block's band
  // (sym_band_count), tile-packed FP32, or NULL
  float* kc = nullptr;
  int kc_owned = 0;  // kc was allocated by the library (else the caller's)
  // column parts of the symmetric product with the stored matrix (on demand)
  float* kc_scratch = nullptr;
  size_t kc_scratch_floats = 0;
};

namespace kop {
// Dimension of the operator's vectors, and that padded to 128 rows.
inline int64_t op_dim(const kop_s* op) { return op->ridge ? op->rp : op->pts.n; }
inline int64_t op_dim_pad(const kop_s* op) { return op->ridge ? ((int64_t)op->rp + 127) / 128 * 128 : op->pts.n_pad; }
// O = A V with the operator's product in `mode` (kernel K(X, X) or X^T X).
int op_apply(kop_s* op, int mode, const float* V, int m, int ldv, float* O, int ldo, cudaStream_t st,
             bool sketch = false);
// FP64 product with the operator (KOP_EXACT arithmetic).
int op_apply_f64(kop_s* op, const double* V, int m, int ldv, double* O, int ldo, cudaStream_t st);
int ridge_apply(const kop_s* op, int mode, const float* V, int m, int ldv, float* O, int ldo, cudaStream_t st);
int ridge_apply_f64(const kop_s* op, const double* V, int m, int ldv, double* O, int ldo, cudaStream_t st);
// The band of block pairs that the symmetric products evaluate: with nb row
// blocks of 128 points, block I takes the blocks J = I + t (mod nb) for
// t = 0 .. sym_band_count(I, nb) - 1, which covers every unordered pair once
// (floor(nb / 2) + 1 blocks; one fewer for I >= nb / 2 when nb is even).
__host__ __device__ inline int sym_band_count(int I, int nb) {
  const int h = nb / 2;
  if (nb & 1) return h + 1;
  return I < h ? h + 1 : h;
}
// Floats of the stored kernel matrix of an n-point operator: nb x
// (floor(nb / 2) + 1) tiles of 128 x 128 (each pair of row blocks once; the
// tile of row block I and band position t at (I (floor(nb / 2) + 1) + t) 128^2,
// row-major within the tile).
inline int64_t check_cache_floats(int64_t n) {
  const int64_t nb = (n + 127) / 128;
  return nb * (nb / 2 + 1) * 128 * 128;
}
// Reserve op->kc for the kernel matrix (KOP_ENOMEM when it does not fit).
int check_cache_reserve(kop_s* op);
// The compensated direct-difference product (KOP_PLAIN_CHECK) of a kernel
// operator with op->kc set, for the solver's checks: V2 (n x 2 cols) holds
// the exact hi / lo FP32 split of cols vectors (columns c and cols + c); T
// (n x 2 cols) receives each product as an unevaluated (sum, error) pair in
// the same two columns.  build = true first computes the stored matrix by
// direct differences.
int check_matvec_cached(kop_s* op, bool build, const float* V2, int cols, float* T, cudaStream_t st);
// The same product without the stored matrix: each pair of row blocks is
// computed once by direct differences (the build's arithmetic) in shared
// memory and used for both of its contributions.  *done = false (and nothing
// launched) when its column-part scratch does not fit in device memory.
int check_matvec_computed(kop_s* op, const float* V2, int cols, float* T, cudaStream_t st, bool* done);
}  // namespace kop

// Stream-ordered device scratch, freed on the same stream when it goes out of scope.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = 0;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

struct nys_s {
  kop_s* op = nullptr;
  int r = 0;
  int64_t n = 0;
  float* U = nullptr;            // device, n_pad x r
  // BF16 splits of U for the tensor-core apply on blocks of columns (built by
  // the first such apply): t-split (U^T V) and r-split (U W)
  __nv_bfloat16* Ut = nullptr;
  __nv_bfloat16* Ur = nullptr;
  double* lam_dev = nullptr;     // device, r (descending)
  double* lam_host = nullptr;    // host copy
  double nu = 0.0;
};
