// Dense helpers (kop_dense.cu): tall-skinny products over the n rows and the
// small r x r FP64 factorizations used by the Nystrom construction.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kop {

// C (p x p, FP64) = A^T A (A: n x p, FP32 row-major) on the CUDA cores with
// exact products and error-free sums within each chunk of rows (about FP64
// accuracy).
int gram_sym(const float* A, int lda, int64_t n, int p, double* C, int ldc, cudaStream_t st);
// w (p, FP64) = U^T v for one vector v (stride ldv).
int utv(const float* U, int ldu, int64_t n, int p, const float* v, int ldv, double* w, cudaStream_t st);
// o = alpha[0] v + U w for one vector (alpha on the device).
int uw(const float* U, int ldu, int64_t n, int p, const float* w, const float* v, int ldv, const float* alpha,
       float* o, int ldo, cudaStream_t st);
// FP64-accurate projections for m <= 8 columns: W = U^T V, and
// O = alpha (.) V + U W (row-major V, O with m columns).
int utv64(const float* U, int ldu, int64_t n, int p, const float* V, int m, double* W, cudaStream_t st);
int uw64(const float* U, int ldu, int64_t n, int p, const double* W, const float* V, int m, const double* alpha,
         float* O, cudaStream_t st);
// Same two projections in float-float arithmetic (error-free FP32 pairs).
int utv_ff(const float* U, int ldu, int64_t n, int p, const float* V, int m, double* W, cudaStream_t st);
int uw_ff(const float* U, int ldu, int64_t n, int p, const float2* W, const float* V, int m, const double* alpha,
          float* O, cudaStream_t st);
// mode 0: M = sym(Goy) + nu Goo;  mode 1: M = Gyy + nu (Goy + Goy^T) + nu^2 Goo.
int combine(const double* Goo, const double* Goy, const double* Gyy, int r, double nu, int mode, double* M,
            cudaStream_t st);
// In-place lower Cholesky; info (device int): 0 ok, k+1 failed pivot k.
int cholesky(double* A, int r, int* info, cudaStream_t st);
// Solve L X = B (trans 0) or L^T X = B (trans 1) for the q columns of B (r x q).
int trsm(const double* L, int r, double* B, int ldb, int q, int trans, cudaStream_t st);
int transpose(const double* A, int r, double* B, int sym, cudaStream_t st);
int power_max_eig(const double* G, int r, int iters, double* out, cudaStream_t st);
// Symmetric eigen-decomposition (parallel Jacobi).  work: 4 re^2 + 160 doubles
// (re = r rounded up to even).  evals (r), evecs (r x r, eigenvectors in columns).
int sym_eig(const double* H, int r, double* work, int* status, double* evals, double* evecs, cudaStream_t st);
void extract_eig(const double* A, const double* V, int r, int re, double* w, double* E, cudaStream_t st);
inline size_t sym_eig_work_doubles(int r) {
  const size_t re = (size_t)(r + (r & 1));
  return 4 * re * re + 160;
}
int sort_desc(const double* w, int r, int* perm, cudaStream_t st);
int nys_finish(const double* w, const double* E, const int* perm, int r, double nu, double* lam, double* Wm,
               cudaStream_t st);
int d2f(const double* a, float* b, int64_t n, cudaStream_t st);
int eye(double* M, int r, cudaStream_t st);

// Tensor-core forms (kop_tcgemm.cu).  Operands are FP32 matrices split
// exactly into three BF16 terms; six partial products give FP32-accurate
// products.  t-split (Gram operands): 3 x ceil(n / 64) x p_pad128 x 64 BF16;
// r-split (row operand of the tall product): 3 x n_pad128 x kp (p rounded up
// to 64).  A2 (optional) is added as A + beta A2 before splitting.
int64_t tsplit_elems(int64_t n, int p);
int64_t rsplit_elems(int64_t n, int p);
int tsplit(const float* A, const float* A2, float beta, int lda, int64_t n, int p, __nv_bfloat16* T,
           cudaStream_t st);
int rsplit(const float* A, const float* A2, float beta, int lda, int64_t n, int p, __nv_bfloat16* R,
           cudaStream_t st);
// C (p x q, FP64, ldc) = A^T B from the t-splits of A and B (sym: B is A).
int gram_tc(const __nv_bfloat16* At, const __nv_bfloat16* Bt, int64_t n, int p, int q, bool sym, double* C, int ldc,
            int* status, cudaStream_t st);
// O (n x q, ldo) = A W (+ alpha_col (.) V) from the r-split of A (n x p) and W
// (p x q, FP32, ldw).
int tall_tc(const __nv_bfloat16* Ar, int64_t n, int p, const float* W, int ldw, int q, const float* V, int ldv,
            const float* alpha_col, float* O, int ldo, int* status, cudaStream_t st);

}  // namespace kop
