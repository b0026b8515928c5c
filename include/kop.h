/*
 * kop.h - C ABI of a single-GPU (B300, sm_103a) Nystrom-preconditioned CG
 * solver for dense regularized kernel systems
 *
 *     (K(X, X) + lam I) x = b,        K_ij = k(x_i, x_j),
 *
 * the problem class of the paper's Sec. 2.1 (Eq. "rlaopt-regularized-linear-
 * system"; kernel ridge regression, Eq. "rlaopt-krr", whose optimality
 * condition is exactly this system with b = y).  K is never formed: every
 * product K V is computed tile by tile by a fused kernel (distances on the
 * tensor cores, kernel function in registers, contraction with V) - the
 * matrix-free linear operator of Sec. 4.3.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices are row-major FP32 unless stated.  X is n x d, a block of vectors
 *   V is n x m (m columns, column c of row i at V[i*m + c]).
 * - Array pointers are DEVICE pointers owned by the caller and borrowed only
 *   for the duration of the call (stream-ordered on `stream`, a cudaStream_t
 *   passed as void*; NULL = legacy default stream).  Arguments documented as
 *   "host" are host pointers.
 * - Handles own device copies of whatever they keep: kop_t keeps the centred
 *   points, their row norms and their BF16 split; nys_t keeps U and the
 *   approximate eigenvalues.  A nys_t must not outlive the kop_t it was built
 *   from.  Handles are not thread-safe; distinct handles may be used from
 *   distinct host threads.
 * - Every call returns a status (enum kop_status).  No C++ exception crosses
 *   the ABI.  On failure kop_last_error() returns a message for the calling
 *   host thread.  Invalid arguments (n < 1, d outside 1..128, bandwidth or
 *   shifts not finite and > 0, null pointers, m < 1) give KOP_EINVAL with
 *   nothing launched.  Device-side waits are bounded: a wait that runs out
 *   makes the call return KOP_ETIMEOUT instead of hanging.
 */
#ifndef KOP_H_
#define KOP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kop_s* kop_t;
typedef struct nys_s* nys_t;

/* Kernel functions.  The paper names only k(x_i, x_j) (Sec. 2.1); the forms
 * follow Rasmussen & Williams (cited there for GP inference), with Euclidean
 * r = ||x_i - x_j|| and bandwidth s (sigma, or the Matern lengthscale):
 *   RBF       exp(-r^2 / (2 s^2))
 *   LAPLACE   exp(-r / s)
 *   MATERN52  (1 + sqrt5 r/s + 5 r^2 / (3 s^2)) exp(-sqrt5 r / s)          */
enum kop_kernel { KOP_RBF = 0, KOP_LAPLACE = 1, KOP_MATERN52 = 2 };

/* Operator precision modes.
 *   KOP_FAST      distances from a 2-term BF16 split (hi + mid) of the centred
 *                 points on the tensor cores (3 MMAs, FP32 accumulation);
 *                 entries accurate to about 2^-15 relative.
 *   KOP_ACCURATE  3-term split (6 MMAs), entries accurate to FP32 rounding;
 *                 used for the periodic true residual of the solver.
 *   KOP_PLAIN     plain FP32 CUDA-core path: direct-difference distances,
 *                 FP32 exp and FMA contraction; no tensor cores.  The speed
 *                 baseline of the fused path.
 *   KOP_EXACT     FP64 CUDA-core path: direct differences of the original
 *                 points, FP64 kernel values and accumulation (the paper's
 *                 float64 residual check, App. B.2).  About two orders of
 *                 magnitude slower than KOP_FAST on a B300; meant for true
 *                 residuals of small or badly conditioned problems.         */
enum kop_mode { KOP_FAST = 0, KOP_ACCURATE = 1, KOP_PLAIN = 2, KOP_EXACT = 3 };

enum kop_status {
  KOP_OK = 0,
  KOP_NOT_CONVERGED = 1, /* warning: maxit reached, outputs written        */
  KOP_EINVAL = -1,       /* invalid argument, nothing launched              */
  KOP_ENOMEM = -2,       /* device allocation failed                        */
  KOP_ECUDA = -3,        /* CUDA runtime/launch error                        */
  KOP_ENOTPD = -4,       /* Cholesky pivot <= 0 or PCG breakdown p^T A p <= 0 */
  KOP_ETIMEOUT = -5      /* a bounded device-side wait ran out              */
};

/* Message describing the last failure on this host thread ("" if none). */
const char* kop_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * host threads; a diagnostic for benchmarks).  Not in the paper: it only
 * reports on the library itself. */
int64_t kop_launch_count(void);

/* Measured SFU throughput of the current device, in operations per second:
 * rates[0] = ex2.approx, rates[1] = sqrt.approx, rates[2] = rsqrt.approx
 * (host array of 3).  The m = 1 operator product is bound by these units, so
 * they are the denominators of its roofline.  Runs each of three short probe
 * kernels four times on `stream` (the first warms up; the fastest of the
 * others gives the rate) and synchronizes it.  Not in the paper: a
 * measurement helper. */
int kop_sfu_rates(double* rates, void* stream);

/* Tile autotuner of the block operator product (m > 8 columns): the column
 * chunk and the ring depths of the fused tensor-core kernel.  When on (the
 * default), the first product of a shape (kernel, log2 n, feature width,
 * columns rounded up to 64, sketch or solver form) runs each candidate (the
 * heuristic's column chunk and the next narrower one, with every X-ring depth
 * that fits in shared memory) once, timed with CUDA events on the caller's stream
 * (which this synchronizes), keeps the fastest for that shape, and returns
 * the product computed with it; later products of the shape reuse it.
 * Candidates differ only in rounding.  Off: a fixed heuristic (widest chunk,
 * deepest rings).  A stream being captured is never tuned.  kop_set_autotune
 * clears the tuned shapes; kop_autotune_shapes returns how many are cached.
 * Not in the paper: a performance control. */
int kop_set_autotune(int32_t enable);
int32_t kop_autotune_shapes(void);

/* ---------------------------------------------------------------------------
 * Kernel operator (the matrix-free linear operator of Sec. 4.3; K of
 * Sec. 2.1 Eq. "rlaopt-krr").
 *
 * kop_create: X (device, n x d FP32) is copied: the column mean is removed
 * (k depends on x_i - x_j only, so K is unchanged), then FP32 row norms and
 * the hi/mid/lo BF16 split are stored, padded to 128 rows and to d' in
 * {16, 32, 64, 128} columns.  Synchronizes `stream` before
 * returning.  1 <= n < 2^31, 1 <= d <= 128.  Device memory held:
 * about n * d' * 10 bytes.                                                  */
int kop_create(const float* X, int64_t n, int32_t d, int32_t kernel, double bandwidth,
               void* stream, kop_t* out);
/* The normal operator A = X^T X of a data matrix X (device, n x p FP32
 * row-major; copied), the operator of ridge regression (X^T X + lam I) w =
 * X^T y in the paper's ridge experiments (Sec. 5.1).  A is applied as
 * X^T (X V) by two passes over X, never formed.  The handle works with
 * kop_matvec (mode KOP_FAST: FP32; KOP_ACCURATE / KOP_PLAIN: error-free
 * float-float sums of exact FP32 products), kop_matvec_f64 (deriv = 0),
 * nys_build, nys_build_adaptive, pcg_solve and pcg_adjoint (dL/dbw = 0); its
 * vectors have p entries.  Entry points of kernel operators only (bandwidth,
 * cross products, point gradients) return KOP_EINVAL.
 * 1 <= n < 2^31, 1 <= p <= 65536.                                          */
int kop_create_ridge(const float* X, int64_t n, int32_t p, void* stream, kop_t* out);
int kop_destroy(kop_t op);
/* Change the bandwidth in place (the points are kept). */
int kop_set_bandwidth(kop_t op, double bandwidth);

/* Keep the kernel matrix of the solver's checks in device memory.  K is
 * symmetric, so each pair of 128-point row blocks is stored once: nb x
 * (floor(nb / 2) + 1) tiles of 128 x 128 FP32, nb = ceil(n / 128) (about
 * n^2 * 2 bytes, 80 GB at n = 200000).  While it is set, the first product of
 * a pcg_solve / pcg_adjoint call with the check operator KOP_PLAIN_CHECK
 * (refine_mode or check_mode KOP_PLAIN) computes those tiles by direct
 * differences as that operator does and stores them, and every check product
 * of the call reads each stored tile once for both of its contributions
 * (K_IJ v_J and K_IJ^T v_I) with the same error-free contraction: about the
 * cost of streaming half of K, instead of recomputing n^2 distances.  The
 * stored values serve that one call only; every call recomputes them.
 * Results equal those without the matrix up to the order of the compensated
 * sums.  A scratch of nb x floor(nb / 2) x 128 x 16 floats at most (the
 * column parts as sum / error pairs) is reserved on first use and freed with
 * the matrix.
 *   enable = 0: stop using it; memory the library reserved is freed (the
 *               device is synchronized first).
 *   enable != 0, buffer = NULL: the library reserves the matrix (kept until
 *               disabled or kop_destroy); KOP_ENOMEM, reserving nothing, when
 *               it and 4 GB of headroom do not fit in the free device memory.
 *   enable != 0, buffer != NULL: the caller's device memory of buffer_floats
 *               >= nb * (floor(nb / 2) + 1) * 16384 floats, 16-byte aligned
 *               (KOP_EINVAL otherwise); the
 *               caller keeps ownership and may free it once the solves that
 *               used it have completed on their streams.
 * Solves on one handle that overlap in time share the matrix: run them one
 * after another while it is set.  KOP_EINVAL for ridge operators.  Not in the
 * paper: a trade of HBM capacity for the check's distance work that a B300's
 * 270 GB makes possible.                                                    */
int kop_set_check_cache(kop_t op, int32_t enable, float* buffer, int64_t buffer_floats);

/* O (n x m) = K(X, X) V for V (n x m).  mode: enum kop_mode.  Asynchronous;
 * the device status of the operator is read by kop_sync(). */
int kop_matvec(kop_t op, const float* V, int32_t m, float* O, int32_t mode, void* stream);

/* Rectangular products against other points Z (device, nz x d FP32; centred
 * with the operator's own column mean):
 *   transpose = 0:  O (nz x m) = K(Z, X) V,     V is n x m
 *   transpose = 1:  O (n x m)  = K(X, Z) V,     V is nz x m
 * deriv = 1 replaces k by dk/d(bandwidth) (used by the adjoint gradient).   */
int kop_cross_matvec(kop_t op, const float* Z, int64_t nz, const float* V, int32_t m, float* O,
                     int32_t transpose, int32_t deriv, int32_t mode, void* stream);

/* FP64 product with the KOP_EXACT operator: O (n x m, FP64) = K V (V FP64),
 * or (dK/d bandwidth) V when deriv != 0. */
int kop_matvec_f64(kop_t op, const double* V, int32_t m, double* O, int32_t deriv, void* stream);

/* O (n x m) = (dK(X, X)/d bandwidth) V. */
int kop_dbw_matvec(kop_t op, const float* V, int32_t m, float* O, int32_t mode, void* stream);

/* Gradient of a^T K(X) b with respect to the points X (the backward product
 * of the operator for its inputs; the paper differentiates through the solve,
 * Sec. 3.2): with c_ij = a_i b_j + a_j b_i and h(r) = -k'(r) / r,
 *   G[i] = d(a^T K b)/dx_i = -sum_j c_ij h(|x_i - x_j|) (x_i - x_j),
 *   RBF h = k / bw^2;  Laplace h = k / (bw r) (0 at r = 0, where k has no
 *   derivative);  Matern-5/2 h = (5 / (3 bw^2)) (1 + a) e^-a, a = sqrt(5) r / bw.
 * a, b: device n FP32;  G: device n x d FP32 row-major (overwritten).
 * mode: KOP_FAST or KOP_ACCURATE (fused tensor-core products on the centred
 * points) or KOP_EXACT (FP64 direct differences); KOP_PLAIN is KOP_EINVAL.
 * Synchronizes `stream`.                                                    */
int kop_grad_points(kop_t op, const float* a, const float* b, int32_t mode, float* G, void* stream);

/* Synchronize `stream` and return the operator's device status (KOP_OK or
 * KOP_ETIMEOUT), clearing it. */
int kop_sync(kop_t op, void* stream);

/* ---------------------------------------------------------------------------
 * Randomized Nystrom preconditioner (Frangella, Tropp & Udell, cited in
 * Sec. 1 and Sec. 2.3; NystromConfig, App. A.5).
 *
 * nys_build: Omega (device, n x r FP32) is the caller's test matrix (the
 * library does not orthonormalize it; Gaussian N(0,1)/sqrt(n) entries are
 * expected).  It is used as given in every step (the KOP_FAST sketch's
 * tensor-core contraction carries it, scaled per column by a power of two,
 * as an FP16 hi + lo pair of 22 significant bits against the kernel values
 * rounded to FP16, about 2^-12 relative per entry).  Steps: Y = K Omega (fused operator, `mode`),
 * nu = nu_rel * ||Y||_2 (nu_rel <= 0 selects 2^-16 for KOP_FAST and 2^-21
 * otherwise), Y_nu = Y + nu Omega, C = chol(sym(Omega^T Y_nu)) in FP64 (on a
 * failed pivot nu grows 10x, at most 3 times, then KOP_ENOTPD),
 * eigen-decomposition of C^-T (Y_nu^T Y_nu) C^-1 = V S^2 V^T in FP64,
 * U = Y_nu C^-1 V S^-1 (re-orthonormalized once), lam_hat = max(0, S^2 - nu)
 * in descending order.  1 <= r <= min(n, 2048).  Synchronizes `stream`.   */
int nys_build(kop_t op, const float* Omega, int32_t r, double nu_rel, int32_t mode, void* stream,
              nys_t* out);
int nys_destroy(nys_t ny);

/* Nystrom approximation with rank adaptation (NystromConfig rank_init,
 * rank_max, num_power_iters, error_tolerance; App. A.5).  The paper lists the
 * controls only; the scheme here is Frangella, Tropp & Udell's adaptive one:
 * r = rank_init; build the rank-r approximation (nys_build) from the first r
 * columns of Omega; estimate its error ||K - U diag(lam_hat) U^T||_2 by
 * power_iters power iterations from the start vector g0; accept r when
 * estimate <= err_tol * lam_hat_1 or r == rank_max, else r = min(2r, rank_max).
 *   Omega      device, n x ld_omega FP32 row-major (ld_omega >= rank_max), the
 *              caller's test matrix as for nys_build
 *   g0         device, n FP32, nonzero (the caller draws it)
 *   nu_rel, mode   as for nys_build (mode also selects the operator of the
 *              error estimate's products K v)
 *   out        the accepted approximation (free with nys_destroy)
 *   rank_out, err_out   host, optional: accepted rank and its error estimate
 *   hist_rank, hist_err, hist_len   host, optional: rank and estimate of each
 *              build, in order (at most hist_len entries are written; at most
 *              1 + ceil(log2(rank_max / rank_init)) builds happen)
 * 1 <= rank_init <= rank_max <= min(n, 2048), 1 <= power_iters <= 1000,
 * err_tol >= 0; otherwise KOP_EINVAL.  Errors of a build are returned as by
 * nys_build.  Synchronizes `stream`.                                         */
int nys_build_adaptive(kop_t op, const float* Omega, int32_t ld_omega, int32_t rank_init, int32_t rank_max,
                       int32_t power_iters, double err_tol, const float* g0, double nu_rel, int32_t mode,
                       void* stream, nys_t* out, int32_t* rank_out, double* err_out, int32_t* hist_rank,
                       double* hist_err, int32_t hist_len);

/* O = P^-1 V column by column, with damping mu[c] (host, m values):
 *   P^-1 v = v / rho + U [ (diag(lam_hat) + mu I)^-1 - I / rho ] U^T v,
 *   rho = lam_hat_r + mu (adaptive != 0) or mu (adaptive == 0).
 * This is the inverse of the damped Nystrom preconditioner of App. A.5
 * ("damping_mode") divided by rho; PCG iterates do not depend on that
 * scale.  V, O: device n x m.  mu[c] must be finite and > 0; mu[c] = 0 is
 * accepted only with adaptive != 0 and lam_hat_r > 0 (else 1 / (lam_k + mu)
 * would divide by zero): KOP_EINVAL otherwise.                              */
int nys_apply(nys_t ny, const double* mu, int32_t adaptive, const float* V, int32_t m, float* O,
              void* stream);

/* Same result as nys_apply for 1 <= m <= 8 columns, but without allocating
 * any device memory.  There is no counterpart in the paper: this exists for
 * callers that cannot allocate on this path (a latency-critical loop that must
 * avoid the device-wide synchronization of cudaMalloc/cudaFree, or an
 * application whose device memory is owned by its own allocator).  Its scratch
 * is a fixed array of 16448 doubles (128.5 KB) inside the library's device
 * image, held on every GPU that loads the library until the process exits;
 * r * m + m must fit in it (r <= 2048 with m <= 8 always does), else
 * KOP_EINVAL.  mu as for nys_apply.  The arithmetic is nys_apply's
 * (float-float projections).  All calls share that array: calls whose GPU work overlaps race,
 * so order them on one stream.  The first call on a device looks up the
 * array's address and should come before any stream capture.               */
int nys_apply_noalloc(nys_t ny, const double* mu, int32_t adaptive, const float* V, int32_t m,
                      float* O, void* stream);

/* Host copies: lam_hat (r doubles, descending), nu (1 double), r (int). */
int nys_eigs(nys_t ny, double* lam_hat, double* nu, int32_t* r);
/* Device copy of U (n x r FP32 row-major) into U_out. */
int nys_factor(nys_t ny, float* U_out, void* stream);

/* ---------------------------------------------------------------------------
 * Preconditioned CG (Hestenes & Stiefel, cited in Sec. 5.1) over a block of
 * independent columns: column c = s * nrhs + j solves
 *     (K + lambdas[s] I) x_c = B[:, j]
 * with its own alpha and beta; each column stops when its recursive residual
 * satisfies ||r|| <= tol ||b|| (PCGStoppingCriteria, App. A.1: the
 * condition must hold for every right-hand side) AND its float64 relative
 * residual ||b - (A + lam I) x|| / ||b|| (the paper's acceptance test,
 * App. B.2) is certified to be <= tol.  Certification: the true residual r
 * is recomputed with `check_mode` on all n rows; unless that is KOP_EXACT,
 * the exact FP64 residual r64 of the rows i_k = floor((2k+1) n / (2s)),
 * k < s, corrects it by the difference estimator
 *     est^2 = sum_i r_i^2 + (n/s) sum_k (r64_ik^2 - r_ik^2)
 * and the column is accepted when est^2 plus three standard errors of the
 * correction is <= tol^2 ||b||^2.  s = n for n <= 4096, else s = 1024
 * (ridge operators: every row); when s = n the FP64 residual of every row is
 * the true residual itself (the test is exact and `check_mode` is not run).
 * The solver's FP64 residuals take kernel values in FP64 from error-free FP32
 * distances (about 2^-44 relative in D^2).  What the check
 * operator missed lowers the column's next candidate threshold; when it is
 * above 0.8 tol^2 ||b||^2 the check operator cannot certify the tolerance and
 * the solve's later checks and refinements use KOP_EXACT.  A periodic
 * refinement with refine_mode == check_mode (not KOP_EXACT) evaluates the
 * same sampled FP64 rows and predicts that miss from the check's difference
 * to them, D = (n/s) sum (r64 - r)^2 plus the estimator's margin at the
 * tolerance, so that the first candidate stop already allows for it.  Every `refine_every` iterations
 * (0 = only at candidate stops and at maxit) the recursive residual is
 * replaced by the true one computed with `refine_mode` (iterative refinement:
 * operator products with `inner_mode`).  Recommended: inner KOP_FAST, refine
 * and check KOP_PLAIN (direct differences with error-free sums), or KOP_EXACT
 * for small badly conditioned systems, refine_every ~30.  A periodic
 * refinement is skipped when every active column's recursive residual is
 * within 8x the tolerance (the candidate stop that follows recomputes the
 * true residual itself).  The refinement
 * operator must be accurate well below the residuals it replaces: the
 * tensor-core KOP_ACCURATE operator's floor on clustered data far from the
 * common centre is ~1e-6, and refining with it there slowed or stopped
 * convergence.  ny = NULL gives plain CG
 * (IdentityConfig, App. A.1).
 * The preconditioner of column c uses damping mu[s] (host; NULL: mu = lambdas).
 *   lambdas      host, n_shifts values > 0
 *   B            device, n x nrhs
 *   X0           device or NULL, n x (nrhs * n_shifts) FP64: warm start (NULL:
 *                x0 = 0; columns with b = 0 return 0).  The first residual is
 *                b - (A + lam I) x0 with `check_mode`; a column whose start
 *                already meets the tolerance returns x0 after 0 iterations.
 *                (The inner solves of ADMM, App. A.4's NysADMM, warm-start
 *                from the previous x with a changing shift rho.)
 *   Xout         device, n x (nrhs * n_shifts), FP64.  The iterate is
 *                accumulated in FP64: FP32 storage of x alone would bound the
 *                attainable FP64 residual near 2^-24 ||A|| ||x|| / ||b||.
 *   iters        host, nrhs * n_shifts ints (operator products per column)
 *   res_hist     host or NULL, (maxit + 1) x cols doubles: recursive
 *                ||r_k|| / ||b|| per iteration (NaN after a column stops)
 *   true_relres  host or NULL, cols doubles: the certified FP64 relative
 *                residual (est / ||b||) of the last check of each column
 * Returns KOP_OK, KOP_NOT_CONVERGED (outputs written), KOP_ENOTPD on a
 * breakdown.  Synchronizes `stream`.                                         */
int pcg_solve(kop_t op, nys_t ny, const double* lambdas, int32_t n_shifts, const double* mu,
              int32_t adaptive, const float* B, int32_t nrhs, const double* X0, double tol, int32_t maxit,
              int32_t refine_every, int32_t inner_mode, int32_t refine_mode, int32_t check_mode,
              double* Xout, int32_t* iters, double* res_hist, double* true_relres, void* stream);

/* Adjoint of one solve (the paper differentiates through the solver,
 * Sec. 3.2, Eq. "rlaopt-bilevel"; here by an adjoint solve instead of
 * unrolling, which gives the same gradient at convergence).  Given the
 * solution x of (K + lam I) x = b and dL/dx (device, n, both FP64), solves
 *     (K + lam I) g = dL/dx
 * with the same preconditioner (mu = lam), writes g (device, n, FP64) and the
 * host scalars
 *     dL/dlam = -g^T x,        dL/dbw|_K = -g^T (dK/dbw) x,
 * (dL/db = g), the derivative product taken with `check_mode`.  iters: host
 * int (may be NULL).                              */
int pcg_adjoint(kop_t op, nys_t ny, double lam, int32_t adaptive, const double* x,
                const double* dLdx, double tol, int32_t maxit, int32_t refine_every,
                int32_t inner_mode, int32_t refine_mode, int32_t check_mode, double* g_out,
                int32_t* iters, double* dLdlam, double* dLdbw, void* stream);

/* Gradient of a validation loss through the solve (the paper's bilevel
 * hyper-parameter problem, Sec. 3.2, Eq. "rlaopt-bilevel", for kernel ridge
 * regression): with x the solution of (K + lam I) x = y (device, n FP64, from
 * pcg_solve) and the validation set (Xval: device nval x d FP32, yval: device
 * nval FP32), all in the library:
 *     e = K(Xval, X) x - yval,            L = e^T e / nval,
 *     dL/dx = (2 / nval) K(X, Xval) e,    g = (K + lam I)^-1 dL/dx (adjoint
 *     PCG with the same preconditioner, mu = lam),
 *     dL/dlam = -g^T x,
 *     dL/dbw  = (2 / nval) e^T (dK(Xval, X)/dbw) x - g^T (dK/dbw) x,
 * (dL/dy = g).  The cross and derivative products use `check_mode` (KOP_PLAIN:
 * direct differences with error-free sums, on the exact two-term split of
 * each FP64 vector; KOP_EXACT: FP64).  Writes g_out (device, n FP64) and the
 * host scalars loss, dLdlam, dLdbw; iters: host int (may be NULL).  Kernel
 * operators only (KOP_EINVAL for ridge).  Returns as pcg_solve for the
 * adjoint solve.  Synchronizes `stream`.                                    */
int pcg_adjoint_val(kop_t op, nys_t ny, double lam, int32_t adaptive, const double* x, const float* Xval,
                    int64_t nval, const float* yval, double tol, int32_t maxit, int32_t refine_every,
                    int32_t inner_mode, int32_t refine_mode, int32_t check_mode, double* g_out, int32_t* iters,
                    double* loss, double* dLdlam, double* dLdbw, void* stream);

/* ---------------------------------------------------------------------------
 * The linear solve inside NysADMM (ADMMConfig, App. A.4: sigma, gamma,
 * preconditioner_update_freq; NysADMM is cited in Sec. 2.3 and Sec. 4.3).
 * The k-th admm_solve call (k = 1, 2, ...) solves
 *     (A + (rho_k + sigma) I) x_k = rhs_k
 * with pcg_solve, warm-started from x_{k-1} (x_0 = 0), to the relative
 * tolerance max(tol_min, k^-gamma), preconditioned by the randomized Nystrom
 * approximation of A built from the handle's copy of Omega (device n x r FP32)
 * in `nys_mode` on call 1 and every update_freq calls after it (update_freq
 * = 0: built once), damped by rho_k + sigma.  The paper lists these controls
 * without formulas; the schedule above is this library's reading.
 * A: any operator (kernel or ridge); the handle must not outlive it.
 * admm_create: 1 <= r <= min(n, 2048), update_freq >= 0, sigma >= 0, gamma >= 0,
 *   0 < tol_min < 1, maxit >= 1, refine_every >= 0, modes as for pcg_solve;
 *   synchronizes `stream`.
 * admm_solve: rhs device n FP32, rho >= 0 with rho + sigma > 0; writes x_out
 *   (device n FP64) and the host values iters, true_relres (the certified FP64
 *   relative residual), tol_used and rebuilt (1 when this call rebuilt the
 *   preconditioner), each optional.  Returns as pcg_solve.                  */
typedef struct admm_s* admm_t;
int admm_create(kop_t op, const float* Omega, int32_t r, int32_t update_freq, double sigma, double gamma,
                double tol_min, int32_t maxit, int32_t refine_every, int32_t nys_mode, int32_t inner_mode,
                int32_t refine_mode, int32_t check_mode, void* stream, admm_t* out);
int admm_solve(admm_t a, const float* rhs, double rho, double* x_out, int32_t* iters, double* true_relres,
               double* tol_used, int32_t* rebuilt, void* stream);
int admm_destroy(admm_t a);

#ifdef __cplusplus
}
#endif
#endif /* KOP_H_ */
