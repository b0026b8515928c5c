// Preconditioned CG over a block of independent columns: pcg_solve and
// pcg_adjoint.
//
// PCG as in Hestenes & Stiefel (cited in the paper's Sec. 5.1), started from
// x0 = 0:  r = b, z = P^-1 r, p = z;  per iteration
//   q = (K + lam I) p,  alpha = r^T z / p^T q,  x += alpha p,  r -= alpha q,
//   stop if ||r|| <= tol ||b||,  z = P^-1 r,  beta = -z^T q / p^T q,
//   p = z + beta p.
// This beta is the flexible (Polak-Ribiere / Notay FCG(1)) form; with an
// exact symmetric preconditioner it equals r^T z_new / r^T z_old, and it
// keeps the recurrence stable when P^-1 is applied inexactly (FP32 blocks).
// Every column has its own alpha and beta and stops on its own (App. A.1: the
// stopping condition must hold for every right-hand side).  The products with
// K use the fast operator; every `refine_every` iterations, and whenever a
// column's recursive residual meets the tolerance, the true residual
// b - (K + lam I) x is recomputed with the accurate operator and replaces the
// recursive one (iterative refinement).  A column stops only when its float64
// relative residual (the paper's acceptance test, App. B.2) is certified to
// meet the tolerance: the check operator's residual over all n rows is
// corrected by the exact FP64 residual of a stride sample of rows (a
// difference estimator with a 3-sigma margin; exact when the sample is every
// row).  Vector updates run in fused passes over the n x cols block with FP64
// per-column reductions; the scalars alpha and beta never leave the device.
#include <cmath>
#include <string>
#include <vector>

#include "kop_dense.h"
#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

constexpr double kNearTol = 8.0;
// Rows of the FP64 residual that certifies a candidate stop: every row when
// n <= kCertAll, else a stride sample of kCertRows rows.
constexpr int64_t kCertAll = 4096;
constexpr int64_t kCertRows = 1024;
// One-sided margin of the certification, in standard errors of the sampled
// correction.
constexpr double kCertSigmas = 3.0;
// A check operator whose certified excess over its own residual is above
// this fraction of tol^2 cannot certify the tolerance: the solve switches
// its checks and refinements to the FP64 operator.
constexpr double kEscalate = 0.8;

enum { OP_INIT = 0, OP_PQ = 1, OP_XR = 2, OP_DOT = 3, OP_P = 4, OP_RES = 5, OP_DOT2 = 6, OP_SPLIT = 7, OP_RES64 = 8 };

// The iterate x is accumulated in FP64 (FP32 storage of x alone would limit
// the attainable FP64 residual to about 2^-24 ||A|| ||x|| / ||b||); p, r, z, q
// are FP32.  The true residual uses K applied to the exact hi/lo FP32 split
// of x (two columns per column of x).
struct VecArgs {
  int64_t n;
  int cols, nrhs;
  double* X;
  float* V2;  // n x 2 cols: [hi | lo] split of X (OP_SPLIT)
  float* R;
  const float* Z;
  float* P;
  float* Q;
  const float* B;  // n x nrhs; column c reads B[:, c % nrhs]
  const float* T;      // n x 2 cols: K applied to the split of X (OP_RES)
  const double* T64;   // n x cols: K X in FP64 (OP_RES64)
  const double* lam;
  const double* alpha;
  const double* beta;
  double* acc;   // per column, pre-zeroed
  double* acc2;  // second reduction (OP_DOT2: q^T z)
};

template <int OP>
KOP_DEV double2 vec_elem(const VecArgs& a, int64_t i, int c) {
  const int64_t e = i * a.cols + c;
  if constexpr (OP == OP_INIT) {
    const float b = a.B[i * a.nrhs + (c % a.nrhs)];
    a.X[e] = 0.0;
    a.R[e] = b;
    return make_double2((double)b * b, 0.0);
  } else if constexpr (OP == OP_PQ) {
    const float p = a.P[e];
    const float q = (float)((double)a.Q[e] + a.lam[c] * (double)p);
    a.Q[e] = q;
    return make_double2((double)p * q, 0.0);
  } else if constexpr (OP == OP_XR) {
    const double al = a.alpha[c];
    a.X[e] = a.X[e] + al * (double)a.P[e];
    const float r = (float)((double)a.R[e] - al * (double)a.Q[e]);
    a.R[e] = r;
    return make_double2((double)r * r, 0.0);
  } else if constexpr (OP == OP_DOT) {
    return make_double2((double)a.R[e] * (double)a.Z[e], 0.0);
  } else if constexpr (OP == OP_DOT2) {
    const double z = (double)a.Z[e];
    return make_double2((double)a.R[e] * z, (double)a.Q[e] * z);
  } else if constexpr (OP == OP_P) {
    a.P[e] = (float)((double)a.Z[e] + a.beta[c] * (double)a.P[e]);
    return make_double2(0.0, 0.0);
  } else if constexpr (OP == OP_SPLIT) {
    const double x = a.X[e];
    const float hi = (float)x;
    a.V2[i * 2 * a.cols + c] = hi;
    a.V2[i * 2 * a.cols + a.cols + c] = (float)(x - (double)hi);
    return make_double2(0.0, 0.0);
  } else if constexpr (OP == OP_RES64) {
    const double r = (double)a.B[i * a.nrhs + (c % a.nrhs)] - a.T64[e] - a.lam[c] * a.X[e];
    a.R[e] = (float)r;
    return make_double2(r * r, 0.0);
  } else {
    const int64_t t = i * 2 * a.cols + c;
    const double kx = (double)a.T[t] + (double)a.T[t + a.cols];
    const double r = (double)a.B[i * a.nrhs + (c % a.nrhs)] - kx - a.lam[c] * a.X[e];
    a.R[e] = (float)r;
    return make_double2(r * r, 0.0);
  }
}

// Several columns: 32 columns x 8 rows per block, row-strided.
template <int OP>
__global__ void __launch_bounds__(256) vec_cols_kernel(VecArgs a) {
  const int c = blockIdx.y * 32 + threadIdx.x;
  double acc = 0.0, acc2 = 0.0;
  if (c < a.cols)
    for (int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.y; i < a.n; i += (int64_t)gridDim.x * 8) {
      const double2 v = vec_elem<OP>(a, i, c);
      acc += v.x;
      acc2 += v.y;
    }
  if (OP == OP_P || OP == OP_SPLIT) return;
  __shared__ double red[2][8][33];
  red[0][threadIdx.y][threadIdx.x] = acc;
  red[1][threadIdx.y][threadIdx.x] = acc2;
  __syncthreads();
  if (threadIdx.y == 0 && c < a.cols) {
    double s = 0.0, s2 = 0.0;
    for (int y = 0; y < 8; ++y) {
      s += red[0][y][threadIdx.x];
      s2 += red[1][y][threadIdx.x];
    }
    atomicAdd(&a.acc[c], s);
    if (OP == OP_DOT2) atomicAdd(&a.acc2[c], s2);
  }
}

// One column: flat grid-stride with a block reduction.
template <int OP>
__global__ void __launch_bounds__(256) vec_one_kernel(VecArgs a) {
  double acc = 0.0, acc2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = vec_elem<OP>(a, i, 0);
    acc += v.x;
    acc2 += v.y;
  }
  if (OP == OP_P || OP == OP_SPLIT) return;
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  }
  __shared__ double red[2][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = acc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, s2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      s += red[0][w];
      s2 += red[1][w];
    }
    atomicAdd(&a.acc[0], s);
    if (OP == OP_DOT2) atomicAdd(&a.acc2[0], s2);
  }
}

template <int OP>
static int vec_launch(const VecArgs& a, cudaStream_t st) {
  if (OP != OP_P && OP != OP_SPLIT) KOP_CUDA_TRY(cudaMemsetAsync(a.acc, 0, sizeof(double) * a.cols, st));
  if (OP == OP_DOT2) KOP_CUDA_TRY(cudaMemsetAsync(a.acc2, 0, sizeof(double) * a.cols, st));
  if (a.cols == 1) {
    int64_t blocks = (a.n + 255) / 256;
    const int64_t cap = 8 * num_sms();
    if (blocks > cap) blocks = cap;
    vec_one_kernel<OP><<<(unsigned)blocks, 256, 0, st>>>(a);
  } else {
    const unsigned gy = (unsigned)((a.cols + 31) / 32);
    int64_t gx = (a.n + 7) / 8;
    const int64_t cap = (8 * num_sms() + gy - 1) / gy;
    if (gx > cap) gx = cap;
    vec_cols_kernel<OP><<<dim3((unsigned)gx, gy), dim3(32, 8), 0, st>>>(a);
  }
  KOP_LAUNCHED();
  return KOP_OK;
}

// alpha_c = rz_c / pq_c for active columns (0 otherwise); p^T q <= 0 on an
// active column is a breakdown.
__global__ void fin_alpha_kernel(int cols, const double* rz, const double* pq, const int* active, double* alpha,
                                 int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double al = 0.0;
  if (active[c]) {
    if (pq[c] > 0.0 && isfinite(pq[c]))
      al = rz[c] / pq[c];
    else
      atomicExch(status, KOP_DEV_BREAKDOWN);
  }
  alpha[c] = al;
}

// beta_c = -q_c^T z_c / p_c^T q_c (flexible form), rz_c <- r_c^T z_c.
__global__ void fin_beta_kernel(int cols, double* rz, const double* rzn, const double* qz, const double* pq,
                                double* beta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  beta[c] = pq[c] > 0.0 ? -qz[c] / pq[c] : 0.0;
  rz[c] = rzn[c];
}

// out += sum_i a_i (b_i + b2_i)   (b2 may be NULL); a in FP64.
__global__ void dot_kernel(const double* a, const float* b, const float* b2, int64_t n, int ldb, double* out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * ((double)b[i * ldb] + (b2 ? (double)b2[i * ldb] : 0.0));
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(out, s);
  }
}

__global__ void dot64_kernel(const double* a, const double* b, int64_t n, double* out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(out, s);
  }
}

// Rows of the certification sample: i_k = floor((2k + 1) n / (2 s)), k < s
// (every row when s = n).
__host__ __device__ inline int64_t cert_row(int64_t k, int64_t n, int64_t s) { return ((2 * k + 1) * n) / (2 * s); }

__global__ void gather_rows_kernel(const float* __restrict__ X, int d, int64_t n, int64_t s, float* __restrict__ Xs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s * d) return;
  const int64_t k = t / d;
  Xs[t] = X[cert_row(k, n, s) * d + (t - k * d)];
}

// Per column c over the sampled rows i: with the FP64 product O64 (s x cols)
// and the check's product T (n x 2 cols, the two columns of x's exact split),
//   r64 = b_i - O64_kc - lam_c x_ic,  rchk = b_i - (T_i,c + T_i,cols+c) - lam_c x_ic,
//   d = r64^2 - rchk^2;   sd_c += d, sd2_c += d^2, sd3_c += (r64 - rchk)^2.
__global__ void __launch_bounds__(256) certify_kernel(int64_t n, int64_t s, int cols, int nrhs,
                                                      const float* __restrict__ B, const double* __restrict__ X,
                                                      const float* __restrict__ T, const double* __restrict__ O64,
                                                      const double* __restrict__ lam, double* sd, double* sd2,
                                                      double* sd3) {
  const int c = blockIdx.y * 32 + threadIdx.x;
  double a = 0.0, a2 = 0.0, a3 = 0.0;
  if (c < cols)
    for (int64_t k = (int64_t)blockIdx.x * 8 + threadIdx.y; k < s; k += (int64_t)gridDim.x * 8) {
      const int64_t i = cert_row(k, n, s);
      const double bx = (double)B[i * nrhs + (c % nrhs)] - lam[c] * X[i * cols + c];
      const double r64 = bx - O64[k * cols + c];
      const int64_t t = i * 2 * cols + c;
      const double rc = bx - ((double)T[t] + (double)T[t + cols]);
      const double dd = (r64 - rc) * (r64 + rc);
      a += dd;
      a2 += dd * dd;
      a3 += (r64 - rc) * (r64 - rc);
    }
  __shared__ double red[3][8][33];
  red[0][threadIdx.y][threadIdx.x] = a;
  red[1][threadIdx.y][threadIdx.x] = a2;
  red[2][threadIdx.y][threadIdx.x] = a3;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    double u = 0.0, u2 = 0.0, u3 = 0.0;
    for (int y = 0; y < 8; ++y) {
      u += red[0][y][threadIdx.x];
      u2 += red[1][y][threadIdx.x];
      u3 += red[2][y][threadIdx.x];
    }
    atomicAdd(sd + c, u);
    atomicAdd(sd2 + c, u2);
    atomicAdd(sd3 + c, u3);
  }
}

// What the check operator will miss at a stop, predicted from its difference
// to the FP64 operator on the current iterate, D = (n / s) sum (r64 - rchk)^2
// (relative to ||b||^2, like tol^2): at a residual near the tolerance the
// certified excess is D plus the one-sided margin of the estimator, whose
// variance is dominated by the cross term 2 rchk (r64 - rchk):
//   D + kCertSigmas * 2 tol sqrt(D) sqrt(1 - s/n) / sqrt(s).
static double predict_excess(double sd3, double nb2, double tol, int64_t n, int64_t s) {
  const double D = (double)n / (double)s * sd3 / nb2;
  if (s >= n) return D;
  const double fpc = 1.0 - (double)s / (double)n;
  return D + kCertSigmas * 2.0 * tol * std::sqrt(D * fpc / (double)s);
}

// The certified squared residual of one column from the check's all-row sum
// S = sum_i rchk_i^2 and the sample sums of d_i = r64_i^2 - rchk_i^2:
//   est2 = S + (n / s) sum d   (the difference estimator of sum_i r64_i^2),
//   ub2  = est2 + kCertSigmas * n sqrt((1 - s/n) var(d) / s),
// exact (ub2 = est2 = sum r64^2) when s = n.
struct Cert {
  double est2, ub2;
};
static Cert certify_column(double S, double sd, double sd2, int64_t n, int64_t s) {
  const double ns = (double)n / (double)s;
  Cert ct;
  ct.est2 = S + ns * sd;
  ct.ub2 = ct.est2;
  if (s < n && s > 1) {
    const double mean = sd / (double)s;
    double var = (sd2 / (double)s - mean * mean) * ((double)s / (double)(s - 1));
    if (var < 0.0) var = 0.0;
    const double fpc = 1.0 - (double)s / (double)n;
    ct.ub2 += kCertSigmas * (double)n * std::sqrt(var * fpc / (double)s);
  }
  if (ct.est2 < 0.0) ct.est2 = 0.0;
  if (ct.ub2 < ct.est2) ct.ub2 = ct.est2;
  return ct;
}

struct PcgProblem {
  kop_s* op = nullptr;
  nys_s* ny = nullptr;
  int cols = 1, nrhs = 1;
  std::vector<double> lam, mu;
  int adaptive = 1;
  const float* B = nullptr;
  const double* X0 = nullptr;  // optional warm start (n x cols FP64)
  double* Xout = nullptr;
  double tol = 1e-6;
  int maxit = 1000, refine_every = 0, inner_mode = KOP_FAST, refine_mode = KOP_ACCURATE, check_mode = KOP_PLAIN;
  int32_t* iters = nullptr;
  double* res_hist = nullptr;
  double* true_relres = nullptr;
};

struct Workspace {
  void* p = nullptr;
  cudaStream_t st = 0;
  ~Workspace() {
    if (p) cudaFreeAsync(p, st);
  }
};

// A column becomes a stop candidate on the device as soon as its recursive
// residual meets the host's threshold thr2 = (tol^2 - excess) ||b||^2: it is
// made inactive (alpha = 0 from then on, so x and r keep that iteration's
// values) and the iteration is recorded for the host, which certifies the
// candidates at its next synchronization.
__global__ void freeze_kernel(int cols, const double* __restrict__ rr, const double* __restrict__ thr2,
                              int* __restrict__ active, int* __restrict__ frozen, int it) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  if (active[c] && rr[c] <= thr2[c]) {
    active[c] = 0;
    frozen[c] = it;
  }
}

// Iterations between host synchronizations: a small system's iteration takes
// less device time than a host round trip, so its iterations run in chunks
// whose residual norms are read back together (a candidate stop is frozen on
// the device at its own iteration, so the chunk costs at most a few idle
// iterations).  Large systems synchronize every iteration.
static int chunk_len(int64_t n, int cols) {
  const double work = (double)n * (double)n * (double)cols;
  if (work <= 268435456.0) return 8;    // e.g. n <= 16384 for one column
  if (work <= 1073741824.0) return 4;   // n <= 32768
  return 1;
}
constexpr int kChunkMax = 8;

static int device_status(kop_s* op, cudaStream_t st, int* h) {
  KOP_CUDA_TRY(cudaMemcpyAsync(h, op->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  return KOP_OK;
}

// X[i][c] = 0 for the columns c that are not active.
__global__ void zero_inactive_kernel(double* __restrict__ X, int64_t nc, int cols, const int* __restrict__ active) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nc && !active[t % cols]) X[t] = 0.0;
}

int pcg_core(PcgProblem& pb, cudaStream_t st) {
  kop_s* op = pb.op;
  const int64_t n = op_dim(op);
  const int cols = pb.cols;
  const size_t nc = (size_t)n * cols;
  const int r = pb.ny ? pb.ny->r : 0;
  Workspace ws;
  ws.st = st;
  const size_t fbytes = sizeof(float) * (8 * nc + (size_t)r * cols + cols);
  const size_t dbytes = sizeof(double) * (12 * (size_t)cols + (size_t)r * cols);
  const size_t ibytes = sizeof(int) * (size_t)cols;
  size_t xbytes = (pb.refine_mode == KOP_EXACT || pb.check_mode == KOP_EXACT) ? sizeof(double) * nc : 0;
  // certification of candidate stops: the sampled rows' points, their FP64
  // product (s x cols; every row of a ridge operator) and two sums per column
  const int64_t s_rows = (op->ridge || n <= kCertAll) ? n : kCertRows;
  const int dpt = op->ridge ? 0 : op->pts.d;
  const size_t cbytes = sizeof(double) * ((size_t)s_rows * cols + 3 * (size_t)cols) +
                        sizeof(float) * (size_t)s_rows * dpt + 64 +
                        sizeof(double) * (size_t)(kChunkMax + 1) * cols + sizeof(int) * (size_t)cols + 64;
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, xbytes + dbytes + fbytes + ibytes + 256, st));
  Workspace wc;
  wc.st = st;
  KOP_CUDA_TRY(cudaMallocAsync(&wc.p, cbytes, st));
  double* O64 = (double*)wc.p;
  double* csd = O64 + (size_t)s_rows * cols;
  double* csd2 = csd + cols;
  double* csd3 = csd2 + cols;
  float* samp_x = (float*)(csd3 + cols);
  // the chunk's squared residual norms, the candidate thresholds, the
  // iteration at which each column froze (0: none)
  double* hist = (double*)(((uintptr_t)(samp_x + (size_t)s_rows * dpt) + 63) & ~(uintptr_t)63);
  double* thr2 = hist + (size_t)kChunkMax * cols;
  int* frozen = (int*)(thr2 + cols);
  PointSet qs;
  if (!op->ridge) {
    qs.n = s_rows;
    qs.d = dpt;
    qs.xorig = samp_x;
    gather_rows_kernel<<<(unsigned)((s_rows * dpt + 255) / 256), 256, 0, st>>>(op->pts.xorig, dpt, n, s_rows, samp_x);
    KOP_LAUNCHED();
  }
  Workspace wx;  // the FP64 product of checks escalated to the exact operator
  wx.st = st;
  double* T64 = xbytes ? (double*)ws.p : nullptr;
  double* lam = (double*)ws.p + (xbytes / sizeof(double));
  double* mu = lam + cols;
  double* alpha = mu + cols;
  double* beta = alpha + cols;
  double* rz = beta + cols;
  double* acc = rz + cols;
  double* acc2 = acc + cols;
  double* pq = acc2 + cols;
  double* qz = pq + cols;
  double* palpha = qz + cols;
  double* spare = palpha + cols;
  double* spare2 = spare + cols;
  double* Wd = spare2 + cols;
  float* R = (float*)(Wd + (size_t)r * cols);
  float* Z = R + nc;
  float* P = Z + nc;
  float* Q = P + nc;
  float* T = Q + nc;      // n x 2 cols
  float* V2 = T + 2 * nc; // n x 2 cols
  float* Wf = V2 + 2 * nc;
  float* acol = Wf + (size_t)r * cols;
  int* active = (int*)(acol + cols);
  double* X = pb.Xout;

  std::vector<int> act(cols, 1);
  std::vector<double> hb(cols), nb(cols), rel(cols, 0.0), hr(cols);
  KOP_CUDA_TRY(cudaMemcpyAsync(lam, pb.lam.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
  KOP_CUDA_TRY(cudaMemcpyAsync(mu, pb.mu.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
  KOP_CUDA_TRY(cudaMemsetAsync(op->status, 0, sizeof(int), st));

  VecArgs va;
  va.n = n;
  va.cols = cols;
  va.nrhs = pb.nrhs;
  va.X = X;
  va.R = R;
  va.Z = Z;
  va.P = P;
  va.Q = Q;
  va.B = pb.B;
  va.T = T;
  va.T64 = T64;
  va.V2 = V2;
  va.lam = lam;
  va.alpha = alpha;
  va.beta = beta;
  va.acc = acc;
  va.acc2 = acc2;
  int rc;
  auto apply_prec = [&]() -> int {
    if (!pb.ny) {
      KOP_CUDA_TRY(cudaMemcpyAsync(Z, R, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));
      return KOP_OK;
    }
    return nys_apply_dev(pb.ny, mu, pb.adaptive, R, cols, Z, Wd, palpha, Wf, acol, st);
  };
  auto matvec = [&](const float* V, float* O, int mode) -> int {
    return op_apply(op, mode, V, cols, cols, O, cols, st);
  };
  auto matvec2 = [&](const float* V, float* O, int mode) -> int {
    return op_apply(op, mode, V, 2 * cols, 2 * cols, O, 2 * cols, st);
  };
  // check products: with the kernel matrix set in HBM, the first one of this
  // solve stores K and later ones multiply the stored K (its contents are
  // never reused across solves)
  bool kc_built = false;
  auto check2 = [&](int mode) -> int {
    if (mode != KOP_PLAIN_CHECK || op->ridge) return matvec2(V2, T, mode);
    if (!op->kc) {
      // no stored matrix: the symmetric product computes each pair of row
      // blocks once, else (its scratch does not fit) every entry is evaluated
      bool done = false;
      const int rc2 = check_matvec_computed(op, V2, cols, T, st, &done);
      if (rc2 || done) return rc2;
      return matvec2(V2, T, mode);
    }
    const int rc2 = check_matvec_cached(op, !kc_built, V2, cols, T, st);
    if (rc2 == KOP_OK) kc_built = true;
    return rc2;
  };

  // certified FP64 residual per column (relative to ||b||): trel = the
  // estimate, urel = its upper bound; excess = (ub2 - S) / ||b||^2, what the
  // check operator's residual S misses, which lowers the column's candidate
  // threshold tol^2 - excess
  std::vector<double> hsd_all(3 * (size_t)cols), trel(cols, 0.0), urel(cols, 0.0), excess(cols, 0.0);
  const double* hsd = hsd_all.data();              // sum d
  const double* hsd2 = hsd_all.data() + cols;      // sum d^2
  const double* hsd3 = hsd_all.data() + 2 * cols;  // sum (r64 - rchk)^2
  // The true residual r = b - (A + lam I) x with the operator `mode` replaces
  // R; with `certify`, a non-FP64 check is corrected by the sampled FP64
  // residual.  Fills trel / urel / excess for the active columns; with
  // `predict` (a refinement far from the tolerance, where the correction's
  // margin would be dominated by the residual itself) excess is instead the
  // prediction of what the check will miss at a stop (predict_excess), so
  // that the first candidate stop already leaves room for it.
  auto true_residual = [&](int mode, bool certify, bool predict = false) -> int {
    int rmode = mode == KOP_PLAIN ? KOP_PLAIN_CHECK : mode;
    // when the certification reads every row anyway (n <= kCertAll, ridge
    // operators), its FP64 product is the true residual itself and the check
    // operator is not run
    const bool exact = rmode == KOP_EXACT || ((certify || predict) && s_rows == n);
    if (exact) {
      if (!T64) {
        KOP_CUDA_TRY(cudaMallocAsync(&wx.p, sizeof(double) * nc, st));
        T64 = (double*)wx.p;
        va.T64 = T64;
      }
      // FP64 product: kernel values in FP64 from error-free FP32 distances
      // (about 2^-44 relative in D^2; FP64 distances are several times
      // slower on this part)
      if (op->ridge) {
        if ((rc = op_apply_f64(op, X, cols, cols, T64, cols, st))) return rc;
      } else {
        if ((rc = cert_matvec(op->pts, op->pts, op->kernel, op->bw, X, cols, cols, T64, cols, st))) return rc;
      }
      if ((rc = vec_launch<OP_RES64>(va, st))) return rc;
    } else {
      if ((rc = vec_launch<OP_SPLIT>(va, st))) return rc;
      if ((rc = check2(rmode))) return rc;
      if ((rc = vec_launch<OP_RES>(va, st))) return rc;
    }
    KOP_CUDA_TRY(cudaMemcpyAsync(hr.data(), acc, sizeof(double) * cols, cudaMemcpyDeviceToHost, st));
    const bool corr = certify && !exact;
    if (corr) {
      if (op->ridge) {
        if ((rc = op_apply_f64(op, X, cols, cols, O64, cols, st))) return rc;
      } else {
        if ((rc = cert_matvec(qs, op->pts, op->kernel, op->bw, X, cols, cols, O64, cols, st))) return rc;
      }
      KOP_CUDA_TRY(cudaMemsetAsync(csd, 0, sizeof(double) * 3 * cols, st));
      const unsigned gy = (unsigned)((cols + 31) / 32);
      int64_t gx = (s_rows + 7) / 8;
      if (gx > 2 * num_sms()) gx = 2 * num_sms();
      certify_kernel<<<dim3((unsigned)gx, gy), dim3(32, 8), 0, st>>>(n, s_rows, cols, pb.nrhs, pb.B, X, T, O64, lam,
                                                                    csd, csd2, csd3);
      KOP_LAUNCHED();
      KOP_CUDA_TRY(cudaMemcpyAsync(hsd_all.data(), csd, sizeof(double) * 3 * cols, cudaMemcpyDeviceToHost, st));
    }
    KOP_CUDA_TRY(cudaStreamSynchronize(st));
    for (int c = 0; c < cols; ++c) {
      if (!act[c]) continue;
      const double nb2 = nb[c] * nb[c];
      Cert ct{hr[c], hr[c]};
      if (corr) ct = certify_column(hr[c], hsd[c], hsd2[c], n, s_rows);
      trel[c] = std::sqrt(ct.est2 / nb2);
      urel[c] = std::sqrt(ct.ub2 / nb2);
      if (corr && predict) excess[c] = predict_excess(hsd3[c], nb2, pb.tol, n, s_rows);
      else if (corr) excess[c] = (ct.ub2 - hr[c]) / nb2 > 0.0 ? (ct.ub2 - hr[c]) / nb2 : 0.0;
      else if (exact) excess[c] = 0.0;
    }
    return KOP_OK;
  };

  // x0 = 0, r0 = b, ||b|| per column
  if ((rc = vec_launch<OP_INIT>(va, st))) return rc;
  KOP_CUDA_TRY(cudaMemcpyAsync(hb.data(), acc, sizeof(double) * cols, cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  bool any = false;
  for (int c = 0; c < cols; ++c) {
    nb[c] = std::sqrt(hb[c]);
    if (pb.res_hist) pb.res_hist[c] = nb[c] > 0.0 ? 1.0 : 0.0;
    if (!(nb[c] > 0.0)) {  // b = 0: x = 0 is exact
      act[c] = 0;
      if (pb.iters) pb.iters[c] = 0;
      if (pb.true_relres) pb.true_relres[c] = 0.0;
    }
    any = any || act[c];
  }
  for (int it = 1; pb.res_hist && it <= pb.maxit; ++it)
    for (int c = 0; c < cols; ++c) pb.res_hist[(size_t)it * cols + c] = NAN;
  KOP_CUDA_TRY(cudaMemcpyAsync(active, act.data(), sizeof(int) * cols, cudaMemcpyHostToDevice, st));
  if (pb.X0 && any) {
    // warm start: x = x0 (columns with b = 0 keep x = 0), r0 = b - (A + lam I) x0
    // with the check operator; a column whose start already meets the
    // tolerance stops after 0 iterations
    KOP_CUDA_TRY(cudaMemcpyAsync(X, pb.X0, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st));
    zero_inactive_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(X, (int64_t)nc, cols, active);
    KOP_LAUNCHED();
    if ((rc = true_residual(pb.check_mode, true))) return rc;
    any = false;
    bool escalate = false;
    for (int c = 0; c < cols; ++c) {
      if (!act[c]) continue;
      if (pb.res_hist) pb.res_hist[c] = trel[c];
      if (pb.true_relres) pb.true_relres[c] = trel[c];
      if (urel[c] <= pb.tol) {
        act[c] = 0;
        if (pb.iters) pb.iters[c] = 0;
      } else if (excess[c] > kEscalate * pb.tol * pb.tol) {
        escalate = true;
      }
      any = any || act[c];
    }
    if (escalate) {
      pb.check_mode = pb.refine_mode = KOP_EXACT;
      for (int c = 0; c < cols; ++c) excess[c] = 0.0;
    }
    KOP_CUDA_TRY(cudaMemcpyAsync(active, act.data(), sizeof(int) * cols, cudaMemcpyHostToDevice, st));
  }
  if ((rc = apply_prec())) return rc;
  va.acc = rz;
  if ((rc = vec_launch<OP_DOT>(va, st))) return rc;
  va.acc = acc;
  KOP_CUDA_TRY(cudaMemcpyAsync(P, Z, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));

  const double tol2 = pb.tol * pb.tol;
  int it = 0;
  bool breakdown = false;
  std::vector<char> cand(cols);
  // candidate thresholds on ||r||^2 for the device: tol^2 - excess, times ||b||^2
  std::vector<double> hthr(cols);
  auto upload_thresholds = [&]() -> int {
    for (int c = 0; c < cols; ++c) hthr[c] = (tol2 - excess[c]) * nb[c] * nb[c];
    KOP_CUDA_TRY(cudaMemcpyAsync(thr2, hthr.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
    return KOP_OK;
  };
  if ((rc = upload_thresholds())) return rc;
  KOP_CUDA_TRY(cudaMemsetAsync(frozen, 0, sizeof(int) * cols, st));
  const int chunk = chunk_len(n, cols);
  std::vector<double> hh((size_t)kChunkMax * cols);
  std::vector<int> hf(cols), stop_it(cols, 0);
  int slot = 0;
  for (it = 1; any && it <= pb.maxit; ++it) {
    if ((rc = matvec(P, Q, pb.inner_mode))) return rc;
    va.acc = pq;
    if ((rc = vec_launch<OP_PQ>(va, st))) return rc;
    fin_alpha_kernel<<<(cols + 127) / 128, 128, 0, st>>>(cols, rz, pq, active, alpha, op->status);
    KOP_LAUNCHED();
    va.acc = hist + (size_t)slot * cols;
    if ((rc = vec_launch<OP_XR>(va, st))) return rc;
    va.acc = acc;
    freeze_kernel<<<(cols + 127) / 128, 128, 0, st>>>(cols, hist + (size_t)slot * cols, thr2, active, frozen, it);
    KOP_LAUNCHED();
    // the host looks at the chunk at its last iteration and wherever a
    // refinement or the last iteration falls
    const bool sync = slot == chunk - 1 || it == pb.maxit || (pb.refine_every > 0 && it % pb.refine_every == 0);
    if (!sync) {
      ++slot;
    } else {
    KOP_CUDA_TRY(cudaMemcpyAsync(hh.data(), hist, sizeof(double) * (size_t)(slot + 1) * cols,
                                 cudaMemcpyDeviceToHost, st));
    KOP_CUDA_TRY(cudaMemcpyAsync(hf.data(), frozen, sizeof(int) * cols, cudaMemcpyDeviceToHost, st));
    int hs = 0;
    if ((rc = device_status(op, st, &hs))) return rc;
    if (hs == KOP_DEV_BREAKDOWN) {
      breakdown = true;
      break;
    }
    if (hs == KOP_DEV_TIMEOUT) return fail(KOP_ETIMEOUT, "pcg: a bounded device wait timed out");
    const int it0 = it - slot;  // first iteration of the chunk
    bool any_cand = false, all_near = true;
    for (int c = 0; c < cols; ++c) {
      cand[c] = 0;
      if (!act[c]) continue;
      // a column frozen at iteration f kept its residual from then on
      const int last = hf[c] > 0 ? hf[c] : it;
      if (pb.res_hist)
        for (int j = it0; j <= last; ++j)
          pb.res_hist[(size_t)j * cols + c] = std::sqrt(hh[(size_t)(j - it0) * cols + c]) / nb[c];
      rel[c] = std::sqrt(hh[(size_t)(last - it0) * cols + c]) / nb[c];
      // a candidate stop once the recursive residual leaves room for what
      // the last certification found the check operator to miss (the
      // device froze the column at that iteration)
      if (hf[c] > 0) {
        cand[c] = 1;
        any_cand = true;
        stop_it[c] = hf[c];
      }
      all_near = all_near && rel[c] <= kNearTol * pb.tol;
    }
    slot = 0;
    // a periodic refinement is skipped when every active column is within
    // kNearTol of the tolerance: its candidate stop, a few iterations later,
    // recomputes the true residual anyway
    const bool periodic = pb.refine_every > 0 && it % pb.refine_every == 0 && !all_near;
    const bool refine = any_cand || periodic || it == pb.maxit;
    if (refine) {
      // the true residual replaces the recursive one: the refinement operator
      // for periodic replacement, the check operator (certified) when a
      // column may stop
      const bool stopping = any_cand || it == pb.maxit;
      // a periodic refinement with the check operator itself also predicts
      // what that operator will miss at the stops
      const bool predict = !stopping && pb.refine_mode == pb.check_mode && pb.check_mode != KOP_EXACT;
      if ((rc = true_residual(stopping ? pb.check_mode : pb.refine_mode, stopping || predict, predict))) return rc;
      any = false;
      bool escalate = false;
      for (int c = 0; c < cols; ++c) {
        if (!act[c]) continue;
        if (stopping && pb.true_relres) pb.true_relres[c] = trel[c];
        if (cand[c] && urel[c] <= pb.tol) {
          act[c] = 0;
          if (pb.iters) pb.iters[c] = stop_it[c];
        } else if ((stopping || predict) && excess[c] > kEscalate * tol2) {
          // any active column, candidate or not: its threshold tol^2 - excess
          // would otherwise leave it no room to become a candidate again
          escalate = true;
        }
        any = any || act[c];
      }
      // the check operator cannot certify the tolerance on this system: later
      // checks and refinements use the FP64 operator
      if (escalate) {
        pb.check_mode = pb.refine_mode = KOP_EXACT;
        for (int c = 0; c < cols; ++c) excess[c] = 0.0;
      }
      // columns whose candidate stop was not certified continue from it
      KOP_CUDA_TRY(cudaMemcpyAsync(active, act.data(), sizeof(int) * cols, cudaMemcpyHostToDevice, st));
      KOP_CUDA_TRY(cudaMemsetAsync(frozen, 0, sizeof(int) * cols, st));
      if ((rc = upload_thresholds())) return rc;
      if (!any) break;
    }
    }  // sync
    if ((rc = apply_prec())) return rc;
    va.acc = acc;
    va.acc2 = qz;
    if ((rc = vec_launch<OP_DOT2>(va, st))) return rc;
    fin_beta_kernel<<<(cols + 127) / 128, 128, 0, st>>>(cols, rz, acc, qz, pq, beta);
    KOP_LAUNCHED();
    va.acc = acc;
    if ((rc = vec_launch<OP_P>(va, st))) return rc;
  }
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  bool all = true;
  for (int c = 0; c < cols; ++c)
    if (act[c]) {
      all = false;
      if (pb.iters) pb.iters[c] = it > pb.maxit ? pb.maxit : it;
    }
  if (breakdown) return fail(KOP_ENOTPD, "pcg: breakdown (p^T A p <= 0)");
  return all ? KOP_OK : KOP_NOT_CONVERGED;
}

}  // namespace kop

using namespace kop;

static bool valid_mode(int m) { return m >= KOP_FAST && m <= KOP_EXACT; }

extern "C" int pcg_solve(kop_t op, nys_t ny, const double* lambdas, int32_t n_shifts, const double* mu,
                         int32_t adaptive, const float* B, int32_t nrhs, const double* X0, double tol,
                         int32_t maxit, int32_t refine_every, int32_t inner_mode, int32_t refine_mode,
                         int32_t check_mode, double* Xout, int32_t* iters, double* res_hist, double* true_relres,
                         void* stream) {
  if (!op || !lambdas || !B || !Xout || !iters) return fail(KOP_EINVAL, "pcg_solve: NULL argument");
  if (ny && ny->op != op) return fail(KOP_EINVAL, "pcg_solve: preconditioner built for another operator");
  if (n_shifts < 1 || nrhs < 1 || (int64_t)n_shifts * nrhs > 4096)
    return fail(KOP_EINVAL, "pcg_solve: need 1 <= nrhs * n_shifts <= 4096");
  if (!(tol > 0.0) || maxit < 1 || refine_every < 0) return fail(KOP_EINVAL, "pcg_solve: bad tol / maxit / refine");
  if (!valid_mode(inner_mode) || !valid_mode(refine_mode) || !valid_mode(check_mode))
    return fail(KOP_EINVAL, "pcg_solve: bad mode");
  PcgProblem pb;
  pb.op = op;
  pb.ny = ny;
  pb.nrhs = nrhs;
  pb.cols = nrhs * n_shifts;
  for (int s = 0; s < n_shifts; ++s) {
    const double l = lambdas[s];
    const double m = mu ? mu[s] : l;
    if (!(l > 0.0) || !std::isfinite(l) || !(m > 0.0) || !std::isfinite(m))
      return fail(KOP_EINVAL, "pcg_solve: shifts and damping must be finite and > 0");
    for (int j = 0; j < nrhs; ++j) {
      pb.lam.push_back(l);
      pb.mu.push_back(m);
    }
  }
  pb.adaptive = adaptive ? 1 : 0;
  pb.B = B;
  pb.X0 = X0;
  pb.Xout = Xout;
  pb.tol = tol;
  pb.maxit = maxit;
  pb.refine_every = refine_every;
  pb.inner_mode = inner_mode;
  pb.refine_mode = refine_mode;
  pb.check_mode = check_mode;
  pb.iters = iters;
  pb.res_hist = res_hist;
  pb.true_relres = true_relres;
  return pcg_core(pb, (cudaStream_t)stream);
}

__global__ void d2f_vec_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// x (FP64) -> [hi | lo] FP32 columns (n x 2).
__global__ void split_vec_kernel(const double* __restrict__ x, float* __restrict__ v2, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float hi = (float)x[i];
  v2[2 * i] = hi;
  v2[2 * i + 1] = (float)(x[i] - (double)hi);
}

namespace kop {

// e_i = a_i + b_i - y_i in FP64 (a, b: the two product columns of an exact
// split, stride 2), and its exact hi/lo FP32 split into e2 (n x 2).
__global__ void residual_split_kernel(const float* __restrict__ t2, const float* __restrict__ y, int64_t n,
                                      double* __restrict__ e, float* __restrict__ e2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = ((double)t2[2 * i] + (double)t2[2 * i + 1]) - (double)y[i];
  e[i] = v;
  const float hi = (float)v;
  e2[2 * i] = hi;
  e2[2 * i + 1] = (float)(v - (double)hi);
}

// e_i = t64_i - y_i (FP64 product) and its split.
__global__ void residual64_split_kernel(const double* __restrict__ t64, const float* __restrict__ y, int64_t n,
                                        double* __restrict__ e, float* __restrict__ e2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = t64[i] - (double)y[i];
  e[i] = v;
  const float hi = (float)v;
  e2[2 * i] = hi;
  e2[2 * i + 1] = (float)(v - (double)hi);
}

// out_i = scale * (a_i + b_i) (two product columns, stride 2) in FP64.
__global__ void combine2_kernel(const float* __restrict__ t2, int64_t n, double scale, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * ((double)t2[2 * i] + (double)t2[2 * i + 1]);
}

__global__ void scale64_kernel(double* __restrict__ a, int64_t n, double s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] *= s;
}

// A product of the operator's kernel family `kf` (k or dk/dbw) between the
// point sets Q and Ks applied to the FP64 vector v (Ks.n entries): O2 (Q.n x
// 2 FP32, the two columns of v's exact split; their sum is the product), or
// in KOP_EXACT mode O64 (Q.n FP64).  split: Ks.n x 2 FP32 scratch.
static int cross_apply64(kop_s* op, const PointSet& Q, const PointSet& Ks, bool self, int kf, int mode,
                         const double* v, float* split, float* O2, double* O64, cudaStream_t st) {
  if (mode == KOP_EXACT) return exact_matvec(Q, Ks, kf, op->bw, v, 1, 1, O64, 1, st);
  split_vec_kernel<<<(unsigned)((Ks.n + 255) / 256), 256, 0, st>>>(v, split, Ks.n);
  KOP_LAUNCHED();
  const KConst kc = kernel_constants(kf, op->bw);
  const int m2 = mode == KOP_PLAIN ? KOP_PLAIN_CHECK : mode;
  return op_matvec(Q, Ks, self, kf, kc, m2, split, 2, 2, O2, 2, op->status, st);
}

// The adjoint solve (K + lam I) g = dL/dx (dLdx: device FP64) with the same
// preconditioner, then dL/dlam = -g^T x and the training term
// dL/dbw|_K = -g^T (dK/dbw) x, the derivative product taken with check_mode.
static int adjoint_core(kop_s* op, nys_s* ny, double lam, int adaptive, const double* x, const double* dLdx,
                        double tol, int maxit, int refine_every, int inner_mode, int refine_mode, int check_mode,
                        double* g_out, int32_t* iters, double* dLdlam, double* dLdbw, cudaStream_t st) {
  const int64_t n = op_dim(op);
  Workspace ws;
  ws.st = st;
  // Bf (n) | V2 (2n) | T2 (2n) floats, t64 (n) and acc (2) doubles
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(float) * 5 * (size_t)n + sizeof(double) * ((size_t)n + 2) + 64, st));
  float* Bf = (float*)ws.p;
  float* V2 = Bf + n;
  float* T2 = V2 + 2 * n;
  double* acc = (double*)(((uintptr_t)(T2 + 2 * n) + 15) & ~(uintptr_t)15);
  double* t64 = acc + 2;
  const unsigned nb = (unsigned)((n + 255) / 256);
  d2f_vec_kernel<<<nb, 256, 0, st>>>(dLdx, Bf, n);
  KOP_LAUNCHED();
  PcgProblem pb;
  pb.op = op;
  pb.ny = ny;
  pb.cols = pb.nrhs = 1;
  pb.lam = {lam};
  pb.mu = {lam};
  pb.adaptive = adaptive ? 1 : 0;
  pb.B = Bf;
  pb.Xout = g_out;
  pb.tol = tol;
  pb.maxit = maxit;
  pb.refine_every = refine_every;
  pb.inner_mode = inner_mode;
  pb.refine_mode = refine_mode;
  pb.check_mode = check_mode;
  int32_t it = 0;
  pb.iters = &it;
  const int rc = pcg_core(pb, st);
  if (iters) *iters = it;
  if (rc < 0) return rc;
  // dL/dlam = -g^T x through the exact split of x; g^T (dK/dbw) x through the
  // two product columns of the split (or one FP64 product in exact mode)
  split_vec_kernel<<<nb, 256, 0, st>>>(x, V2, n);
  KOP_LAUNCHED();
  KOP_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  dot_kernel<<<4 * num_sms(), 256, 0, st>>>(g_out, V2, V2 + 1, n, 2, acc);
  KOP_LAUNCHED();
  if (op->ridge) {
    // X^T X has no bandwidth: dL/dbw = 0
  } else {
    int r2 = cross_apply64(op, op->pts, op->pts, true, op->kernel + 3, check_mode, x, V2, T2, t64, st);
    if (r2) return r2;
    if (check_mode == KOP_EXACT)
      dot64_kernel<<<4 * num_sms(), 256, 0, st>>>(g_out, t64, n, acc + 1);
    else
      dot_kernel<<<4 * num_sms(), 256, 0, st>>>(g_out, T2, T2 + 1, n, 2, acc + 1);
    KOP_LAUNCHED();
  }
  double h[2];
  KOP_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  const int s = kop_sync(op, (void*)st);
  if (s != KOP_OK) return s;
  *dLdlam = -h[0];
  *dLdbw = -h[1];
  return rc;
}

static int adjoint_args(kop_t op, nys_t ny, double lam, double tol, int32_t maxit, int32_t refine_every,
                        int32_t inner_mode, int32_t refine_mode, int32_t check_mode, const char* where) {
  const std::string w(where);
  if (ny && ny->op != op) return fail(KOP_EINVAL, w + ": preconditioner built for another operator");
  if (!(lam > 0.0) || !std::isfinite(lam)) return fail(KOP_EINVAL, w + ": lam must be > 0");
  if (!(tol > 0.0) || maxit < 1 || refine_every < 0) return fail(KOP_EINVAL, w + ": bad tol / maxit");
  if (!valid_mode(inner_mode) || !valid_mode(refine_mode) || !valid_mode(check_mode))
    return fail(KOP_EINVAL, w + ": bad mode");
  return KOP_OK;
}

}  // namespace kop

extern "C" int pcg_adjoint(kop_t op, nys_t ny, double lam, int32_t adaptive, const double* x, const double* dLdx,
                           double tol, int32_t maxit, int32_t refine_every, int32_t inner_mode, int32_t refine_mode,
                           int32_t check_mode, double* g_out, int32_t* iters, double* dLdlam, double* dLdbw,
                           void* stream) {
  if (!op || !x || !dLdx || !g_out || !dLdlam || !dLdbw) return fail(KOP_EINVAL, "pcg_adjoint: NULL argument");
  if (int rc = adjoint_args(op, ny, lam, tol, maxit, refine_every, inner_mode, refine_mode, check_mode,
                            "pcg_adjoint"))
    return rc;
  return adjoint_core(op, ny, lam, adaptive, x, dLdx, tol, maxit, refine_every, inner_mode, refine_mode, check_mode,
                      g_out, iters, dLdlam, dLdbw, (cudaStream_t)stream);
}

extern "C" int pcg_adjoint_val(kop_t op, nys_t ny, double lam, int32_t adaptive, const double* x,
                               const float* Xval, int64_t nval, const float* yval, double tol, int32_t maxit,
                               int32_t refine_every, int32_t inner_mode, int32_t refine_mode, int32_t check_mode,
                               double* g_out, int32_t* iters, double* loss, double* dLdlam, double* dLdbw,
                               void* stream) {
  if (!op || !x || !Xval || !yval || !g_out || !loss || !dLdlam || !dLdbw)
    return fail(KOP_EINVAL, "pcg_adjoint_val: NULL argument");
  if (op->ridge) return fail(KOP_EINVAL, "pcg_adjoint_val: not defined for a ridge (X^T X) operator");
  if (nval < 1 || nval >= (int64_t(1) << 31)) return fail(KOP_EINVAL, "pcg_adjoint_val: nval must be in [1, 2^31)");
  if (int rc = adjoint_args(op, ny, lam, tol, maxit, refine_every, inner_mode, refine_mode, check_mode,
                            "pcg_adjoint_val"))
    return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = op->pts.n;
  const int kf = op->kernel;
  const double s2 = 2.0 / (double)nval;
  PointSet zs;  // the validation points, centred with the operator's mean
  int rc = pointset_alloc(zs, nval, op->pts.d, st);
  if (rc) return rc;
  struct Free {
    PointSet* z;
    cudaStream_t st;
    ~Free() { pointset_free(*z, st); }
  } free_zs{&zs, st};
  if ((rc = pointset_fill(zs, Xval, op->mean, st))) return rc;
  Workspace ws;
  ws.st = st;
  // e (nval), t64v (nval), dLdx (n), t64 (n) doubles | split (2 max(n, nval)), tv2 (2 nval), tn2 (2 n) floats,
  // acc (2) doubles
  const size_t nm = (size_t)(n > nval ? n : nval);
  KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(double) * (2 * (size_t)nval + 2 * (size_t)n + 2) +
                                          sizeof(float) * (2 * nm + 2 * (size_t)nval + 2 * (size_t)n) + 64, st));
  double* e = (double*)ws.p;
  double* t64v = e + nval;
  double* dLdx = t64v + nval;
  double* t64 = dLdx + n;
  double* acc = t64 + n;
  float* split = (float*)(acc + 2);
  float* tv2 = split + 2 * nm;
  float* tn2 = tv2 + 2 * nval;
  const unsigned bv = (unsigned)((nval + 255) / 256), bn = (unsigned)((n + 255) / 256);
  // e = K(Xval, X) x - yval, loss = e^T e / nval
  if ((rc = cross_apply64(op, zs, op->pts, false, kf, check_mode, x, split, tv2, t64v, st))) return rc;
  if (check_mode == KOP_EXACT)
    residual64_split_kernel<<<bv, 256, 0, st>>>(t64v, yval, nval, e, split);
  else
    residual_split_kernel<<<bv, 256, 0, st>>>(tv2, yval, nval, e, split);
  KOP_LAUNCHED();
  KOP_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  dot64_kernel<<<4 * num_sms(), 256, 0, st>>>(e, e, nval, acc);
  KOP_LAUNCHED();
  // dL/dx = (2 / nval) K(X, Xval) e, from e's exact split (already in `split`)
  if (check_mode == KOP_EXACT) {
    if ((rc = exact_matvec(op->pts, zs, kf, op->bw, e, 1, 1, dLdx, 1, st))) return rc;
    scale64_kernel<<<bn, 256, 0, st>>>(dLdx, n, s2);
  } else {
    const KConst kc = kernel_constants(kf, op->bw);
    const int m2 = check_mode == KOP_PLAIN ? KOP_PLAIN_CHECK : check_mode;
    if ((rc = op_matvec(op->pts, zs, false, kf, kc, m2, split, 2, 2, tn2, 2, op->status, st))) return rc;
    combine2_kernel<<<bn, 256, 0, st>>>(tn2, n, s2, dLdx);
  }
  KOP_LAUNCHED();
  // validation term of dL/dbw: (2 / nval) e^T (dK(Xval, X)/dbw) x
  if ((rc = cross_apply64(op, zs, op->pts, false, kf + 3, check_mode, x, split, tv2, t64v, st)))
    return rc;
  if (check_mode == KOP_EXACT)
    dot64_kernel<<<4 * num_sms(), 256, 0, st>>>(e, t64v, nval, acc + 1);
  else
    dot_kernel<<<4 * num_sms(), 256, 0, st>>>(e, tv2, tv2 + 1, nval, 2, acc + 1);
  KOP_LAUNCHED();
  double h[2];
  KOP_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  KOP_CUDA_TRY(cudaStreamSynchronize(st));
  double dlam = 0.0, dbw_k = 0.0;
  rc = adjoint_core(op, ny, lam, adaptive, x, dLdx, tol, maxit, refine_every, inner_mode, refine_mode, check_mode,
                    g_out, iters, &dlam, &dbw_k, st);
  if (rc < 0) return rc;
  *loss = h[0] / (double)nval;
  *dLdlam = dlam;
  *dLdbw = s2 * h[1] + dbw_k;
  return rc;
}
