// Gradient of a^T K(X) b with respect to the points: kop_grad_points.
//
// The backward pass of the kernel operator for the inputs X (the paper
// differentiates through the solve, Sec. 3.2; for a loss L(x) of the solution
// x = (K + lam I)^-1 y the X-part of dL/dX is -d(g^T K(X) x)/dX with the
// adjoint g).  With h(r) = -k'(r) / r (the radial derivative; kop_epilogue.cuh)
// and c_ij = a_i b_j + a_j b_i,
//   d(a^T K b)/dx_i = -sum_j c_ij h_ij (x_i - x_j)
//                   = -[ x_i (a_i (H b)_i + b_i (H a)_i) - a_i (H (b.X))_i - b_i (H (a.X))_i ],
// H_ij = h(|x_i - x_j|), (b.X) the rows b_j x_j.  So one product of H with the
// n x (2 + 2d) block [b, a, b.X, a.X] (the fused operator with the h
// epilogue; d > 3 makes it a tensor-core contraction in the FAST mode), then
// an elementwise combine in FP64.  K is translation invariant, so the
// gradient taken in the centred coordinates of the point set is the gradient
// in the caller's coordinates.
#include <cmath>

#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

// V (n x (2 + 2d)) = [b, a, b x_k, a x_k] from coordinates P (n x d, ldp).
template <typename T>
__global__ void grad_block_kernel(const float* __restrict__ P, int ldp, int64_t n, int d, const float* __restrict__ a,
                                  const float* __restrict__ b, T* __restrict__ V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = 2 + 2 * d;
  if (t >= n * m) return;
  const int64_t i = t / m;
  const int c = (int)(t - i * m);
  T v;
  if (c == 0) v = (T)b[i];
  else if (c == 1) v = (T)a[i];
  else if (c < 2 + d) v = (T)b[i] * (T)P[i * ldp + (c - 2)];
  else v = (T)a[i] * (T)P[i * ldp + (c - 2 - d)];
  V[t] = v;
}

// G[i][k] = -(x_ik (a_i O_i0 + b_i O_i1) - a_i O_i,2+k - b_i O_i,2+d+k), in FP64.
template <typename T>
__global__ void grad_combine_kernel(const float* __restrict__ P, int ldp, int64_t n, int d,
                                    const float* __restrict__ a, const float* __restrict__ b,
                                    const T* __restrict__ O, float* __restrict__ G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int64_t i = t / d;
  const int k = (int)(t - i * d);
  const int m = 2 + 2 * d;
  const T* o = O + i * m;
  const double ai = a[i], bi = b[i];
  const double s = ai * (double)o[0] + bi * (double)o[1];
  const double g = (double)P[i * ldp + k] * s - ai * (double)o[2 + k] - bi * (double)o[2 + d + k];
  G[t] = (float)(-g);
}

}  // namespace kop

using namespace kop;

extern "C" int kop_grad_points(kop_t op, const float* a, const float* b, int32_t mode, float* G, void* stream) {
  if (!op || !a || !b || !G) return fail(KOP_EINVAL, "kop_grad_points: NULL argument");
  if (op->ridge) return fail(KOP_EINVAL, "kop_grad_points: not defined for a ridge (X^T X) operator");
  if (mode != KOP_FAST && mode != KOP_ACCURATE && mode != KOP_EXACT)
    return fail(KOP_EINVAL, "kop_grad_points: mode must be KOP_FAST, KOP_ACCURATE or KOP_EXACT");
  cudaStream_t st = (cudaStream_t)stream;
  const PointSet& ps = op->pts;
  const int64_t n = ps.n;
  const int d = ps.d;
  const int m = 2 + 2 * d;
  const int kf = op->kernel + KF_GRBF;
  const int64_t nm = n * m, nd = n * d;
  DevBuf ws;
  ws.st = st;
  int rc = KOP_OK;
  if (mode == KOP_EXACT) {
    // FP64 direct differences of the caller's coordinates
    KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(double) * 2 * (size_t)nm, st));
    double* V = (double*)ws.p;
    double* O = V + nm;
    grad_block_kernel<double><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(ps.xorig, d, n, d, a, b, V);
    KOP_LAUNCHED();
    if ((rc = exact_matvec(ps, ps, kf, op->bw, V, m, m, O, m, st))) return rc;
    grad_combine_kernel<double><<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(ps.xorig, d, n, d, a, b, O, G);
    KOP_LAUNCHED();
  } else {
    // fused operator on the centred coordinates
    KOP_CUDA_TRY(cudaMallocAsync(&ws.p, sizeof(float) * 2 * (size_t)nm, st));
    float* V = (float*)ws.p;
    float* O = V + nm;
    grad_block_kernel<float><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(ps.xc, ps.dp, n, d, a, b, V);
    KOP_LAUNCHED();
    const KConst kc = kernel_constants(kf, op->bw);
    if ((rc = op_matvec(ps, ps, true, kf, kc, mode, V, m, m, O, m, op->status, st))) return rc;
    grad_combine_kernel<float><<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(ps.xc, ps.dp, n, d, a, b, O, G);
    KOP_LAUNCHED();
  }
  return kop_sync(op, stream);
}
