// Operand preparation (once per point set) and shared host utilities.
//
// The kernels of Sec. 2.1 depend on x_i - x_j only, so the points are centred
// by their column mean before anything else: this keeps |x|^2 small and the
// norm identity |x_i - x_j|^2 = |x_i|^2 + |x_j|^2 - 2 x_i.x_j well conditioned.
// Each centred FP32 value x is then split exactly into BF16 parts
//   hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)
// (both differences are exact in FP32), so hi + mid carries about 16 bits and
// hi + mid + lo about 24 bits of x.
#include <atomic>
#include <mutex>
#include <string>

#include "kop_device.cuh"
#include "kop_internal.h"

namespace kop {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KOP_ENOMEM : KOP_ECUDA;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

KConst kernel_constants(int kind, double bw) {
  const double log2e = 1.4426950408889634;
  KConst k{0.f, 0.f, bw};
  double scale = 0.0;
  switch (kind) {
    case KF_RBF:
    case KF_DRBF:
      scale = -log2e / (2.0 * bw * bw);
      k.c2 = (float)(1.0 / (scale * bw * bw * bw));
      break;
    case KF_LAPLACE:
    case KF_DLAPLACE:
      scale = (log2e / bw) * (log2e / bw);
      k.c2 = (float)(1.0 / ((log2e / bw) * bw * bw));
      break;
    case KF_GRBF:
      scale = -log2e / (2.0 * bw * bw);
      k.c2 = (float)(1.0 / (bw * bw));
      break;
    case KF_GLAPLACE:
      scale = (log2e / bw) * (log2e / bw);
      k.c2 = (float)(log2e / (bw * bw));
      break;
    case KF_GMATERN:
      scale = 5.0 / (bw * bw);
      k.c2 = (float)(5.0 / (3.0 * bw * bw));
      break;
    default:
      scale = 5.0 / (bw * bw);
      k.c2 = (float)(1.0 / bw);
      break;
  }
  k.scale = (float)scale;
  return k;
}

__global__ void scale_norms_kernel(const float* __restrict__ nrm, int64_t n, float s, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = s * nrm[i];
}

int ensure_scaled_norms(PointSet& ps, float scale, cudaStream_t st) {
  if (ps.snorm && ps.snorm_scale == scale) return KOP_OK;
  if (!ps.snorm) KOP_CUDA_TRY(cudaMallocAsync((void**)&ps.snorm, sizeof(float) * ps.n_pad, st));
  scale_norms_kernel<<<(unsigned)((ps.n_pad + 255) / 256), 256, 0, st>>>(ps.norms, ps.n_pad, scale, ps.snorm);
  KOP_LAUNCHED();
  ps.snorm_scale = scale;
  return KOP_OK;
}

int padded_dim(int d) {
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  return ((d + 63) / 64) * 64;
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2-D BF16 tensor map over a row-major rows x cols array; boxes of
// box_cols x box_rows with the swizzle matching the box row width.
int encode_tmap_bf16(CUtensorMap* map, const void* base, int64_t rows, int cols, int box_cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(KOP_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const int row_bytes = box_cols * 2;
  CUtensorMapSwizzle swz = row_bytes == 128   ? CU_TENSOR_MAP_SWIZZLE_128B
                           : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(KOP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return KOP_OK;
}

// ------------------------------------------------------------ point sets
int pointset_alloc(PointSet& ps, int64_t n, int d, cudaStream_t st) {
  ps.n = n;
  ps.d = d;
  ps.dp = padded_dim(d);
  ps.n_pad = ((n + 127) / 128) * 128;
  const size_t nx = (size_t)ps.n_pad * ps.dp;
  const size_t bytes = nx * 4 + (size_t)ps.n_pad * 4 + 3 * nx * 2 + (size_t)n * d * 4 + 2048;
  void* p = nullptr;
  KOP_CUDA_TRY(cudaMallocAsync(&p, bytes, st));
  ps.block = p;
  uint8_t* b = (uint8_t*)p;
  ps.xc = (float*)b;
  b += nx * 4;
  ps.norms = (float*)b;
  b += (size_t)ps.n_pad * 4;
  b = (uint8_t*)(((uintptr_t)b + 255) & ~(uintptr_t)255);
  for (int s = 0; s < 3; ++s) {
    ps.sp[s] = (__nv_bfloat16*)b;
    b += nx * 2;
  }
  b = (uint8_t*)(((uintptr_t)b + 255) & ~(uintptr_t)255);
  ps.xorig = (float*)b;
  const int box_cols = ps.dp >= 64 ? 64 : ps.dp;
  for (int s = 0; s < 3; ++s) {
    int rc = encode_tmap_bf16(&ps.tm[s][0], ps.sp[s], ps.n_pad, ps.dp, box_cols, 128);
    if (rc == KOP_OK) rc = encode_tmap_bf16(&ps.tm[s][1], ps.sp[s], ps.n_pad, ps.dp, box_cols, 64);
    if (rc != KOP_OK) {
      pointset_free(ps, st);
      return rc;
    }
  }
  return KOP_OK;
}

void pointset_free(PointSet& ps, cudaStream_t st) {
  if (ps.block) cudaFreeAsync(ps.block, st);
  if (ps.snorm) cudaFreeAsync(ps.snorm, st);
  if (ps.sym_scratch) cudaFreeAsync(ps.sym_scratch, st);
  ps.sym_scratch = nullptr;
  ps.sym_scratch_floats = 0;
  ps.snorm = nullptr;
  ps.snorm_scale = 0.0f;
  ps.block = nullptr;
  ps.xc = ps.norms = ps.xorig = nullptr;
  ps.sp[0] = ps.sp[1] = ps.sp[2] = nullptr;
}

__global__ void colsum_kernel(const float* __restrict__ X, int64_t n, int d, int64_t rows_per_block,
                              double* __restrict__ sum) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) s += (double)X[i * d + c];
    atomicAdd(&sum[c], s);
  }
}

__global__ void scale_kernel(double* v, int d, double f) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < d) v[c] *= f;
}

int column_mean(const float* X, int64_t n, int d, double* mean, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemsetAsync(mean, 0, sizeof(double) * d, st));
  const int64_t rpb = 512;
  const int64_t blocks = (n + rpb - 1) / rpb;
  colsum_kernel<<<(unsigned)blocks, 128, 0, st>>>(X, n, d, rpb, mean);
  KOP_LAUNCHED();
  scale_kernel<<<(d + 127) / 128, 128, 0, st>>>(mean, d, 1.0 / (double)n);
  KOP_LAUNCHED();
  return KOP_OK;
}

// One warp per padded row: centre, split, and the FP64 row norm (rounded
// once to FP32).  Rows >= n and columns >= d are zero.
__global__ void fill_kernel(const float* __restrict__ X, const double* __restrict__ mean, int64_t n, int d, int dp,
                            int64_t n_pad, float* __restrict__ xc, float* __restrict__ norms,
                            __nv_bfloat16* __restrict__ s0, __nv_bfloat16* __restrict__ s1,
                            __nv_bfloat16* __restrict__ s2) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_pad) return;
  double nrm = 0.0;
  for (int c = lane; c < dp; c += 32) {
    float x = 0.0f;
    if (row < n && c < d) x = (float)((double)X[row * d + c] - mean[c]);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
    const int64_t o = row * dp + c;
    xc[o] = x;
    s0[o] = hi;
    s1[o] = mid;
    s2[o] = lo;
    nrm += (double)x * (double)x;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0) norms[row] = (float)nrm;
}

int pointset_fill(PointSet& ps, const float* X, const double* mean, cudaStream_t st) {
  KOP_CUDA_TRY(cudaMemcpyAsync(ps.xorig, X, sizeof(float) * (size_t)ps.n * ps.d, cudaMemcpyDeviceToDevice, st));
  const int64_t threads = ps.n_pad * 32;
  const int bs = 256;
  fill_kernel<<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(X, mean, ps.n, ps.d, ps.dp, ps.n_pad, ps.xc,
                                                                   ps.norms, ps.sp[0], ps.sp[1], ps.sp[2]);
  KOP_LAUNCHED();
  return KOP_OK;
}

}  // namespace kop

extern "C" const char* kop_last_error(void) { return kop::g_last_error.c_str(); }

extern "C" int64_t kop_launch_count(void) { return (int64_t)kop::g_launches.load(std::memory_order_relaxed); }
