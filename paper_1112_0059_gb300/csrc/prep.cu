// Index and query preparation kernels: exact BF16 operands and the
// K-extension that carries the squared norms (and, for location-weighted
// rows, the location cross terms) into the tensor-core contraction.
//
// Coordinates are centred, x' = x - 128 in [-128, 127]: x' and -2q' are exact
// in BF16 (8 significant bits), ||q' - r'|| = ||q - r||, and every partial sum
// of the contraction stays far below 2^24, so the FP32 accumulator holds the
// exact distance whatever the summation order:
//   the positive terms add up to at most ||q'||^2 + ||r'||^2 + 2 sum |q'_t r'_t|
//   <= 4 * 128 * 128^2 = 8,388,608 for the 128 appearance coordinates, plus
//   for a location weight w <= 48 at most 4 * 2 * w * 128^2 + 2 * 2 * 255 * 128
//   = 6,422,016 for the location terms (norms and the digit-split cross
//   terms below): 14,810,624 in all, < 2^24 = 16,777,216.
//
// K-extension (16 BF16 columns), reference row:
//   (d0, d1, d2, 1, 256, 65536, x_r', x_r', y_r', y_r', 0 ...)
// query row:
//   (1, 256, 65536, e0, e1, e2, -512 hx, -2 lx, -512 hy, -2 ly, 0 ...)
// with (d0, d1, d2) and (e0, e1, e2) the base-256 digits of the norms
// ||r'||^2 + w ||l_r'||^2 and ||q'||^2 + w ||l_q'||^2 (l' the centred location),
// and w x_q' = 256 hx + lx (0 <= lx < 256, |hx| <= 24), so that the
// location columns add -2 w (x_q' x_r' + y_q' y_r').  Every value is exact in
// BF16.  Rows without a location (128 bytes) have zeros there.
#include "internal.cuh"

namespace lnbnn {
namespace {

// 16 threads per row, 8 coordinates per thread.
constexpr int kThreadsPerRow = 16;
constexpr int kRowsPerBlock = 16;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// 16 extension values as two 16-byte stores.
__device__ __forceinline__ void store_ext(__nv_bfloat16* dst, const float (&v)[kExt]) {
  uint4 a, b;
  uint32_t* pa = reinterpret_cast<uint32_t*>(&a);
  uint32_t* pb = reinterpret_cast<uint32_t*>(&b);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    pa[t] = pack_bf16x2(v[2 * t], v[2 * t + 1]);
    pb[t] = pack_bf16x2(v[8 + 2 * t], v[9 + 2 * t]);
  }
  reinterpret_cast<uint4*>(dst)[0] = a;
  reinterpret_cast<uint4*>(dst)[1] = b;
}

// Eight appearance bytes of a row (row_bytes 128: one aligned 8-byte load;
// 130: byte loads, the rows are only 2-byte aligned).
__device__ __forceinline__ void load8(const uint8_t* p, int row_bytes, uint8_t (&b)[8]) {
  if (row_bytes == kDim) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    memcpy(b, &raw, 8);
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t) b[t] = p[t];
  }
}

__global__ void prep_ref_kernel(const uint8_t* __restrict__ ref, int64_t n_ref, int64_t n_pad, int row_bytes,
                                int loc_w, __nv_bfloat16* __restrict__ ref_bf, float* __restrict__ rnorm,
                                __nv_bfloat16* __restrict__ ref_ext) {
  const int sub = threadIdx.x % kThreadsPerRow;
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kThreadsPerRow;
  if (row >= n_pad) return;
  const bool real = row < n_ref;
  uint8_t b[8] = {128, 128, 128, 128, 128, 128, 128, 128};  // padding rows: x' = 0
  if (real) load8(ref + row * row_bytes + sub * 8, row_bytes, b);
  int32_t ss = 0;
  uint4 out;
  uint32_t* o = reinterpret_cast<uint32_t*>(&out);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int32_t x0 = (int32_t)b[2 * t] - 128, x1 = (int32_t)b[2 * t + 1] - 128;
    ss += x0 * x0 + x1 * x1;
    o[t] = pack_bf16x2((float)x0, (float)x1);
  }
  *reinterpret_cast<uint4*>(ref_bf + row * kDim + sub * 8) = out;
#pragma unroll
  for (int off = kThreadsPerRow / 2; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if (sub != 0) return;
  int32_t lx = 0, ly = 0;
  if (real && row_bytes > kDim) {
    lx = (int32_t)ref[row * row_bytes + kDim] - 128;
    ly = (int32_t)ref[row * row_bytes + kDim + 1] - 128;
  }
  const int32_t norm = real ? ss + loc_w * (lx * lx + ly * ly) : (int32_t)kPadNorm;
  rnorm[row] = (float)norm;
  // base-256 digits: d2 <= 56 for real rows, 512 for padding rows
  const float v[kExt] = {(float)(norm & 255), (float)((norm >> 8) & 255), (float)(norm >> 16), 1.0f, 256.0f,
                         65536.0f, (float)lx, (float)lx, (float)ly, (float)ly, 0, 0, 0, 0, 0, 0};
  store_ext(ref_ext + row * kExt, v);
}

// w x' = 256 h + l with 0 <= l < 256.
__device__ __forceinline__ void split256(int32_t v, int32_t* h, int32_t* l) {
  *h = v >> 8;  // arithmetic shift: floor division
  *l = v - (*h << 8);
}

__global__ void prep_query_kernel(const uint8_t* __restrict__ q, int64_t m, int64_t m_pad, int row_bytes, int loc_w,
                                  int32_t* __restrict__ qnorm, __nv_bfloat16* __restrict__ qbf,
                                  __nv_bfloat16* __restrict__ qext) {
  const int sub = threadIdx.x % kThreadsPerRow;
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kThreadsPerRow;
  if (row >= m_pad) return;
  const bool real = row < m;
  uint8_t b[8] = {128, 128, 128, 128, 128, 128, 128, 128};  // padding rows: x' = 0
  if (real) load8(q + row * row_bytes + sub * 8, row_bytes, b);
  int32_t ss = 0;
  uint4 out;
  uint32_t* o = reinterpret_cast<uint32_t*>(&out);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int32_t x0 = (int32_t)b[2 * t] - 128, x1 = (int32_t)b[2 * t + 1] - 128;
    ss += x0 * x0 + x1 * x1;
    o[t] = pack_bf16x2(-2.0f * (float)x0, -2.0f * (float)x1);
  }
  if (qbf) *reinterpret_cast<uint4*>(qbf + row * kDim + sub * 8) = out;
#pragma unroll
  for (int off = kThreadsPerRow / 2; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if (sub != 0) return;
  int32_t lx = 0, ly = 0;
  if (real && row_bytes > kDim) {
    lx = (int32_t)q[row * row_bytes + kDim] - 128;
    ly = (int32_t)q[row * row_bytes + kDim + 1] - 128;
  }
  const int32_t norm = ss + loc_w * (lx * lx + ly * ly);
  if (real) qnorm[row] = norm;
  if (!qext) return;
  int32_t hx, lox, hy, loy;
  split256(loc_w * lx, &hx, &lox);
  split256(loc_w * ly, &hy, &loy);
  // weights for the reference's norm digits, this query's norm digits, then
  // the location cross terms: the MMA yields ||r - q||^2 (+ w ||l_r - l_q||^2)
  const float v[kExt] = {1.0f, 256.0f, 65536.0f, (float)(norm & 255), (float)((norm >> 8) & 255), (float)(norm >> 16),
                         -512.0f * (float)hx, -2.0f * (float)lox, -512.0f * (float)hy, -2.0f * (float)loy,
                         0, 0, 0, 0, 0, 0};
  store_ext(qext + row * kExt, v);
}

__global__ void label_hist_kernel(const int32_t* __restrict__ labels, int64_t n, int32_t C,
                                  unsigned long long* __restrict__ counts, uint32_t* __restrict__ bad) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = labels[j];
    if (c < 0 || c >= C) {
      atomicOr(bad, 1u);
    } else {
      atomicAdd(counts + c, 1ull);
    }
  }
}

__global__ void gather_ref_kernel(const int64_t* __restrict__ perm, int64_t n, const __nv_bfloat16* __restrict__ src_bf,
                                  __nv_bfloat16* __restrict__ dst_bf, const __nv_bfloat16* __restrict__ src_ext,
                                  __nv_bfloat16* __restrict__ dst_ext, const float* __restrict__ src_norm,
                                  float* __restrict__ dst_norm, const int32_t* __restrict__ src_lab,
                                  int32_t* __restrict__ dst_lab) {
  // one warp per row: 32 lanes x 8 bytes of bf16
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const int64_t from = perm[row];
  reinterpret_cast<uint2*>(dst_bf + row * kDim)[lane] = reinterpret_cast<const uint2*>(src_bf + from * kDim)[lane];
  if (lane < 2)
    reinterpret_cast<uint4*>(dst_ext + row * kExt)[lane] = reinterpret_cast<const uint4*>(src_ext + from * kExt)[lane];
  if (lane == 0) {
    dst_norm[row] = src_norm[from];
    dst_lab[row] = src_lab[from];
  }
}

__global__ void fill_float_kernel(float* __restrict__ dst, int64_t n, float v) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = v;
}

}  // namespace

cudaError_t launch_fill_float(float* dst, int64_t n, float v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  fill_float_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, v);
  return cudaGetLastError();
}

cudaError_t launch_prep_ref(const uint8_t* ref, int64_t n_ref, int64_t n_pad, int row_bytes, int loc_w,
                            __nv_bfloat16* ref_bf, float* rnorm, __nv_bfloat16* ref_ext, cudaStream_t s) {
  if (!row_layout_ok(row_bytes, loc_w)) return cudaErrorInvalidValue;
  const int64_t blocks = (n_pad + kRowsPerBlock - 1) / kRowsPerBlock;
  prep_ref_kernel<<<(unsigned)blocks, kRowsPerBlock * kThreadsPerRow, 0, s>>>(ref, n_ref, n_pad, row_bytes, loc_w,
                                                                               ref_bf, rnorm, ref_ext);
  return cudaGetLastError();
}

cudaError_t launch_prep_query(const uint8_t* q, int64_t m, int64_t m_pad, int row_bytes, int loc_w, int32_t* qnorm,
                              __nv_bfloat16* qbf, __nv_bfloat16* qext, cudaStream_t s) {
  if (m_pad == 0) return cudaSuccess;
  if (!row_layout_ok(row_bytes, loc_w)) return cudaErrorInvalidValue;
  const int64_t blocks = (m_pad + kRowsPerBlock - 1) / kRowsPerBlock;
  prep_query_kernel<<<(unsigned)blocks, kRowsPerBlock * kThreadsPerRow, 0, s>>>(q, m, m_pad, row_bytes, loc_w, qnorm,
                                                                                 qbf, qext);
  return cudaGetLastError();
}

cudaError_t launch_label_hist(const int32_t* labels, int64_t n, int32_t C, unsigned long long* counts,
                              uint32_t* bad, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  label_hist_kernel<<<(unsigned)blocks, 256, 0, s>>>(labels, n, C, counts, bad);
  return cudaGetLastError();
}

cudaError_t launch_gather_ref(const int64_t* perm, int64_t n, const __nv_bfloat16* src_bf, __nv_bfloat16* dst_bf,
                              const __nv_bfloat16* src_ext,
                              __nv_bfloat16* dst_ext, const float* src_norm, float* dst_norm,
                              const int32_t* src_lab, int32_t* dst_lab, cudaStream_t s) {
  const int64_t blocks = (n * 32 + 255) / 256;
  gather_ref_kernel<<<(unsigned)blocks, 256, 0, s>>>(perm, n, src_bf, dst_bf, src_ext, dst_ext, src_norm, dst_norm,
                                                     src_lab, dst_lab);
  return cudaGetLastError();
}

}  // namespace lnbnn
