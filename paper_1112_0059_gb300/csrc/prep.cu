// Index and query preparation kernels: exact BF16 operand copies and squared
// norms.  Every uint8 value 0..255 is exact in BF16 (8 significant bits), and
// so is -2q (a power-of-two scale), so the tensor-core contraction of these
// operands reproduces the integer dot products exactly.
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

__device__ __forceinline__ uint32_t bf16_bits(float v) {
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return (uint32_t)*reinterpret_cast<unsigned short*>(&b);
}

// First 8 BF16 values of a K-extension row: (a, b, c, d, e, f, 0, 0); the
// other 8 values of the row are zero.
__device__ __forceinline__ uint4 ext_head(float a, float b, float c, float d, float e, float f) {
  return make_uint4(bf16_bits(a) | (bf16_bits(b) << 16), bf16_bits(c) | (bf16_bits(d) << 16),
                    bf16_bits(e) | (bf16_bits(f) << 16), 0u);
}

__global__ void prep_ref_kernel(const uint8_t* __restrict__ ref, int64_t n_ref, int64_t n_pad,
                                __nv_bfloat16* __restrict__ ref_bf, float* __restrict__ rnorm,
                                __nv_bfloat16* __restrict__ ref_ext) {
  const int sub = threadIdx.x % kThreadsPerRow;
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kThreadsPerRow;
  if (row >= n_pad) return;
  uint2 raw = make_uint2(0, 0);
  if (row < n_ref) raw = *reinterpret_cast<const uint2*>(ref + row * kDim + sub * 8);
  const uint8_t* b = reinterpret_cast<const uint8_t*>(&raw);
  int32_t ss = 0;
  uint4 out;
  uint32_t* o = reinterpret_cast<uint32_t*>(&out);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int32_t x0 = b[2 * t], x1 = b[2 * t + 1];
    ss += x0 * x0 + x1 * x1;
    o[t] = pack_bf16x2((float)x0, (float)x1);
  }
  *reinterpret_cast<uint4*>(ref_bf + row * kDim + sub * 8) = out;
#pragma unroll
  for (int off = kThreadsPerRow / 2; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  const int32_t norm = row < n_ref ? ss : (int32_t)kPadNorm;
  if (sub == 0) rnorm[row] = (float)norm;
  // K-extension (d0, d1, d2, 1, 256, 65536): base-256 digits of the norm,
  // d0 + 256 d1 + 65536 d2 (d2 <= 127 for real rows, 512 for padding rows),
  // then the weights that pick up the query's norm digits; all exact in BF16
  uint4* ext = reinterpret_cast<uint4*>(ref_ext + row * kExt);
  if (sub == 0)
    ext[0] = ext_head((float)(norm & 255), (float)((norm >> 8) & 255), (float)(norm >> 16), 1.0f, 256.0f, 65536.0f);
  if (sub == 1) ext[1] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void prep_query_kernel(const uint8_t* __restrict__ q, int64_t m, int64_t m_pad,
                                  int32_t* __restrict__ qnorm, __nv_bfloat16* __restrict__ qbf,
                                  __nv_bfloat16* __restrict__ qext) {
  const int sub = threadIdx.x % kThreadsPerRow;
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kThreadsPerRow;
  if (row >= m_pad) return;
  uint2 raw = make_uint2(0, 0);
  if (row < m) raw = *reinterpret_cast<const uint2*>(q + row * kDim + sub * 8);
  const uint8_t* b = reinterpret_cast<const uint8_t*>(&raw);
  int32_t ss = 0;
  uint4 out;
  uint32_t* o = reinterpret_cast<uint32_t*>(&out);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int32_t x0 = b[2 * t], x1 = b[2 * t + 1];
    ss += x0 * x0 + x1 * x1;
    o[t] = pack_bf16x2(-2.0f * (float)x0, -2.0f * (float)x1);
  }
  if (qbf) *reinterpret_cast<uint4*>(qbf + row * kDim + sub * 8) = out;
#pragma unroll
  for (int off = kThreadsPerRow / 2; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if (sub == 0 && row < m) qnorm[row] = ss;
  if (qext && sub < 2) {
    // K-extension (1, 256, 65536, e0, e1, e2): weights for the reference's norm
    // digits, then the base-256 digits of this query's norm, so the MMA yields
    // ||r||^2 + ||q||^2 - 2 q.r, the exact squared distance
    uint4* ext = reinterpret_cast<uint4*>(qext + row * kExt);
    ext[sub] = sub == 0 ? ext_head(1.0f, 256.0f, 65536.0f, (float)(ss & 255), (float)((ss >> 8) & 255),
                                   (float)(ss >> 16))
                        : make_uint4(0u, 0u, 0u, 0u);
  }
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

cudaError_t launch_prep_ref(const uint8_t* ref, int64_t n_ref, int64_t n_pad, __nv_bfloat16* ref_bf,
                            float* rnorm, __nv_bfloat16* ref_ext, cudaStream_t s) {
  const int64_t blocks = (n_pad + kRowsPerBlock - 1) / kRowsPerBlock;
  prep_ref_kernel<<<(unsigned)blocks, kRowsPerBlock * kThreadsPerRow, 0, s>>>(ref, n_ref, n_pad, ref_bf, rnorm,
                                                                               ref_ext);
  return cudaGetLastError();
}

cudaError_t launch_prep_query(const uint8_t* q, int64_t m, int64_t m_pad, int32_t* qnorm, __nv_bfloat16* qbf,
                              __nv_bfloat16* qext, cudaStream_t s) {
  if (m_pad == 0) return cudaSuccess;
  const int64_t blocks = (m_pad + kRowsPerBlock - 1) / kRowsPerBlock;
  prep_query_kernel<<<(unsigned)blocks, kRowsPerBlock * kThreadsPerRow, 0, s>>>(q, m, m_pad, qnorm, qbf, qext);
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
