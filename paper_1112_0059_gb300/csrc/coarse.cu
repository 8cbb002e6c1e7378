// FP8 E4M3 shortlist search, the two steps around the tensor-core coarse
// pass: operand preparation and the exact rerank.
//
// Coarse operands: every coordinate is shifted, x' = x - 64, and rounded to
// E4M3 (3 mantissa bits, round to nearest even); queries are stored as
// -2 E4M3(q'), which E4M3 holds exactly (|q'| <= 191 rounds to at most 192,
// and 384 <= 448).  The K-extension carries the unrounded squared norms
// ||r'||^2 and ||q'||^2 + kCoarseBias as base-256 digits (exact in BF16).
// The shift puts the 30% zero coordinates of SIFT-like data (x' = -64) and
// the common mid-range values on exactly representable or finely spaced
// E4M3 values.
//
// Rerank: one warp per query row computes the exact squared distance of
// every shortlisted row (uint8 rows, integer SIMD) and keeps the K1 smallest
// (distance, row) keys, the same keys the exact search produces.
#include <cuda_fp8.h>

#include "internal.cuh"

namespace lnbnn {
namespace {

constexpr int kThreadsPerRow = 16;  // 8 coordinates per thread
constexpr int kRowsPerBlock = 16;
constexpr int kShift = 64;

__device__ __forceinline__ uint32_t e4m3_bits(int32_t x) {
  return (uint32_t)__nv_cvt_float_to_fp8((float)x, __NV_SATFINITE, __NV_E4M3);
}

// E4M3 bits of -2v for the E4M3 value v with bits b: flip the sign and add one
// to the exponent field (bits 3-6); v = 0 stays 0.  Valid for |v| <= 192.
__device__ __forceinline__ uint32_t e4m3_neg2(uint32_t b) { return b == 0 ? 0u : ((b + 0x08u) ^ 0x80u) & 0xFFu; }

__device__ __forceinline__ uint32_t bf16_bits(float v) {
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return (uint32_t)*reinterpret_cast<unsigned short*>(&b);
}

__device__ __forceinline__ uint4 ext_head(float a, float b, float c, float d, float e, float f) {
  return make_uint4(bf16_bits(a) | (bf16_bits(b) << 16), bf16_bits(c) | (bf16_bits(d) << 16),
                    bf16_bits(e) | (bf16_bits(f) << 16), 0u);
}

// rows >= n are padding: zero operand bytes, extension (0, 0, 512, 1, 256,
// 65536) for references (a norm of 2^25 keeps them out of every shortlist),
// all zero for queries.
template <bool kQuery>
__global__ void prep_e4m3_kernel(const uint8_t* __restrict__ x, int64_t n, int64_t n_pad, uint8_t* __restrict__ f8,
                                 __nv_bfloat16* __restrict__ ext) {
  const int sub = threadIdx.x % kThreadsPerRow;
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kThreadsPerRow;
  if (row >= n_pad) return;
  const bool real = row < n;
  uint2 raw = make_uint2(0, 0);
  if (real) raw = *reinterpret_cast<const uint2*>(x + row * kDim + sub * 8);
  const uint8_t* b = reinterpret_cast<const uint8_t*>(&raw);
  int32_t ss = 0;
  uint32_t w[2] = {0u, 0u};
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int32_t v = (int32_t)b[t] - kShift;
    ss += v * v;
    uint32_t bits = e4m3_bits(v);
    if (kQuery) bits = e4m3_neg2(bits);
    w[t >> 2] |= (real ? bits : 0u) << (8 * (t & 3));
  }
  *reinterpret_cast<uint2*>(f8 + row * kDim + sub * 8) = make_uint2(w[0], w[1]);
#pragma unroll
  for (int off = kThreadsPerRow / 2; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if (sub >= 2) return;
  uint4* e = reinterpret_cast<uint4*>(ext + row * kExt);
  if (sub == 1) {
    e[1] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  if (kQuery) {
    // (1, 256, 65536, e0, e1, e2): weights of the reference digits, then the
    // digits of ||q'||^2 + kCoarseBias (< 2^23)
    const int32_t v = ss + kCoarseBias;
    e[0] = real ? ext_head(1.0f, 256.0f, 65536.0f, (float)(v & 255), (float)((v >> 8) & 255), (float)(v >> 16))
                : make_uint4(0u, 0u, 0u, 0u);
  } else {
    // (d0, d1, d2, 1, 256, 65536): digits of ||r'||^2 (<= 128 * 191^2 < 2^23)
    const int32_t v = real ? ss : (int32_t)kPadNorm;
    e[0] = ext_head((float)(v & 255), (float)((v >> 8) & 255), (float)(v >> 16), 1.0f, 256.0f, 65536.0f);
  }
}

constexpr int kRerankWarps = 8;
constexpr int kMaxPerLane = (LNBNN_MAX_K + 1 + 31) / 32;  // shortlist entries per lane, at most

// ||q - r||^2 over one 128-byte row, 16 bytes at a time.
__device__ __forceinline__ uint32_t sqdist_u8(const uint4 (&q)[8], const uint8_t* __restrict__ r) {
  uint32_t acc = 0;
  const uint4* rv = reinterpret_cast<const uint4*>(r);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint4 b = __ldg(rv + i);
    uint32_t d;
    d = __vabsdiffu4(q[i].x, b.x);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(q[i].y, b.y);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(q[i].z, b.z);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(q[i].w, b.w);
    acc = __dp4a(d, d, acc);
  }
  return acc;
}

__global__ void __launch_bounds__(32 * kRerankWarps)
    rerank_kernel(const uint64_t* __restrict__ shortlist, int64_t m, int M1, const uint8_t* __restrict__ q,
                  const uint8_t* __restrict__ ref, int64_t n_ref, int K1, uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kRerankWarps + (threadIdx.x >> 5);
  if (row >= m) return;
  uint4 qv[8];
  const uint4* qrow = reinterpret_cast<const uint4*>(q + row * kDim);
#pragma unroll
  for (int i = 0; i < 8; ++i) qv[i] = __ldg(qrow + i);
  // lane l scores shortlist entries l, l + 32, ...
  uint64_t key[kMaxPerLane];
#pragma unroll
  for (int c = 0; c < kMaxPerLane; ++c) {
    const int at = c * 32 + lane;
    key[c] = kEmptyKey;
    if (at < M1) {
      const uint64_t s = shortlist[row * M1 + at];
      // (a padding row can only be shortlisted when fewer than M1 real rows
      // exist, which the caller rules out; it is skipped all the same)
      if (s != kEmptyKey && (int64_t)key_row(s) < n_ref) {
        const uint32_t j = key_row(s);
        key[c] = make_key(sqdist_u8(qv, ref + (int64_t)j * kDim), j);
      }
    }
  }
  // the K1 smallest keys, in order: repeated warp minimum; each key is unique
  for (int r = 0; r < K1; ++r) {
    uint64_t mn = key[0];
#pragma unroll
    for (int c = 1; c < kMaxPerLane; ++c) mn = min(mn, key[c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    if (lane == 0) out[row * K1 + r] = mn;
    if (mn == kEmptyKey) continue;
#pragma unroll
    for (int c = 0; c < kMaxPerLane; ++c)
      if (key[c] == mn) key[c] = kEmptyKey;
  }
}

}  // namespace

cudaError_t launch_prep_ref_e4m3(const uint8_t* ref, int64_t n_ref, int64_t n_pad, uint8_t* ref_f8,
                                 __nv_bfloat16* ref_ext, cudaStream_t s) {
  if (n_pad == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n_pad + kRowsPerBlock - 1) / kRowsPerBlock);
  prep_e4m3_kernel<false><<<blocks, kThreadsPerRow * kRowsPerBlock, 0, s>>>(ref, n_ref, n_pad, ref_f8, ref_ext);
  return cudaGetLastError();
}

cudaError_t launch_prep_query_e4m3(const uint8_t* q, int64_t m, int64_t m_pad, uint8_t* qf8, __nv_bfloat16* qext,
                                   cudaStream_t s) {
  if (m_pad == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((m_pad + kRowsPerBlock - 1) / kRowsPerBlock);
  prep_e4m3_kernel<true><<<blocks, kThreadsPerRow * kRowsPerBlock, 0, s>>>(q, m, m_pad, qf8, qext);
  return cudaGetLastError();
}

cudaError_t launch_rerank(const uint64_t* shortlist, int64_t m, int M1, const uint8_t* q, const uint8_t* ref,
                          int64_t n_ref, int K1, uint64_t* out, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  if (M1 < 1 || M1 > LNBNN_MAX_K + 1 || K1 < 1 || K1 > M1) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((m + kRerankWarps - 1) / kRerankWarps);
  rerank_kernel<<<blocks, 32 * kRerankWarps, 0, s>>>(shortlist, m, M1, q, ref, n_ref, K1, out);
  return cudaGetLastError();
}

}  // namespace lnbnn
