// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (see include/lnbnn.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lnbnn.h"

namespace lnbnn {

constexpr int kDim = LNBNN_DIM;
// A list slot with no neighbour yet; sorts after every real (distance, row) key.
constexpr uint64_t kEmptyKey = ~0ull;
// Squared norm given to padding rows of the reference operand: larger than any
// real squared distance (<= 128 * 255^2 = 8,323,200) plus its query norm, and
// exactly representable in fp32, so a padding row never enters a top-k list
// while real rows remain.
constexpr float kPadNorm = 33554432.0f;  // 2^25
// Reference rows are padded to a multiple of this (the widest reference tile).
constexpr int kRefPad = 256;
// Query rows are padded to a multiple of this (the 128-row query tile of the
// tensor-core search).
constexpr int kQueryPad = 128;

// Width of the K-extension that carries ||r||^2 into the tensor-core
// contraction: a reference row gets the base-256 digits (d0, d1, d2) of its
// squared norm, a query row the constants (1, 256, 65536), zero-padded to one
// MMA K-step of 16 BF16 columns.  All these values are exact in BF16.
constexpr int kExt = 16;

// Added to every coarse value of the FP8 shortlist search so that it stays
// positive (float bit patterns then order like the values).
constexpr int32_t kCoarseBias = 1 << 21;

// Bits of the per-index device error word.
enum : uint32_t { kDevErrTimeout = 1u, kDevErrOffsets = 2u };

// Neighbour key: (squared distance, reference row) packed so that one unsigned
// compare orders by distance first, then by the lower row.
__host__ __device__ __forceinline__ uint64_t make_key(uint32_t dist, uint32_t row) {
  return (static_cast<uint64_t>(dist) << 32) | row;
}
__host__ __device__ __forceinline__ uint32_t key_dist(uint64_t k) { return static_cast<uint32_t>(k >> 32); }
__host__ __device__ __forceinline__ uint32_t key_row(uint64_t k) { return static_cast<uint32_t>(k); }

// ----------------------------------------------------------- kernels (launchers)
// Each launcher returns cudaGetLastError() after the launch.

// Rows of descriptors are kDim bytes (appearance), or kDim + 2 with a location
// (x, y) weighted by loc_w in [0, LNBNN_MAX_LOCATION_WEIGHT].
__host__ __device__ __forceinline__ bool row_layout_ok(int row_bytes, int loc_w) {
  return (row_bytes == kDim && loc_w == 0) ||
         (row_bytes == LNBNN_LOCATED_DIM && loc_w >= 0 && loc_w <= LNBNN_MAX_LOCATION_WEIGHT);
}

// Reference preparation (rows of row_bytes bytes): exact BF16 copy of the
// centred appearance coordinates x - 128 (padding rows up to n_pad: zero),
// squared norms as fp32 (padding rows get kPadNorm) and the K-extension
// [n_pad, kExt] (norm digits, location columns).
cudaError_t launch_prep_ref(const uint8_t* ref, int64_t n_ref, int64_t n_pad, int row_bytes, int loc_w,
                            __nv_bfloat16* ref_bf, float* rnorm, __nv_bfloat16* ref_ext, cudaStream_t s);
// Query preparation: squared norms (int32) and, when qbf != nullptr, the BF16
// operand -2 (q - 128) (padding rows up to m_pad: zero) and its K-extension
// [m_pad, kExt] (the weights of the reference's norm digits, the query's norm
// digits, the location cross-term columns).
cudaError_t launch_prep_query(const uint8_t* q, int64_t m, int64_t m_pad, int row_bytes, int loc_w, int32_t* qnorm,
                              __nv_bfloat16* qbf, __nv_bfloat16* qext, cudaStream_t s);
// Label histogram; sets *bad when a label is outside [0, C).
cudaError_t launch_label_hist(const int32_t* labels, int64_t n, int32_t C, unsigned long long* counts,
                              uint32_t* bad, cudaStream_t s);
// Gather rows: dst[i] = src[perm[i]] for bf16 operand rows, norm-digit rows,
// norms and labels.
cudaError_t launch_gather_ref(const int64_t* perm, int64_t n, const __nv_bfloat16* src_bf, __nv_bfloat16* dst_bf,
                              const __nv_bfloat16* src_ext,
                              __nv_bfloat16* dst_ext, const float* src_norm, float* dst_norm,
                              const int32_t* src_lab, int32_t* dst_lab, cudaStream_t s);

// dst[0..n) = v
cudaError_t launch_fill_float(float* dst, int64_t n, float v, cudaStream_t s);

// Merge `splits` sorted lists per row into one sorted list of K1 keys
// (at most 32 * kMaxListsPerLane lists).  With `chain.done` set (the scan's
// per-work-item flags of a launch whose splits carried their lists), a row
// whose last split reports 2 merges only that split's lists_per_split lists.
constexpr int kMaxListsPerLane = 20;
struct MergeChain {
  const uint32_t* done = nullptr;
  int64_t T = 0;              // query-tile groups: work item x + y T is split y of group x
  int64_t rows_per_item = 0;  // query rows per group
  int lists_per_split = 0;
};
cudaError_t launch_merge_lists(const uint64_t* lists, int splits, int64_t m, int64_t list_stride_rows,
                               int K1, uint64_t* out, cudaStream_t s, const MergeChain& chain = MergeChain{});
// knn_search output: first k entries of each sorted list as (row, distance).
cudaError_t launch_extract_knn(const uint64_t* lists, int64_t m, int K1, int k, int32_t* idx,
                               int32_t* dist, cudaStream_t s);
// Alg. 2 per-descriptor update: totals[img][C] += dist_C - dist_B (rows whose
// list is incomplete, which only a search that gave up leaves, are skipped).
cudaError_t launch_lnbnn_score(const uint64_t* lists, int64_t m, int K1, int k, const int32_t* labels, int64_t n_ref,
                               const int64_t* offsets, int64_t n_img, int32_t C, int64_t* totals,
                               uint32_t* dev_err, cudaStream_t s);
// Alg. 1 sum: totals[img][c] = sum of mins[row][c] over the image's rows.
cudaError_t launch_nbnn_sum(const int32_t* mins, int64_t m, int32_t C, const int64_t* offsets, int64_t n_img,
                            int64_t* totals, cudaStream_t s);
// Offsets validation (0 = o[0] <= ... <= o[n_img] = m); flags kDevErrOffsets.
cudaError_t launch_check_offsets(const int64_t* offsets, int64_t n_img, int64_t m, uint32_t* dev_err,
                                 cudaStream_t s);
// FP8 shortlist search: E4M3 operands of the coarse pass (see coarse.cu).
// ref_f8 [n_pad, 128] bytes of E4M3(r - 64), ref_ext [n_pad, kExt] digits of
// ||r - 64||^2; qf8 [m_pad, 128] bytes of -2 E4M3(q - 64), qext [m_pad, kExt]
// digits of ||q - 64||^2 + kCoarseBias.
cudaError_t launch_prep_ref_e4m3(const uint8_t* ref, int64_t n_ref, int64_t n_pad, uint8_t* ref_f8,
                                 __nv_bfloat16* ref_ext, cudaStream_t s);
cudaError_t launch_prep_query_e4m3(const uint8_t* q, int64_t m, int64_t m_pad, uint8_t* qf8, __nv_bfloat16* qext,
                                   cudaStream_t s);
// Exact rerank: for each query row, the K1 smallest exact (distance, row) keys
// among the rows of its shortlist [m, M1] (kEmptyKey entries are no row).
cudaError_t launch_rerank(const uint64_t* shortlist, int64_t m, int M1, const uint8_t* q, const uint8_t* ref,
                          int64_t n_ref, int K1, uint64_t* out, cudaStream_t s);
// NBNN as a sum of log-odds increments (logodds.cu).  Per descriptor row of the
// [m, C] class-minimum table, the statistics of its posterior (32 bytes a row);
// then per image and class the sum of the increments (all, or only those > 0)
// in row order, and per image the number of increments added (counts may be
// null; it is added to, so the caller zeroes it).
constexpr int kLogoddsRowStatBytes = 32;
cudaError_t launch_logodds_rowstat(const int32_t* mins, int64_t m, int32_t C, double beta, void* rowstat,
                                   cudaStream_t s);
cudaError_t launch_logodds_sum(const int32_t* mins, const void* rowstat, int64_t m, int32_t C, double beta,
                               bool positive_only, const int64_t* offsets, int64_t n_img, double* totals,
                               int64_t* counts, cudaStream_t s);
// argmax over classes per image, lowest class on ties.
cudaError_t launch_argmax_f64(const double* totals, int64_t n_img, int32_t C, int32_t* classes, cudaStream_t s);
// argmin over classes per image, lowest class on ties.
cudaError_t launch_argmin(const int64_t* totals, int64_t n_img, int32_t C, int32_t* classes, cudaStream_t s);

}  // namespace lnbnn
