// Host-side interface of the tensor-core (tcgen05) search kernels.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace lnbnn {

// References per tile of the tensor-core kernels (the MMA N extent).
constexpr int kTcRefTile = 256;
// Query rows per CTA (the MMA M extent) and CTAs per cluster; the query
// operand must be padded to kTcQueryTile * kTcCluster rows.
constexpr int kTcQueryTile = 128;
constexpr int kTcCluster = 1;
static_assert(kQueryPad % (kTcQueryTile * kTcCluster) == 0, "query padding must cover whole clusters");
// Epilogue warps per TMEM lane quarter.  Each owns a column slice of every
// tile and keeps its own top-K1 list per query row, so one reference split
// yields this many sorted lists per row (merged afterwards).
constexpr int kTcListsPerSplit = 2;
// Largest K1 kept in registers; larger lists live in global memory.  The
// coarse pass also has a 32-entry register list (its shortlists are longer).
constexpr int kTcRegListMax = 16;
constexpr int kTcCoarseRegListMax = 32;
static_assert(kTcListsPerSplit > 1, "the shortlist search merges into a buffer apart from the lists");

// TMA descriptors over an index's BF16 reference operands (caller's row order
// and class-sorted order).  Encoded once at index creation.
struct TcTensorMaps {
  CUtensorMap ref, ref_ext;    // BF16 [n_pad,128] (128-byte swizzle) and norm digits [n_pad,16] (32-byte swizzle)
  CUtensorMap sref, sref_ext;  // the same over the class-sorted copy
  CUtensorMap f8, f8_ext;      // E4M3 coarse operand [n_pad,128] and its extension [n_pad,16]
};

// Sets the kernels' shared-memory size on the current device; call once per
// device before launching (and before any stream capture).
cudaError_t prepare_tc_kernels();

bool make_tc_tensor_maps(const __nv_bfloat16* ref_bf, const __nv_bfloat16* sref_bf, const __nv_bfloat16* ref_ext,
                         const __nv_bfloat16* sref_ext, int64_t n_pad, TcTensorMaps* out);

bool make_tc_tensor_maps_e4m3(const uint8_t* ref_f8, const __nv_bfloat16* ref_f8_ext, int64_t n_pad,
                              TcTensorMaps* out);

// Exact top-K1 search on tensor cores.  qbf: BF16 -2q operand [m_pad, 128];
// qext: its K-extension [m_pad, 16].  Split s scans reference rows
// [s * split_len, min((s+1) * split_len, n_ref)) and writes kTcListsPerSplit
// sorted lists per query row i, list w at lists[((s * kTcListsPerSplit + w) *
// stride + i) * K1]; the K1 smallest keys of their union are the split's answer.
cudaError_t launch_knn_tc(const TcTensorMaps& maps, bool sorted_copy, const __nv_bfloat16* qbf,
                          const __nv_bfloat16* qext, int64_t m, int64_t m_pad, int64_t n_ref, int splits,
                          int64_t split_len, int K1, uint64_t* lists, int64_t stride, uint32_t* dev_err,
                          unsigned long long* stats, cudaStream_t s);
// Coarse pass of the FP8 shortlist search: the same scan over the E4M3
// operands (qf8 [m_pad, 128] bytes of -2 E4M3(q - 64), qext its extension),
// keeping the K1 smallest (coarse + 2^21, row) keys per list in the same
// layout as launch_knn_tc.
cudaError_t launch_coarse_tc(const TcTensorMaps& maps, const uint8_t* qf8, const __nv_bfloat16* qext, int64_t m,
                             int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int K1, uint64_t* lists,
                             int64_t stride, uint32_t* dev_err, unsigned long long* stats, cudaStream_t s);
// Original NBNN on the same tensor-core scan over the class-sorted copy:
// mins [m_pad, C] (int32, filled with INT32_MAX-like values beforehand) gets
// atomicMin(mins[i][c], ||q_i - r||^2) over every reference r of class c that
// split's range covers, so after all splits mins[i][c] = NN_c(q_i).
cudaError_t launch_nbnn_tc(const TcTensorMaps& maps, const __nv_bfloat16* qbf, const __nv_bfloat16* qext, int64_t m,
                           int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int32_t* mins, int32_t C,
                           const int64_t* class_off, uint32_t* dev_err, unsigned long long* stats, cudaStream_t s);
// stats (may be null): the MMA thread of every CTA adds its SM cycles,
// globaltimer nanoseconds and tile count to stats[0..2] and 1 to stats[3].

}  // namespace lnbnn
