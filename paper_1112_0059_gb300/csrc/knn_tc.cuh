// Host-side interface of the tensor-core (tcgen05) search kernels.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace lnbnn {

// References per tile of the tensor-core kernels (the MMA N extent).
constexpr int kTcRefTile = 256;

// TMA descriptors over an index's BF16 reference operands (caller's row order
// and class-sorted order).  Encoded once at index creation.
struct TcTensorMaps {
  CUtensorMap ref, ref_ext;    // BF16 [n_pad,128] (128-byte swizzle) and norm digits [n_pad,16] (32-byte swizzle)
  CUtensorMap sref, sref_ext;  // the same over the class-sorted copy
};

bool make_tc_tensor_maps(const __nv_bfloat16* ref_bf, const __nv_bfloat16* sref_bf, const __nv_bfloat16* ref_ext,
                         const __nv_bfloat16* sref_ext, int64_t n_pad, TcTensorMaps* out);

// Exact top-K1 search on tensor cores.  qbf: BF16 -2q operand [m_pad, 128];
// qext: its K-extension [m_pad, 16].  Split s scans reference rows
// [s * split_len, min((s+1) * split_len, n_ref)); its sorted list for query row i
// is written at lists[(s * stride + i) * K1].
cudaError_t launch_knn_tc(const TcTensorMaps& maps, bool sorted_copy, const __nv_bfloat16* qbf,
                          const __nv_bfloat16* qext, int64_t m, int64_t m_pad, const int32_t* qnorm, int64_t n_ref,
                          int splits, int64_t split_len, int K1, uint64_t* lists, int64_t stride, uint32_t* dev_err,
                          cudaStream_t s);

}  // namespace lnbnn
