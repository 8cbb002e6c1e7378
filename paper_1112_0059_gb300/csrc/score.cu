// Split merge, knn_search output, the Local NBNN class update (Alg. 2), the
// offsets check and the per-image argmin (Alg. 1 and Alg. 2, last line).
#include "internal.cuh"

namespace lnbnn {
namespace {

constexpr int kMaxSplitsMerge = 64;

// Row i's `splits` partial lists live at lists[(s * stride + i) * K1]; each is
// sorted ascending.  Writes the K1 smallest keys of their union, ascending.
__global__ void merge_lists_kernel(const uint64_t* __restrict__ lists, int splits, int64_t m, int64_t stride,
                                   int K1, uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int pos[kMaxSplitsMerge];
  for (int s = 0; s < splits; ++s) pos[s] = 0;
  for (int t = 0; t < K1; ++t) {
    uint64_t best = kEmptyKey;
    int bs = -1;
    for (int s = 0; s < splits; ++s) {
      if (pos[s] < K1) {
        const uint64_t v = lists[((int64_t)s * stride + i) * K1 + pos[s]];
        if (v < best) {
          best = v;
          bs = s;
        }
      }
    }
    if (bs >= 0) ++pos[bs];
    out[i * K1 + t] = best;
  }
}

__global__ void extract_knn_kernel(const uint64_t* __restrict__ lists, int64_t m, int K1, int k,
                                   int32_t* __restrict__ idx, int32_t* __restrict__ dist) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t i = e / k;
  const int t = (int)(e - i * k);
  const uint64_t key = lists[i * K1 + t];
  idx[e] = (int32_t)key_row(key);
  dist[e] = (int32_t)key_dist(key);
}

// Image owning descriptor row i: the last image whose first row is <= i.
__device__ __forceinline__ int64_t image_of(const int64_t* __restrict__ offsets, int64_t n_img, int64_t i) {
  int64_t lo = 0, hi = n_img;  // answer in [0, n_img)
  while (lo + 1 < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Alg. 2 for one descriptor row i, given its k+1 nearest neighbours sorted by
// (distance, row): dist_B = distance of the (k+1)-th; every class found among
// the first k is updated once with dist_C - dist_B, where dist_C is the
// distance of its first (hence nearest) occurrence in the sorted list.
__global__ void lnbnn_score_kernel(const uint64_t* __restrict__ lists, int64_t m, int K1, int k,
                                   const int32_t* __restrict__ labels, const int64_t* __restrict__ offsets,
                                   int64_t n_img, int32_t C, int64_t* __restrict__ totals,
                                   uint32_t* __restrict__ dev_err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t img = image_of(offsets, n_img, i);
  if (i < offsets[img] || i >= offsets[img + 1]) {  // only with invalid offsets
    atomicOr(dev_err, kDevErrOffsets);
    return;
  }
  const uint64_t* L = lists + i * K1;
  const int64_t dist_B = (int64_t)key_dist(L[k]);
  unsigned long long* t = reinterpret_cast<unsigned long long*>(totals + img * C);
  for (int a = 0; a < k; ++a) {
    const uint64_t ka = L[a];
    const int32_t c = labels[key_row(ka)];
    bool seen = false;
    for (int b = 0; b < a && !seen; ++b) seen = labels[key_row(L[b])] == c;
    if (seen) continue;
    const int64_t delta = (int64_t)key_dist(ka) - dist_B;  // <= 0
    if (delta != 0) atomicAdd(t + c, (unsigned long long)delta);
  }
}

// Alg. 1's sum for image img and class c: totals[img][c] = sum over the image's
// descriptor rows of mins[row][c] (= NN_c of that descriptor).  Rows outside
// [0, m) are skipped (they only arise from invalid offsets, flagged elsewhere).
__global__ void nbnn_sum_kernel(const int32_t* __restrict__ mins, int64_t m, int32_t C,
                                const int64_t* __restrict__ offsets, int64_t* __restrict__ totals) {
  const int64_t img = blockIdx.x;
  const int32_t c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int64_t r0 = max(offsets[img], (int64_t)0), r1 = min(offsets[img + 1], m);
  int64_t acc = 0;
  for (int64_t r = r0; r < r1; ++r) acc += mins[r * C + c];
  totals[img * C + c] = acc;
}

__global__ void check_offsets_kernel(const int64_t* __restrict__ offsets, int64_t n_img, int64_t m,
                                     uint32_t* __restrict__ dev_err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_img) return;
  bool bad = false;
  if (i == 0) bad = offsets[0] != 0;
  if (i == n_img) bad = bad || offsets[n_img] != m;
  if (i < n_img) bad = bad || offsets[i + 1] < offsets[i];
  if (bad) atomicOr(dev_err, kDevErrOffsets);
}

// One warp per image; lanes scan classes lane, lane+32, ...; ties -> lowest class.
__global__ void argmin_kernel(const int64_t* __restrict__ totals, int64_t n_img, int32_t C,
                              int32_t* __restrict__ classes) {
  const int64_t img = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (img >= n_img) return;
  const int64_t* t = totals + img * C;
  int64_t best = INT64_MAX;
  int32_t bc = INT32_MAX;
  for (int32_t c = lane; c < C; c += 32) {
    const int64_t v = t[c];
    if (v < best) {  // c increases, so the first minimum seen is the lowest
      best = v;
      bc = c;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int64_t ov = __shfl_xor_sync(0xffffffffu, best, off);
    const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (ov < best || (ov == best && oc < bc)) {
      best = ov;
      bc = oc;
    }
  }
  if (lane == 0) classes[img] = bc;
}

}  // namespace

cudaError_t launch_merge_lists(const uint64_t* lists, int splits, int64_t m, int64_t stride, int K1, uint64_t* out,
                               cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  if (splits > kMaxSplitsMerge) return cudaErrorInvalidValue;
  merge_lists_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(lists, splits, m, stride, K1, out);
  return cudaGetLastError();
}

cudaError_t launch_extract_knn(const uint64_t* lists, int64_t m, int K1, int k, int32_t* idx, int32_t* dist,
                               cudaStream_t s) {
  const int64_t n = m * k;
  if (n == 0) return cudaSuccess;
  extract_knn_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lists, m, K1, k, idx, dist);
  return cudaGetLastError();
}

cudaError_t launch_lnbnn_score(const uint64_t* lists, int64_t m, int K1, int k, const int32_t* labels,
                               const int64_t* offsets, int64_t n_img, int32_t C, int64_t* totals, uint32_t* dev_err,
                               cudaStream_t s) {
  if (m == 0 || n_img == 0) return cudaSuccess;
  lnbnn_score_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(lists, m, K1, k, labels, offsets, n_img, C, totals,
                                                                  dev_err);
  return cudaGetLastError();
}

cudaError_t launch_nbnn_sum(const int32_t* mins, int64_t m, int32_t C, const int64_t* offsets, int64_t n_img,
                            int64_t* totals, cudaStream_t s) {
  if (n_img == 0) return cudaSuccess;
  dim3 grid((unsigned)n_img, (unsigned)((C + 127) / 128));
  nbnn_sum_kernel<<<grid, 128, 0, s>>>(mins, m, C, offsets, totals);
  return cudaGetLastError();
}

cudaError_t launch_check_offsets(const int64_t* offsets, int64_t n_img, int64_t m, uint32_t* dev_err,
                                 cudaStream_t s) {
  check_offsets_kernel<<<(unsigned)((n_img + 1 + 255) / 256), 256, 0, s>>>(offsets, n_img, m, dev_err);
  return cudaGetLastError();
}

cudaError_t launch_argmin(const int64_t* totals, int64_t n_img, int32_t C, int32_t* classes, cudaStream_t s) {
  if (n_img == 0) return cudaSuccess;
  argmin_kernel<<<(unsigned)((n_img * 32 + 255) / 256), 256, 0, s>>>(totals, n_img, C, classes);
  return cudaGetLastError();
}

}  // namespace lnbnn
