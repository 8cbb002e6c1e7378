// Split merge, knn_search output, the Local NBNN class update (Alg. 2), the
// offsets check and the per-image argmin (Alg. 1 and Alg. 2, last line).
#include "internal.cuh"

namespace lnbnn {
namespace {

// Row i's `n_lists` partial lists live at lists[(l * stride + i) * K1]; each is
// sorted ascending.  One warp per row writes the K1 smallest keys of their
// union, ascending: lane j holds the heads of lists j, j + 32, ...; each round
// the warp minimum is written and the list that held it advances.  A key
// names one reference row; it can sit in several lists of a row when a split
// started from the previous split's list, and is written once (a key equal to
// the last one written only advances its lists).
constexpr int kMergeWarps = 4;
// Up to this many lists a thread merges a row on its own (few lists: the
// warp form would leave most lanes idle).
constexpr int kThreadMergeLists = 8;

// The first list of row i to merge: all of them, or only the last split's
// when that split's work item says its lists hold every earlier split's keys
// (the scan's done flag 2).  Work item x + y T covers query rows
// [x rows_per_item, (x + 1) rows_per_item) of split y.
__device__ __forceinline__ int first_list(const MergeChain& c, int64_t i, int n_lists) {
  if (c.done == nullptr) return 0;
  const int splits = n_lists / c.lists_per_split;
  const int64_t w = i / c.rows_per_item + (int64_t)(splits - 1) * c.T;
  return c.done[w] == 2u ? n_lists - c.lists_per_split : 0;
}

__global__ void merge_lists_thread_kernel(const uint64_t* __restrict__ lists, int n_lists, int64_t m, int64_t stride,
                                          int K1, MergeChain chain, uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int l0 = first_list(chain, i, n_lists);
  lists += (int64_t)l0 * stride * K1;
  n_lists -= l0;
  int pos[kThreadMergeLists];
  uint64_t head[kThreadMergeLists];
#pragma unroll
  for (int l = 0; l < kThreadMergeLists; ++l) {
    pos[l] = 0;
    head[l] = l < n_lists ? lists[((int64_t)l * stride + i) * K1] : kEmptyKey;
  }
  uint64_t last = kEmptyKey;
  for (int t = 0; t < K1;) {
    uint64_t best = head[0];
    int bl = 0;
#pragma unroll
    for (int l = 1; l < kThreadMergeLists; ++l)
      if (head[l] < best) {
        best = head[l];
        bl = l;
      }
    const bool dup = best != kEmptyKey && best == last;
    if (!dup) {
      out[i * K1 + t] = best;
      ++t;
      last = best;
    }
    if (best == kEmptyKey) continue;
#pragma unroll
    for (int l = 0; l < kThreadMergeLists; ++l)
      if (l == bl) {
        ++pos[l];
        head[l] = pos[l] < K1 ? lists[((int64_t)l * stride + i) * K1 + pos[l]] : kEmptyKey;
      }
  }
}

__global__ void __launch_bounds__(32 * kMergeWarps)
    merge_lists_kernel(const uint64_t* __restrict__ lists, int n_lists, int64_t m, int64_t stride, int K1,
                       MergeChain chain, uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kMergeWarps + (threadIdx.x >> 5);
  if (i >= m) return;
  const int l0 = first_list(chain, i, n_lists);  // the same for the whole warp (one row)
  lists += (int64_t)l0 * stride * K1;
  n_lists -= l0;
  uint64_t head[kMaxListsPerLane];
  int pos[kMaxListsPerLane];
#pragma unroll
  for (int c = 0; c < kMaxListsPerLane; ++c) {
    const int l = c * 32 + lane;
    pos[c] = 0;
    head[c] = l < n_lists ? lists[((int64_t)l * stride + i) * K1] : kEmptyKey;
  }
  uint64_t last = kEmptyKey;
  for (int t = 0; t < K1;) {
    uint64_t best = kEmptyKey;
    int bc = 0;
#pragma unroll
    for (int c = 0; c < kMaxListsPerLane; ++c)
      if (head[c] < best) {
        best = head[c];
        bc = c;
      }
    uint64_t wmin = best;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, off));
    const bool dup = wmin != kEmptyKey && wmin == last;  // warp-uniform
    if (!dup) {
      if (lane == 0) out[i * K1 + t] = wmin;
      ++t;
      last = wmin;
    }
    if (wmin != kEmptyKey && best == wmin) {
#pragma unroll
      for (int c = 0; c < kMaxListsPerLane; ++c)
        if (c == bc) {
          const int l = c * 32 + lane;
          ++pos[c];
          head[c] = pos[c] < K1 ? lists[((int64_t)l * stride + i) * K1 + pos[c]] : kEmptyKey;
        }
    }
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
// Thread per row; the adds are aggregated per warp: at each neighbour rank
// the lanes that update the same (image, class) are grouped, and one of them
// adds the group's sum (int64 addition, exact in any order).
constexpr int kScoreThreads = 128;
__global__ void __launch_bounds__(kScoreThreads)
    lnbnn_score_kernel(const uint64_t* __restrict__ lists, int64_t m, int K1, int k,
                       const int32_t* __restrict__ labels, int64_t n_ref, const int64_t* __restrict__ offsets,
                       int64_t n_img, int32_t C, int64_t* __restrict__ totals, uint32_t* __restrict__ dev_err) {
  __shared__ int64_t part[kScoreThreads];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int64_t* wpart = part + (threadIdx.x & ~31);
  bool ok = i < m;
  int64_t img = 0;
  if (ok) {
    img = image_of(offsets, n_img, i);
    if (i < offsets[img] || i >= offsets[img + 1]) {  // only with invalid offsets
      atomicOr(dev_err, kDevErrOffsets);
      ok = false;
    }
  }
  const uint64_t* L = lists + (ok ? i : 0) * K1;
  // A complete list holds k+1 real rows.  Only a search that gave up (a
  // timeout, reported by lnbnn_sync) leaves empty keys: skip such a row
  // rather than gather labels[] at an empty key's row.
  if (ok)
    for (int a = 0; a <= k; ++a)
      if ((int64_t)key_row(L[a]) >= n_ref) ok = false;
  const int64_t dist_B = ok ? (int64_t)key_dist(L[k]) : 0;
  unsigned long long* t = reinterpret_cast<unsigned long long*>(totals);
  for (int a = 0; a < k; ++a) {  // every lane of the warp takes every step
    long long slot = -1;          // img * C + class of this lane's update, or none
    int64_t delta = 0;
    if (ok) {
      const uint64_t ka = L[a];
      const int32_t c = labels[key_row(ka)];
      bool seen = false;
      for (int b = 0; b < a && !seen; ++b) seen = labels[key_row(L[b])] == c;
      if (!seen) {
        delta = (int64_t)key_dist(ka) - dist_B;  // <= 0
        if (delta != 0) slot = img * C + c;
      }
    }
    const unsigned act = __ballot_sync(0xffffffffu, slot >= 0);
    if (slot >= 0) {
      const unsigned grp = __match_any_sync(act, (unsigned long long)slot);
      wpart[lane] = delta;
      __syncwarp(act);
      if (lane == __ffs(grp) - 1) {
        int64_t sum = 0;
        for (unsigned g = grp; g; g &= g - 1) sum += wpart[__ffs(g) - 1];
        atomicAdd(t + slot, (unsigned long long)sum);
      }
      __syncwarp(act);  // the leaders have read the slots before the next step writes them
    }
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
                               cudaStream_t s, const MergeChain& chain) {
  if (m == 0) return cudaSuccess;
  if (splits < 1 || splits > 32 * kMaxListsPerLane) return cudaErrorInvalidValue;
  if (chain.done != nullptr &&
      (chain.lists_per_split < 1 || splits % chain.lists_per_split != 0 || chain.T < 1 || chain.rows_per_item < 1))
    return cudaErrorInvalidValue;
  if (splits <= kThreadMergeLists) {
    merge_lists_thread_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(lists, splits, m, stride, K1, chain, out);
    return cudaGetLastError();
  }
  merge_lists_kernel<<<(unsigned)((m + kMergeWarps - 1) / kMergeWarps), 32 * kMergeWarps, 0, s>>>(
      lists, splits, m, stride, K1, chain, out);
  return cudaGetLastError();
}

cudaError_t launch_extract_knn(const uint64_t* lists, int64_t m, int K1, int k, int32_t* idx, int32_t* dist,
                               cudaStream_t s) {
  const int64_t n = m * k;
  if (n == 0) return cudaSuccess;
  extract_knn_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lists, m, K1, k, idx, dist);
  return cudaGetLastError();
}

cudaError_t launch_lnbnn_score(const uint64_t* lists, int64_t m, int K1, int k, const int32_t* labels, int64_t n_ref,
                               const int64_t* offsets, int64_t n_img, int32_t C, int64_t* totals, uint32_t* dev_err,
                               cudaStream_t s) {
  if (m == 0 || n_img == 0) return cudaSuccess;
  lnbnn_score_kernel<<<(unsigned)((m + kScoreThreads - 1) / kScoreThreads), kScoreThreads, 0, s>>>(
      lists, m, K1, k, labels, n_ref, offsets, n_img, C, totals, dev_err);
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
