// Original NBNN on CUDA cores (dp4a): the per-class nearest distance NN_C of
// Alg. 1.  One thread owns one query row; reference tiles are staged in
// shared memory and read by broadcast.  ||q - r||^2 = ||q||^2 + ||r||^2 - 2 q.r,
// all exact in 32-bit integers.
#include "internal.cuh"

namespace lnbnn {
namespace {

constexpr int kThreads = 128;  // query rows per block
constexpr int kTile = 32;      // references per shared-memory tile

__device__ __forceinline__ void load_query(const uint8_t* __restrict__ q, int64_t row, bool active, uint32_t (&qw)[32]) {
  const uint4* src = reinterpret_cast<const uint4*>(q + row * kDim);
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    uint4 x = active ? src[v] : make_uint4(0, 0, 0, 0);
    qw[4 * v + 0] = x.x;
    qw[4 * v + 1] = x.y;
    qw[4 * v + 2] = x.z;
    qw[4 * v + 3] = x.w;
  }
}

__device__ __forceinline__ void stage_tile(const uint8_t* __restrict__ ref, int64_t j0, int64_t j1,
                                           uint4 (*tile)[8]) {
  // kTile rows x 8 uint4 = 256 uint4, two per thread
  for (int e = threadIdx.x; e < kTile * 8; e += kThreads) {
    const int r = e >> 3, v = e & 7;
    const int64_t j = j0 + r;
    tile[r][v] = j < j1 ? reinterpret_cast<const uint4*>(ref + j * kDim)[v] : make_uint4(0, 0, 0, 0);
  }
}

__device__ __forceinline__ uint32_t dot_u8(const uint32_t (&qw)[32], const uint4 (&r)[8]) {
  uint32_t acc = 0;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const uint4 x = r[v];
    acc = __dp4a(qw[4 * v + 0], x.x, acc);
    acc = __dp4a(qw[4 * v + 1], x.y, acc);
    acc = __dp4a(qw[4 * v + 2], x.z, acc);
    acc = __dp4a(qw[4 * v + 3], x.w, acc);
  }
  return acc;
}

// Alg. 1 per class over the class-sorted copy: block (bx, g) scans the
// references of classes [groups.cls[g], groups.cls[g+1]) and, at the end of
// each class, adds the row's minimum distance to totals[image][class].
__global__ void __launch_bounds__(kThreads) nbnn_simt_kernel(const uint8_t* __restrict__ q, int64_t m,
                                                             const int32_t* __restrict__ qnorm,
                                                             const uint8_t* __restrict__ sref,
                                                             const float* __restrict__ srnorm,
                                                             const int64_t* __restrict__ class_off, ClassGroups groups,
                                                             const int64_t* __restrict__ offsets, int64_t n_img,
                                                             int32_t C, int64_t* __restrict__ totals) {
  __shared__ uint4 tile[kTile][8];
  __shared__ int32_t tnorm[kTile];
  const int64_t row = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool active = row < m;
  uint32_t qw[32];
  load_query(q, row, active, qw);
  const int32_t qn = active ? qnorm[row] : 0;
  int64_t img = 0;
  if (active) {
    int64_t lo = 0, hi = n_img;
    while (lo + 1 < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= row) lo = mid; else hi = mid;
    }
    img = lo;
  }
  unsigned long long* t = reinterpret_cast<unsigned long long*>(totals + img * C);
  const int32_t c_begin = groups.cls[blockIdx.y], c_end = groups.cls[blockIdx.y + 1];
  for (int32_t c = c_begin; c < c_end; ++c) {
    const int64_t j_begin = class_off[c], j_end = class_off[c + 1];
    int32_t best = INT32_MAX;
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kTile) {
      __syncthreads();
      stage_tile(sref, j0, j_end, tile);
      if (threadIdx.x < kTile) tnorm[threadIdx.x] = j0 + threadIdx.x < j_end ? (int32_t)srnorm[j0 + threadIdx.x] : 0;
      __syncthreads();
      const int nt = (int)min((int64_t)kTile, j_end - j0);
      for (int r = 0; r < nt; ++r) {
        const int32_t d = qn + tnorm[r] - 2 * (int32_t)dot_u8(qw, tile[r]);
        best = min(best, d);
      }
    }
    if (active && j_end > j_begin) atomicAdd(t + c, (unsigned long long)(int64_t)best);
  }
}

}  // namespace

cudaError_t launch_nbnn_simt(const uint8_t* q, int64_t m, const int32_t* qnorm, const uint8_t* sref,
                             const float* srnorm, const int32_t* slabels, const int64_t* class_off,
                             const ClassGroups& groups, const int64_t* offsets, int64_t n_img, int32_t C,
                             int64_t* totals, cudaStream_t s) {
  (void)slabels;
  if (m == 0 || n_img == 0) return cudaSuccess;
  dim3 grid((unsigned)((m + kThreads - 1) / kThreads), (unsigned)groups.n);
  nbnn_simt_kernel<<<grid, kThreads, 0, s>>>(q, m, qnorm, sref, srnorm, class_off, groups, offsets, n_img, C, totals);
  return cudaGetLastError();
}

}  // namespace lnbnn
