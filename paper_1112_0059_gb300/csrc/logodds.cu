// NBNN as a sum of log-odds increments (Section 3.1): each query descriptor d
// changes the log-odds of every class C by
//
//   inc(d, C) = log [P(C|d) P(Cbar)] / [P(Cbar|d) P(C)]            Eq. (eqn:log-odds)
//
// with equal priors P(C) = 1/|classes| and the posterior of the NBNN Gaussian
// kernel on each class's nearest neighbour, P(C|d) ~ exp(-beta D_C),
// D_C = ||d - NN_C(d)||^2, beta = 1/(2 sigma^2).  The image goes to the class
// with the largest sum (Eq. (eqn:log-increments)); the "positive increments
// only" variant (Table 1) adds only increments > 0.
//
// Written without the normalisation, which cancels:
//   inc(d, C) = -beta D_C - log sum_{C' != C} exp(-beta D_C') + log(|classes| - 1).
// Shifting by the row minimum Dmin keeps every exponential <= 1 and the sums
// >= 1, so nothing underflows into a log(0):
//   * C not the unique nearest class: with x = beta (D_C - Dmin) and
//     S = sum_C' exp(-beta (D_C' - Dmin)) >= 1 + exp(-x),
//       inc = -x - log(S - exp(-x)) + log(|classes| - 1);
//   * C the unique nearest class, D2 the second smallest distance and
//     S2 = sum_{C' != C} exp(-beta (D_C' - D2)) >= 1,
//       inc = beta (D2 - Dmin) - log S2 + log(|classes| - 1).
// All of it is float64.  The input is the [m, C] table of NN_C distances that
// the tensor-core scan of the class-sorted references fills for Alg. 1.
#include <math.h>

#include "internal.cuh"

namespace lnbnn {
namespace {

struct RowStat {
  double s;       // sum over classes of exp(-beta (D_C - Dmin)), in [1, |classes|]
  double log_s2;  // log of the sum over the other classes of exp(-beta (D_C - D2)) (unique minimum only)
  int32_t dmin;   // smallest class distance of the row
  int32_t d2;     // smallest distance of the other classes (unique minimum only)
  int32_t cstar;  // the unique nearest class, or -1 when two or more classes tie at Dmin
  int32_t pad;
};
static_assert(sizeof(RowStat) == kLogoddsRowStatBytes, "row statistics layout");

__device__ __forceinline__ double warp_sum(double v) {
  // xor butterfly: both partners add the same two values, so every lane ends
  // with the same bits and the order is fixed
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// One warp per descriptor row: its minimum, the lowest class attaining it and
// how many do, the sum S, and for a unique minimum D2 and log S2.
__global__ void logodds_rowstat_kernel(const int32_t* __restrict__ mins, int64_t m, int32_t C, double beta,
                                       RowStat* __restrict__ st) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const int32_t* d = mins + row * C;
  int32_t best = INT32_MAX, bc = INT32_MAX, ties = 0;
  for (int32_t c = lane; c < C; c += 32) {
    const int32_t v = d[c];
    if (v < best) {
      best = v;
      bc = c;
      ties = 1;
    } else if (v == best) {
      ++ties;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int32_t ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
    const int32_t ot = __shfl_xor_sync(0xffffffffu, ties, off);
    if (ob < best) {
      best = ob;
      bc = oc;
      ties = ot;
    } else if (ob == best) {
      bc = min(bc, oc);
      ties += ot;
    }
  }
  double s = 0.0;
  int32_t sec = INT32_MAX;
  for (int32_t c = lane; c < C; c += 32) {
    const int32_t v = d[c];
    s += exp(-beta * (double)(v - best));
    if (c != bc) sec = min(sec, v);
  }
  s = warp_sum(s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sec = min(sec, __shfl_xor_sync(0xffffffffu, sec, off));
  double log_s2 = 0.0;
  if (ties == 1) {
    double s2 = 0.0;
    for (int32_t c = lane; c < C; c += 32)
      if (c != bc) s2 += exp(-beta * (double)(d[c] - sec));
    log_s2 = log(warp_sum(s2));
  }
  if (lane == 0) {
    RowStat r;
    r.s = s;
    r.log_s2 = log_s2;
    r.dmin = best;
    r.d2 = ties == 1 ? sec : best;
    r.cstar = ties == 1 ? bc : -1;
    r.pad = 0;
    st[row] = r;
  }
}

// Block (image, 128 classes): thread c adds the increments of class c over the
// image's rows in row order (so the sums are deterministic); the block's count
// of added increments goes to counts[img] (integer atomics: order-free).
__global__ void logodds_sum_kernel(const int32_t* __restrict__ mins, const RowStat* __restrict__ st, int64_t m,
                                   int32_t C, double beta, double log_c1, int positive_only,
                                   const int64_t* __restrict__ offsets, double* __restrict__ totals,
                                   unsigned long long* __restrict__ counts) {
  const int64_t img = blockIdx.x;
  const int32_t c = blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t r0 = max(offsets[img], (int64_t)0), r1 = min(offsets[img + 1], m);
  double acc = 0.0;
  unsigned long long n = 0;
  if (c < C) {
    for (int64_t r = r0; r < r1; ++r) {
      const RowStat t = st[r];
      double inc;
      if (c == t.cstar) {
        inc = beta * (double)(t.d2 - t.dmin) - t.log_s2 + log_c1;
      } else {
        const double x = beta * (double)(mins[r * C + c] - t.dmin);
        inc = -x - log(t.s - exp(-x)) + log_c1;
      }
      if (!positive_only || inc > 0.0) {
        acc += inc;
        ++n;
      }
    }
    totals[img * C + c] = acc;
  }
  if (counts) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(0xffffffffu, n, off);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(counts + img, n);
  }
}

// One warp per image: argmax over classes, lowest class on ties.
__global__ void argmax_f64_kernel(const double* __restrict__ totals, int64_t n_img, int32_t C,
                                  int32_t* __restrict__ classes) {
  const int64_t img = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (img >= n_img) return;
  const double* t = totals + img * C;
  double best = -INFINITY;
  int32_t bc = INT32_MAX;
  for (int32_t c = lane; c < C; c += 32) {
    const double v = t[c];
    if (v > best || bc == INT32_MAX) {  // c increases: the first maximum seen is the lowest
      best = v;
      bc = c;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, off);
    const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (oc != INT32_MAX && (bc == INT32_MAX || ov > best || (ov == best && oc < bc))) {
      best = ov;
      bc = oc;
    }
  }
  if (lane == 0) classes[img] = bc;
}

}  // namespace

cudaError_t launch_logodds_rowstat(const int32_t* mins, int64_t m, int32_t C, double beta, void* rowstat,
                                   cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  logodds_rowstat_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(mins, m, C, beta,
                                                                          static_cast<RowStat*>(rowstat));
  return cudaGetLastError();
}

cudaError_t launch_logodds_sum(const int32_t* mins, const void* rowstat, int64_t m, int32_t C, double beta,
                               bool positive_only, const int64_t* offsets, int64_t n_img, double* totals,
                               int64_t* counts, cudaStream_t s) {
  if (n_img == 0) return cudaSuccess;
  dim3 grid((unsigned)n_img, (unsigned)((C + 127) / 128));
  logodds_sum_kernel<<<grid, 128, 0, s>>>(mins, static_cast<const RowStat*>(rowstat), m, C, beta,
                                          log((double)(C - 1)), positive_only ? 1 : 0, offsets, totals,
                                          reinterpret_cast<unsigned long long*>(counts));
  return cudaGetLastError();
}

cudaError_t launch_argmax_f64(const double* totals, int64_t n_img, int32_t C, int32_t* classes, cudaStream_t s) {
  if (n_img == 0) return cudaSuccess;
  argmax_f64_kernel<<<(unsigned)((n_img * 32 + 255) / 256), 256, 0, s>>>(totals, n_img, C, classes);
  return cudaGetLastError();
}

}  // namespace lnbnn
