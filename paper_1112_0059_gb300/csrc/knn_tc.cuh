// Host-side interface of the tensor-core (tcgen05) search kernels.
#pragma once

#include <cuda.h>

#include <algorithm>

#include "internal.cuh"

namespace lnbnn {

// References per tile of the tensor-core kernels (the MMA N extent).
constexpr int kTcRefTile = 256;
// Query rows per CTA (the MMA M extent); the query operand is padded to
// whole tiles.  Every kernel runs single CTAs: each loads its own reference
// tiles, and concurrently running CTAs share them through L2.
constexpr int kTcQueryTile = 128;
static_assert(kQueryPad % kTcQueryTile == 0, "query padding must cover whole tiles");
// Lists of the k+1 (or shortlist) nearest per query row: up to 16 entries a
// 16-entry register list (the fewest registers), up to 24 a 24-entry one (a
// narrower insertion network than 32), up to 32 a 32-entry one, up
// to 64 a 64-entry list in shared memory with warp-cooperative inserts (in
// registers for an exact scan of long splits), longer ones a heap in global
// memory.
constexpr int kTcRegListMax = 16;
constexpr int kTcMidRegListMax = 24;
constexpr int kTcCoarseRegListMax = 32;
constexpr int kTcWideRegListMax = 64;
// Epilogue warps per TMEM lane quarter.  Each owns a column slice of every
// tile and keeps its own top-K1 list per query row, so one reference split
// yields this many sorted lists per row (merged afterwards).  Two, except for
// the 64-entry register lists, which need one warp per quarter (all 256
// columns of a tile) to have the registers.
// With two query tiles per CTA (qt = 2) each epilogue warp takes all 128
// columns of its own query tile's block, so a split yields one list per row.
inline int tc_lists_per_split(int K1, int qt = 1) {
  return qt == 2 || (K1 > kTcCoarseRegListMax && K1 <= kTcWideRegListMax) ? 1 : 2;
}

// Longest reference split for which the exact scan keeps 33..64-entry lists
// in shared memory rather than registers (shared-memory lists leave room for
// a two-stage ring only; measured on the 256-class data at k = 50, shared
// memory is faster while a split holds up to 5.76M references, registers at
// 11.52M).
constexpr int64_t kSmemListMaxRefs = int64_t(8) << 20;

// Where a scan keeps its per-row lists of K1 keys.
enum class ListKind { Reg16, Reg24, Reg32, Smem64, Reg64, Heap };
inline ListKind tc_list_kind(int K1, int64_t split_len, bool coarse) {
  if (K1 <= kTcRegListMax) return ListKind::Reg16;
  if (K1 <= kTcMidRegListMax) return ListKind::Reg24;
  if (K1 <= kTcCoarseRegListMax) return ListKind::Reg32;
  if (K1 <= kTcWideRegListMax) return coarse || split_len <= kSmemListMaxRefs ? ListKind::Smem64 : ListKind::Reg64;
  return ListKind::Heap;
}

// TMA descriptors over an index's BF16 reference operands (caller's row order
// and class-sorted order).  Encoded once at index creation; boxes of 256
// reference rows (one query tile per CTA) and, the "_h" maps, of 128 rows
// (two query tiles per CTA).
struct TcTensorMaps {
  CUtensorMap ref, ref_ext;    // BF16 [n_pad,128] (128-byte swizzle) and norm digits [n_pad,16] (32-byte swizzle)
  CUtensorMap sref, sref_ext;  // the same over the class-sorted copy
  CUtensorMap f8, f8_ext;      // E4M3 coarse operand [n_pad,128] and its extension [n_pad,16]
  CUtensorMap ref_h, ref_ext_h, sref_h, sref_ext_h, f8_h, f8_ext_h;
};

// How one scan launch is laid out (never what it computes).
struct TcSched {
  int qt = 1;                  // query tiles per CTA: 1 (steps of 128 x 256 pairs) or 2 (256 x 128)
  int persistent_ctas = 0;     // > 0: a persistent grid of that many CTAs taking work items from *queue
  uint32_t* queue = nullptr;   // the item counter of a persistent launch, zeroed before it
  bool bound_per_tile = true;  // with row_thr: share the row bound every tile, or at item start and end
  // kNN lists with several splits run one after another: per work item a
  // flag (zeroed before the launch) set once its lists are written; the
  // same rows' next split, if it finds the flag set when it starts, begins
  // from those lists (so a row's lists carry its best keys across splits and
  // the merge drops the duplicates).  Null: every item starts empty.
  uint32_t* done = nullptr;
  // > 0: the claimed-chunk form for launches of few query-tile groups:
  // `group` CTAs per group, each keeping the group's query tiles and its own
  // lists for the whole launch and claiming reference chunks of split_len
  // rows in increasing order from the group's counter queue[group index]
  // (T counters zeroed before the launch); the launch writes `group` x lists
  // per CTA lists per query row.  kNN register lists and heaps only; never
  // with `done`.
  int group = 0;
};

// Split-N schedule of one scan launch over T query-tile groups (qt 128-row
// query tiles per CTA) keeping lists of K1 keys: s reference splits make
// T * s work items, run one per SM in waves of sm_count.  Modelled device
// time:
//   ceil(T * s / sm_count) * (a * qt * tiles_per_item(s) + b + e * K1) + c * T * s,
// tiles_per_item(s) = ceil(ceil(n_ref / s) / kTcRefTile): a is the time of one
// step of 128 x 256 query-reference pairs, b the fixed time of a wave (start,
// drain, epilogue store), e the time per list entry of filling an item's lists
// (a list of K1 takes about K1 (1 + ln(n / K1)) inserts, most of them at the
// start of the item), c the merge time per (query-tile group, split).
// lnbnn_autotune fits a, b, c, e on the device; these defaults are in step
// units.
struct SplitModel {
  double a = 1.0, b = 64.0, c = 0.02, e = 0.5;
};

// Largest split count considered for T query-tile groups: at most four waves
// of CTAs (so workspace sizes do not depend on the fitted model), at least
// 4,096 references per split, at most max_splits.
inline int64_t max_splits_for(int64_t T, int64_t n_ref, int sm_count, int64_t max_splits) {
  int64_t hi = (4 * (int64_t)sm_count + T - 1) / T;
  hi = std::min<int64_t>(hi, std::max<int64_t>(1, n_ref / 4096));
  return std::max<int64_t>(1, std::min<int64_t>(hi, max_splits));
}

inline double split_cost(const SplitModel& md, int64_t T, int64_t s, int64_t n_ref, int sm_count, int qt = 1,
                         int K1 = 0) {
  const int64_t tiles = ((n_ref + s - 1) / s + kTcRefTile - 1) / kTcRefTile;
  const int64_t waves = (T * s + sm_count - 1) / sm_count;
  return (double)waves * (md.a * (double)(qt * tiles) + md.b + md.e * (double)K1) + md.c * (double)(T * s);
}

// The split count of least modelled time (the smaller one on ties).
inline int choose_splits_model(const SplitModel& md, int64_t T, int64_t n_ref, int sm_count, int64_t max_splits,
                               int qt = 1, int K1 = 0) {
  const int64_t hi = max_splits_for(T, n_ref, sm_count, max_splits);
  int64_t best = 1;
  double best_cost = split_cost(md, T, 1, n_ref, sm_count, qt, K1);
  for (int64_t s = 2; s <= hi; ++s) {
    const double c = split_cost(md, T, s, n_ref, sm_count, qt, K1);
    if (c < best_cost * (1.0 - 1e-9)) {
      best_cost = c;
      best = s;
    }
  }
  return (int)best;
}

// Sets the kernels' shared-memory size on the current device; call once per
// device before launching (and before any stream capture).
cudaError_t prepare_tc_kernels();

bool make_tc_tensor_maps(const __nv_bfloat16* ref_bf, const __nv_bfloat16* sref_bf, const __nv_bfloat16* ref_ext,
                         const __nv_bfloat16* sref_ext, int64_t n_pad, TcTensorMaps* out);

bool make_tc_tensor_maps_e4m3(const uint8_t* ref_f8, const __nv_bfloat16* ref_f8_ext, int64_t n_pad,
                              TcTensorMaps* out);

// Exact top-K1 search on tensor cores.  qbf: BF16 -2q operand [m_pad, 128];
// qext: its K-extension [m_pad, 16].  Split s scans reference rows
// [s * split_len, min((s+1) * split_len, n_ref)) and writes L =
// tc_lists_per_split(K1, sched.qt) sorted lists per query row i, list w at
// lists[((s * L + w) * stride + i) * K1]; the K1 smallest keys of their union
// are the split's answer.
// row_thr (null, or [m_pad] int32 filled with the bytes 0x7F beforehand) is
// the per-row bound the lists of a row share: each list may leave out columns
// that cannot be among the row's K1 nearest over all lists, so only the union
// of a row's lists (merged) is the answer, not each list by itself.
cudaError_t launch_knn_tc(const TcTensorMaps& maps, bool sorted_copy, const __nv_bfloat16* qbf,
                          const __nv_bfloat16* qext, int64_t m, int64_t m_pad, int64_t n_ref, int splits,
                          int64_t split_len, int K1, uint64_t* lists, int64_t stride, int32_t* row_thr,
                          uint32_t* dev_err, unsigned long long* stats, const uint32_t* gate, const TcSched& sched,
                          cudaStream_t s);
// Coarse pass of the FP8 shortlist search: the same scan over the E4M3
// operands (qf8 [m_pad, 128] bytes of -2 E4M3(q - 64), qext its extension),
// keeping the K1 smallest (coarse + 2^21, row) keys per list in the same
// layout as launch_knn_tc.
cudaError_t launch_coarse_tc(const TcTensorMaps& maps, const uint8_t* qf8, const __nv_bfloat16* qext,
                             int64_t m, int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int K1,
                             uint64_t* lists, int64_t stride, int32_t* row_thr, uint32_t* dev_err,
                             unsigned long long* stats, const uint32_t* gate, const TcSched& sched, cudaStream_t s);
// Original NBNN on the same tensor-core scan over the class-sorted copy:
// mins [m_pad, C] (int32, filled with INT32_MAX-like values beforehand) gets
// atomicMin(mins[i][c], ||q_i - r||^2) over every reference r of class c that
// split's range covers, so after all splits mins[i][c] = NN_c(q_i).
cudaError_t launch_nbnn_tc(const TcTensorMaps& maps, const __nv_bfloat16* qbf, const __nv_bfloat16* qext, int64_t m,
                           int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int32_t* mins, int32_t C,
                           const int64_t* class_off, uint32_t* dev_err, unsigned long long* stats,
                           const uint32_t* gate, const TcSched& sched, cudaStream_t s);
// stats (may be null): the MMA thread of every CTA adds its SM cycles,
// globaltimer nanoseconds and tile count to stats[0..2] and 1 to stats[3].
// gate (may be null): each CTA's producer waits, at most 1 s, until *gate is
// nonzero before it loads anything; on expiry the launch reports a timeout
// like any other wait (lnbnn_set_start_gate).

}  // namespace lnbnn
