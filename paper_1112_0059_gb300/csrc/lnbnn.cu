// The C ABI of include/lnbnn.h: index ownership, argument checks, workspace
// and the launch sequence of each call.  All arithmetic runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"
#include "knn_tc.cuh"

using namespace lnbnn;

struct lnbnn_index {
  int device = 0;
  int sm_count = 0;
  int64_t n_ref = 0;
  int64_t n_pad = 0;
  int32_t n_classes = 0;
  int32_t row_bytes = kDim;  // bytes per descriptor row: 128, or 130 with a location
  int32_t loc_w = 0;         // weight of the location term (130-byte rows)
  // merged reference set, caller's row order
  uint8_t* ref_u8 = nullptr;         // [n_ref, row_bytes] the descriptors as given
  __nv_bfloat16* ref_bf = nullptr;   // [n_pad, 128] exact BF16 copy, zero padding rows
  __nv_bfloat16* ref_ext = nullptr;  // [n_pad, 16] squared-norm digits (K-extension)
  float* rnorm = nullptr;            // [n_pad] squared norms, kPadNorm on padding rows
  int32_t* labels = nullptr;        // [n_ref]
  // class-sorted view (aliases the above when the labels are already grouped)
  bool sorted = true;
  __nv_bfloat16* sref_bf = nullptr;
  __nv_bfloat16* sref_ext = nullptr;
  float* srnorm = nullptr;
  int32_t* slabels = nullptr;
  std::vector<int64_t> class_off_h;  // [C+1]
  int64_t* class_off_d = nullptr;
  bool has_empty_class = false;
  uint32_t* dev_err = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* stage = nullptr;  // device staging for the _host calls
  size_t stage_bytes = 0;
  // E4M3 operand of the FP8 shortlist search (lnbnn_index_prepare_fp8)
  uint8_t* ref_f8 = nullptr;             // [n_pad, 128]
  __nv_bfloat16* ref_f8_ext = nullptr;   // [n_pad, 16]
  bool fp8 = false;
  TcTensorMaps tc;  // tensor maps over ref_bf / sref_bf (and ref_f8) for the tensor-core kernels
  SplitModel split_model;  // split-N schedule (defaults, or fitted by lnbnn_autotune)
  lnbnn_schedule sched{0, 0, -1, -1};  // lnbnn_set_schedule: fixed choices (0 / -1: automatic)
  // large-batch forms per scan kind (exact, coarse, NBNN), chosen by lnbnn_autotune
  int auto_qt[3] = {1, 2, 1};
  int auto_persistent[3] = {0, 0, 0};
  const uint32_t* gate = nullptr;  // lnbnn_set_start_gate: search kernels wait for *gate != 0
  // optional device-time profile (lnbnn_profile_enable)
  struct CallEvents {
    cudaEvent_t e[4];
  };
  bool prof_on = false;
  lnbnn_profile prof{};
  unsigned long long* prof_stats = nullptr;  // [4] device counters of the search kernel
  std::vector<CallEvents> prof_pending, prof_free;
};

struct lnbnn_workspace {
  const lnbnn_index* index = nullptr;
  void* base = nullptr;
  size_t bytes = 0;
};

namespace {

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return status_of(e_);       \
  } while (0)

lnbnn_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return LNBNN_OK;
  if (getenv("LNBNN_DEBUG")) fprintf(stderr, "lnbnn: CUDA error: %s\n", cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return LNBNN_ERR_OOM;
  (void)cudaGetLastError();
  return LNBNN_ERR_CUDA;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Allocations the test hook lnbnn_debug_fail_allocations still has to fail.
std::atomic<int> g_fail_allocs{0};

// Every device allocation of the library goes through here.
cudaError_t lib_malloc(void** p, size_t bytes) {
  *p = nullptr;
  for (int n = g_fail_allocs.load(); n > 0;)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  return lib_malloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void free_index(lnbnn_index* ix) {
  if (!ix) return;
  for (auto* v : {&ix->prof_pending, &ix->prof_free})
    for (auto& ce : *v)
      for (cudaEvent_t e : ce.e) cudaEventDestroy(e);
  if (!ix->sorted) {
    cudaFree(ix->sref_bf);
    cudaFree(ix->sref_ext);
    cudaFree(ix->srnorm);
    cudaFree(ix->slabels);
  }
  cudaFree(ix->ref_f8);
  cudaFree(ix->ref_f8_ext);
  cudaFree(ix->ref_u8);
  cudaFree(ix->ref_bf);
  cudaFree(ix->ref_ext);
  cudaFree(ix->rnorm);
  cudaFree(ix->labels);
  cudaFree(ix->class_off_d);
  cudaFree(ix->dev_err);
  cudaFree(ix->prof_stats);
  cudaFree(ix->ws);
  cudaFree(ix->stage);
  delete ix;
}

// An NVTX range for the duration of a scope: calls and their phases show up
// by name on a profiler's timeline (nothing is recorded without a tool).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Carves aligned sub-buffers out of one allocation.
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

// Events of one call: e[0] start, e[1] before the search kernel, e[2] after
// it, e[3] end.  Inactive unless profiling is enabled on the index.
struct CallProfile {
  lnbnn_index* ix;
  cudaStream_t s;
  lnbnn_index::CallEvents ev{};
  bool on;
  int marked = 0;
  CallProfile(lnbnn_index* i, cudaStream_t st) : ix(i), s(st), on(i->prof_on) {
    if (!on) return;
    if (!ix->prof_free.empty()) {
      ev = ix->prof_free.back();
      ix->prof_free.pop_back();
    } else {
      for (auto& e : ev.e)
        if (cudaEventCreate(&e) != cudaSuccess) {
          on = false;
          return;
        }
    }
    mark(0);
  }
  void mark(int i) {
    if (on && cudaEventRecord(ev.e[i], s) == cudaSuccess) marked |= 1 << i;
  }
  void launched(int n, bool search = false) {
    if (!on) return;
    ix->prof.kernel_launches += n;
    if (search) ix->prof.search_launches += n;
  }
  ~CallProfile() {
    if (!on) return;
    mark(3);
    if (marked == 15) {
      ix->prof_pending.push_back(ev);
      ix->prof.calls += 1;
    } else {
      ix->prof_free.push_back(ev);
    }
  }
};

cudaError_t ensure(void** buf, size_t* have, size_t need) {
  if (*have >= need) return cudaSuccess;
  if (*buf) {
    cudaError_t e = cudaFree(*buf);  // synchronises the device
    *buf = nullptr;
    *have = 0;
    if (e != cudaSuccess) return e;
  }
  need = (need + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
  cudaError_t e = lib_malloc(buf, need);
  if (e == cudaSuccess) *have = need;
  return e;
}

bool k_ok(const lnbnn_index* ix, int32_t k, int extra) {
  return k >= 1 && k <= LNBNN_MAX_K && (int64_t)k + extra <= ix->n_ref;
}

// Most reference splits of one launch: two CTAs per SM for a single query
// tile, within what the list merge takes (two lists per split).
int64_t max_splits(const lnbnn_index* ix) {
  return std::min<int64_t>(2 * (int64_t)ix->sm_count, 32 * kMaxListsPerLane / 2);
}

// What a scan computes: kNN lists over the exact BF16 operand, kNN lists over
// the E4M3 coarse operand, or NBNN's class minima.
enum class ScanKind { Exact, Coarse, Nbnn };

// Reference operand bytes a scan streams per reference row.
int64_t op_row_bytes(ScanKind k) { return k == ScanKind::Coarse ? kDim + 2 * kExt : 2 * (kDim + kExt); }

// Reference bytes one split may stream for the CTAs running at the same time
// to find every tile in L2 (129 MB), with room for the next split and the
// other traffic.
constexpr int64_t kL2SplitBytes = int64_t(48) << 20;

// Schedule rules (measured on the 256-class data; see the schedule
// measurements in the design notes).  A launch with at least a full wave of
// query-tile groups streams its references in splits of at most
// kL2SplitBytes for the coarse pass, which otherwise re-reads most of its
// operand from DRAM once per wave.
bool l2_splits_for(ScanKind k) { return k == ScanKind::Coarse; }
// The large-batch form of a scan kind (query tiles per CTA, persistent grid)
// for launches of at least a full wave of query tiles, unless lnbnn_autotune
// measured another form faster on this index.  Defaults, measured on the
// 256-class data (750k query rows): one query tile per CTA for the exact and
// NBNN scans (exact 1,229 ms a classify call against 1,263 with two, whose
// steps take fewer cycles, 1,305 against 1,341, at a lower SM clock); two
// for the FP8 coarse pass (shortlist 24, lists carried across the 37
// L2-sized splits: 860 against 899 ms); one CTA per work item (persistent
// grids within 0.2%).
// The exact scan with lists longer than 16 entries takes two query tiles
// per CTA whatever the tuned k+1 = 11 form is: one list per row and split
// instead of two column halves halves the list work (256-class data, 750k
// query rows: k = 20 1,277 against 1,303 ms, k = 100 with heaps 2,225
// against 3,571 ms).
int auto_query_tiles(const lnbnn_index* ix, ScanKind k, int64_t T1, int K1) {
  if (T1 < ix->sm_count) return 1;
  if (k == ScanKind::Exact && K1 > kTcRegListMax) return 2;
  return ix->auto_qt[(int)k];
}
bool auto_persistent(const lnbnn_index* ix, ScanKind k, int64_t T1) {
  return T1 >= ix->sm_count && ix->auto_persistent[(int)k] == 1;
}

// Splits for the exact scan of a launch of at least a full wave whose lists
// are dearer than the 16-entry ones: with the splits run one after another
// and their lists carried across, the later splits insert little, and the
// shorter reference ranges stay in L2.  Measured on the 256-class data (300k
// query rows): k = 20 (24-entry lists) 1 / 4 splits 556 / 527 ms; k = 100
// (heaps) 1 / 2 / 4 / 8 splits 1,493 / 1,464 / 1,437 / 1,413 ms.  The
// 64-entry lists keep one split (at shorter splits they move to shared
// memory, 2,660 against 2,367 cycles per step at k = 50).
int long_list_splits(const lnbnn_index* ix, int K1) {
  int want = 1;
  if (K1 > kTcRegListMax && K1 <= kTcCoarseRegListMax) want = 4;
  if (K1 > kTcWideRegListMax) want = 8;
  return (int)std::min<int64_t>(want, std::max<int64_t>(1, ix->n_ref / (int64_t(1) << 20)));
}

int64_t l2_splits(const lnbnn_index* ix, ScanKind k) {
  const int64_t bytes = ix->n_ref * op_row_bytes(k);
  return std::min<int64_t>(max_splits(ix), std::max<int64_t>(1, (bytes + kL2SplitBytes - 1) / kL2SplitBytes));
}

// Largest split count a launch over T query-tile groups may use (workspaces
// are sized for it).
int64_t splits_bound(const lnbnn_index* ix, int64_t T, ScanKind k) {
  int64_t hi = max_splits_for(T, ix->n_ref, ix->sm_count, max_splits(ix));
  if (T >= ix->sm_count) hi = std::max<int64_t>(hi, std::max<int64_t>(l2_splits(ix, k), 8));
  return hi;
}

struct KnnPlan {
  int64_t m_pad;
  int splits;
  int lists;  // sorted lists per query row the search writes (merged when > 1)
  int64_t split_len;
  int K1;
  int qt;               // 128-row query tiles per CTA
  bool persistent;      // a persistent grid taking items from a queue
  bool bound_per_tile;  // with several splits: the row bound shared every tile (else at item start/end)
  bool seeded;          // each split's lists may start from the same rows' previous split's lists
  int group;            // > 0: the claimed-chunk form (`splits` = CTAs per query-tile group, split_len = chunk)
  int64_t items;        // work items of the launch (query-tile groups x splits)
  size_t off_qnorm, off_qbf, off_qext, off_lists, off_merged, off_rowthr, off_queue, off_done, bytes;
  TcSched sched(char* ws, int sm_count) const {
    TcSched t;
    t.qt = qt;
    t.persistent_ctas = persistent ? sm_count : 0;
    t.queue = reinterpret_cast<uint32_t*>(ws + off_queue);
    t.bound_per_tile = bound_per_tile;
    t.done = seeded ? reinterpret_cast<uint32_t*>(ws + off_done) : nullptr;
    t.group = group;
    return t;
  }
  // Clears what a launch needs zeroed: the work counter of a persistent
  // launch, the per-item flags of a seeded one.
  cudaError_t clear(char* ws, cudaStream_t s) const {
    cudaError_t e = cudaSuccess;
    if (persistent) e = cudaMemsetAsync(ws + off_queue, 0, sizeof(uint32_t) * (size_t)(group > 0 ? items / splits : 1), s);
    if (e == cudaSuccess && seeded) e = cudaMemsetAsync(ws + off_done, 0, sizeof(uint32_t) * (size_t)items, s);
    return e;
  }
  // The merge's view of a seeded launch: rows whose last split holds every
  // split's keys merge only that split's lists.
  MergeChain chain(char* ws) const {
    MergeChain c;
    if (!seeded) return c;
    c.done = reinterpret_cast<const uint32_t*>(ws + off_done);
    c.T = items / splits;
    c.rows_per_item = (int64_t)kTcQueryTile * qt;
    c.lists_per_split = lists / splits;
    return c;
  }
};

// The launch schedule of a scan over m queries keeping K1 keys per row:
// tile shape, split count, bound mode and grid form, each from the index's
// fixed choices (lnbnn_set_schedule) or else the rules and split model above.
// splits > 0 fixes the split count (an upper bound after rounding the split
// length to whole tiles).
KnnPlan plan_knn(const lnbnn_index* ix, int64_t m, int K1, ScanKind kind, int splits = 0) {
  KnnPlan p{};
  const lnbnn_schedule& o = ix->sched;
  const int P = ix->sm_count;
  p.m_pad = round_up(m, kQueryPad);
  p.K1 = K1;
  const int64_t T1 = p.m_pad / kTcQueryTile;
  const bool qt2_ok = kind == ScanKind::Nbnn || K1 <= kTcCoarseRegListMax || K1 > kTcWideRegListMax;
  p.qt = qt2_ok && (o.query_tiles == 2 || (o.query_tiles == 0 && auto_query_tiles(ix, kind, T1, K1) == 2)) ? 2 : 1;
  const int64_t T = (T1 + p.qt - 1) / p.qt;
  if (splits <= 0) splits = o.splits;
  // The claimed-chunk form for launches of fewer query-tile groups than SMs
  // (automatic split count; register lists or heaps): on a class-sorted
  // index the few reference ranges that hold a query's own class carry most
  // of the list inserts, and with fixed splits the CTAs that draw them set
  // the launch's time.  Instead each of P / T CTAs per group keeps the
  // group's lists for the whole launch and claims short reference chunks, in
  // increasing order, from the group's counter: the near-class chunks are
  // shared by whichever CTAs are free.
  // The coarse pass, whose shortlist inserts are dear, takes it while there
  // are at least 8 CTAs per query tile (256-class data, shortlist 24, one
  // image of 100 / 256 / 512 / 768 / 1,280 / 2,000 descriptors: 0.42-0.54 /
  // 0.71-0.76 / 1.07-1.13 / 1.38-1.50 / 2.11-2.32 / 2.93-3.44 ms against
  // 0.55-0.66 / 0.84-0.89 / 1.14-1.27 / 1.69-1.74 / 2.41-2.47 / 3.28-3.53
  // with splits; 4,000: slower, 4 CTAs per tile leave SMs idle); the exact
  // scan, whose inserts are few, for a lone query tile only (0.53 against
  // 0.55 ms at 100 descriptors; 2 and 3 tiles were 7-30% slower, 4 to 10
  // tiles 1-12% faster).
  const bool claim_kind = kind != ScanKind::Nbnn && (K1 <= kTcCoarseRegListMax || K1 > kTcWideRegListMax) &&
                          (kind == ScanKind::Coarse ? T * 8 <= P : T == 1);
  const int64_t ref_tiles = (ix->n_ref + kTcRefTile - 1) / kTcRefTile;
  p.group = splits <= 0 && T < P && p.qt == 1 && claim_kind && o.persistent != 0 && o.bound_per_tile != 0
                // chunks of >= 4 tiles each, and no more lists than the split
                // form may write (workspaces are sized for that)
                ? (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(P / T, ref_tiles / 4),
                                                              max_splits_for(T, ix->n_ref, P, max_splits(ix))))
                : 0;
  if (p.group > 0) {
    const int64_t tiles = ref_tiles;
    const int64_t chunk_tiles = std::max<int64_t>(4, (tiles + 8 * (int64_t)p.group - 1) / (8 * (int64_t)p.group));
    p.split_len = chunk_tiles * kTcRefTile;  // about eight chunks per CTA
    p.splits = p.group;
    p.persistent = true;
    p.bound_per_tile = true;
  } else {
    if (splits <= 0) {
      splits = choose_splits_model(ix->split_model, T, ix->n_ref, P, max_splits(ix), p.qt, K1);
      if (T >= P && l2_splits_for(kind)) splits = (int)std::max<int64_t>(splits, l2_splits(ix, kind));
      if (T >= P && kind == ScanKind::Exact) splits = std::max(splits, long_list_splits(ix, K1));
    }
    p.split_len = round_up((ix->n_ref + splits - 1) / splits, kTcRefTile);
    p.splits = (int)((ix->n_ref + p.split_len - 1) / p.split_len);
    p.persistent = o.persistent == 1 || (o.persistent == -1 && auto_persistent(ix, kind, T1));
    p.bound_per_tile = o.bound_per_tile >= 0 ? o.bound_per_tile == 1 : T < P;
  }
  p.items = T * p.splits;
  p.seeded = kind != ScanKind::Nbnn && p.splits > 1 && !p.bound_per_tile;
  Carve c;
  p.off_qnorm = c.take<int32_t>(p.m_pad);
  p.off_qbf = c.take<__nv_bfloat16>(p.m_pad * kDim);
  p.off_qext = c.take<__nv_bfloat16>(p.m_pad * kExt);
  p.lists = p.splits * tc_lists_per_split(K1, p.qt);
  p.off_lists = c.take<uint64_t>(kind == ScanKind::Nbnn ? 0 : (size_t)p.lists * p.m_pad * K1);
  p.off_merged = c.take<uint64_t>(kind == ScanKind::Nbnn ? 0 : (size_t)p.m_pad * K1);  // apart from the lists (rerank)
  p.off_rowthr = c.take<int32_t>(p.m_pad);                // the bound a row's lists share
  p.off_queue = c.take<uint32_t>((size_t)T);             // the work counter(s) of a persistent launch
  p.off_done = c.take<uint32_t>((size_t)p.items);        // per-item "lists written" flags
  p.bytes = c.off;
  return p;
}

// Device scratch of one call: the caller's workspace (fixed size, nothing is
// allocated) or else the index's grow-only workspace.
struct Scratch {
  lnbnn_index* ix;
  lnbnn_workspace* w;
  lnbnn_status get(size_t need, char** out) {
    if (w) {
      if (need > w->bytes) return LNBNN_ERR_SCRATCH_LIMIT;
      *out = static_cast<char*>(w->base);
      return LNBNN_OK;
    }
    CK(ensure(&ix->ws, &ix->ws_bytes, need));
    *out = static_cast<char*>(ix->ws);
    return LNBNN_OK;
  }
};

struct NbnnPlan {
  KnnPlan k;
  size_t off_qnorm, off_qbf, off_qext, off_mins, off_rowstat, off_queue, bytes;
};

NbnnPlan plan_nbnn(const lnbnn_index* ix, int64_t m, int splits = 0) {
  NbnnPlan p{};
  p.k = plan_knn(ix, m, 1, ScanKind::Nbnn, splits);
  Carve c;
  p.off_qnorm = c.take<int32_t>(p.k.m_pad);
  p.off_qbf = c.take<__nv_bfloat16>(p.k.m_pad * kDim);
  p.off_qext = c.take<__nv_bfloat16>(p.k.m_pad * kExt);
  p.off_mins = c.take<int32_t>((size_t)p.k.m_pad * ix->n_classes);
  p.off_rowstat = c.take<char>((size_t)p.k.m_pad * kLogoddsRowStatBytes);  // log-odds rule only
  p.off_queue = c.take<uint32_t>(1);
  p.k.off_queue = p.off_queue;
  p.k.seeded = false;
  p.bytes = c.off;
  return p;
}

// Largest scratch any call with at most max_q queries and lists of K1 needs.
// The lists grow with the split count, so the bound takes the largest count
// the schedule may choose (for either tile shape), whatever model
// lnbnn_autotune fits later.
size_t scratch_bound(const lnbnn_index* ix, int64_t max_q, int K1) {
  size_t b = 0;
  for (int64_t m = kQueryPad; m < max_q + kQueryPad; m += kQueryPad) {
    const int64_t mm = std::min(m, max_q);
    const int64_t T1 = round_up(mm, kQueryPad) / kTcQueryTile;
    for (ScanKind k : {ScanKind::Exact, ScanKind::Coarse, ScanKind::Nbnn}) {
      const int64_t hi = std::max(splits_bound(ix, T1, k), splits_bound(ix, (T1 + 1) / 2, k));
      if (k == ScanKind::Nbnn)
        b = std::max(b, plan_nbnn(ix, mm, (int)hi).bytes);
      else
        b = std::max(b, plan_knn(ix, mm, K1, k, (int)hi).bytes);
    }
  }
  return b;
}

// Runs the exact search; *lists receives m sorted lists of K1 keys.
lnbnn_status run_knn(lnbnn_index* ix, Scratch& scratch, const uint8_t* q, int64_t m, int K1, cudaStream_t s,
                     const uint64_t** lists, CallProfile& prof, int force_splits = 0) {
  KnnPlan p = plan_knn(ix, m, K1, ScanKind::Exact, force_splits);
  char* ws = nullptr;
  lnbnn_status st = scratch.get(p.bytes, &ws);
  if (st != LNBNN_OK) return st;
  int32_t* qnorm = reinterpret_cast<int32_t*>(ws + p.off_qnorm);
  __nv_bfloat16* qbf = reinterpret_cast<__nv_bfloat16*>(ws + p.off_qbf);
  __nv_bfloat16* qext = reinterpret_cast<__nv_bfloat16*>(ws + p.off_qext);
  uint64_t* part = reinterpret_cast<uint64_t*>(ws + p.off_lists);
  uint64_t* merged = reinterpret_cast<uint64_t*>(ws + p.off_merged);
  int32_t* row_thr = reinterpret_cast<int32_t*>(ws + p.off_rowthr);
  Range range("lnbnn: exact k+1 search");
  CK(launch_prep_query(q, m, p.m_pad, ix->row_bytes, ix->loc_w, qnorm, qbf, qext, s));
  CK(cudaMemsetAsync(row_thr, 0x7F, sizeof(int32_t) * (size_t)p.m_pad, s));
  const TcSched sched = p.sched(ws, ix->sm_count);
  CK(p.clear(ws, s));
  prof.launched(1);
  prof.mark(1);
  CK(launch_knn_tc(ix->tc, /*sorted_copy=*/false, qbf, qext, m, p.m_pad, ix->n_ref, p.splits, p.split_len, K1, part,
                   p.m_pad, p.splits > 1 ? row_thr : nullptr, ix->dev_err, ix->prof_on ? ix->prof_stats : nullptr,
                   ix->gate, sched, s));
  prof.launched(1, true);
  prof.mark(2);
  if (p.lists > 1) {
    CK(launch_merge_lists(part, p.lists, m, p.m_pad, K1, merged, s, p.chain(ws)));
    prof.launched(1);
  }
  *lists = p.lists > 1 ? merged : part;
  return LNBNN_OK;
}

// The FP8 shortlist search: coarse pass keeping the M1 smallest coarse keys,
// merge, exact rerank; *lists receives m sorted lists of K1 exact keys.
lnbnn_status run_knn_fp8(lnbnn_index* ix, Scratch& scratch, const uint8_t* q, int64_t m, int K1, int M1,
                         cudaStream_t s, const uint64_t** lists, CallProfile& prof) {
  KnnPlan p = plan_knn(ix, m, M1, ScanKind::Coarse);
  char* ws = nullptr;
  lnbnn_status st = scratch.get(p.bytes, &ws);
  if (st != LNBNN_OK) return st;
  // the BF16 query operand's space holds the E4M3 bytes (half its size)
  uint8_t* qf8 = reinterpret_cast<uint8_t*>(ws + p.off_qbf);
  __nv_bfloat16* qext = reinterpret_cast<__nv_bfloat16*>(ws + p.off_qext);
  uint64_t* part = reinterpret_cast<uint64_t*>(ws + p.off_lists);
  uint64_t* merged = reinterpret_cast<uint64_t*>(ws + p.off_merged);
  int32_t* row_thr = reinterpret_cast<int32_t*>(ws + p.off_rowthr);
  Range range("lnbnn: FP8 shortlist search");
  CK(launch_prep_query_e4m3(q, m, p.m_pad, qf8, qext, s));
  CK(cudaMemsetAsync(row_thr, 0x7F, sizeof(int32_t) * (size_t)p.m_pad, s));
  const TcSched sched = p.sched(ws, ix->sm_count);
  CK(p.clear(ws, s));
  prof.launched(1);
  prof.mark(1);
  CK(launch_coarse_tc(ix->tc, qf8, qext, m, p.m_pad, ix->n_ref, p.splits, p.split_len, M1, part, p.m_pad,
                      p.splits > 1 ? row_thr : nullptr, ix->dev_err, ix->prof_on ? ix->prof_stats : nullptr,
                      ix->gate, sched, s));
  prof.launched(1, true);
  prof.mark(2);
  // the shortlist is the merged lists (or the one list); the reranked lists
  // go to the other buffer
  if (p.lists > 1) {
    CK(launch_merge_lists(part, p.lists, m, p.m_pad, M1, merged, s, p.chain(ws)));
    CK(launch_rerank(merged, m, M1, q, ix->ref_u8, ix->n_ref, K1, part, s));
    prof.launched(2);
    *lists = part;
  } else {
    CK(launch_rerank(part, m, M1, q, ix->ref_u8, ix->n_ref, K1, merged, s));
    prof.launched(1);
    *lists = merged;
  }
  return LNBNN_OK;
}

// Shortlist length of an FP8 call needing K1 neighbours: K1 <= shortlist <=
// LNBNN_MAX_K + 1; more than n_ref means all references.
bool shortlist_ok(const lnbnn_index* ix, int32_t shortlist, int K1, int* M1) {
  if (shortlist < K1 || shortlist > LNBNN_MAX_K + 1) return false;
  *M1 = (int)std::min<int64_t>(shortlist, ix->n_ref);
  return true;
}

bool device_ok(int* sm_count, int* dev) {
  if (cudaGetDevice(dev) != cudaSuccess) return false;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, *dev) != cudaSuccess) return false;
  *sm_count = prop.multiProcessorCount;
  return prop.major == 10 && prop.minor == 3;
}

}  // namespace

extern "C" {

const char* lnbnn_status_string(lnbnn_status st) {
  switch (st) {
    case LNBNN_OK: return "ok";
    case LNBNN_ERR_INVALID_ARG: return "invalid argument";
    case LNBNN_ERR_LABEL_RANGE: return "label outside [0, n_classes)";
    case LNBNN_ERR_EMPTY_CLASS: return "a class has no reference descriptor";
    case LNBNN_ERR_K_RANGE: return "k out of range (need 1 <= k <= LNBNN_MAX_K and k + 1 <= n_ref)";
    case LNBNN_ERR_OOM: return "device out of memory";
    case LNBNN_ERR_CUDA: return "CUDA error";
    case LNBNN_ERR_TIMEOUT: return "device wait timed out";
    case LNBNN_ERR_UNSUPPORTED: return "unsupported device (needs compute capability 10.3)";
    case LNBNN_ERR_OFFSETS: return "invalid image offsets";
    case LNBNN_ERR_SCRATCH_LIMIT: return "problem larger than the fixed scratch (workspace or knn_search_noalloc)";
    case LNBNN_ERR_NO_FP8: return "the index has no FP8 operand (call lnbnn_index_prepare_fp8 first)";
    case LNBNN_ERR_IO: return "file could not be written or read, or is not an intact index file";
  }
  return "unknown status";
}

static lnbnn_status create_index(const uint8_t* ref, const int32_t* labels, int64_t n_ref, int32_t n_classes,
                                 int32_t row_bytes, int32_t loc_w, void* stream, lnbnn_index** out) {
  Range range("lnbnn: lnbnn_index_create");
  if (!out) return LNBNN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ref || !labels || n_ref < 1 || n_classes < 1 || n_ref > (int64_t)INT32_MAX - kRefPad ||
      !row_layout_ok(row_bytes, loc_w))
    return LNBNN_ERR_INVALID_ARG;
  int sm = 0, dev = 0;
  if (!device_ok(&sm, &dev)) return LNBNN_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lnbnn_index* ix = new (std::nothrow) lnbnn_index();
  if (!ix) return LNBNN_ERR_OOM;
  ix->device = dev;
  ix->sm_count = sm;
  ix->n_ref = n_ref;
  ix->n_pad = round_up(n_ref, kRefPad);
  ix->n_classes = n_classes;
  ix->row_bytes = row_bytes;
  ix->loc_w = loc_w;
  lnbnn_status st = LNBNN_OK;
  unsigned long long* counts = nullptr;
  uint32_t* bad = nullptr;
  int64_t* perm_d = nullptr;
  auto fail = [&](lnbnn_status e) {
    cudaFree(counts);
    cudaFree(bad);
    cudaFree(perm_d);
    free_index(ix);
    return e;
  };
#define CKF(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return fail(status_of(e_)); \
  } while (0)
  CKF(dmalloc(&ix->ref_u8, (size_t)n_ref * row_bytes));
  CKF(dmalloc(&ix->ref_bf, (size_t)ix->n_pad * kDim));
  CKF(dmalloc(&ix->ref_ext, (size_t)ix->n_pad * kExt));
  CKF(dmalloc(&ix->rnorm, (size_t)ix->n_pad));
  CKF(dmalloc(&ix->labels, (size_t)n_ref));
  CKF(dmalloc(&ix->dev_err, 1));
  CKF(dmalloc(&counts, (size_t)n_classes));
  CKF(dmalloc(&bad, 1));
  CKF(cudaMemsetAsync(ix->dev_err, 0, sizeof(uint32_t), s));
  CKF(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * n_classes, s));
  CKF(cudaMemsetAsync(bad, 0, sizeof(uint32_t), s));
  CKF(cudaMemcpyAsync(ix->ref_u8, ref, (size_t)n_ref * row_bytes, cudaMemcpyDeviceToDevice, s));
  CKF(cudaMemcpyAsync(ix->labels, labels, sizeof(int32_t) * n_ref, cudaMemcpyDeviceToDevice, s));
  CKF(launch_label_hist(ix->labels, n_ref, n_classes, counts, bad, s));
  CKF(launch_prep_ref(ix->ref_u8, n_ref, ix->n_pad, row_bytes, loc_w, ix->ref_bf, ix->rnorm, ix->ref_ext, s));
  std::vector<unsigned long long> cnt(n_classes);
  uint32_t bad_h = 0;
  std::vector<int32_t> lab_h(n_ref);
  CKF(cudaMemcpyAsync(cnt.data(), counts, sizeof(unsigned long long) * n_classes, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(&bad_h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(lab_h.data(), ix->labels, sizeof(int32_t) * n_ref, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (bad_h) return fail(LNBNN_ERR_LABEL_RANGE);
  ix->class_off_h.assign(n_classes + 1, 0);
  for (int32_t c = 0; c < n_classes; ++c) {
    ix->class_off_h[c + 1] = ix->class_off_h[c] + (int64_t)cnt[c];
    if (cnt[c] == 0) ix->has_empty_class = true;
  }
  CKF(dmalloc(&ix->class_off_d, (size_t)n_classes + 1));
  CKF(cudaMemcpyAsync(ix->class_off_d, ix->class_off_h.data(), sizeof(int64_t) * (n_classes + 1),
                      cudaMemcpyHostToDevice, s));
  ix->sorted = std::is_sorted(lab_h.begin(), lab_h.end());
  if (ix->sorted) {
    ix->sref_bf = ix->ref_bf;
    ix->sref_ext = ix->ref_ext;
    ix->srnorm = ix->rnorm;
    ix->slabels = ix->labels;
  } else {
    // stable counting sort by class: rows of one class keep their order
    std::vector<int64_t> next(ix->class_off_h.begin(), ix->class_off_h.end() - 1);
    std::vector<int64_t> perm(n_ref);
    for (int64_t j = 0; j < n_ref; ++j) perm[next[lab_h[j]]++] = j;
    CKF(dmalloc(&perm_d, (size_t)n_ref));
    CKF(dmalloc(&ix->sref_bf, (size_t)ix->n_pad * kDim));
    CKF(dmalloc(&ix->sref_ext, (size_t)ix->n_pad * kExt));
    CKF(dmalloc(&ix->srnorm, (size_t)ix->n_pad));
    CKF(dmalloc(&ix->slabels, (size_t)n_ref));
    CKF(cudaMemcpyAsync(perm_d, perm.data(), sizeof(int64_t) * n_ref, cudaMemcpyHostToDevice, s));
    CKF(launch_gather_ref(perm_d, n_ref, ix->ref_bf, ix->sref_bf, ix->ref_ext, ix->sref_ext, ix->rnorm, ix->srnorm,
                          ix->labels, ix->slabels, s));
    // padding rows are the same in both orders
    CKF(cudaMemcpyAsync(ix->sref_bf + (size_t)n_ref * kDim, ix->ref_bf + (size_t)n_ref * kDim,
                        sizeof(__nv_bfloat16) * (size_t)(ix->n_pad - n_ref) * kDim, cudaMemcpyDeviceToDevice, s));
    CKF(cudaMemcpyAsync(ix->sref_ext + (size_t)n_ref * kExt, ix->ref_ext + (size_t)n_ref * kExt,
                        sizeof(__nv_bfloat16) * (size_t)(ix->n_pad - n_ref) * kExt, cudaMemcpyDeviceToDevice, s));
    CKF(launch_fill_float(ix->srnorm + n_ref, ix->n_pad - n_ref, kPadNorm, s));
    CKF(cudaStreamSynchronize(s));  // perm (host vector) must outlive the copy
  }
  if (!make_tc_tensor_maps(ix->ref_bf, ix->sref_bf, ix->ref_ext, ix->sref_ext, ix->n_pad, &ix->tc))
    return fail(LNBNN_ERR_CUDA);
  CKF(prepare_tc_kernels());
  CKF(cudaStreamSynchronize(s));
  cudaFree(counts);
  cudaFree(bad);
  cudaFree(perm_d);
  *out = ix;
  return st;
#undef CKF
}

lnbnn_status lnbnn_index_create(const uint8_t* ref, const int32_t* labels, int64_t n_ref, int32_t n_classes,
                                void* stream, lnbnn_index** out) {
  return create_index(ref, labels, n_ref, n_classes, kDim, 0, stream, out);
}

lnbnn_status lnbnn_index_create_located(const uint8_t* ref, const int32_t* labels, int64_t n_ref, int32_t n_classes,
                                        int32_t location_weight, void* stream, lnbnn_index** out) {
  if (out) *out = nullptr;
  if (location_weight < 0 || location_weight > LNBNN_MAX_LOCATION_WEIGHT) return LNBNN_ERR_INVALID_ARG;
  return create_index(ref, labels, n_ref, n_classes, LNBNN_LOCATED_DIM, location_weight, stream, out);
}

lnbnn_status lnbnn_index_layout(const lnbnn_index* index, int32_t* row_bytes, int32_t* location_weight) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  if (row_bytes) *row_bytes = index->row_bytes;
  if (location_weight) *location_weight = index->loc_w;
  return LNBNN_OK;
}

void lnbnn_index_destroy(lnbnn_index* index) { free_index(index); }

// ------------------------------------------------------------ persistence

namespace {

constexpr char kFileMagic[8] = {'L', 'N', 'B', 'N', 'N', 'I', 'X', '1'};
constexpr uint32_t kFileVersion = 1;
constexpr size_t kFileChunk = size_t(64) << 20;  // bytes staged through host memory at a time

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t dim;
  int64_t n_ref;
  int32_t n_classes;
  uint32_t location_weight;  // 0 for 128-byte rows
};
static_assert(sizeof(FileHeader) == 32, "the file header is 32 bytes");

// FNV-1a, 64-bit.
struct Fnv64 {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  }
};

struct File {
  FILE* f = nullptr;
  File(const char* path, const char* mode) : f(fopen(path, mode)) {}
  ~File() {
    if (f) fclose(f);
  }
};

// Copies `bytes` of device memory to the file through a host buffer, hashing them.
bool write_device(FILE* f, const void* dev, size_t bytes, std::vector<unsigned char>& buf, Fnv64& h) {
  for (size_t off = 0; off < bytes; off += kFileChunk) {
    const size_t n = std::min(kFileChunk, bytes - off);
    if (cudaMemcpy(buf.data(), static_cast<const unsigned char*>(dev) + off, n, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return false;
    h.add(buf.data(), n);
    if (fwrite(buf.data(), 1, n, f) != n) return false;
  }
  return true;
}

}  // namespace

lnbnn_status lnbnn_index_save(const lnbnn_index* index, const char* path) {
  if (!index || !path) return LNBNN_ERR_INVALID_ARG;
  Range range("lnbnn: lnbnn_index_save");
  File file(path, "wb");
  if (!file.f) return LNBNN_ERR_IO;
  FileHeader hd{};
  memcpy(hd.magic, kFileMagic, sizeof kFileMagic);
  hd.version = kFileVersion;
  hd.dim = (uint32_t)index->row_bytes;
  hd.location_weight = (uint32_t)index->loc_w;
  hd.n_ref = index->n_ref;
  hd.n_classes = index->n_classes;
  Fnv64 h;
  h.add(&hd, sizeof hd);
  if (fwrite(&hd, sizeof hd, 1, file.f) != 1) return LNBNN_ERR_IO;
  std::vector<unsigned char> buf(kFileChunk);
  if (!write_device(file.f, index->ref_u8, (size_t)index->n_ref * index->row_bytes, buf, h) ||
      !write_device(file.f, index->labels, sizeof(int32_t) * (size_t)index->n_ref, buf, h))
    return LNBNN_ERR_IO;
  if (fwrite(&h.h, sizeof h.h, 1, file.f) != 1 || fflush(file.f) != 0) return LNBNN_ERR_IO;
  return LNBNN_OK;
}

lnbnn_status lnbnn_index_load(const char* path, void* stream, lnbnn_index** out) {
  if (!out) return LNBNN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!path) return LNBNN_ERR_INVALID_ARG;
  Range range("lnbnn: lnbnn_index_load");
  File file(path, "rb");
  if (!file.f) return LNBNN_ERR_IO;
  FileHeader hd{};
  if (fread(&hd, sizeof hd, 1, file.f) != 1) return LNBNN_ERR_IO;
  if (memcmp(hd.magic, kFileMagic, sizeof kFileMagic) != 0 || hd.version != kFileVersion ||
      hd.dim > (uint32_t)LNBNN_LOCATED_DIM || hd.location_weight > (uint32_t)LNBNN_MAX_LOCATION_WEIGHT ||
      !row_layout_ok((int)hd.dim, (int)hd.location_weight) || hd.n_ref < 1 ||
      hd.n_ref > (int64_t)INT32_MAX - kRefPad || hd.n_classes < 1)
    return LNBNN_ERR_IO;
  // the whole payload is read and its hash checked before the device is touched
  const size_t ref_bytes = (size_t)hd.n_ref * hd.dim, lab_bytes = sizeof(int32_t) * (size_t)hd.n_ref;
  std::vector<unsigned char> ref, lab;
  try {
    ref.resize(ref_bytes);
    lab.resize(lab_bytes);
  } catch (const std::bad_alloc&) {
    return LNBNN_ERR_OOM;
  }
  Fnv64 h;
  h.add(&hd, sizeof hd);
  uint64_t stored = 0;
  if (fread(ref.data(), 1, ref_bytes, file.f) != ref_bytes || fread(lab.data(), 1, lab_bytes, file.f) != lab_bytes ||
      fread(&stored, sizeof stored, 1, file.f) != 1 || fgetc(file.f) != EOF)
    return LNBNN_ERR_IO;
  h.add(ref.data(), ref_bytes);
  h.add(lab.data(), lab_bytes);
  if (h.h != stored) return LNBNN_ERR_IO;
  uint8_t* ref_d = nullptr;
  int32_t* lab_d = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lnbnn_status st = LNBNN_OK;
  cudaError_t e = dmalloc(&ref_d, ref_bytes);
  if (e == cudaSuccess) e = dmalloc(&lab_d, (size_t)hd.n_ref);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ref_d, ref.data(), ref_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lab_d, lab.data(), lab_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  st = e == cudaSuccess ? create_index(ref_d, lab_d, hd.n_ref, hd.n_classes, (int32_t)hd.dim,
                                        (int32_t)hd.location_weight, stream, out)
                        : status_of(e);
  cudaFree(ref_d);
  cudaFree(lab_d);
  return st;
}

void lnbnn_debug_fail_allocations(int32_t count) { g_fail_allocs.store(count > 0 ? count : 0); }

lnbnn_status lnbnn_set_start_gate(lnbnn_index* index, const uint32_t* gate) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  index->gate = gate;
  return LNBNN_OK;
}

lnbnn_status lnbnn_plan_splits(const lnbnn_index* index, int64_t n_queries, int32_t* splits) {
  if (!index || !splits || n_queries < 1) return LNBNN_ERR_INVALID_ARG;
  *splits = plan_knn(index, n_queries, 1, ScanKind::Exact).splits;
  return LNBNN_OK;
}

lnbnn_status lnbnn_set_schedule(lnbnn_index* index, const lnbnn_schedule* schedule) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  if (!schedule) {
    index->sched = lnbnn_schedule{0, 0, -1, -1};
    return LNBNN_OK;
  }
  const lnbnn_schedule& o = *schedule;
  if (o.splits < 0 || o.splits > max_splits(index) || o.query_tiles < 0 || o.query_tiles > 2 ||
      o.persistent < -1 || o.persistent > 1 || o.bound_per_tile < -1 || o.bound_per_tile > 1)
    return LNBNN_ERR_INVALID_ARG;
  index->sched = o;
  return LNBNN_OK;
}

lnbnn_status lnbnn_plan_search(const lnbnn_index* index, int64_t n_queries, int32_t k1, int32_t fp8,
                               lnbnn_search_plan* out) {
  if (!index || !out || n_queries < 1) return LNBNN_ERR_INVALID_ARG;
  if (k1 < 1 || k1 > LNBNN_MAX_K + 1 || (int64_t)k1 > index->n_ref) return LNBNN_ERR_K_RANGE;
  if (fp8 && !index->fp8) return LNBNN_ERR_NO_FP8;
  const KnnPlan p = plan_knn(index, n_queries, k1, fp8 ? ScanKind::Coarse : ScanKind::Exact);
  lnbnn_search_plan r{};
  r.splits = p.splits;
  r.lists_per_row = p.lists;
  r.split_len = p.split_len;
  switch (tc_list_kind(k1, p.split_len, fp8 != 0)) {
    case ListKind::Reg16: r.list_storage = 0; r.list_capacity = kTcRegListMax; break;
    case ListKind::Reg24: r.list_storage = 0; r.list_capacity = kTcMidRegListMax; break;
    case ListKind::Reg32: r.list_storage = 0; r.list_capacity = kTcCoarseRegListMax; break;
    case ListKind::Smem64: r.list_storage = 1; r.list_capacity = kTcWideRegListMax; break;
    case ListKind::Reg64: r.list_storage = 0; r.list_capacity = kTcWideRegListMax; break;
    case ListKind::Heap: r.list_storage = 2; r.list_capacity = k1; break;
  }
  r.tile_m = kTcQueryTile * p.qt;
  r.tile_n = kTcRefTile / p.qt;
  r.persistent = p.persistent ? 1 : 0;
  r.bound_per_tile = p.splits > 1 ? (p.bound_per_tile ? 1 : 0) : -1;
  r.chunked = p.group > 0 ? 1 : 0;
  *out = r;
  return LNBNN_OK;
}

lnbnn_status lnbnn_autotune(lnbnn_index* index, void* stream, lnbnn_tuning* out) {
  Range range("lnbnn: lnbnn_autotune");
  if (!index) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = index->sm_count;
  const int64_t n_ref = index->n_ref;
  lnbnn_tuning res{};
  res.exact_persistent = res.coarse_persistent = -1;
  // query tiles up to 64 (a few waves of CTAs with few splits), copied from
  // reference rows spread over the set, so their neighbour structure is real
  const int64_t t_max = std::min<int64_t>(64, n_ref / kTcQueryTile);
  if (t_max < 1) {  // too few references for a whole query tile: keep the defaults
    if (out) *out = res;
    return LNBNN_OK;
  }
  struct Run {
    int64_t T, splits;
    int K1;
    double ms;
  };
  std::vector<Run> runs;
  for (int K1 : {11, 51}) {
    if (K1 > n_ref) continue;
    for (int64_t T = 1; T <= t_max; T *= (K1 == 11 ? 2 : 4)) {
      const int64_t hi = max_splits_for(T, n_ref, P, max_splits(index));
      int64_t last = 0;
      for (int64_t w : {1, 2, 4}) {
        const int64_t sp = std::min<int64_t>(hi, std::max<int64_t>(1, w * P / T));
        if (sp != last) runs.push_back({T, sp, K1, 0.0});
        last = sp;
      }
    }
  }
  // large-batch forms: two waves of query tiles, when the references hold that many rows
  const int64_t t_big = (int64_t)2 * P;
  const bool forms = n_ref >= t_big * kTcQueryTile;
  struct Form {
    ScanKind kind;
    int qt, persistent;
    double ms;
  };
  std::vector<Form> cand;
  if (forms)
    for (ScanKind k : {ScanKind::Exact, ScanKind::Coarse}) {
      if (k == ScanKind::Coarse && !index->fp8) continue;
      for (int qt : {1, 2})
        for (int pe : {0, 1}) cand.push_back({k, qt, pe, 0.0});
    }
  const int64_t m_max = std::max(t_max, forms ? t_big : int64_t(0)) * kTcQueryTile;
  const lnbnn_schedule saved = index->sched;
  size_t need = 0;
  index->sched = lnbnn_schedule{0, 0, 0, -1};
  for (const Run& r : runs)
    need = std::max(need, plan_knn(index, r.T * kTcQueryTile, r.K1, ScanKind::Exact, (int)r.splits).bytes);
  for (const Form& f : cand) {
    index->sched = lnbnn_schedule{0, f.qt, f.persistent, -1};
    need = std::max(need, plan_knn(index, t_big * kTcQueryTile, f.kind == ScanKind::Coarse ? 32 : 11, f.kind).bytes);
  }
  index->sched = saved;
  lnbnn_workspace w;
  w.index = index;
  w.bytes = need;
  uint8_t* q = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lnbnn_status st = LNBNN_OK;
  const bool prof_was_on = index->prof_on;
  auto cleanup = [&]() {  // idempotent
    index->sched = saved;
    index->prof_on = prof_was_on;
    cudaFree(q);
    cudaFree(w.base);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    q = nullptr;
    w.base = nullptr;
    e0 = e1 = nullptr;
  };
#define CKA(call)                         \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      st = status_of(e_);                 \
      cleanup();                          \
      return st;                          \
    }                                     \
  } while (0)
  const int32_t rb = index->row_bytes;
  CKA(dmalloc(&q, (size_t)m_max * rb));
  CKA(lib_malloc(&w.base, need));
  CKA(cudaEventCreate(&e0));
  CKA(cudaEventCreate(&e1));
  const int64_t step = n_ref / m_max;  // >= 1
  CKA(cudaMemcpy2DAsync(q, rb, index->ref_u8, (size_t)step * rb, rb, (size_t)m_max, cudaMemcpyDeviceToDevice, s));
  index->prof_on = false;
  // the best of two timed calls after a warm-up
  auto time_call = [&](auto&& call, double* ms_out) -> lnbnn_status {
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaError_t e = cudaEventRecord(e0, s);
      if (e != cudaSuccess) return status_of(e);
      const lnbnn_status cs = call();
      if (cs != LNBNN_OK) return cs;
      e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) return status_of(e);
      if (rep == 1 || (rep > 1 && ms < best)) best = ms;
    }
    *ms_out = best;
    return LNBNN_OK;
  };
  // split-model runs: one query tile per CTA, one CTA per item
  index->sched = lnbnn_schedule{0, 1, 0, -1};
  for (Run& r : runs) {
    st = time_call([&]() {
      Scratch scratch{index, &w};
      CallProfile prof(index, s);
      const uint64_t* lists = nullptr;
      return run_knn(index, scratch, q, r.T * kTcQueryTile, r.K1, s, &lists, prof, (int)r.splits);
    }, &r.ms);
    if (st != LNBNN_OK) {
      cleanup();
      return st;
    }
  }
  // large-batch forms at the automatic split count of each
  for (Form& f : cand) {
    index->sched = lnbnn_schedule{0, f.qt, f.persistent, -1};
    st = time_call([&]() {
      Scratch scratch{index, &w};
      CallProfile prof(index, s);
      const uint64_t* lists = nullptr;
      return f.kind == ScanKind::Coarse
                 ? run_knn_fp8(index, scratch, q, t_big * kTcQueryTile, 11, 32, s, &lists, prof)
                 : run_knn(index, scratch, q, t_big * kTcQueryTile, 11, s, &lists, prof);
    }, &f.ms);
    if (st != LNBNN_OK) {
      cleanup();
      return st;
    }
  }
  cleanup();
#undef CKA
  // the fastest form of each kind (the first, one query tile per CTA and one
  // CTA per item, unless another is faster by more than 2%)
  for (ScanKind k : {ScanKind::Exact, ScanKind::Coarse}) {
    const Form* best = nullptr;
    for (const Form& f : cand)
      if (f.kind == k && (!best || f.ms < best->ms * 0.98)) best = &f;
    if (!best) continue;
    index->auto_qt[(int)k] = best->qt;
    index->auto_persistent[(int)k] = best->persistent;
    (k == ScanKind::Exact ? res.exact_query_tiles : res.coarse_query_tiles) = best->qt;
    (k == ScanKind::Exact ? res.exact_persistent : res.coarse_persistent) = best->persistent;
  }
  for (size_t i = 0; i < cand.size() && i < 8; ++i) {
    const int slot = (cand[i].kind == ScanKind::Coarse ? 4 : 0) + 2 * (cand[i].qt - 1) + cand[i].persistent;
    res.form_ms[slot] = cand[i].ms;
  }
  res.form_runs = (int32_t)cand.size();
  // least squares for ms = a * waves * tiles + b * waves + c * T * splits + e * waves * K1 + d,
  // dropping a term whose coefficient comes out negative
  constexpr int NF = 5;
  bool use[NF] = {true, true, true, true, true};
  double coef[NF] = {0, 0, 0, 0, 0};
  auto feat = [&](const Run& r, int j) {
    const int64_t split_len = round_up((n_ref + r.splits - 1) / r.splits, kTcRefTile);
    const int64_t sp = (n_ref + split_len - 1) / split_len;
    const double waves = (double)((r.T * sp + P - 1) / P);
    const double tiles = (double)(split_len / kTcRefTile);
    switch (j) {
      case 0: return waves * tiles;
      case 1: return waves;
      case 2: return (double)(r.T * sp);
      case 3: return waves * (double)r.K1;
      default: return 1.0;
    }
  };
  for (int pass = 0; pass < NF; ++pass) {
    double A[NF][NF + 1] = {};
    for (const Run& r : runs)
      for (int i = 0; i < NF; ++i)
        for (int j = 0; j < NF; ++j) A[i][j] += use[i] && use[j] ? feat(r, i) * feat(r, j) : 0.0;
    for (const Run& r : runs)
      for (int i = 0; i < NF; ++i) A[i][NF] += use[i] ? feat(r, i) * r.ms : 0.0;
    for (int i = 0; i < NF; ++i)
      if (!use[i]) A[i][i] = 1.0;
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < NF; ++c) {
      int piv = c;
      for (int r = c + 1; r < NF; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
      for (int j = 0; j <= NF; ++j) std::swap(A[c][j], A[piv][j]);
      if (std::fabs(A[c][c]) < 1e-300) continue;
      for (int r = 0; r < NF; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int j = c; j <= NF; ++j) A[r][j] -= f * A[c][j];
      }
    }
    for (int i = 0; i < NF; ++i) coef[i] = use[i] && std::fabs(A[i][i]) > 1e-300 ? A[i][NF] / A[i][i] : 0.0;
    int worst = -1;
    for (int i = 0; i < NF - 1; ++i)
      if (use[i] && coef[i] < 0 && (worst < 0 || coef[i] < coef[worst])) worst = i;
    if (worst < 0) break;
    use[worst] = false;
  }
  res.runs = (int32_t)runs.size();
  if (coef[0] <= 0) {  // measurements no schedule model explains: keep the current model
    if (out) *out = res;
    return LNBNN_OK;
  }
  index->split_model.a = coef[0];
  index->split_model.b = std::max(0.0, coef[1]);
  index->split_model.c = std::max(0.0, coef[2]);
  index->split_model.e = std::max(0.0, coef[3]);
  res.tile_ms = coef[0];
  res.wave_ms = index->split_model.b;
  res.list_ms = index->split_model.c;
  res.entry_ms = index->split_model.e;
  double worst = 0;
  for (const Run& r : runs) {
    const double pred = coef[4] + coef[0] * feat(r, 0) + index->split_model.b * feat(r, 1) +
                        index->split_model.c * feat(r, 2) + index->split_model.e * feat(r, 3);
    worst = std::max(worst, std::fabs(pred - r.ms) / r.ms);
  }
  res.max_rel_error = worst;
  if (out) *out = res;
  return LNBNN_OK;
}

lnbnn_status lnbnn_index_prepare_fp8(lnbnn_index* index, void* stream) {
  Range range("lnbnn: lnbnn_index_prepare_fp8");
  if (!index) return LNBNN_ERR_INVALID_ARG;
  if (index->row_bytes != kDim) return LNBNN_ERR_UNSUPPORTED;  // the coarse operand has no location term
  if (index->fp8) return LNBNN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto undo = [&](lnbnn_status st) {  // a failed preparation keeps nothing
    cudaFree(index->ref_f8);
    cudaFree(index->ref_f8_ext);
    index->ref_f8 = nullptr;
    index->ref_f8_ext = nullptr;
    return st;
  };
  cudaError_t e = dmalloc(&index->ref_f8, (size_t)index->n_pad * kDim);
  if (e == cudaSuccess) e = dmalloc(&index->ref_f8_ext, (size_t)index->n_pad * kExt);
  if (e == cudaSuccess)
    e = launch_prep_ref_e4m3(index->ref_u8, index->n_ref, index->n_pad, index->ref_f8, index->ref_f8_ext, s);
  if (e != cudaSuccess) return undo(status_of(e));
  if (!make_tc_tensor_maps_e4m3(index->ref_f8, index->ref_f8_ext, index->n_pad, &index->tc)) {
    cudaStreamSynchronize(s);
    return undo(LNBNN_ERR_CUDA);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return undo(status_of(e));
  index->fp8 = true;
  return LNBNN_OK;
}

lnbnn_status lnbnn_index_info(const lnbnn_index* index, int64_t* n_ref, int32_t* n_classes) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  if (n_ref) *n_ref = index->n_ref;
  if (n_classes) *n_classes = index->n_classes;
  return LNBNN_OK;
}

static lnbnn_status do_knn_search(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries, int64_t n_queries,
                                  int32_t k, int32_t* idx, int32_t* dist, void* stream) {
  Range range("lnbnn: knn_search");
  if (!index || n_queries < 0) return LNBNN_ERR_INVALID_ARG;
  if (!k_ok(index, k, 0)) return LNBNN_ERR_K_RANGE;
  if (n_queries == 0) return LNBNN_OK;
  if (!queries || !idx || !dist) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallProfile prof(index, s);
  Scratch scratch{index, w};
  const uint64_t* lists = nullptr;
  lnbnn_status st = run_knn(index, scratch, queries, n_queries, k, s, &lists, prof);
  if (st != LNBNN_OK) return st;
  CK(launch_extract_knn(lists, n_queries, k, k, idx, dist, s));
  prof.launched(1);
  return LNBNN_OK;
}

static lnbnn_status do_knn_search_fp8(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                      int64_t n_queries, int32_t k, int32_t shortlist, int32_t* idx, int32_t* dist,
                                      void* stream) {
  Range range("lnbnn: knn_search_fp8");
  if (!index || n_queries < 0) return LNBNN_ERR_INVALID_ARG;
  int M1 = 0;
  if (!k_ok(index, k, 0) || !shortlist_ok(index, shortlist, k, &M1)) return LNBNN_ERR_K_RANGE;
  if (!index->fp8) return LNBNN_ERR_NO_FP8;
  if (n_queries == 0) return LNBNN_OK;
  if (!queries || !idx || !dist) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallProfile prof(index, s);
  Scratch scratch{index, w};
  const uint64_t* lists = nullptr;
  lnbnn_status st = run_knn_fp8(index, scratch, queries, n_queries, k, M1, s, &lists, prof);
  if (st != LNBNN_OK) return st;
  CK(launch_extract_knn(lists, n_queries, k, k, idx, dist, s));
  prof.launched(1);
  return LNBNN_OK;
}

// shortlist = 0: exact search; otherwise the FP8 shortlist search.
static lnbnn_status do_lnbnn_classify(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                      int64_t n_queries, const int64_t* offsets, int64_t n_images, int32_t k,
                                      int32_t shortlist, int64_t* totals, int32_t* classes, void* stream) {
  Range range("lnbnn: lnbnn_classify");
  if (!index || n_queries < 0 || n_images < 0) return LNBNN_ERR_INVALID_ARG;
  if (!k_ok(index, k, 1)) return LNBNN_ERR_K_RANGE;
  int M1 = 0;
  if (shortlist != 0) {
    if (!shortlist_ok(index, shortlist, k + 1, &M1)) return LNBNN_ERR_K_RANGE;
    if (!index->fp8) return LNBNN_ERR_NO_FP8;
  }
  if (n_images == 0) return n_queries == 0 ? LNBNN_OK : LNBNN_ERR_OFFSETS;
  if (!offsets || !totals || !classes || (n_queries > 0 && !queries)) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallProfile prof(index, s);
  const int32_t C = index->n_classes;
  CK(cudaMemsetAsync(totals, 0, sizeof(int64_t) * (size_t)n_images * C, s));
  CK(launch_check_offsets(offsets, n_images, n_queries, index->dev_err, s));
  prof.launched(1);
  if (n_queries > 0) {
    Scratch scratch{index, w};
    const uint64_t* lists = nullptr;
    lnbnn_status st = shortlist ? run_knn_fp8(index, scratch, queries, n_queries, k + 1, M1, s, &lists, prof)
                                : run_knn(index, scratch, queries, n_queries, k + 1, s, &lists, prof);
    if (st != LNBNN_OK) return st;
    CK(launch_lnbnn_score(lists, n_queries, k + 1, k, index->labels, index->n_ref, offsets, n_images, C, totals,
                          index->dev_err, s));
    prof.launched(1);
  } else {
    prof.mark(1);
    prof.mark(2);
  }
  CK(launch_argmin(totals, n_images, C, classes, s));
  prof.launched(1);
  return LNBNN_OK;
}

// The [m_pad, C] table of class minima NN_C(d), one row per query row, filled
// by the tensor-core scan of the class-sorted references (Alg. 1's inner
// loop).  Sets *mins and, when rowstat is given, the row-statistics buffer of
// the same workspace.
static lnbnn_status scan_class_minima(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                      int64_t n_queries, cudaStream_t s, CallProfile& prof, int32_t** mins,
                                      void** rowstat) {
  const NbnnPlan np = plan_nbnn(index, n_queries);
  const KnnPlan& p = np.k;
  Scratch scratch{index, w};
  char* ws = nullptr;
  lnbnn_status st = scratch.get(np.bytes, &ws);
  if (st != LNBNN_OK) return st;
  int32_t* qnorm = reinterpret_cast<int32_t*>(ws + np.off_qnorm);
  __nv_bfloat16* qbf = reinterpret_cast<__nv_bfloat16*>(ws + np.off_qbf);
  __nv_bfloat16* qext = reinterpret_cast<__nv_bfloat16*>(ws + np.off_qext);
  *mins = reinterpret_cast<int32_t*>(ws + np.off_mins);
  if (rowstat) *rowstat = ws + np.off_rowstat;
  CK(launch_prep_query(queries, n_queries, p.m_pad, index->row_bytes, index->loc_w, qnorm, qbf, qext, s));
  CK(cudaMemsetAsync(*mins, 0x7F, sizeof(int32_t) * (size_t)p.m_pad * index->n_classes, s));  // > any distance
  const TcSched sched = p.sched(ws, index->sm_count);
  CK(p.clear(ws, s));
  prof.launched(1);
  prof.mark(1);
  CK(launch_nbnn_tc(index->tc, qbf, qext, n_queries, p.m_pad, index->n_ref, p.splits, p.split_len, *mins,
                    index->n_classes, index->class_off_d, index->dev_err,
                    index->prof_on ? index->prof_stats : nullptr, index->gate, sched, s));
  prof.launched(1, true);
  prof.mark(2);
  return LNBNN_OK;
}

static lnbnn_status do_nbnn_classify(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                     int64_t n_queries, const int64_t* offsets, int64_t n_images, int64_t* totals,
                                     int32_t* classes, void* stream) {
  Range range("lnbnn: nbnn_classify");
  if (!index || n_queries < 0 || n_images < 0) return LNBNN_ERR_INVALID_ARG;
  if (index->has_empty_class) return LNBNN_ERR_EMPTY_CLASS;
  if (n_images == 0) return n_queries == 0 ? LNBNN_OK : LNBNN_ERR_OFFSETS;
  if (!offsets || !totals || !classes || (n_queries > 0 && !queries)) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallProfile prof(index, s);
  const int32_t C = index->n_classes;
  CK(cudaMemsetAsync(totals, 0, sizeof(int64_t) * (size_t)n_images * C, s));
  CK(launch_check_offsets(offsets, n_images, n_queries, index->dev_err, s));
  prof.launched(1);
  if (n_queries == 0) {
    prof.mark(1);
    prof.mark(2);
  } else {
    int32_t* mins = nullptr;
    lnbnn_status st = scan_class_minima(index, w, queries, n_queries, s, prof, &mins, nullptr);
    if (st != LNBNN_OK) return st;
    CK(launch_nbnn_sum(mins, n_queries, C, offsets, n_images, totals, s));
    prof.launched(1);
  }
  CK(launch_argmin(totals, n_images, C, classes, s));
  prof.launched(1);
  return LNBNN_OK;
}

static lnbnn_status do_nbnn_logodds_classify(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                             int64_t n_queries, const int64_t* offsets, int64_t n_images,
                                             double beta, bool positive_only, double* totals, int32_t* classes,
                                             int64_t* n_increments, void* stream) {
  Range range("lnbnn: nbnn_logodds_classify");
  if (!index || n_queries < 0 || n_images < 0) return LNBNN_ERR_INVALID_ARG;
  if (!(beta >= 0.0 && beta <= 1e250) || index->n_classes < 2) return LNBNN_ERR_INVALID_ARG;
  if (index->has_empty_class) return LNBNN_ERR_EMPTY_CLASS;
  if (n_images == 0) return n_queries == 0 ? LNBNN_OK : LNBNN_ERR_OFFSETS;
  if (!offsets || !totals || !classes || (n_queries > 0 && !queries)) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallProfile prof(index, s);
  const int32_t C = index->n_classes;
  CK(cudaMemsetAsync(totals, 0, sizeof(double) * (size_t)n_images * C, s));
  if (n_increments) CK(cudaMemsetAsync(n_increments, 0, sizeof(int64_t) * (size_t)n_images, s));
  CK(launch_check_offsets(offsets, n_images, n_queries, index->dev_err, s));
  prof.launched(1);
  if (n_queries == 0) {
    prof.mark(1);
    prof.mark(2);
  } else {
    int32_t* mins = nullptr;
    void* rowstat = nullptr;
    lnbnn_status st = scan_class_minima(index, w, queries, n_queries, s, prof, &mins, &rowstat);
    if (st != LNBNN_OK) return st;
    CK(launch_logodds_rowstat(mins, n_queries, C, beta, rowstat, s));
    CK(launch_logodds_sum(mins, rowstat, n_queries, C, beta, positive_only, offsets, n_images, totals,
                          n_increments, s));
    prof.launched(2);
  }
  CK(launch_argmax_f64(totals, n_images, C, classes, s));
  prof.launched(1);
  return LNBNN_OK;
}

lnbnn_status knn_search(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, int32_t k, int32_t* idx,
                        int32_t* dist, void* stream) {
  return do_knn_search(index, nullptr, queries, n_queries, k, idx, dist, stream);
}

lnbnn_status lnbnn_classify(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, const int64_t* offsets,
                            int64_t n_images, int32_t k, int64_t* totals, int32_t* classes, void* stream) {
  return do_lnbnn_classify(index, nullptr, queries, n_queries, offsets, n_images, k, 0, totals, classes, stream);
}

lnbnn_status knn_search_fp8(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, int32_t k,
                            int32_t shortlist, int32_t* idx, int32_t* dist, void* stream) {
  return do_knn_search_fp8(index, nullptr, queries, n_queries, k, shortlist, idx, dist, stream);
}

lnbnn_status lnbnn_classify_fp8(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, const int64_t* offsets,
                                int64_t n_images, int32_t k, int32_t shortlist, int64_t* totals, int32_t* classes,
                                void* stream) {
  if (shortlist == 0) return LNBNN_ERR_K_RANGE;
  return do_lnbnn_classify(index, nullptr, queries, n_queries, offsets, n_images, k, shortlist, totals, classes,
                           stream);
}

lnbnn_status nbnn_classify(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, const int64_t* offsets,
                           int64_t n_images, int64_t* totals, int32_t* classes, void* stream) {
  return do_nbnn_classify(index, nullptr, queries, n_queries, offsets, n_images, totals, classes, stream);
}

lnbnn_status nbnn_logodds_classify(lnbnn_index* index, const uint8_t* queries, int64_t n_queries,
                                   const int64_t* offsets, int64_t n_images, double beta, int32_t positive_only,
                                   double* totals, int32_t* classes, int64_t* n_increments, void* stream) {
  return do_nbnn_logodds_classify(index, nullptr, queries, n_queries, offsets, n_images, beta, positive_only != 0,
                                  totals, classes, n_increments, stream);
}

lnbnn_status lnbnn_workspace_create(lnbnn_index* index, int64_t max_queries, int32_t max_k, lnbnn_workspace** out) {
  if (!out) return LNBNN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!index || max_queries < 1) return LNBNN_ERR_INVALID_ARG;
  if (!k_ok(index, max_k, 0)) return LNBNN_ERR_K_RANGE;
  lnbnn_workspace* w = new (std::nothrow) lnbnn_workspace();
  if (!w) return LNBNN_ERR_OOM;
  w->index = index;
  w->bytes = scratch_bound(index, max_queries, std::min<int>(max_k + 1, LNBNN_MAX_K + 1));
  cudaError_t e = lib_malloc(&w->base, w->bytes);
  if (e != cudaSuccess) {
    delete w;
    return status_of(e);
  }
  *out = w;
  return LNBNN_OK;
}

void lnbnn_workspace_destroy(lnbnn_workspace* w) {
  if (!w) return;
  cudaFree(w->base);
  delete w;
}

lnbnn_status knn_search_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries, int64_t n_queries,
                           int32_t k, int32_t* idx, int32_t* dist, void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  return do_knn_search(index, w, queries, n_queries, k, idx, dist, stream);
}

lnbnn_status lnbnn_classify_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries, int64_t n_queries,
                               const int64_t* offsets, int64_t n_images, int32_t k, int64_t* totals, int32_t* classes,
                               void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  return do_lnbnn_classify(index, w, queries, n_queries, offsets, n_images, k, 0, totals, classes, stream);
}

lnbnn_status knn_search_fp8_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries, int64_t n_queries,
                               int32_t k, int32_t shortlist, int32_t* idx, int32_t* dist, void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  return do_knn_search_fp8(index, w, queries, n_queries, k, shortlist, idx, dist, stream);
}

lnbnn_status lnbnn_classify_fp8_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                   int64_t n_queries, const int64_t* offsets, int64_t n_images, int32_t k,
                                   int32_t shortlist, int64_t* totals, int32_t* classes, void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  if (shortlist == 0) return LNBNN_ERR_K_RANGE;
  return do_lnbnn_classify(index, w, queries, n_queries, offsets, n_images, k, shortlist, totals, classes, stream);
}

lnbnn_status nbnn_classify_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries, int64_t n_queries,
                              const int64_t* offsets, int64_t n_images, int64_t* totals, int32_t* classes,
                              void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  return do_nbnn_classify(index, w, queries, n_queries, offsets, n_images, totals, classes, stream);
}

lnbnn_status nbnn_logodds_classify_ws(lnbnn_index* index, lnbnn_workspace* w, const uint8_t* queries,
                                      int64_t n_queries, const int64_t* offsets, int64_t n_images, double beta,
                                      int32_t positive_only, double* totals, int32_t* classes,
                                      int64_t* n_increments, void* stream) {
  if (!w || w->index != index) return LNBNN_ERR_INVALID_ARG;
  return do_nbnn_logodds_classify(index, w, queries, n_queries, offsets, n_images, beta, positive_only != 0, totals,
                                  classes, n_increments, stream);
}

static lnbnn_status classify_host(lnbnn_index* index, bool local, const uint8_t* queries, int64_t n_queries,
                                  const int64_t* offsets, int64_t n_images, int32_t k, int32_t shortlist,
                                  int64_t* totals, int32_t* classes, void* stream) {
  Range range("lnbnn: classify_host");
  if (!index || n_queries < 0 || n_images < 0) return LNBNN_ERR_INVALID_ARG;
  if (n_images == 0) return n_queries == 0 ? LNBNN_OK : LNBNN_ERR_OFFSETS;
  if (!offsets || !totals || !classes || (n_queries > 0 && !queries)) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t C = index->n_classes;
  Carve c;
  const size_t oq = c.take<uint8_t>((size_t)n_queries * index->row_bytes);
  const size_t oo = c.take<int64_t>((size_t)n_images + 1);
  const size_t ot = c.take<int64_t>((size_t)n_images * C);
  const size_t oc = c.take<int32_t>((size_t)n_images);
  CK(ensure(&index->stage, &index->stage_bytes, c.off));
  char* b = static_cast<char*>(index->stage);
  uint8_t* dq = reinterpret_cast<uint8_t*>(b + oq);
  int64_t* doff = reinterpret_cast<int64_t*>(b + oo);
  int64_t* dtot = reinterpret_cast<int64_t*>(b + ot);
  int32_t* dcls = reinterpret_cast<int32_t*>(b + oc);
  if (n_queries > 0)
    CK(cudaMemcpyAsync(dq, queries, (size_t)n_queries * index->row_bytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(doff, offsets, sizeof(int64_t) * (n_images + 1), cudaMemcpyHostToDevice, s));
  lnbnn_status st =
      local ? do_lnbnn_classify(index, nullptr, dq, n_queries, doff, n_images, k, shortlist, dtot, dcls, stream)
            : nbnn_classify(index, dq, n_queries, doff, n_images, dtot, dcls, stream);
  if (st != LNBNN_OK) return st;
  CK(cudaMemcpyAsync(totals, dtot, sizeof(int64_t) * (size_t)n_images * C, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(classes, dcls, sizeof(int32_t) * (size_t)n_images, cudaMemcpyDeviceToHost, s));
  return lnbnn_sync(index, stream);
}

lnbnn_status lnbnn_classify_host(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, const int64_t* offsets,
                                 int64_t n_images, int32_t k, int64_t* totals, int32_t* classes, void* stream) {
  if (index && !k_ok(index, k, 1)) return LNBNN_ERR_K_RANGE;
  return classify_host(index, true, queries, n_queries, offsets, n_images, k, 0, totals, classes, stream);
}

lnbnn_status lnbnn_classify_fp8_host(lnbnn_index* index, const uint8_t* queries, int64_t n_queries,
                                     const int64_t* offsets, int64_t n_images, int32_t k, int32_t shortlist,
                                     int64_t* totals, int32_t* classes, void* stream) {
  int M1 = 0;
  if (index && (!k_ok(index, k, 1) || !shortlist_ok(index, shortlist, k + 1, &M1))) return LNBNN_ERR_K_RANGE;
  if (index && !index->fp8) return LNBNN_ERR_NO_FP8;
  return classify_host(index, true, queries, n_queries, offsets, n_images, k, shortlist, totals, classes, stream);
}

lnbnn_status nbnn_classify_host(lnbnn_index* index, const uint8_t* queries, int64_t n_queries, const int64_t* offsets,
                                int64_t n_images, int64_t* totals, int32_t* classes, void* stream) {
  if (index && index->has_empty_class) return LNBNN_ERR_EMPTY_CLASS;
  return classify_host(index, false, queries, n_queries, offsets, n_images, 0, 0, totals, classes, stream);
}

lnbnn_status lnbnn_profile_enable(lnbnn_index* index, int enable) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  for (auto& ce : index->prof_pending) {
    cudaEventSynchronize(ce.e[3]);
    index->prof_free.push_back(ce);
  }
  index->prof_pending.clear();
  index->prof = lnbnn_profile{};
  index->prof_on = enable != 0;
  if (index->prof_on) {
    if (!index->prof_stats) CK(dmalloc(&index->prof_stats, 4));
    CK(cudaMemset(index->prof_stats, 0, 4 * sizeof(unsigned long long)));
  }
  return LNBNN_OK;
}

lnbnn_status lnbnn_profile_read(lnbnn_index* index, lnbnn_profile* out) {
  if (!index || !out) return LNBNN_ERR_INVALID_ARG;
  for (auto& ce : index->prof_pending) {
    CK(cudaEventSynchronize(ce.e[3]));
    float a = 0.f, b = 0.f, c = 0.f;
    CK(cudaEventElapsedTime(&a, ce.e[0], ce.e[1]));
    CK(cudaEventElapsedTime(&b, ce.e[1], ce.e[2]));
    CK(cudaEventElapsedTime(&c, ce.e[2], ce.e[3]));
    index->prof.other_ms += (double)a + (double)c;
    index->prof.search_ms += (double)b;
    index->prof_free.push_back(ce);
  }
  index->prof_pending.clear();
  if (index->prof_stats) {
    unsigned long long st[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(st, index->prof_stats, sizeof st, cudaMemcpyDeviceToHost));
    index->prof.search_sm_clock_ghz = st[1] ? (double)st[0] / (double)st[1] : 0.0;
    index->prof.search_cycles_per_tile = st[2] ? (double)st[0] / (double)st[2] : 0.0;
  }
  *out = index->prof;
  return LNBNN_OK;
}

lnbnn_status lnbnn_sync(lnbnn_index* index, void* stream) {
  if (!index) return LNBNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t err = 0;
  CK(cudaMemcpyAsync(&err, index->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err) {
    CK(cudaMemsetAsync(index->dev_err, 0, sizeof(uint32_t), s));
    CK(cudaStreamSynchronize(s));
  }
  if (err & kDevErrTimeout) return LNBNN_ERR_TIMEOUT;
  if (err & kDevErrOffsets) return LNBNN_ERR_OFFSETS;
  return LNBNN_OK;
}

}  // extern "C"
