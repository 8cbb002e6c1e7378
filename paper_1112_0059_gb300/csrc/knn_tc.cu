// Exact k+1 nearest-neighbour search (the NN(d, k+1) of Alg. 2) on the sm_103a
// tensor cores.
//
// For a tile of 128 query rows and 256 reference rows the MMA computes, in
// FP32 TMEM accumulators,
//     acc[i][j] = sum_t (-2 q_it) r_jt + (1, 256, 65536, e0, e1, e2)_i . (d0, d1, d2, 1, 256, 65536)_j
//               = ||r_j||^2 + ||q_i||^2 - 2 q_i . r_j = ||q_i - r_j||^2,
// the last term being a 16-wide K-extension that carries both squared norms as
// base-256 digits.  BF16 holds 0..255, -2q and the digits exactly; every
// product and partial sum is an integer below 2^24 in magnitude, so acc is the
// exact squared distance.  Non-negative floats order like their bit patterns,
// so the epilogue tests 32 columns with one compare of their minimum, which
// the TMEM load itself returns (tcgen05.ld.red ... .min.u32), against the
// row's current (k+1)-th distance, and keeps the k+1 smallest (distance, row)
// pairs.  The distance matrix never leaves the SM.
//
// The same scan runs the coarse pass of the FP8 shortlist search: operands
// are the E4M3 roundings of the coordinates shifted by -64 (queries scaled by
// -2, exact in E4M3), one 128-byte K-chunk per tile and four kind::f8f6f4
// MMAs (K = 32 each), and the K-extension carries ||q'||^2 + 2^21 and ||r'||^2
// of the shifted (unrounded) coordinates.  The accumulator then holds
//     coarse = ||q'||^2 + ||r'||^2 - 2 q~ . r~ + 2^21,
// an integer: the bias keeps it positive (E4M3 rounding is within 2^-4 of
// each coordinate, so 2 q~.r~ is within 2 * 0.129 * 128 * 191^2 < 1.21e6 of
// 2 q'.r'), and with the extension issued first every partial sum stays in
// [0, 2^24), so FP32 holds it exactly.
//
// Work: a launch covers T groups of QT query tiles (128 rows each) x S
// reference splits as T x S work items, split-major; a CTA takes one item, or
// (persistent form) items from a queue one after another (see Work below).
//
// Roles (one CTA = QT query tiles x one reference split at a time):
//   warp 0, one thread : TMA producer (the item's query tiles; reference
//                        K-chunks into a ring, the K-extension riding with
//                        the last chunk of each tile)
//   warp 1, one thread : tcgen05.mma issuer (9 MMAs of 128x256x16 per tile);
//                        warp 1 also owns the TMEM allocation; with QT = 2 a
//                        second issuer (the warp after the epilogue warps)
//                        issues the second query tile's MMAs
//   warps 2-9          : epilogue: two warps per TMEM lane quarter, each
//                        taking a 128-column half of every tile (QT = 2: its
//                        query tile's 128 x 128 block) with one thread per
//                        query row (TMEM lane); each keeps its own sorted
//                        list of the k+1 nearest (in registers for k+1 <= 64,
//                        otherwise a heap in global memory; for 33..64 one
//                        warp per quarter takes all 256 columns, to have the
//                        registers); two 256-column FP32 accumulators in
//                        flight; each 32-column load also returns the
//                        columns' minimum
// Every wait is bounded; on expiry the CTA records a timeout in the index's
// device error word, drains what it issued and returns.
#include <cudaTypedefs.h>

#include "knn_tc.cuh"
#include "sm103.cuh"
#include "topk.cuh"

namespace lnbnn {
namespace {

using namespace sm103;

constexpr int kBM = kTcQueryTile;         // query rows per query tile (MMA M)
constexpr int kBK = 64;                   // BF16 K elements per 128-byte swizzle row
constexpr int kKChunks = kDim / kBK;      // K-chunks of the BF16 operand (shared memory is laid out for these)
constexpr int kMmaPerChunk = 4;           // 32-byte K-steps per 128-byte chunk (16 BF16 or 32 E4M3)
constexpr uint32_t kAChunkBytes = kBM * kBK * 2;     // 16 KB
constexpr uint32_t kAExtBytes = kBM * kExt * 2;      // 4 KB

// Tile shapes: a CTA computes QT query tiles (128 rows each) against a tile
// of 256 / QT references per step, so every step is 128 x 256 query-reference
// pairs and its FP32 accumulator takes 256 TMEM columns (QT = 2: the two
// query tiles' 128 x 128 blocks side by side).  QT = 2 loads each reference
// tile once for 256 query rows: half the reference bytes per pair.
template <int QT>
struct Shape {
  static_assert(QT == 1 || QT == 2, "one or two query tiles per CTA");
  static constexpr int kTileN = kTcRefTile / QT;                 // references per tile (MMA N)
  static constexpr uint32_t kBChunkBytes = kTileN * kBK * 2;     // 32 or 16 KB
  static constexpr uint32_t kBExtBytes = kTileN * kExt * 2;      // 8 or 4 KB
  static constexpr uint32_t kStageBytes = kBChunkBytes + kBExtBytes;
};

// Threads of a CTA whose epilogue has `epq` warps per TMEM lane quarter and
// which computes `qt` query tiles: the producer warp, one MMA warp per query
// tile (the second after the epilogue warps) and 4 * epq epilogue warps.
constexpr int warps_for(int epq, int qt) { return 1 + qt + 4 * epq; }
constexpr int threads_for(int epq, int qt) { return 32 * warps_for(epq, qt); }
// Registers per thread above which the CTA's warps cannot share one SM (the
// sub-partition holding the most warps has 16,384 registers).
constexpr int max_regs_for(int epq, int qt) {
  return (16384 / (32 * ((warps_for(epq, qt) + 3) / 4))) / 8 * 8 > 255
             ? 255
             : (16384 / (32 * ((warps_for(epq, qt) + 3) / 4))) / 8 * 8;
}
constexpr uint32_t kAccCols = kTcRefTile;  // FP32 columns per accumulator (one step)
constexpr uint32_t kTmemCols = 2 * kAccCols;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per wait

// Shared-memory layout of one CTA: QT query tiles (each AChunks
// 128-byte-swizzle chunks + the 32-byte-swizzle extension), the reference
// ring (Stages stages, each room for one K-chunk of a reference tile and its
// extension), the mbarriers, the TMEM address, abort flag and work-item
// slots, and ListBytes for an epilogue that keeps its lists in shared memory.
template <int AChunks, int Stages, uint32_t ListBytes, int QT>
struct Layout {
  using S = Shape<QT>;
  static constexpr int kStages = Stages;
  static constexpr uint32_t kAQueryBytes = AChunks * kAChunkBytes + 1024 * ((kAExtBytes + 1023) / 1024);
  static constexpr uint32_t kOffA = 0;  // query tile q at kOffA + q * kAQueryBytes; its extension after its chunks
  static constexpr uint32_t kOffB = QT * kAQueryBytes;
  static constexpr uint32_t kOffBar = kOffB + Stages * S::kStageBytes;
  // full, empty per stage; tmem full, tmem empty per accumulator; A full, A
  // empty, drain; item full, item empty per item slot; lists written
  static constexpr int kNumBars = 2 * Stages + 2 + 2 + 3 + 2 + 2 + 1;
  // TMEM address, abort flag, 2 item slots, 2 "an earlier split was not carried" words
  static constexpr uint32_t kOffMisc = kOffBar + 8 * kNumBars;
  static constexpr uint32_t kOffList = (kOffMisc + 48 + 1023) / 1024 * 1024;
  static constexpr uint32_t kSmemBytes = kOffList + ListBytes + 1024;  // + alignment slack
  static_assert(Stages % AChunks == 0, "a tile's chunks map to fixed stage parities");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

// Operand formats.  Either way one K-chunk is one 128-byte (swizzled) row
// per operand row and one MMA consumes 32 bytes of it.
struct FmtBf16 {  // exact search: 128 BF16 coordinates, two chunks
  static constexpr int kChunks = 2;
  static constexpr bool kExtFirst = false;
  template <int N>
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    mma_bf16(d, a, b, idesc_bf16_f32(kBM, N), acc);
  }
};
struct FmtE4m3 {  // coarse pass: 128 E4M3 coordinates, one chunk
  static constexpr int kChunks = 1;
  static constexpr bool kExtFirst = true;
  template <int N>
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    mma_f8(d, a, b, idesc_e4m3_f32(kBM, N), acc);
  }
};

template <int kStages>
struct Bars {
  uint32_t base;
  __device__ uint32_t full(int s) const { return base + 8 * s; }
  __device__ uint32_t empty(int s) const { return base + 8 * (kStages + s); }
  __device__ uint32_t tfull(int b) const { return base + 8 * (2 * kStages + b); }
  __device__ uint32_t tempty(int b) const { return base + 8 * (2 * kStages + 2 + b); }
  __device__ uint32_t afull() const { return base + 8 * (2 * kStages + 4); }
  __device__ uint32_t aempty() const { return base + 8 * (2 * kStages + 5); }
  __device__ uint32_t drain() const { return base + 8 * (2 * kStages + 6); }
  __device__ uint32_t ifull(int i) const { return base + 8 * (2 * kStages + 7 + i); }
  __device__ uint32_t iempty(int i) const { return base + 8 * (2 * kStages + 9 + i); }
  __device__ uint32_t lists_done() const { return base + 8 * (2 * kStages + 11); }
};

// The layout of a kernel instantiation: the format's query chunks; ring
// stages for two tiles of 256 references (BF16: four chunks, E4M3: two), as
// many as fit when the epilogue's lists take shared memory (BF16 two, E4M3
// three), and three or four times as many tiles of 128 references for QT = 2
// (BF16 six stages, E4M3 eight).
template <class Fmt, class Epilogue, int QT>
using LayoutOf = Layout<Fmt::kChunks,
                        QT == 2 ? (Fmt::kChunks == 2 ? 6 : 8)
                                : (Epilogue::kListBytes ? (Fmt::kChunks == 2 ? 2 : 3) : 4),
                        Epilogue::kListBytes, QT>;

__device__ __forceinline__ void flag_timeout(volatile uint32_t* abort_flag, uint32_t* dev_err) {
  *abort_flag = 1u;
  atomicOr(dev_err, kDevErrTimeout);
}

// Wait until the gate word is nonzero, for at most limit_ns, giving up early
// once another role of the CTA has given up.  Returns false on expiry.
__device__ __forceinline__ bool wait_gate(const uint32_t* gate, uint64_t limit_ns,
                                          const volatile uint32_t* abort_flag) {
  const volatile uint32_t* g = gate;
  if (*g != 0u) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (*g != 0u) return true;
    if ((it & 255u) == 0 && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) return false;
  }
}

// Sorted list of the K1 smallest (distance, row) pairs seen so far, held in
// registers: ascending in slots [KMAX-K1, KMAX); the slots below hold the
// distance -1, which no real distance displaces, so the list always has K1
// live entries and its largest is slot KMAX-1.  Every list receives its
// columns in increasing row order, so comparing distances strictly is exact
// for (distance, row) order: a later row at an equal distance sorts after.
template <int KMAX>
struct RegList {
  int32_t d[KMAX];
  uint32_t r[KMAX];

  __device__ __forceinline__ void init(int K1) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      d[i] = i < KMAX - K1 ? -1 : INT32_MAX;
      r[i] = 0xFFFFFFFFu;
    }
  }
  __device__ __forceinline__ int32_t worst() const { return d[KMAX - 1]; }
  // Start from a finished list of K1 ascending keys (kEmptyKey: no entry).
  __device__ __forceinline__ void seed(const uint64_t* src, int K1) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      if (i >= KMAX - K1) {
        const uint64_t k = __ldcg(src + (i - (KMAX - K1)));
        d[i] = k == kEmptyKey ? INT32_MAX : (int32_t)key_dist(k);
        r[i] = key_row(k);
      }
      // at most four keys in flight: the list itself holds the registers
      if ((i & 3) == 3) asm volatile("" ::: "memory");
    }
  }
  // new[i] = old[i-1] if x sorts before it, else min(x, old[i]); requires x < worst().
  __device__ __forceinline__ void insert(int32_t x, uint32_t row) {
#pragma unroll
    for (int i = KMAX - 1; i > 0; --i) {
      const bool shift = x < d[i - 1];
      const bool place = !shift && x < d[i];
      const int32_t nd = shift ? d[i - 1] : (place ? x : d[i]);
      const uint32_t nr = shift ? r[i - 1] : (place ? row : r[i]);
      d[i] = nd;
      r[i] = nr;
    }
    if (x < d[0]) {
      d[0] = x;
      r[0] = row;
    }
  }
  // Writes the K1 live entries ascending (unfilled slots as kEmptyKey).
  __device__ __forceinline__ void store(uint64_t* out, int K1) const {
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
      if (i >= KMAX - K1) out[i - (KMAX - K1)] = d[i] == INT32_MAX ? kEmptyKey : make_key((uint32_t)d[i], r[i]);
  }
};

// Bits of a non-negative float (or -0) as int32; ordered like the float.
__device__ __forceinline__ int32_t thr_bits(int32_t dist) { return __float_as_int((float)dist); }

// v[j] for a run-time j without dynamic register indexing (no local memory):
// a 5-level select tree on the bits of j.
__device__ __forceinline__ int32_t select32(const uint32_t (&v)[32], int j) {
  uint32_t t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = (j & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = (j & 2) ? t[2 * i + 1] : t[2 * i];
#pragma unroll
  for (int i = 0; i < 4; ++i) t[i] = (j & 4) ? t[2 * i + 1] : t[2 * i];
#pragma unroll
  for (int i = 0; i < 2; ++i) t[i] = (j & 8) ? t[2 * i + 1] : t[2 * i];
  return (int32_t)((j & 16) ? t[1] : t[0]);
}

// Bit j set when column j's distance is below the threshold.
__device__ __forceinline__ uint32_t hit_mask(const uint32_t (&v)[32], int32_t thr) {
  uint32_t mask = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) mask |= ((int32_t)v[j] < thr ? 1u : 0u) << j;
  return mask;
}

template <>
struct RegList<0> {
  __device__ __forceinline__ void init(int) {}
};

// KMAX > 0: per-row lists in registers (K1 <= KMAX); KMAX = 0: heaps in global memory.
// What the epilogue writes (see the two epilogues below).
struct ScanOut {
  uint64_t* lists;           // kNN: sorted lists, [splits * lists per split][stride][K1]
  int64_t stride;
  int K1;
  int32_t* mins;             // NBNN: per (query row, class) minimum distance, [m_pad][C], atomicMin
  int32_t C;
  const int64_t* class_off;  // NBNN: class c owns sorted rows [class_off[c], class_off[c+1])
  const uint32_t* gate;      // null, or a word the producer waits to see nonzero before loading
  int32_t* row_thr;          // kNN: per query row, a shared bound (below), or null
  bool bound_per_tile;       // row_thr read and published every tile, or at a work item's start and end
  uint32_t* done;            // kNN with splits run one after another: per work item, nonzero once its
                             // lists are written, 2 if they also hold every earlier split's keys (zero
                             // before the launch), or null
  int64_t T;                 // query-tile groups of the launch (work item w - T is the same rows' previous split)
  int lists_per_split;
};

// kNN epilogue: the K1 smallest (distance, row) keys of the columns one
// thread sees (Alg. 2's NN(d, k+1) restricted to a slice of the references).
//
// The lists (here and in KnnSmemEpilogue) share a bound per query row with the other lists of that row
// (the other column half, the other reference splits): row_thr[row] holds the
// bit pattern of a distance at or below which some list already holds K1
// entries, so a column farther than it cannot be among the row's K1 nearest
// and is not offered (a column at exactly the bound still is: it may win on
// its row).  When the lists of a row run at the same time (few query tiles,
// many splits), a full list publishes its K1-th distance with an atomic
// minimum after each tile that improved it, and reads the word once per tile
// (the read issued at the end of one tile is taken in at the end of the
// next).  When they run one after another (many query tiles: the splits of a
// row are work items far apart), a list reads the word once when it starts
// and publishes once when it ends.  Which columns a list drops depends on
// timing; the K1 nearest of the row never are, so the merged result does not.
template <int KMAX>
struct KnnEpilogue {
  static constexpr int kWarpsPerQuarter = KMAX == kTcWideRegListMax ? 1 : 2;
  static constexpr bool kSeeds = true;  // can start from the previous split's list of its rows
  static constexpr bool kClaimsChunks = true;  // can keep its lists across claimed reference chunks
  static constexpr uint32_t kListBytes = 0;
  RegList<KMAX> L;
  TopK top;
  int32_t thr;      // bit pattern of this list's K1-th distance (INT32_MAX's while not full)
  int32_t shared;   // the row's shared bound as last read (bit pattern)
  int32_t pending;  // the read in flight for the next tile
  int32_t* rthr;    // the row's shared bound, or null
  bool per_tile;    // share the bound every tile (else at start and end)
  bool active;
  int K1;
  uint64_t* out;
  __device__ __forceinline__ KnnEpilogue(const ScanOut& o, int list, int64_t row, bool act, int64_t, uint8_t*, int)
      : top(o.lists + ((int64_t)list * o.stride + (act ? row : 0)) * o.K1, o.K1),
        thr(thr_bits(INT32_MAX)),
        shared(kNoBound),
        pending(kNoBound),
        rthr(act && o.row_thr ? o.row_thr + row : nullptr),
        per_tile(o.bound_per_tile),
        active(act),
        K1(o.K1),
        out(o.lists + ((int64_t)list * o.stride + (act ? row : 0)) * o.K1) {
    L.init(K1);
    if (rthr && !per_tile) shared = __ldcg(rthr);
  }
  static constexpr int32_t kNoBound = 0x7F7F7F7F;  // the word's initial value: above every distance
  // One 32-column group: one compare of the group's minimum bit pattern (mn,
  // from the reducing TMEM load); on a hit, the columns below the limit are
  // offered in column order, each checked again as the limit tightens.  A
  // column at exactly the list's K1-th distance cannot enter: its row is
  // higher than every kept row's.
  __device__ __forceinline__ void group(const uint32_t (&v)[32], uint32_t mn, int64_t col0) {
    int32_t lim = min(thr, shared + 1);  // strictly below: own K1-th, at or below: the shared bound
    const bool hit = active && (int32_t)mn < lim;
    if (__any_sync(0xffffffffu, hit)) {
      if (hit) {
        for (uint32_t mask = hit_mask(v, lim); mask; mask &= mask - 1) {
          const int j = __ffs(mask) - 1;
          const int32_t bits = select32(v, j);
          if (bits < lim) {
            const int32_t d = __float2int_rn(__int_as_float(bits));
            if constexpr (KMAX > 0) {
              L.insert(d, (uint32_t)(col0 + j));
              thr = thr_bits(L.worst());
            } else {
              top.push(make_key((uint32_t)d, (uint32_t)(col0 + j)));
              thr = thr_bits(top.threshold);
            }
            lim = min(thr, shared + 1);
          }
        }
      }
      __syncwarp();
    }
  }
  // Start from the same rows' finished list of the previous split (K1
  // ascending keys of lower reference rows than any column to come, so the
  // strict distance tests keep exact (distance, row) order): the list then
  // holds the best keys so far and offers only columns that improve on them.
  __device__ __forceinline__ void seed(const uint64_t* src) {
    if (!active) return;
    if constexpr (KMAX > 0) {
      L.seed(src, K1);
      thr = thr_bits(L.worst());
    } else {
      for (int i = 0; i < K1; ++i) {
        const uint64_t k = __ldcg(src + i);
        if (k != kEmptyKey) top.push(k);
      }
      thr = thr_bits(top.threshold);
    }
  }
  __device__ __forceinline__ bool full() const {
    if constexpr (KMAX > 0) {
      return L.worst() != INT32_MAX;
    } else {
      return top.size == top.cap;
    }
  }
  // After each tile: publish an improved K1-th distance of a full list, take
  // in the bound read a tile ago (its latency hidden behind a whole tile), and
  // start the next read.
  __device__ __forceinline__ void tile_end() {
    if (rthr && per_tile) {
      if (full() && thr < shared) {
        atomicMin(rthr, thr);
        shared = thr;
      }
      shared = min(shared, pending);
      pending = __ldcg(rthr);
    }
  }
  __device__ __forceinline__ void finish() {
    if (!active) return;
    if (rthr && !per_tile && full() && thr < shared) atomicMin(rthr, thr);
    if constexpr (KMAX > 0) {
      L.store(out, K1);
    } else {
      top.finish();
    }
  }
};

// kNN epilogue with the lists in shared memory, for lists of up to KM = 64
// entries on the one-warp-per-quarter layout (register lists that long leave
// the insert as the bottleneck: a 64-wide insertion network per list and
// only four warps to hide it).  Each epilogue warp keeps its 32 rows' lists
// in shared memory, list by list, as float bit patterns and rows, and inserts
// with the whole warp: lane i computes entries i and i + 32 of the list
// (shifted, the new key, or unchanged) from their predecessors, so an insert
// is a few instructions per lane whatever the list length.  Candidates are
// taken lane by lane (the lowest lane with a hit first) and, within a lane,
// in column order, so each list still receives its columns in increasing row
// order.
template <int KM>
struct KnnSmemEpilogue {
  static constexpr int kWarpsPerQuarter = 1;
  static constexpr bool kSeeds = false;
  static constexpr bool kClaimsChunks = false;
  static constexpr int kPerLane = KM / 32;  // list entries each lane computes in an insert
  static constexpr uint32_t kListBytes = 4 * kWarpsPerQuarter * 32 * KM * 8;
  static constexpr int32_t kInf = 0x7F800000;  // bits of +inf, above every distance
  static constexpr int32_t kNoBound = 0x7F7F7F7F;  // the shared bound's initial value
  static_assert(KM % 32 == 0 && KM <= 64, "entries i and i + 32 per lane");
  __device__ __forceinline__ void seed(const uint64_t*) {}
  uint32_t* D;  // this warp's lists: D[list * KM + i] bit patterns, R[list * KM + i] rows
  uint32_t* R;
  int32_t thr;      // bit pattern of this lane's list's K1-th entry
  int32_t shared;   // the row's shared bound as last read (as in KnnEpilogue)
  int32_t pending;  // the read in flight
  int32_t* rthr;    // the row's shared bound, or null
  bool per_tile;    // share the bound every tile (else at start and end)
  bool active;
  int K1;
  int lane;
  uint64_t* out;
  __device__ __forceinline__ KnnSmemEpilogue(const ScanOut& o, int list, int64_t row, bool act, int64_t,
                                             uint8_t* smem_list, int epi_warp)
      : D(reinterpret_cast<uint32_t*>(smem_list) + (size_t)epi_warp * 32 * KM * 2),
        R(D + 32 * KM),
        thr(kInf),
        shared(kNoBound),
        pending(kNoBound),
        rthr(act && o.row_thr ? o.row_thr + row : nullptr),
        per_tile(o.bound_per_tile),
        active(act),
        K1(o.K1),
        lane((int)(threadIdx.x & 31)),
        out(o.lists + ((int64_t)list * o.stride + (act ? row : 0)) * o.K1) {
    if (rthr && !per_tile) shared = __ldcg(rthr);
    __syncwarp();  // the previous work item's lists have been read out
    for (int l = 0; l < 32; ++l)
#pragma unroll
      for (int e = 0; e < kPerLane; ++e) {
        D[l * KM + e * 32 + lane] = (uint32_t)kInf;
        R[l * KM + e * 32 + lane] = 0xFFFFFFFFu;
      }
    __syncwarp();
  }
  // Insert (x, row) into list L; every lane takes part.  Requires x below the
  // list's K1-th entry.
  __device__ __forceinline__ void insert(int L, int32_t x, uint32_t row) {
    uint32_t* d = D + L * KM;
    uint32_t* r = R + L * KM;
    int32_t a[kPerLane];
    uint32_t ra[kPerLane];
#pragma unroll
    for (int e = 0; e < kPerLane; ++e) {
      a[e] = (int32_t)d[e * 32 + lane];
      ra[e] = r[e * 32 + lane];
    }
    int32_t nd[kPerLane];
#pragma unroll
    for (int e = 0; e < kPerLane; ++e) {
      // predecessor of entry e * 32 + lane: lane - 1 of the same half, or
      // lane 31 of the previous half for lane 0
      const int32_t up = __shfl_up_sync(0xffffffffu, a[e], 1);
      const uint32_t upr = __shfl_up_sync(0xffffffffu, ra[e], 1);
      int32_t b = up;
      uint32_t rb = upr;
      bool has_pred = lane > 0;
      if (e > 0) {
        const int32_t w = __shfl_sync(0xffffffffu, a[e - 1], 31);
        const uint32_t wr = __shfl_sync(0xffffffffu, ra[e - 1], 31);
        if (lane == 0) {
          b = w;
          rb = wr;
          has_pred = true;
        }
      }
      const bool shift = has_pred && x < b;
      const bool place = !shift && x < a[e];
      nd[e] = shift ? b : (place ? x : a[e]);
      const uint32_t nr = shift ? rb : (place ? row : ra[e]);
      if (e * 32 + lane < K1) {
        d[e * 32 + lane] = (uint32_t)nd[e];
        r[e * 32 + lane] = nr;
      }
    }
    // the list's new K1-th entry
    const int last = K1 - 1;
    int32_t v = nd[0];
#pragma unroll
    for (int e = 1; e < kPerLane; ++e)
      if ((last >> 5) == e) v = nd[e];
    const int32_t nt = __shfl_sync(0xffffffffu, v, last & 31);
    if (lane == L) thr = nt;
    __syncwarp();
  }
  __device__ __forceinline__ void group(const uint32_t (&v)[32], uint32_t mn, int64_t col0) {
    // strictly below the list's K1-th entry, at or below the row's shared bound
    const bool hit = active && (int32_t)mn < min(thr, shared + 1);
    if (!__any_sync(0xffffffffu, hit)) return;
    uint32_t mask = hit ? hit_mask(v, min(thr, shared + 1)) : 0u;
    for (;;) {
      const uint32_t who = __ballot_sync(0xffffffffu, mask != 0u);
      if (who == 0u) break;
      const int L = __ffs(who) - 1;
      const int j = mask ? __ffs(mask) - 1 : 0;
      const int32_t x = __shfl_sync(0xffffffffu, select32(v, j), L);
      const int jl = __shfl_sync(0xffffffffu, j, L);
      const int32_t tl = __shfl_sync(0xffffffffu, min(thr, shared + 1), L);
      if (lane == L) mask &= mask - 1;
      if (x < tl) insert(L, x, (uint32_t)(col0 + jl));  // warp-uniform
    }
  }
  // As in KnnEpilogue: publish a full list's improved K1-th entry, take in the
  // read from a tile ago, start the next one.
  __device__ __forceinline__ void tile_end() {
    if (rthr && per_tile) {
      if (thr != kInf && thr < shared) {
        atomicMin(rthr, thr);
        shared = thr;
      }
      shared = min(shared, pending);
      pending = __ldcg(rthr);
    }
  }
  __device__ __forceinline__ void finish() {
    __syncwarp();
    if (!active) return;
    if (rthr && !per_tile && thr != kInf && thr < shared) atomicMin(rthr, thr);
    for (int i = 0; i < K1; ++i) {
      const uint32_t bits = D[lane * KM + i];
      out[i] = (int32_t)bits == kInf ? kEmptyKey
                                      : make_key((uint32_t)__float2int_rn(__uint_as_float(bits)), R[lane * KM + i]);
    }
  }
};

// NBNN epilogue (Alg. 1's NN_C for every class C): the columns are the
// class-sorted references; each thread keeps the minimum over the current
// class and, when the class ends, folds it into mins[row][class] with an
// atomic minimum (other column slices and splits see other parts of the
// class).  All lanes of a warp see the same columns, so the class bookkeeping
// is uniform across the warp.
struct NbnnEpilogue {
  static constexpr int kWarpsPerQuarter = 2;
  static constexpr bool kSeeds = false;
  static constexpr bool kClaimsChunks = false;
  __device__ __forceinline__ void seed(const uint64_t*) {}
  static constexpr uint32_t kListBytes = 0;
  __device__ __forceinline__ void tile_end() {}
  int32_t* dst;          // mins + row * C
  const int64_t* class_off;
  int64_t n_ref;
  int32_t C;
  int32_t cls;           // class of the current column
  int64_t next;          // first row of the next class
  int32_t run;           // float bits of the running minimum over cls
  bool active;
  __device__ __forceinline__ NbnnEpilogue(const ScanOut& o, int, int64_t row, bool act, int64_t j_begin, uint8_t*,
                                          int)
      : dst(o.mins + (act ? row : 0) * (int64_t)o.C), class_off(o.class_off), n_ref(o.class_off[o.C]), C(o.C),
        run(INT32_MAX), active(act) {
    // class of j_begin: the last c with class_off[c] <= j_begin
    int32_t lo = 0, hi = C;
    while (lo + 1 < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (class_off[mid] <= j_begin) lo = mid; else hi = mid;
    }
    cls = lo;
    next = class_off[cls + 1];
  }
  __device__ __forceinline__ void flush() {
    if (active && run != INT32_MAX) atomicMin(dst + cls, __float2int_rn(__int_as_float(run)));
    run = INT32_MAX;
  }
  __device__ __forceinline__ void group(const uint32_t (&v)[32], uint32_t mn, int64_t col0) {
    if (col0 + 32 <= next) {  // the whole group lies in class cls
      run = min(run, (int32_t)mn);
      return;
    }
#pragma unroll 1
    for (int j = 0; j < 32; ++j) {
      const int64_t col = col0 + j;
      if (col >= n_ref) return;  // padding rows past the last class
      while (col >= next) {      // class boundaries (empty classes skipped)
        flush();
        ++cls;
        next = class_off[cls + 1];
      }
      run = min(run, select32(v, j));
    }
  }
  __device__ __forceinline__ void finish() { flush(); }
};

// The work of one launch: T query-tile groups (QT query tiles each) x S
// reference splits = n_items items; item w is group w % T of split w / T
// (split-major, so the CTAs that run at the same time scan the same split and
// L2 serves its tiles to all of them).  queue == null: one CTA per item,
// item = blockIdx.x.  Otherwise a persistent grid: each CTA's producer takes
// the next item from *queue (zero at launch) with an atomic add and hands it
// to the CTA's other roles through a two-slot ring in shared memory; no CTA
// ever waits for another.
struct Work {
  int64_t T;
  int64_t n_items;
  int64_t split_len;
  uint32_t* queue;
  // 0: work items are (query-tile group, reference split) pairs.  > 0 (the
  // claimed-chunk form, persistent): `group` CTAs serve each query-tile
  // group, CTA c the group c / group; each keeps that group's query tiles
  // and its lists for the whole launch and claims reference chunks of
  // split_len rows, in increasing order, from the group's counter
  // queue[c / group]; n_items is then the number of chunks.
  int group;
};

// Claim: the claimed-chunk form (Work::group > 0), a separate instantiation
// so that the split form's kernels carry none of its code.
template <class Fmt, class Epilogue, int QT, bool Claim>
__global__ void __launch_bounds__(threads_for(Epilogue::kWarpsPerQuarter, QT), 1)
    tc_scan_kernel(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_qe,
                   const __grid_constant__ CUtensorMap tmap_r, const __grid_constant__ CUtensorMap tmap_re, int64_t m,
                   int64_t n_ref, Work work, ScanOut out, uint32_t* __restrict__ dev_err,
                   unsigned long long* __restrict__ stats) {
  using Sh = Shape<QT>;
  constexpr int KC = Fmt::kChunks;
  constexpr int kTileN = Sh::kTileN;
  using L = LayoutOf<Fmt, Epilogue, QT>;
  constexpr int kStages = L::kStages;
  // The epilogue learns that a tile's MMAs are done from the commit that
  // frees the tile's last ring stage, where that stage is not reused within
  // two tiles (its next phase then needs this tile's accumulator back, so a
  // parity wait cannot miss a phase); a separate accumulator-full commit per
  // tile cost the MMA thread 2-10% of a step.  With a two-stage ring the
  // stage comes back within a tile and the separate commit stays.
  constexpr bool kStageSignalsTile = kStages >= 2 * KC;
  constexpr int kEpiPerQuarter = Epilogue::kWarpsPerQuarter;  // epilogue warps per TMEM lane quarter
  constexpr int kEpiWarps = 4 * kEpiPerQuarter;
  constexpr int kEpiCols = kAccCols / kEpiPerQuarter;  // accumulator columns per epilogue warp
  constexpr int kRounds = kEpiCols / 64;               // rounds of two 32-column loads per tile
  static_assert(QT == 1 || kEpiPerQuarter == 2, "two query tiles need one epilogue warp per tile and quarter");
  static_assert(KC <= kKChunks, "the query tile fits the chunks shared memory is laid out for");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const Bars<kStages> bars{sbase + L::kOffBar};
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffMisc);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  volatile int64_t* item_slot = reinterpret_cast<volatile int64_t*>(smem + L::kOffMisc + 16);
  volatile uint32_t* chain_broken = reinterpret_cast<volatile uint32_t*>(smem + L::kOffMisc + 32);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool persistent = work.queue != nullptr;
  // MMA issuers: one thread per query tile (warp 1, and for QT = 2 the warp
  // after the epilogue warps), each issuing its tile's MMAs into its half of
  // the accumulator, so that no single thread issues all of a step's MMAs.
  constexpr int kIssuers = QT;
  constexpr int kSecondIssuerWarp = 2 + kEpiWarps;
  const bool issuer = warp == 1 || (kIssuers == 2 && warp == kSecondIssuerWarp);
  // A timeout reported earlier and not yet collected by lnbnn_sync: scan no
  // tiles (every item's lists are still written, empty).
  const bool stale_timeout = (*reinterpret_cast<volatile uint32_t*>(dev_err) & kDevErrTimeout) != 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), kIssuers);  // the MMA completions that free the stage
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars.tfull(b), kIssuers);
      mbar_init(bars.tempty(b), kEpiWarps);  // one arrival per epilogue warp
      mbar_init(bars.ifull(b), 1);
      mbar_init(bars.iempty(b), kIssuers + kEpiWarps);  // the MMA threads and each epilogue warp
    }
    mbar_init(bars.afull(), 1);
    mbar_init(bars.aempty(), kIssuers);
    mbar_init(bars.drain(), kIssuers);
    mbar_init(bars.lists_done(), kEpiWarps);
    *abort_flag = 0u;
    chain_broken[0] = chain_broken[1] = 0u;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // Item i of this CTA for the MMA and epilogue roles (the producer publishes
  // it in the persistent form); n_items means no more work.
  auto consume_item = [&](int i, int64_t* w) -> bool {
    if (!persistent) {
      *w = i == 0 ? (int64_t)blockIdx.x : work.n_items;
      return true;
    }
    const int slot = i & 1;
    if (!mbar_wait(bars.ifull(slot), (uint32_t)((i >> 1) & 1), kWaitLimitNs, abort_flag)) return false;
    *w = item_slot[slot];
    return true;
  };
  static_assert(!Claim || (QT == 1 && Epilogue::kClaimsChunks), "the claimed-chunk form: one query tile per CTA, kNN lists");
  constexpr bool chunked = Claim;
  auto item_tiles = [&](int64_t w, int64_t* m0, int64_t* j_begin) -> int {
    const int64_t x = chunked ? (int64_t)blockIdx.x / work.group : w % work.T;
    const int64_t y = chunked ? w : w / work.T;
    *m0 = x * (int64_t)(kBM * QT);
    *j_begin = y * work.split_len;
    const int64_t j_end = min(*j_begin + work.split_len, n_ref);
    return stale_timeout ? 0 : (int)((j_end - *j_begin + kTileN - 1) / kTileN);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      // an optional start gate; with nothing loaded the other roles' waits
      // run out on the abort flag
      bool go = true;
      if (out.gate != nullptr && !stale_timeout && !wait_gate(out.gate, kWaitLimitNs, abort_flag)) {
        flag_timeout(abort_flag, dev_err);
        go = false;
      }
      prefetch_tmap(&tmap_q);
      prefetch_tmap(&tmap_qe);
      prefetch_tmap(&tmap_r);
      prefetch_tmap(&tmap_re);
      int it = 0;       // reference K-chunks issued
      int a_loads = 0;  // query tiles issued
      for (int i = 0; go; ++i) {
        int64_t w;
        if (persistent) {
          const int slot = i & 1;
          if (i >= 2 && !mbar_wait(bars.iempty(slot), (uint32_t)(((i >> 1) - 1) & 1), kWaitLimitNs, abort_flag)) {
            flag_timeout(abort_flag, dev_err);
            break;
          }
          w = *abort_flag ? work.n_items
                          : (int64_t)atomicAdd(work.queue + (chunked ? blockIdx.x / work.group : 0u), 1u);
          if (w > work.n_items) w = work.n_items;
          item_slot[slot] = w;
          mbar_arrive(bars.ifull(slot));
        } else {
          w = i == 0 ? (int64_t)blockIdx.x : work.n_items;
        }
        if (w >= work.n_items) break;
        int64_t m0, j_begin;
        const int ntiles = item_tiles(w, &m0, &j_begin);
        // the query tiles: once the previous item's MMAs have read theirs (in
        // the claimed-chunk form, once for the whole launch)
        if (!chunked || a_loads == 0) {
          if (a_loads > 0 && !mbar_wait(bars.aempty(), (uint32_t)((a_loads - 1) & 1), kWaitLimitNs, abort_flag)) {
            flag_timeout(abort_flag, dev_err);
            break;
          }
          mbar_arrive_expect_tx(bars.afull(), QT * (KC * kAChunkBytes + kAExtBytes));
          for (int q = 0; q < QT; ++q) {
            const uint32_t a = sbase + L::kOffA + q * L::kAQueryBytes;
            const int32_t qrow = (int32_t)(m0 + q * kBM);
            for (int kc = 0; kc < KC; ++kc) tma_load_2d(a + kc * kAChunkBytes, &tmap_q, kc * kBK, qrow, bars.afull());
            tma_load_2d(a + KC * kAChunkBytes, &tmap_qe, 0, qrow, bars.afull());
          }
          ++a_loads;
        }
        bool ok = true;
        for (int t = 0; ok && t < ntiles && !*abort_flag; ++t) {
          const int32_t row = (int32_t)(j_begin + (int64_t)t * kTileN);
          for (int kc = 0; kc < KC; ++kc, ++it) {
            const int s = it % kStages;
            const uint32_t round = (uint32_t)(it / kStages);
            if (!mbar_wait(bars.empty(s), (round & 1u) ^ 1u, kWaitLimitNs, abort_flag)) {
              flag_timeout(abort_flag, dev_err);
              ok = false;
              break;
            }
            const uint32_t dst = sbase + L::kOffB + s * Sh::kStageBytes;
            const bool last = kc == KC - 1;
            mbar_arrive_expect_tx(bars.full(s), Sh::kBChunkBytes + (last ? Sh::kBExtBytes : 0u));
            tma_load_2d(dst, &tmap_r, kc * kBK, row, bars.full(s));
            if (last) tma_load_2d(dst + Sh::kBChunkBytes, &tmap_re, 0, row, bars.full(s));
          }
        }
        if (!ok || *abort_flag) break;
      }
      // every load issued must land before the CTA may exit
      const uint32_t never = 0;
      if (a_loads > 0) mbar_wait(bars.afull(), (uint32_t)((a_loads - 1) & 1), kWaitLimitNs, &never);
      for (int s = 0; s < kStages; ++s) {
        const int issued = it / kStages + (s < it % kStages ? 1 : 0);
        if (issued > 0) mbar_wait(bars.full(s), (uint32_t)((issued - 1) & 1), kWaitLimitNs, &never);
      }
    }
  } else if (issuer) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issuers
      const int q_first = kIssuers == QT ? (warp == 1 ? 0 : 1) : 0;  // this thread's query tiles
      const int q_last = kIssuers == QT ? q_first + 1 : QT;
      const long long clk0 = clock64();
      const uint64_t ns0 = globaltimer_ns();
      int it = 0;       // reference K-chunks consumed
      int tg = 0;       // tiles over all items (accumulator use)
      int64_t tiles_done = 0;
      bool ok = true;
      for (int i = 0; ok; ++i) {
        int64_t w;
        if (!consume_item(i, &w)) {
          flag_timeout(abort_flag, dev_err);
          break;
        }
        if (w >= work.n_items) break;
        int64_t m0, j_begin;
        const int ntiles = item_tiles(w, &m0, &j_begin);
        if ((!chunked || i == 0) && !mbar_wait(bars.afull(), (uint32_t)(i & 1), kWaitLimitNs, abort_flag)) {
          flag_timeout(abort_flag, dev_err);
          break;
        }
        tc_fence_after();
        // no abort-flag read per tile here: shared-memory loads are slow on
        // this thread while the MMAs stream their operands (the per-tile
        // read cost 2% of the FP8 pass), and a role that gives up stops
        // completing barriers, so the next wait below sees the flag
        for (int t = 0; ok && t < ntiles; ++t, ++tg) {
          const int b = tg & 1;
          const uint32_t use = (uint32_t)(tg >> 1);
          if (!mbar_wait(bars.tempty(b), (use & 1u) ^ 1u, kWaitLimitNs, abort_flag)) {
            flag_timeout(abort_flag, dev_err);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + b * kAccCols;
          for (int kc = 0; kc < KC; ++kc, ++it) {
            const int s = it % kStages;
            const uint32_t round = (uint32_t)(it / kStages);
            if (!mbar_wait(bars.full(s), round & 1u, kWaitLimitNs, abort_flag)) {
              flag_timeout(abort_flag, dev_err);
              ok = false;
              break;
            }
            tc_fence_after();
            // descriptors are built once per stage and advanced by adding the
            // byte offset >> 4 to their start-address field (14 bits of
            // addr >> 4; every shared address is below 256 KB, so the sum
            // never carries out of the field): the MMA thread's issue loop is
            // on the critical path of the N = 128 shape, which issues twice
            // as many MMAs per step
            const uint32_t b_base = sbase + L::kOffB + s * Sh::kStageBytes;
            const uint64_t b_desc = sw128_kmajor_desc(b_base);
            const uint64_t b_ext = sw32_kmajor_desc(b_base + Sh::kBChunkBytes);
            const bool last = kc == KC - 1;  // the norms' K-extension rides with the last chunk
#pragma unroll
            for (int q = 0; q < QT; ++q) {
              if (q < q_first || q >= q_last) continue;
              const uint32_t a_q = sbase + L::kOffA + q * L::kAQueryBytes;
              const uint64_t a_desc = sw128_kmajor_desc(a_q) + (uint64_t)((kc * kAChunkBytes) >> 4);
              const uint64_t a_ext = sw32_kmajor_desc(a_q + KC * kAChunkBytes);
              const uint32_t d_q = d_tmem + q * kTileN;
              if (Fmt::kExtFirst && last) mma_bf16(d_q, a_ext, b_ext, idesc_bf16_f32(kBM, kTileN), kc != 0 ? 1u : 0u);
#pragma unroll
              for (int kk = 0; kk < kMmaPerChunk; ++kk)  // K-steps of 32 bytes
                Fmt::template mma<kTileN>(d_q, a_desc + (uint64_t)(2 * kk), b_desc + (uint64_t)(2 * kk),
                                          (kc | kk) != 0 || (Fmt::kExtFirst && last) ? 1u : 0u);
              if (!Fmt::kExtFirst && last) mma_bf16(d_q, a_ext, b_ext, idesc_bf16_f32(kBM, kTileN), 1u);
            }
            mma_commit(bars.empty(s));  // the producer may refill this stage
          }
          if constexpr (!kStageSignalsTile) {
            if (ok) mma_commit(bars.tfull(b));
          }
        }
        tiles_done += ntiles;
        if (!chunked) mma_commit(bars.aempty());  // the query tiles may be replaced once these MMAs are done
        if (persistent) mbar_arrive(bars.iempty(i & 1));
      }
      // all MMAs issued by this thread must finish before TMEM is released
      const uint32_t never = 0;
      mma_commit(bars.drain());
      mbar_wait(bars.drain(), 0, kWaitLimitNs, &never);
      if (stats && warp == 1) {
        atomicAdd(stats + 0, (unsigned long long)(clock64() - clk0));
        atomicAdd(stats + 1, (unsigned long long)(globaltimer_ns() - ns0));
        atomicAdd(stats + 2, (unsigned long long)tiles_done);
        atomicAdd(stats + 3, 1ull);
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int quarter = warp & 3;          // this warp may read TMEM lanes [32*quarter, 32*quarter+32)
    const int half = (warp - 2) >> 2;      // QT = 1: its column half of every tile; QT = 2: its query tile
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    int tg = 0;
    // the tiles of one work item into the lists of `e`; false if a wait ran out
    auto scan_tiles = [&](auto& e, int ntiles, int64_t col_base) -> bool {
      for (int t = 0; t < ntiles; ++t, ++tg) {
        const int b = tg & 1;
        bool done;
        if constexpr (kStageSignalsTile) {
          const int itl = tg * KC + KC - 1;  // the tile's last K-chunk
          done = mbar_wait(bars.empty(itl % kStages), (uint32_t)(itl / kStages) & 1u, kWaitLimitNs, abort_flag);
        } else {
          done = mbar_wait(bars.tfull(b), (uint32_t)(tg >> 1) & 1u, kWaitLimitNs, abort_flag);
        }
        if (!done) {
          flag_timeout(abort_flag, dev_err);
          return false;
        }
        tc_fence_after();
        // rounds of 64 columns; the accumulator goes back as soon as the last
        // round is in registers
        const uint32_t taddr = tmem_base + lane_addr + b * kAccCols + half * kEpiCols;
        const int64_t col0 = col_base + (int64_t)t * kTileN;
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
          uint32_t v0[32], v1[32], mn0, mn1;
          tmem_ld_min_32x32b_x32(taddr + 64 * r, v0, mn0);
          tmem_ld_min_32x32b_x32(taddr + 64 * r + 32, v1, mn1);
          tmem_ld_wait(v0, mn0);
          reg_fence(v1);
          asm volatile("" : "+r"(mn1));
          if (r == kRounds - 1) {
            // every lane's loads are complete (waited above); one arrival
            // per warp after a warp barrier (256 single-thread arrivals on
            // one barrier, while the MMAs read their operands from shared
            // memory, delayed the accumulator's return by ~100 cycles a step)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.tempty(b));
          }
          e.group(v0, mn0, col0 + 64 * r);
          e.group(v1, mn1, col0 + 64 * r + 32);
        }
        e.tile_end();
      }
      return true;
    };
    if constexpr (Claim) {
      {
        // claimed-chunk form: one query-tile group and one set of lists for
        // the whole launch (list = this CTA's rank in the group's CTAs x the
        // lists per CTA), written once every claimed chunk is scanned
        const int rank = (int)(blockIdx.x % (unsigned)work.group);
        const int64_t row =
            (int64_t)(blockIdx.x / (unsigned)work.group) * (kBM * QT) + (QT == 2 ? half * kBM : 0) + quarter * 32 + lane;
        const int64_t c_off = QT == 2 ? 0 : half * kEpiCols;
        const int list = QT == 2 ? rank : rank * kEpiPerQuarter + half;
        const bool active = row < m;
        Epilogue epi(out, list, row, active, c_off, smem + L::kOffList, warp - 2);
        for (int i = 0;; ++i) {
          int64_t w;
          if (!consume_item(i, &w)) {
            flag_timeout(abort_flag, dev_err);
            break;
          }
          if (w >= work.n_items) break;
          int64_t m0, j_begin;
          const int ntiles = item_tiles(w, &m0, &j_begin);
          if (!scan_tiles(epi, ntiles, j_begin + c_off)) break;
          __syncwarp();
          if (lane == 0) mbar_arrive(bars.iempty(i & 1));
        }
        epi.finish();
      }
    }
    for (int i = 0; !chunked; ++i) {
      int64_t w;
      if (!consume_item(i, &w)) {
        flag_timeout(abort_flag, dev_err);
        break;
      }
      if (w >= work.n_items) break;
      int64_t m0, j_begin;
      const int ntiles = item_tiles(w, &m0, &j_begin);
      const int64_t y = w / work.T;
      const int64_t row = m0 + (QT == 2 ? half * kBM : 0) + quarter * 32 + lane;
      const int64_t c_off = QT == 2 ? 0 : half * kEpiCols;  // this warp's first column within a tile
      const int list = QT == 2 ? (int)y : (int)y * kEpiPerQuarter + half;
      const bool active = row < m;
      Epilogue epi(out, list, row, active, j_begin + c_off, smem + L::kOffList, warp - 2);
      // the previous split of these rows, if it has finished: start from its
      // list.  Its flag says 2 when every earlier split of the rows was
      // carried into it; a warp that cannot say the same of this item marks
      // the item's slot (cleared by the thread that publishes the slot's
      // previous item before that item's slot is released)
      if (Epilogue::kSeeds && out.done != nullptr) {
        const uint32_t prev = y > 0 && ntiles > 0 ? ld_acquire_gpu(out.done + (w - out.T)) : 0u;
        if (prev != 0u)
          epi.seed(out.lists + ((int64_t)(list - out.lists_per_split) * out.stride + (active ? row : 0)) * out.K1);
        if (lane == 0 && y > 0 && prev != 2u) chain_broken[i & 1] = 1u;
      }
      const bool ok = scan_tiles(epi, ntiles, j_begin + c_off);
      epi.finish();
      if (Epilogue::kSeeds && out.done != nullptr) {
        // this item's lists are complete once every epilogue warp has written
        // its rows' lists; one thread then marks the item done: 2 if its
        // lists hold every earlier split's keys (each split of the rows
        // started from the one before), else 1 (if the wait runs out nothing
        // is marked and a later split simply starts empty)
        __threadfence();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars.lists_done());
        if (warp == 2 && lane == 0 && ok &&
            mbar_wait(bars.lists_done(), (uint32_t)(i & 1), kWaitLimitNs, abort_flag)) {
          // the item index again (from its slot, which the producer refills
          // only after this warp's release below), not kept live across the tiles
          const int64_t wd = persistent ? item_slot[i & 1] : (int64_t)blockIdx.x;
          const uint32_t flag = chain_broken[i & 1] != 0u ? 1u : 2u;
          chain_broken[i & 1] = 0u;
          __threadfence();
          st_release_gpu(out.done + wd, flag);
        }
      }
      if (!ok) break;
      if (persistent) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bars.iempty(i & 1));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// BF16 [rows, cols] row-major, boxes of box_cols x box_rows with the given swizzle.
bool encode_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint32_t cols, uint32_t box_cols,
                 uint32_t box_rows, CUtensorMapSwizzle swizzle) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// E4M3 bytes [rows, 128] row-major, boxes of 128 x box_rows, 128-byte swizzle.
bool encode_e4m3(CUtensorMap* map, const void* base, uint64_t rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)kDim, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kDim};
  cuuint32_t box[2] = {(cuuint32_t)kDim, box_rows};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), gdim, gstride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Main operand (128 K-columns, 64-column boxes, 128-byte swizzle) and its
// 16-column K-extension (32-byte swizzle).
bool encode_operand(CUtensorMap* main, CUtensorMap* ext, const void* bf, const void* ext_base, uint64_t rows,
                    uint32_t box_rows) {
  return encode_bf16(main, bf, rows, kDim, kBK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B) &&
         encode_bf16(ext, ext_base, rows, kExt, kExt, box_rows, CU_TENSOR_MAP_SWIZZLE_32B);
}

}  // namespace

bool make_tc_tensor_maps(const __nv_bfloat16* ref_bf, const __nv_bfloat16* sref_bf, const __nv_bfloat16* ref_ext,
                         const __nv_bfloat16* sref_ext, int64_t n_pad, TcTensorMaps* out) {
  return encode_operand(&out->ref, &out->ref_ext, ref_bf, ref_ext, (uint64_t)n_pad, Shape<1>::kTileN) &&
         encode_operand(&out->sref, &out->sref_ext, sref_bf, sref_ext, (uint64_t)n_pad, Shape<1>::kTileN) &&
         encode_operand(&out->ref_h, &out->ref_ext_h, ref_bf, ref_ext, (uint64_t)n_pad, Shape<2>::kTileN) &&
         encode_operand(&out->sref_h, &out->sref_ext_h, sref_bf, sref_ext, (uint64_t)n_pad, Shape<2>::kTileN);
}

bool make_tc_tensor_maps_e4m3(const uint8_t* ref_f8, const __nv_bfloat16* ref_f8_ext, int64_t n_pad,
                              TcTensorMaps* out) {
  return encode_e4m3(&out->f8, ref_f8, (uint64_t)n_pad, Shape<1>::kTileN) &&
         encode_bf16(&out->f8_ext, ref_f8_ext, (uint64_t)n_pad, kExt, kExt, Shape<1>::kTileN,
                     CU_TENSOR_MAP_SWIZZLE_32B) &&
         encode_e4m3(&out->f8_h, ref_f8, (uint64_t)n_pad, Shape<2>::kTileN) &&
         encode_bf16(&out->f8_ext_h, ref_f8_ext, (uint64_t)n_pad, kExt, kExt, Shape<2>::kTileN,
                     CU_TENSOR_MAP_SWIZZLE_32B);
}

namespace {

template <class Fmt, class Epilogue, int QT>
cudaError_t launch_scan(const CUtensorMap& tr, const CUtensorMap& tre, const void* qop,
                        const __nv_bfloat16* qext, int64_t m, int64_t m_pad, int64_t n_ref, int splits,
                        int64_t split_len, const ScanOut& out, uint32_t* dev_err, unsigned long long* stats,
                        const TcSched& sched, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  if (m_pad % kBM != 0 || split_len % kTcRefTile != 0 || splits < 1) return cudaErrorInvalidValue;
  if (sched.persistent_ctas > 0 && sched.queue == nullptr) return cudaErrorInvalidValue;
  CUtensorMap tq, tqe;
  const bool ok = Fmt::kChunks == 1
                      ? encode_e4m3(&tq, qop, (uint64_t)m_pad, kBM) &&
                            encode_bf16(&tqe, qext, (uint64_t)m_pad, kExt, kExt, kBM, CU_TENSOR_MAP_SWIZZLE_32B)
                      : encode_operand(&tq, &tqe, qop, qext, (uint64_t)m_pad, kBM);
  if (!ok) return cudaErrorInvalidValue;
  Work work;
  work.T = (m_pad + kBM * QT - 1) / (kBM * QT);
  work.n_items = work.T * splits;
  work.split_len = split_len;
  work.queue = sched.persistent_ctas > 0 ? sched.queue : nullptr;
  work.group = 0;
  ScanOut o = out;
  o.done = splits > 1 ? sched.done : nullptr;
  o.T = work.T;
  o.lists_per_split = QT == 2 ? 1 : Epilogue::kWarpsPerQuarter;
  int64_t grid = work.queue ? std::min<int64_t>(work.n_items, sched.persistent_ctas) : work.n_items;
  if (sched.group > 0) {
    // the claimed-chunk form: `splits` is the CTAs per query-tile group (the
    // lists' "split" index is the CTA's rank), split_len the chunk length
    if (!Epilogue::kClaimsChunks || sched.queue == nullptr || o.done != nullptr || sched.group != splits)
      return cudaErrorInvalidValue;
    work.group = sched.group;
    work.queue = sched.queue;
    work.n_items = (n_ref + split_len - 1) / split_len;
    grid = work.T * sched.group;
  }
  if (work.n_items > (int64_t)INT32_MAX || grid > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  if constexpr (QT == 1 && Epilogue::kClaimsChunks) {
    if (work.group > 0) {
      tc_scan_kernel<Fmt, Epilogue, QT, true>
          <<<(unsigned)grid, threads_for(Epilogue::kWarpsPerQuarter, QT), LayoutOf<Fmt, Epilogue, QT>::kSmemBytes,
             s>>>(tq, tqe, tr, tre, m, n_ref, work, o, dev_err, stats);
      return cudaGetLastError();
    }
  }
  if (work.group > 0) return cudaErrorInvalidValue;
  tc_scan_kernel<Fmt, Epilogue, QT, false>
      <<<(unsigned)grid, threads_for(Epilogue::kWarpsPerQuarter, QT), LayoutOf<Fmt, Epilogue, QT>::kSmemBytes, s>>>(
          tq, tqe, tr, tre, m, n_ref, work, o, dev_err, stats);
  return cudaGetLastError();
}

template <class Fmt, class Epilogue, int QT, bool Claim>
cudaError_t prepare_kernel() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, tc_scan_kernel<Fmt, Epilogue, QT, Claim>);
  if (e != cudaSuccess) return e;
  if (a.numRegs > max_regs_for(Epilogue::kWarpsPerQuarter, QT)) return cudaErrorInvalidKernelImage;
  return cudaFuncSetAttribute(tc_scan_kernel<Fmt, Epilogue, QT, Claim>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)LayoutOf<Fmt, Epilogue, QT>::kSmemBytes);
}

template <class Fmt, class Epilogue, int QT>
cudaError_t prepare_one() {
  cudaError_t e = prepare_kernel<Fmt, Epilogue, QT, false>();
  if constexpr (QT == 1 && Epilogue::kClaimsChunks) {
    if (e == cudaSuccess) e = prepare_kernel<Fmt, Epilogue, QT, true>();
  }
  return e;
}

// One list kind's kernel for the tile shape the schedule asks for (two query
// tiles per CTA only where the epilogue has two warps per lane quarter).
template <class Fmt, class Epilogue>
cudaError_t launch_shape(const TcTensorMaps& maps, bool sorted_copy, const void* qop, const __nv_bfloat16* qext,
                         int64_t m, int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, const ScanOut& out,
                         uint32_t* dev_err, unsigned long long* stats, const TcSched& sched, cudaStream_t s) {
  constexpr bool coarse = Fmt::kChunks == 1;
  if constexpr (Epilogue::kWarpsPerQuarter == 2) {
    if (sched.qt == 2) {
      const CUtensorMap& tr = coarse ? maps.f8_h : (sorted_copy ? maps.sref_h : maps.ref_h);
      const CUtensorMap& tre = coarse ? maps.f8_ext_h : (sorted_copy ? maps.sref_ext_h : maps.ref_ext_h);
      return launch_scan<Fmt, Epilogue, 2>(tr, tre, qop, qext, m, m_pad, n_ref, splits, split_len, out, dev_err,
                                           stats, sched, s);
    }
  }
  if (sched.qt != 1) return cudaErrorInvalidValue;
  const CUtensorMap& tr = coarse ? maps.f8 : (sorted_copy ? maps.sref : maps.ref);
  const CUtensorMap& tre = coarse ? maps.f8_ext : (sorted_copy ? maps.sref_ext : maps.ref_ext);
  return launch_scan<Fmt, Epilogue, 1>(tr, tre, qop, qext, m, m_pad, n_ref, splits, split_len, out, dev_err, stats,
                                       sched, s);
}

template <class Fmt, class Epilogue>
cudaError_t prepare_both() {
  cudaError_t e = prepare_one<Fmt, Epilogue, 1>();
  if constexpr (Epilogue::kWarpsPerQuarter == 2) {
    if (e == cudaSuccess) e = prepare_one<Fmt, Epilogue, 2>();
  }
  return e;
}

// The kNN scan with the list kind for K1 and the split length.
template <class Fmt>
cudaError_t launch_lists(const TcTensorMaps& maps, bool sorted_copy, const void* qop, const __nv_bfloat16* qext,
                         int64_t m, int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int K1,
                         const ScanOut& out, uint32_t* dev_err, unsigned long long* stats, const TcSched& sched,
                         cudaStream_t s) {
  switch (tc_list_kind(K1, split_len, Fmt::kChunks == 1)) {
    case ListKind::Reg16:
      return launch_shape<Fmt, KnnEpilogue<kTcRegListMax>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref, splits,
                                                           split_len, out, dev_err, stats, sched, s);
    case ListKind::Reg24:
      return launch_shape<Fmt, KnnEpilogue<kTcMidRegListMax>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref, splits,
                                                              split_len, out, dev_err, stats, sched, s);
    case ListKind::Reg32:
      return launch_shape<Fmt, KnnEpilogue<kTcCoarseRegListMax>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref,
                                                                 splits, split_len, out, dev_err, stats, sched, s);
    case ListKind::Smem64:
      return launch_shape<Fmt, KnnSmemEpilogue<kTcWideRegListMax>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref,
                                                                   splits, split_len, out, dev_err, stats, sched, s);
    case ListKind::Reg64:
      if constexpr (Fmt::kChunks == 2)
        return launch_shape<Fmt, KnnEpilogue<kTcWideRegListMax>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref,
                                                                 splits, split_len, out, dev_err, stats, sched, s);
      return cudaErrorInvalidValue;
    case ListKind::Heap:
      break;
  }
  return launch_shape<Fmt, KnnEpilogue<0>>(maps, sorted_copy, qop, qext, m, m_pad, n_ref, splits, split_len, out,
                                           dev_err, stats, sched, s);
}

}  // namespace

cudaError_t prepare_tc_kernels() {
  cudaError_t e = prepare_both<FmtBf16, KnnEpilogue<kTcRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, KnnEpilogue<kTcMidRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtE4m3, KnnEpilogue<kTcMidRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, KnnEpilogue<kTcCoarseRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, KnnSmemEpilogue<kTcWideRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, KnnEpilogue<kTcWideRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, KnnEpilogue<0>>();
  if (e == cudaSuccess) e = prepare_both<FmtBf16, NbnnEpilogue>();
  if (e == cudaSuccess) e = prepare_both<FmtE4m3, KnnEpilogue<kTcRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtE4m3, KnnEpilogue<kTcCoarseRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtE4m3, KnnSmemEpilogue<kTcWideRegListMax>>();
  if (e == cudaSuccess) e = prepare_both<FmtE4m3, KnnEpilogue<0>>();
  return e;
}

cudaError_t launch_knn_tc(const TcTensorMaps& maps, bool sorted_copy, const __nv_bfloat16* qbf,
                          const __nv_bfloat16* qext, int64_t m, int64_t m_pad, int64_t n_ref, int splits,
                          int64_t split_len, int K1, uint64_t* lists, int64_t stride, int32_t* row_thr,
                          uint32_t* dev_err, unsigned long long* stats, const uint32_t* gate, const TcSched& sched,
                          cudaStream_t s) {
  ScanOut out{};
  out.gate = gate;
  out.row_thr = row_thr;
  out.bound_per_tile = sched.bound_per_tile;
  out.lists = lists;
  out.stride = stride;
  out.K1 = K1;
  return launch_lists<FmtBf16>(maps, sorted_copy, qbf, qext, m, m_pad, n_ref, splits, split_len, K1, out, dev_err,
                               stats, sched, s);
}

cudaError_t launch_coarse_tc(const TcTensorMaps& maps, const uint8_t* qf8, const __nv_bfloat16* qext,
                             int64_t m, int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int K1,
                             uint64_t* lists, int64_t stride, int32_t* row_thr, uint32_t* dev_err,
                             unsigned long long* stats, const uint32_t* gate, const TcSched& sched, cudaStream_t s) {
  ScanOut out{};
  out.gate = gate;
  out.row_thr = row_thr;
  out.bound_per_tile = sched.bound_per_tile;
  out.lists = lists;
  out.stride = stride;
  out.K1 = K1;
  return launch_lists<FmtE4m3>(maps, false, qf8, qext, m, m_pad, n_ref, splits, split_len, K1, out, dev_err, stats,
                               sched, s);
}

cudaError_t launch_nbnn_tc(const TcTensorMaps& maps, const __nv_bfloat16* qbf, const __nv_bfloat16* qext, int64_t m,
                           int64_t m_pad, int64_t n_ref, int splits, int64_t split_len, int32_t* mins, int32_t C,
                           const int64_t* class_off, uint32_t* dev_err, unsigned long long* stats,
                           const uint32_t* gate, const TcSched& sched, cudaStream_t s) {
  ScanOut out{};
  out.gate = gate;
  out.mins = mins;
  out.C = C;
  out.class_off = class_off;
  return launch_shape<FmtBf16, NbnnEpilogue>(maps, true, qbf, qext, m, m_pad, n_ref, splits, split_len, out, dev_err,
                                             stats, sched, s);
}

}  // namespace lnbnn
