/*
 * lnbnn.h -- C ABI of the GB300 Local Naive Bayes Nearest Neighbor library.
 *
 * Method: McCann & Lowe, "Local Naive Bayes Nearest Neighbor for Image
 * Classification".  Original NBNN is Alg. 1 (Section 1) with the decision
 * rule of Eq. (eqn:nbnn) (Section 3); Local NBNN is Alg. 2 (Section 4).
 *
 * Conventions for every call:
 *   - Descriptors are 128-dimensional uint8, row-major, 128 bytes per row;
 *     an index made by lnbnn_index_create_located takes 130-byte rows (the
 *     128 appearance bytes, then a 2-byte location) for its references and
 *     for every query.
 *   - Unless a name ends in _host, every array argument is a DEVICE pointer
 *     (cudaMalloc / PyTorch CUDA storage) owned by the caller; the library
 *     never frees or keeps it beyond the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device calls are asynchronous on that stream: argument
 *     errors are returned at once; a device-side timeout is recorded in the
 *     index and returned by lnbnn_sync().  Until it is collected, search
 *     kernels of that index skip their work, so results of calls made between
 *     the timeout and lnbnn_sync() are invalid.
 *   - Distances are exact squared Euclidean distances of the raw uint8
 *     values (plus the weighted location term of a located index), as int32;
 *     totals are exact int64 sums.
 *   - Neighbours are ordered by (distance, reference row) ascending, so equal
 *     distances go to the lower row of the reference set given to create.
 *   - Calls without a workspace argument share the index's own workspace:
 *     issue them on one stream, or serialise them; two such calls on one
 *     index that overlap on the GPU race.  Calls that may overlap (several
 *     streams) each use their own lnbnn_workspace.
 *   - No call throws; every failure is a status code.
 */
#ifndef LNBNN_H
#define LNBNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LNBNN_API __attribute__((visibility("default")))
#else
#define LNBNN_API
#endif

#define LNBNN_DIM 128
/* row bytes of a located descriptor: 128 appearance bytes, then (x, y) */
#define LNBNN_LOCATED_DIM 130
/* largest location weight (keeps the tensor-core distances exact) */
#define LNBNN_MAX_LOCATION_WEIGHT 48
/* largest neighbourhood size k (the search keeps k + 1 neighbours) */
#define LNBNN_MAX_K 255

typedef struct lnbnn_index lnbnn_index;

typedef enum lnbnn_status {
  LNBNN_OK = 0,
  LNBNN_ERR_INVALID_ARG = 1,  /* null pointer, negative size, bad handle */
  LNBNN_ERR_LABEL_RANGE = 2,  /* a label outside [0, n_classes) */
  LNBNN_ERR_EMPTY_CLASS = 3,  /* a class with no reference (NN_C undefined) */
  LNBNN_ERR_K_RANGE = 4,      /* k < 1, k > LNBNN_MAX_K or k + 1 > n_ref */
  LNBNN_ERR_OOM = 5,          /* device allocation failed */
  LNBNN_ERR_CUDA = 6,         /* a CUDA runtime call or launch failed */
  LNBNN_ERR_TIMEOUT = 7,      /* a bounded device wait expired */
  LNBNN_ERR_UNSUPPORTED = 8,  /* device is not compute capability 10.3 (sm_103); FP8 on a located index */
  LNBNN_ERR_OFFSETS = 9,      /* offsets not 0 = o[0] <= ... <= o[n_images] = n_queries */
  LNBNN_ERR_SCRATCH_LIMIT = 10, /* problem larger than a workspace or the scratch of knn_search_noalloc */
  LNBNN_ERR_NO_FP8 = 11,        /* an FP8 call on an index without lnbnn_index_prepare_fp8 */
  LNBNN_ERR_IO = 12             /* a file could not be written or read, or is not an intact index file */
} lnbnn_status;

/*
 * Build the merged reference index of Alg. 2 ("a nearest neighbor index
 * comprising all descriptors" plus the class lookup Class(p), Section 4; the
 * class of each descriptor stored beside it, Section 5.1).  The same index
 * also serves original NBNN (Alg. 1), which needs NN_C for every class.
 *
 *   ref      device uint8 [n_ref * 128], row j = reference descriptor j
 *   labels   device int32 [n_ref], labels[j] = class of row j, in [0, n_classes)
 *   n_ref    >= 1;  n_classes >= 1
 *   stream   work is issued on it; the call synchronises it before returning
 *   out      receives the handle (set to NULL on failure)
 *
 * The index copies what it needs (the descriptors, an exact BF16 operand copy
 * with a 16-column norm extension, squared norms, labels, and a class-sorted
 * operand copy when the labels are not already grouped by class), so the
 * caller may free ref and labels afterwards.  Device memory: about 424 bytes
 * per reference (plus about 296 more when the labels are not grouped).
 * Errors: INVALID_ARG, LABEL_RANGE, OOM, CUDA, UNSUPPORTED.  A class with no
 * reference is accepted here; nbnn_classify then returns EMPTY_CLASS.
 */
LNBNN_API lnbnn_status lnbnn_index_create(const uint8_t *ref, const int32_t *labels, int64_t n_ref,
                                int32_t n_classes, void *stream, lnbnn_index **out);

/*
 * The same index over location-weighted descriptors: the alpha weighting of
 * descriptor location that Section 5 fixes at 1.6 for its experiments (an
 * option of the original NBNN, where the location is appended to the
 * descriptor).  Each row is 130 bytes: 128 appearance coordinates, then the
 * descriptor's location (x, y) on a 0..255 grid of the image, and
 *   distance(q, r) = sum_{t<128} (q_t - r_t)^2
 *                  + location_weight * ((q_x - r_x)^2 + (q_y - r_y)^2),
 * the squared Euclidean distance with the location appended at scale
 * sqrt(location_weight) (so location_weight = alpha^2 in grid units).  Every
 * call on this index takes 130-byte query rows; the distances stay exact.
 *
 *   ref              device uint8 [n_ref * 130]
 *   location_weight  0 <= location_weight <= LNBNN_MAX_LOCATION_WEIGHT
 * Other arguments as lnbnn_index_create.  The FP8 shortlist search is not
 * offered for such an index (lnbnn_index_prepare_fp8 returns UNSUPPORTED);
 * knn_search_noalloc takes 128-byte rows only.
 * Errors: as lnbnn_index_create, plus INVALID_ARG for a weight out of range.
 */
LNBNN_API lnbnn_status lnbnn_index_create_located(const uint8_t *ref, const int32_t *labels, int64_t n_ref,
                                                  int32_t n_classes, int32_t location_weight, void *stream,
                                                  lnbnn_index **out);

/* Row layout of an index: bytes per descriptor row (128 or 130) and the
 * location weight (0 for 128-byte rows).  Either pointer may be NULL. */
LNBNN_API lnbnn_status lnbnn_index_layout(const lnbnn_index *index, int32_t *row_bytes, int32_t *location_weight);

/* Release the index and all device memory it owns.  NULL is accepted. */
LNBNN_API void lnbnn_index_destroy(lnbnn_index *index);

/* Sizes of an index (any output pointer may be NULL). */
LNBNN_API lnbnn_status lnbnn_index_info(const lnbnn_index *index, int64_t *n_ref, int32_t *n_classes);

/*
 * NN(d, k) of Alg. 2 for every query descriptor: the k nearest references in
 * the merged set, exact, ordered by (distance, reference row).
 *
 *   queries   device uint8 [n_queries * 128]
 *   k         1 <= k <= LNBNN_MAX_K, k <= n_ref
 *   idx       device int32 [n_queries * k], row-major, reference rows
 *   dist      device int32 [n_queries * k], exact squared distances
 * n_queries = 0 is a no-op.  Errors: INVALID_ARG, K_RANGE, OOM, CUDA, TIMEOUT.
 */
LNBNN_API lnbnn_status knn_search(lnbnn_index *index, const uint8_t *queries, int64_t n_queries, int32_t k,
                        int32_t *idx, int32_t *dist, void *stream);

/*
 * LocalNBNN(Q, k), Alg. 2, for a batch of query images.  For each descriptor
 * d of image i: {p_1..p_{k+1}} = NN(d, k+1); dist_B = ||d - p_{k+1}||^2; for
 * each class C among p_1..p_k, dist_C = min ||d - p_j||^2 over those of class
 * C, and totals[i][C] += dist_C - dist_B.  classes[i] = argmin_C totals[i][C]
 * (lowest class on ties).  The background-class discount is the one Section 4
 * describes: classes not among the k nearest are not updated.
 *
 *   queries   device uint8 [n_queries * 128], all images' descriptors, flattened
 *   offsets   device int64 [n_images + 1]; image i owns rows offsets[i] ..
 *             offsets[i+1]-1; offsets[0] = 0, nondecreasing, offsets[n_images] = n_queries
 *   k         1 <= k <= LNBNN_MAX_K and k + 1 <= n_ref
 *   totals    device int64 [n_images * n_classes] (overwritten; every entry <= 0)
 *   classes   device int32 [n_images]
 * An image with no descriptors gets all-zero totals and class 0.  Invalid
 * offsets are detected on the device and reported as OFFSETS by lnbnn_sync.
 * Errors: INVALID_ARG, K_RANGE, OOM, CUDA, TIMEOUT, OFFSETS.
 */
LNBNN_API lnbnn_status lnbnn_classify(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                            const int64_t *offsets, int64_t n_images, int32_t k, int64_t *totals,
                            int32_t *classes, void *stream);

/*
 * NBNN(Q), Alg. 1: totals[i][C] = sum over descriptors d of image i of
 * ||d - NN_C(d)||^2, classes[i] = argmin_C totals[i][C] (lowest class on
 * ties); the rule of Eq. (eqn:nbnn).  Arguments as lnbnn_classify without k.
 * Errors: as lnbnn_classify, plus EMPTY_CLASS when a class has no reference.
 */
LNBNN_API lnbnn_status nbnn_classify(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                           const int64_t *offsets, int64_t n_images, int64_t *totals,
                           int32_t *classes, void *stream);

/*
 * Workspaces: the device scratch of one call (query operand copies, the
 * per-row neighbour lists, the NBNN minima table), sized once for at most
 * max_queries query descriptors and neighbourhoods up to max_k.  A call given a
 * workspace allocates nothing, so it may be captured into a CUDA graph, and
 * calls with distinct workspaces may run concurrently on different streams
 * (the index itself is only read).  A workspace belongs to the index it was
 * created for.  A call larger than its workspace returns SCRATCH_LIMIT.
 * The profile (lnbnn_profile_*) is not for captured calls.
 */
typedef struct lnbnn_workspace lnbnn_workspace;

LNBNN_API lnbnn_status lnbnn_workspace_create(lnbnn_index *index, int64_t max_queries, int32_t max_k,
                                              lnbnn_workspace **out);
LNBNN_API void lnbnn_workspace_destroy(lnbnn_workspace *workspace);

/* knn_search, lnbnn_classify and nbnn_classify with an explicit workspace. */
LNBNN_API lnbnn_status knn_search_ws(lnbnn_index *index, lnbnn_workspace *workspace, const uint8_t *queries,
                                     int64_t n_queries, int32_t k, int32_t *idx, int32_t *dist, void *stream);
LNBNN_API lnbnn_status lnbnn_classify_ws(lnbnn_index *index, lnbnn_workspace *workspace, const uint8_t *queries,
                                         int64_t n_queries, const int64_t *offsets, int64_t n_images, int32_t k,
                                         int64_t *totals, int32_t *classes, void *stream);
LNBNN_API lnbnn_status nbnn_classify_ws(lnbnn_index *index, lnbnn_workspace *workspace, const uint8_t *queries,
                                        int64_t n_queries, const int64_t *offsets, int64_t n_images,
                                        int64_t *totals, int32_t *classes, void *stream);

/*
 * NBNN as a sum of log-odds increments, Section 3.1.  Each descriptor d of
 * image i adds to every class C
 *   inc(d, C) = log [P(C|d) P(Cbar)] / [P(Cbar|d) P(C)]           Eq. (eqn:log-odds)
 * (Cbar: all other classes; equal priors P(C) = 1 / n_classes, so the prior
 * term of Eq. (eqn:log-increments) is dropped), with the posterior of the NBNN
 * Gaussian kernel on each class's nearest neighbour:
 *   P(C|d) = exp(-beta ||d - NN_C(d)||^2) / sum_C' exp(-beta ||d - NN_C'(d)||^2),
 * beta = 1 / (2 sigma^2); the paper leaves sigma unstated, so beta is the
 * caller's.  totals[i][C] = sum of the increments (positive_only != 0: only
 * those > 0, the variant of Table 1), classes[i] = argmax_C totals[i][C]
 * (lowest class on ties); n_increments[i] (optional) = how many increments
 * were added (n_classes per descriptor for the full rule).
 *
 *   beta          0 <= beta <= 1e250 (finite); 0 makes every increment 0
 *   totals        device float64 [n_images * n_classes], overwritten; each
 *                 image's sums are taken in descriptor order (deterministic)
 *   classes       device int32 [n_images]
 *   n_increments  device int64 [n_images] or NULL
 * Other arguments as nbnn_classify.  An empty image gets all-zero totals,
 * class 0 and no increments.  The distances NN_C(d) are exact (the scan of
 * nbnn_classify); the increments are float64 (device exp and log).
 * Errors: as nbnn_classify, plus INVALID_ARG for beta outside the range or an
 * index with fewer than two classes.
 */
LNBNN_API lnbnn_status nbnn_logodds_classify(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                                             const int64_t *offsets, int64_t n_images, double beta,
                                             int32_t positive_only, double *totals, int32_t *classes,
                                             int64_t *n_increments, void *stream);
LNBNN_API lnbnn_status nbnn_logodds_classify_ws(lnbnn_index *index, lnbnn_workspace *workspace,
                                                const uint8_t *queries, int64_t n_queries, const int64_t *offsets,
                                                int64_t n_images, double beta, int32_t positive_only,
                                                double *totals, int32_t *classes, int64_t *n_increments,
                                                void *stream);

/*
 * FP8 shortlist search: an approximate search of this library's own design,
 * in the place the paper fills with an approximate kd-tree search (Section
 * 5, "Approximate nearest neighbors"); the paper has no FP8 step.  A coarse
 * tensor-core pass over FP8 E4M3 operands ranks every reference by
 *     coarse(q, r) = ||q'||^2 + ||r'||^2 - 2 E4M3(q') . E4M3(r'),
 * x' = x - 64 per coordinate, E4M3 = round to nearest even on 3 mantissa bits;
 * the `shortlist` smallest (coarse, row) pairs are then reranked by their
 * exact squared distance, and the k (knn) or k + 1 (classify) smallest exact
 * (distance, row) pairs of the shortlist are the neighbours.  Distances and
 * totals are therefore exact for the neighbours found; a true neighbour
 * outside the shortlist is missed (recall < 1).  With shortlist >= n_ref the
 * result equals the exact search.  The result of a query does not depend on
 * the other queries of the call.
 *
 * lnbnn_index_prepare_fp8 builds the E4M3 operand once (about 160 bytes per
 * reference) and synchronises `stream`; until then the FP8 calls return
 * NO_FP8.  Repeated calls are no-ops.
 *
 *   shortlist   knn: k <= shortlist; classify: k + 1 <= shortlist; at most
 *               LNBNN_MAX_K + 1 (K_RANGE otherwise)
 * Other arguments, outputs and errors as knn_search / lnbnn_classify.  A
 * workspace serves an FP8 call when max_queries >= n_queries and
 * max_k + 1 >= shortlist.
 */
LNBNN_API lnbnn_status lnbnn_index_prepare_fp8(lnbnn_index *index, void *stream);
LNBNN_API lnbnn_status knn_search_fp8(lnbnn_index *index, const uint8_t *queries, int64_t n_queries, int32_t k,
                                      int32_t shortlist, int32_t *idx, int32_t *dist, void *stream);
LNBNN_API lnbnn_status lnbnn_classify_fp8(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                                          const int64_t *offsets, int64_t n_images, int32_t k, int32_t shortlist,
                                          int64_t *totals, int32_t *classes, void *stream);
LNBNN_API lnbnn_status knn_search_fp8_ws(lnbnn_index *index, lnbnn_workspace *workspace, const uint8_t *queries,
                                         int64_t n_queries, int32_t k, int32_t shortlist, int32_t *idx,
                                         int32_t *dist, void *stream);
LNBNN_API lnbnn_status lnbnn_classify_fp8_ws(lnbnn_index *index, lnbnn_workspace *workspace,
                                             const uint8_t *queries, int64_t n_queries, const int64_t *offsets,
                                             int64_t n_images, int32_t k, int32_t shortlist, int64_t *totals,
                                             int32_t *classes, void *stream);

/*
 * Search schedule.  Each search launch runs ceil(n_queries / (128 qt)) groups
 * of qt query tiles (qt = 1 or 2) x `splits` reference ranges as work items,
 * one CTA per item or a persistent grid that takes items from a queue, and
 * merges the splits' lists; the split count is chosen per call by a
 * device-time model
 *   waves(groups * splits) * (a * qt * tiles_per_item + b + e * k1)
 *     + c * groups * splits,
 * where the term e * k1 (k1 = list length) is the cost of filling one item's
 * lists, so longer lists favour fewer splits.  A launch with at least one
 * wave of query tiles also takes at least as many splits as keep each
 * split's reference bytes in L2 for the FP8 coarse pass (48 MB a split), and
 * 4 (lists of 17..32 entries) or 8 (heaps) for the exact scan; the splits of
 * a row then run one after another, and each starts from the row's lists of
 * the previous split when that split has finished (the results never depend
 * on whether it has).  A launch of few query tiles with an automatic split
 * count takes the claimed-chunk form instead of splits (the FP8 coarse pass
 * while there are at least 8 SMs per query tile, the exact scan for a lone
 * query tile; lists of up to 32 entries or heaps): each of P / T CTAs per
 * query tile keeps that tile's lists for the whole launch and claims short
 * reference chunks, in increasing order, from a counter the tile's CTAs
 * share, so that the reference ranges holding a query's own class, where
 * most list inserts fall on a class-sorted index, are shared by whichever
 * CTAs are free (lnbnn_plan_search reports chunked = 1; `splits` is then the
 * CTAs per query tile and split_len the chunk length).  lnbnn_autotune times about
 * thirty search launches of 1 to 64 query tiles (query rows copied from the
 * index's own references) with several split counts and two list lengths
 * (k1 = 11 and 51) on `stream` and fits a, b, c, e by least squares; then, on
 * indexes with enough references for two waves of query tiles, it times the
 * four large-batch forms of the exact scan (k1 = 11) and, when the index has
 * its FP8 operand, of the coarse pass (k1 = 32): one or two query tiles per
 * CTA, one CTA per item or persistent; the fastest form of each is then used
 * for launches of at least a full wave of query tiles (without tuning: one
 * query tile per CTA for the NBNN scan and the exact scan of lists of up to
 * 16 entries, two for longer exact lists and the coarse pass, one CTA per
 * item; longer exact lists take two query tiles after tuning too).  It keeps
 * all of this
 * in the index; it synchronises `stream`, allocates and frees its own
 * scratch, and changes no result (every schedule gives bit-identical output),
 * only speed.  Call it outside stream capture.  out (may be NULL) receives
 * the fitted milliseconds per 128 x 256 step, per wave, per (query-tile
 * group, split) and per list entry and wave, the number of timed split-model
 * runs and the largest relative error of that fit (tile_ms = 0: no fit, the
 * model is unchanged), the chosen large-batch forms (query tiles per CTA 1 or
 * 2, persistent 0 or 1; 0 and -1 when not timed) and the timed milliseconds
 * of the candidates, [0..3] exact and [4..7] coarse, in the order (1, grid),
 * (1, persistent), (2, grid), (2, persistent) (0 when not timed).
 * lnbnn_plan_splits reports the split count a call with n_queries query
 * descriptors would use.  Workspaces are sized for the largest split count
 * any model may choose, so they stay valid after tuning.
 */
typedef struct lnbnn_tuning {
  double tile_ms;
  double wave_ms;
  double list_ms;
  double max_rel_error;
  int32_t runs;
  int32_t exact_query_tiles;
  double entry_ms;
  int32_t exact_persistent;
  int32_t coarse_query_tiles;
  int32_t coarse_persistent;
  int32_t form_runs;
  double form_ms[8];
} lnbnn_tuning;

LNBNN_API lnbnn_status lnbnn_autotune(lnbnn_index *index, void *stream, lnbnn_tuning *out);
LNBNN_API lnbnn_status lnbnn_plan_splits(const lnbnn_index *index, int64_t n_queries, int32_t *splits);

/*
 * lnbnn_plan_search reports how a search of the k1 nearest references of each
 * of n_queries query descriptors would be launched on this index (the search
 * step of Alg. 2, NN(d, k+1)): the exact scan (fp8 == 0; knn_search with
 * k = k1, or a Local NBNN classify call with k + 1 = k1) or the coarse pass
 * of the FP8 shortlist search (fp8 != 0; k1 = the shortlist length).  Nothing
 * is launched.  Fields: the reference splits of the launch and references per
 * split; the sorted lists per query row the scan writes (merged afterwards
 * when more than one); where each list lives (list_storage 0: registers, 1:
 * shared memory, 2: a heap in global memory) and how many entries it holds
 * (16, 24, 32 or 64; k1 for a heap); the tile of query rows x references one CTA
 * computes per step (tile_m query rows x tile_n references); persistent = 1
 * when a fixed grid of CTAs takes (query tiles, split) work items from a
 * queue instead of one CTA per item; bound_per_tile: how the lists of a row
 * share their bound when there are several splits (1: every tile, as the
 * splits of a row run at the same time; 0: read when a list starts and
 * published when it ends, as they run one after another; -1: one split);
 * chunked = 1 for the claimed-chunk form of launches with fewer query-tile
 * groups than SMs: `splits` CTAs per group each keep that group's lists for
 * the whole launch and claim reference chunks of split_len rows, in
 * increasing order, from a counter the group's CTAs share (so the reference
 * ranges that hold a query's own class, where most list inserts fall, are
 * shared by whichever CTAs are free).
 * Errors: INVALID_ARG (null pointers, n_queries < 1), K_RANGE (k1 outside
 * [1, LNBNN_MAX_K + 1] or above n_ref), NO_FP8 (fp8 != 0 on an index without
 * the FP8 operand).
 */
typedef struct lnbnn_search_plan {
  int32_t splits;
  int32_t lists_per_row;
  int64_t split_len;
  int32_t list_storage;
  int32_t list_capacity;
  int32_t tile_m;
  int32_t tile_n;
  int32_t persistent;
  int32_t bound_per_tile;
  int32_t chunked;
} lnbnn_search_plan;

LNBNN_API lnbnn_status lnbnn_plan_search(const lnbnn_index *index, int64_t n_queries, int32_t k1, int32_t fp8,
                                         lnbnn_search_plan *out);

/*
 * lnbnn_set_schedule fixes parts of the launch schedule of this index's
 * search scans (every later call; NULL restores the automatic choice of
 * everything).  It changes speed only, never a result: every schedule gives
 * bit-identical output.  Fields: splits > 0 fixes the reference split count
 * (rounded to whole 256-row tiles; 0: automatic); query_tiles 1 or 2 fixes the
 * tile shape (128 x 256 or 256 x 128 query rows x references per step; 2 is
 * taken only where the list kind allows it, i.e. not for lists of 33..64
 * entries; 0: automatic); persistent 1 / 0 a persistent grid with a work
 * queue / one CTA per work item (-1: automatic); bound_per_tile 1 / 0 how
 * the lists of a row share their bound (-1: automatic).  A fixed split count
 * above the automatic range may need more scratch than a workspace made
 * earlier holds (those calls then return SCRATCH_LIMIT).  Meant for tuning
 * and tests.  Errors: INVALID_ARG (null index, a field out of range).
 */
typedef struct lnbnn_schedule {
  int32_t splits;
  int32_t query_tiles;
  int32_t persistent;
  int32_t bound_per_tile;
} lnbnn_schedule;

LNBNN_API lnbnn_status lnbnn_set_schedule(lnbnn_index *index, const lnbnn_schedule *schedule);

/*
 * Host-buffer forms of the classifiers: queries, offsets, totals and
 * classes are HOST pointers.  The call copies the inputs to the device
 * (into the index's device staging buffer), classifies, copies the
 * results back and synchronises `stream` before returning.  Pinned (page-locked)
 * host buffers give the fastest copies.
 */
LNBNN_API lnbnn_status lnbnn_classify_host(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                                 const int64_t *offsets, int64_t n_images, int32_t k,
                                 int64_t *totals, int32_t *classes, void *stream);
LNBNN_API lnbnn_status nbnn_classify_host(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                                const int64_t *offsets, int64_t n_images, int64_t *totals,
                                int32_t *classes, void *stream);
LNBNN_API lnbnn_status lnbnn_classify_fp8_host(lnbnn_index *index, const uint8_t *queries, int64_t n_queries,
                                               const int64_t *offsets, int64_t n_images, int32_t k,
                                               int32_t shortlist, int64_t *totals, int32_t *classes, void *stream);

/*
 * Wait for `stream`, then report (and clear) any device-side error recorded
 * for this index since the last report: TIMEOUT when a bounded wait inside a
 * kernel expired, OFFSETS when a classify call got invalid offsets.
 */
LNBNN_API lnbnn_status lnbnn_sync(lnbnn_index *index, void *stream);

/*
 * Device-time profile of an index's calls (an aid for measurement; no part
 * of the method).  While enabled, every classify / search call records CUDA
 * events on its own stream around its phases: "search" is the exact search
 * kernel (the tensor-core k+1 nearest-neighbour kernel, or the per-class
 * NBNN kernel); "other" is everything else the call launches (query
 * preparation, split merge, class update, argmin).  lnbnn_profile_read waits
 * for the recorded events and returns the sums since the last enable.
 * kernel_launches counts every kernel the library launched in those calls.
 */
typedef struct lnbnn_profile {
  int64_t calls;
  int64_t kernel_launches;
  int64_t search_launches;
  double search_ms;
  double other_ms;
  /* tensor-core kNN search only: mean SM clock seen by its CTAs (GHz) and SM
   * cycles per 128 x 256 tile, from clock64/globaltimer at each CTA's start
   * and end (0 when no such launch was profiled) */
  double search_sm_clock_ghz;
  double search_cycles_per_tile;
} lnbnn_profile;

LNBNN_API lnbnn_status lnbnn_profile_enable(lnbnn_index *index, int enable);
LNBNN_API lnbnn_status lnbnn_profile_read(lnbnn_index *index, lnbnn_profile *out);

/*
 * knn_search_noalloc -- the exact k nearest neighbours of knn_search for
 * callers that must not allocate device memory: code running inside a host
 * framework that owns every device allocation (a fixed memory pool or arena,
 * a plugin whose host forbids cudaMalloc), or a caller that cannot afford the
 * implicit device synchronisation cudaMalloc and cudaFree bring.  The paper
 * has no counterpart; this is a deployment variant of the same search.
 *
 * No index is needed: ref and queries are the caller's device uint8 arrays
 * ([n_ref * 128] and [n_queries * 128]), idx and dist its device int32 outputs
 * ([n_queries * k], as knn_search); all four must be memory of the current
 * device (INVALID_ARG otherwise).  Every intermediate (BF16 operand copies,
 * squared norms, per-row neighbour lists and their shared bounds, the error
 * word) lives in one fixed-size array in device global memory that the
 * library defines at file scope: LNBNN_NOALLOC_SCRATCH_BYTES (64 MiB),
 * reserved on a device once the library's device code is loaded there (at
 * the latest by the first call there) and held until the process exits.  The
 * call makes no cudaMalloc, cudaFree or other allocating call.  n_ref or
 * n_queries above 262,144 (the rows whose BF16 copy alone fills the array),
 * or a problem whose intermediates do not fit (roughly n_ref + n_queries
 * above about 200,000 rows at k = 10), is rejected with
 * LNBNN_ERR_SCRATCH_LIMIT before any work is issued.
 *
 * The first call on each device looks up that device's address of the array
 * (once, with the device current); make that first call before any stream
 * capture begins.  That set-up belongs to the device's primary context: after
 * cudaDeviceReset the entry point must not be used again in the process.  All
 * calls share the one array and find the previous call's contents in it; two
 * calls whose work overlaps on the GPU (different streams, or threads without
 * ordering) race and corrupt each other.  The call waits for `stream` before
 * returning, to report device-side errors.
 * Errors: INVALID_ARG, K_RANGE, SCRATCH_LIMIT, UNSUPPORTED, CUDA, TIMEOUT.
 */
#define LNBNN_NOALLOC_SCRATCH_BYTES (64ull << 20)
LNBNN_API lnbnn_status knn_search_noalloc(const uint8_t *ref, int64_t n_ref, const uint8_t *queries,
                                          int64_t n_queries, int32_t k, int32_t *idx, int32_t *dist,
                                          void *stream);

/*
 * Index persistence (no part of the method; lets a server restart without
 * the original arrays).  lnbnn_index_save writes what lnbnn_index_create was
 * given — the reference descriptors and their labels — to the file `path`:
 * a 32-byte header (the 8 bytes "LNBNNIX1", uint32 format version 1, uint32
 * row bytes 128 or 130, int64 n_ref, int32 n_classes, uint32 location weight
 * (0 for 128-byte rows)), the uint8 descriptors [n_ref * row bytes], the
 * int32 labels [n_ref], and an 8-byte FNV-1a
 * 64-bit hash of everything before it; all integers little-endian.  The call
 * waits for the device copies.  lnbnn_index_load checks the header, sizes and
 * hash before it touches the device, then builds the index exactly as
 * lnbnn_index_create would (the same results; derived operands, the FP8
 * operand and a fitted schedule are rebuilt, not stored).
 * Errors: INVALID_ARG, IO (cannot open, short read or write, wrong magic,
 * version or sizes, hash mismatch), and those of lnbnn_index_create.
 */
LNBNN_API lnbnn_status lnbnn_index_save(const lnbnn_index *index, const char *path);
LNBNN_API lnbnn_status lnbnn_index_load(const char *path, void *stream, lnbnn_index **out);

/*
 * Test hooks for the failure paths (no part of the method).
 *
 * lnbnn_debug_fail_allocations: the library's next `count` device allocations
 * (in any call: index creation, workspaces, the index's own scratch, FP8
 * preparation, autotuning) fail as if the device were out of memory, so the
 * call returns OOM and frees what it had allocated.  count <= 0 clears it.
 * Process-wide; needs no device.
 *
 * lnbnn_set_start_gate: search kernels of this index wait, before loading any
 * operand, until the device word *gate is nonzero; gate = NULL (the default)
 * removes the wait.  The wait is bounded like every other wait in the search
 * kernels (1 s): a gate that nothing opens makes the call's kernels give up,
 * record a timeout and return, and lnbnn_sync then reports TIMEOUT.  The
 * pointer must stay valid while calls may run.
 */
LNBNN_API void lnbnn_debug_fail_allocations(int32_t count);
LNBNN_API lnbnn_status lnbnn_set_start_gate(lnbnn_index *index, const uint32_t *gate);

/* Static English text for a status code. */
LNBNN_API const char *lnbnn_status_string(lnbnn_status status);

#ifdef __cplusplus
}
#endif

#endif /* LNBNN_H */
