/*
 * CPU oracle for Local Naive Bayes Nearest Neighbor (McCann & Lowe,
 * "Local Naive Bayes Nearest Neighbor for Image Classification").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  It shares no code, header, table
 * or helper with the CUDA library, and only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.
 *
 * Readings taken where the paper is silent (each is repeated where it is used):
 *   - distance is the squared Euclidean distance on the raw uint8 values
 *     (||d_i - p||^2 in Alg. 1 and Alg. 2), exact in integers;
 *   - "the k+1 nearest neighbours" are ordered by (distance, reference index)
 *     ascending, so equal distances go to the lower index;
 *   - dist_C in Alg. 2 is the minimum over the first k neighbours of class C
 *     (the (k+1)-th cannot lower it for a class already present);
 *   - argmin over classes returns the lowest class index among equal totals;
 *   - an image with no descriptors has all-zero totals and class 0;
 *   - k >= 1 and k + 1 <= N are required (Alg. 2 reads the (k+1)-th neighbour);
 *   - original NBNN needs every class to own at least one reference (NN_C).
 *
 * Location-weighted descriptors (the alpha weighting of descriptor location
 * that Section 5 fixes at 1.6 for its experiments, an option of the original
 * NBNN): a descriptor row may carry 2 location bytes after its 128
 * appearance bytes (130 bytes a row), and the distance is then
 *   sum over the 128 appearance coordinates of (q_t - r_t)^2
 *   + w * sum over the 2 location coordinates of (q_t - r_t)^2,
 * with an integer weight w >= 0: the squared Euclidean distance of the
 * descriptors with the location appended at scale sqrt(w) (alpha^2 = w in
 * the units of the location grid).  The FP8 shortlist form is 128-byte only.
 *
 * Work is split across threads only over query descriptors, which Alg. 1 and
 * Alg. 2 treat independently; every per-descriptor step runs as written.
 *
 * The coarse-shortlist form (an approximate search of this project's own
 * design, standing where the paper uses an approximate kd-tree search,
 * Section 5) is stated here as:
 *   - every coordinate is shifted, x' = x - 64, and rounded to the nearest
 *     FP8 E4M3 value (3 mantissa bits, ties to even mantissa), x~;
 *   - coarse(q, r) = ||q'||^2 + ||r'||^2 - 2 sum_t q~_t r~_t, an integer;
 *   - the shortlist of a query is the m smallest (coarse, index) pairs;
 *   - its exact distances are computed and the kk smallest (distance, index)
 *     pairs of the shortlist are the neighbours; Alg. 2 then runs unchanged.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_D 128
#define ORACLE_LOC 2

/* Row layout and weight of the distance: stride ORACLE_D (appearance only) or
 * ORACLE_D + ORACLE_LOC (appearance, then location weighted by w). */
typedef struct {
  int32_t stride;
  int64_t w;
} metric_t;

static const metric_t plain_metric = {ORACLE_D, 0};

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_ARG = -1,
  ORACLE_ERR_LABEL = -2,
  ORACLE_ERR_K = -3,
  ORACLE_ERR_EMPTY_CLASS = -4,
  ORACLE_ERR_OFFSETS = -5,
  ORACLE_ERR_NOMEM = -6,
};

/* ||a - b||^2 over the 128 appearance coordinates (each term at most 255^2,
 * the sum at most 128 * 255^2 = 8,323,200 < 2^31, so 32-bit sums are exact),
 * plus w times the squared difference of the location coordinates, if any. */
static int64_t sqdist(const uint8_t *a, const uint8_t *b, const metric_t *mt) {
  int32_t s = 0;
  for (int t = 0; t < ORACLE_D; ++t) {
    int32_t e = (int32_t)a[t] - (int32_t)b[t];
    s += e * e;
  }
  int64_t loc = 0;
  for (int t = ORACLE_D; t < mt->stride; ++t) {
    int32_t e = (int32_t)a[t] - (int32_t)b[t];
    loc += e * e;
  }
  return (int64_t)s + mt->w * loc;
}

/* (d1, j1) comes before (d2, j2): smaller distance, then smaller index. */
static int before(int64_t d1, int64_t j1, int64_t d2, int64_t j2) {
  return d1 < d2 || (d1 == d2 && j1 < j2);
}

/* NN(q, kk): the kk references with the smallest (distance, index), ascending.
 * Scans every reference and keeps the kk best seen so far in a sorted list. */
static void knn_one(const uint8_t *ref, int64_t N, const uint8_t *q, int32_t kk,
                    int64_t *od, int64_t *oj, const metric_t *mt) {
  int32_t len = 0;
  for (int64_t j = 0; j < N; ++j) {
    int64_t d = sqdist(q, ref + j * mt->stride, mt);
    if (len == kk && !before(d, j, od[kk - 1], oj[kk - 1])) continue;
    int32_t p = (len < kk) ? len++ : kk - 1; /* slot freed at the end of the list */
    while (p > 0 && before(d, j, od[p - 1], oj[p - 1])) {
      od[p] = od[p - 1];
      oj[p] = oj[p - 1];
      --p;
    }
    od[p] = d;
    oj[p] = j;
  }
}

/* NN_C(q) for every class C: the smallest distance to a reference of class C
 * (Alg. 1's per-class search).  Classes without references keep INT64_MAX. */
static void class_min_one(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                          const uint8_t *q, int64_t *cmin, const metric_t *mt) {
  for (int32_t c = 0; c < C; ++c) cmin[c] = INT64_MAX;
  for (int64_t j = 0; j < N; ++j) {
    int64_t d = sqdist(q, ref + j * mt->stride, mt);
    if (d < cmin[labels[j]]) cmin[labels[j]] = d;
  }
}

/* Alg. 2, body of the loop over descriptors, for one descriptor:
 *   {p_1..p_{k+1}} = NN(d, k+1); dist_B = ||d - p_{k+1}||^2;
 *   for every class C among p_1..p_k:
 *     dist_C = min over p_j of class C of ||d - p_j||^2;
 *     totals[C] += dist_C - dist_B.
 * nd, nj: scratch of k+1 entries. */
static void score_one(const int32_t *labels, int32_t k, const int64_t *nd, const int64_t *nj,
                      int64_t *totals) {
  const int64_t dist_B = nd[k];
  for (int32_t a = 0; a < k; ++a) {
    const int32_t c = labels[nj[a]];
    int seen = 0;
    for (int32_t b = 0; b < a; ++b)
      if (labels[nj[b]] == c) seen = 1;
    if (seen) continue; /* each class found among the k is updated once */
    int64_t dist_C = nd[a];
    for (int32_t b = 0; b < k; ++b)
      if (labels[nj[b]] == c && nd[b] < dist_C) dist_C = nd[b];
    totals[c] += dist_C - dist_B;
  }
}

static void lnbnn_one(const uint8_t *ref, const int32_t *labels, int64_t N, const uint8_t *q,
                      int32_t k, int64_t *nd, int64_t *nj, int64_t *totals, const metric_t *mt) {
  knn_one(ref, N, q, k + 1, nd, nj, mt);
  score_one(labels, k, nd, nj, totals);
}

/* ------------------------------------------------------ coarse shortlist */

#define ORACLE_SHIFT 64

/* Nearest FP8 E4M3 value to the integer x (|x| <= 448), ties to the even
 * mantissa.  E4M3 holds every integer below 16; from 2^p (p >= 4) up to
 * 2^(p+1) its values are 2^(p-3) apart.  The result is an integer. */
static int32_t e4m3_round(int32_t x) {
  const int32_t a = x < 0 ? -x : x;
  if (a < 16) return x;
  int32_t p = 4;
  while (a >= (1 << (p + 1))) ++p;
  const int32_t step = 1 << (p - 3);
  int32_t n = a / step, rem = a % step;
  if (2 * rem > step || (2 * rem == step && (n & 1))) ++n;
  const int32_t r = n * step;
  return x < 0 ? -r : r;
}

/* E4M3 rounding of every shifted coordinate value, x~ = e4m3_round(x - 64)
 * for x = 0..255: a table of e4m3_round, filled before any search starts
 * (the searches only read it), so that a pair costs no more than a lookup
 * per coordinate. */
static int32_t rounded_shifted[256];

static void fill_rounded_shifted(void) {
  for (int x = 0; x < 256; ++x) rounded_shifted[x] = e4m3_round(x - ORACLE_SHIFT);
}

/* coarse(q, r) = ||q'||^2 + ||r'||^2 - 2 q~ . r~  with x' = x - 64 and x~ its
 * E4M3 rounding. */
static int64_t coarse(const uint8_t *q, const uint8_t *r) {
  int64_t nq = 0, nr = 0, dot = 0;
  for (int t = 0; t < ORACLE_D; ++t) {
    const int32_t qs = (int32_t)q[t] - ORACLE_SHIFT, rs = (int32_t)r[t] - ORACLE_SHIFT;
    nq += qs * qs;
    nr += rs * rs;
    dot += (int64_t)rounded_shifted[q[t]] * rounded_shifted[r[t]];
  }
  return nq + nr - 2 * dot;
}

/* The kk nearest of q among its coarse shortlist: the m smallest
 * (coarse, index) pairs over all N references (m >= kk; m > N means all),
 * reranked by exact (distance, index).  cd, cj: scratch of m entries. */
static void knn_coarse_one(const uint8_t *ref, int64_t N, const uint8_t *q, int32_t kk, int32_t m,
                           int64_t *cd, int64_t *cj, int64_t *od, int64_t *oj) {
  if ((int64_t)m > N) m = (int32_t)N;
  int32_t len = 0;
  for (int64_t j = 0; j < N; ++j) {
    const int64_t c = coarse(q, ref + j * ORACLE_D);
    if (len == m && !before(c, j, cd[m - 1], cj[m - 1])) continue;
    int32_t p = (len < m) ? len++ : m - 1;
    while (p > 0 && before(c, j, cd[p - 1], cj[p - 1])) {
      cd[p] = cd[p - 1];
      cj[p] = cj[p - 1];
      --p;
    }
    cd[p] = c;
    cj[p] = j;
  }
  /* rerank: exact distance of each candidate, keep the kk smallest */
  int32_t n = 0;
  for (int32_t a = 0; a < m; ++a) {
    const int64_t j = cj[a], d = sqdist(q, ref + j * ORACLE_D, &plain_metric);
    if (n == kk && !before(d, j, od[kk - 1], oj[kk - 1])) continue;
    int32_t p = (n < kk) ? n++ : kk - 1;
    while (p > 0 && before(d, j, od[p - 1], oj[p - 1])) {
      od[p] = od[p - 1];
      oj[p] = oj[p - 1];
      --p;
    }
    od[p] = d;
    oj[p] = j;
  }
}

static int cmp_i64(const void *x, const void *y) {
  int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
  return (a > b) - (a < b);
}

/* The same Local NBNN totals by a second route.  Every reference strictly
 * closer than the (k+1)-th neighbour is among the first k, so a class C is
 * found among the k nearest with dist_C = NN_C(d) exactly when
 * NN_C(d) < dist_B, and otherwise contributes nothing; a class whose nearest
 * member ties dist_B adds 0 either way.  Hence
 *   totals[C] += min(0, NN_C(d) - dist_B(d)),
 * with dist_B the (k+1)-th smallest of all N distances (values only). */
static int closed_form_one(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                           const uint8_t *q, int32_t k, int64_t *all, int64_t *cmin,
                           int64_t *totals, const metric_t *mt) {
  for (int64_t j = 0; j < N; ++j) all[j] = sqdist(q, ref + j * mt->stride, mt);
  for (int32_t c = 0; c < C; ++c) cmin[c] = INT64_MAX;
  for (int64_t j = 0; j < N; ++j)
    if (all[j] < cmin[labels[j]]) cmin[labels[j]] = all[j];
  qsort(all, (size_t)N, sizeof(int64_t), cmp_i64);
  const int64_t dist_B = all[k];
  for (int32_t c = 0; c < C; ++c)
    if (cmin[c] != INT64_MAX && cmin[c] < dist_B) totals[c] += cmin[c] - dist_B;
  return ORACLE_OK;
}

/* argmin over classes; the lowest class wins ties */
static int32_t argmin_lowest(const int64_t *t, int32_t C) {
  int32_t best = 0;
  for (int32_t c = 1; c < C; ++c)
    if (t[c] < t[best]) best = c;
  return best;
}

/* ------------------------------------------------------------------ checks */

static int check_ref(int64_t N, int32_t C, const int32_t *labels) {
  if (N < 1 || C < 1) return ORACLE_ERR_ARG;
  if (labels)
    for (int64_t j = 0; j < N; ++j)
      if (labels[j] < 0 || labels[j] >= C) return ORACLE_ERR_LABEL;
  return ORACLE_OK;
}

static int check_offsets(const int64_t *offsets, int64_t n_img, int64_t M) {
  if (n_img < 0 || offsets[0] != 0) return ORACLE_ERR_OFFSETS;
  for (int64_t i = 0; i < n_img; ++i)
    if (offsets[i + 1] < offsets[i]) return ORACLE_ERR_OFFSETS;
  if (offsets[n_img] != M) return ORACLE_ERR_OFFSETS;
  return ORACLE_OK;
}

/* -------------------------------------------------------------- threading */

enum { JOB_KNN, JOB_CLASS_MIN, JOB_LNBNN, JOB_CLOSED, JOB_NBNN, JOB_KNN_COARSE, JOB_LNBNN_COARSE };

typedef struct {
  int kind;
  const uint8_t *ref;
  const int32_t *labels;
  int64_t N;
  int32_t C;
  const uint8_t *q;
  int64_t M;
  int32_t k;             /* kk for JOB_KNN, k for the classifiers */
  int32_t m;             /* shortlist length of the coarse jobs */
  metric_t mt;           /* row stride and location weight (coarse jobs: plain) */
  const int64_t *img_of; /* descriptor -> image, classifiers only */
  int64_t n_img;
  int64_t *out_d;        /* JOB_KNN [M*kk]; JOB_CLASS_MIN [M*C] */
  int64_t *out_j;        /* JOB_KNN [M*kk] */
  int64_t next;          /* next descriptor to hand out */
  int nthreads;
  int64_t *partial;      /* classifiers: [nthreads][n_img*C] */
  int status;
} job_t;

typedef struct {
  job_t *job;
  int tid;
} worker_t;

static void *worker(void *arg) {
  worker_t *w = (worker_t *)arg;
  job_t *J = w->job;
  const int64_t chunk = 4;
  int64_t *s1 = NULL, *s2 = NULL;
  int64_t *s3 = NULL, *s4 = NULL;
  if (J->kind == JOB_KNN_COARSE || J->kind == JOB_LNBNN_COARSE) {
    s3 = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->m);
    s4 = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->m);
    if (!s3 || !s4) goto oom;
  }
  if (J->kind == JOB_LNBNN || J->kind == JOB_LNBNN_COARSE) {
    s1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(J->k + 1));
    s2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(J->k + 1));
  } else if (J->kind == JOB_CLOSED) {
    s1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->N);
    s2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->C);
  } else if (J->kind == JOB_NBNN) {
    s1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->C);
  }
  if ((J->kind == JOB_LNBNN || J->kind == JOB_CLOSED || J->kind == JOB_LNBNN_COARSE) && (!s1 || !s2)) goto oom;
  if (J->kind == JOB_NBNN && !s1) goto oom;
  int64_t *mine = J->partial ? J->partial + (size_t)w->tid * (size_t)(J->n_img * J->C) : NULL;
  for (;;) {
    int64_t i0 = __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
    if (i0 >= J->M) break;
    int64_t i1 = i0 + chunk < J->M ? i0 + chunk : J->M;
    for (int64_t i = i0; i < i1; ++i) {
      const uint8_t *qi = J->q + i * J->mt.stride;
      switch (J->kind) {
        case JOB_KNN:
          knn_one(J->ref, J->N, qi, J->k, J->out_d + i * J->k, J->out_j + i * J->k, &J->mt);
          break;
        case JOB_CLASS_MIN:
          class_min_one(J->ref, J->labels, J->N, J->C, qi, J->out_d + i * J->C, &J->mt);
          break;
        case JOB_LNBNN:
          lnbnn_one(J->ref, J->labels, J->N, qi, J->k, s1, s2, mine + J->img_of[i] * J->C, &J->mt);
          break;
        case JOB_CLOSED:
          closed_form_one(J->ref, J->labels, J->N, J->C, qi, J->k, s1, s2,
                          mine + J->img_of[i] * J->C, &J->mt);
          break;
        case JOB_KNN_COARSE:
          knn_coarse_one(J->ref, J->N, qi, J->k, J->m, s3, s4, J->out_d + i * J->k, J->out_j + i * J->k);
          break;
        case JOB_LNBNN_COARSE:
          knn_coarse_one(J->ref, J->N, qi, J->k + 1, J->m, s3, s4, s1, s2);
          score_one(J->labels, J->k, s1, s2, mine + J->img_of[i] * J->C);
          break;
        case JOB_NBNN: {
          /* Alg. 1: totals[C] += ||d_i - NN_C(d_i)||^2 for every class C */
          class_min_one(J->ref, J->labels, J->N, J->C, qi, s1, &J->mt);
          int64_t *t = mine + J->img_of[i] * J->C;
          for (int32_t c = 0; c < J->C; ++c) t[c] += s1[c];
          break;
        }
      }
    }
  }
  free(s1);
  free(s2);
  free(s3);
  free(s4);
  return NULL;
oom:
  free(s1);
  free(s2);
  free(s3);
  free(s4);
  __atomic_store_n(&J->status, ORACLE_ERR_NOMEM, __ATOMIC_RELAXED);
  return NULL;
}

static int run(job_t *J, int nthreads) {
  if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  J->nthreads = nthreads;
  J->next = 0;
  J->status = ORACLE_OK;
  pthread_t th[256];
  worker_t ws[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    ws[t].job = J;
    ws[t].tid = t;
    if (pthread_create(&th[t], NULL, worker, &ws[t]) != 0) break;
    ++started;
  }
  if (started == 0) worker(&ws[0]); /* no thread could start: run inline */
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return J->status;
}

/* Classifier driver: per-thread partial totals, summed (integer sums are
 * exact in any order), then the per-image argmin. */
static int classify(int kind, const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                    const uint8_t *q, const int64_t *offsets, int64_t n_img, int32_t k, int32_t m,
                    int64_t *totals, int32_t *classes, int nthreads, metric_t mt) {
  int st = check_ref(N, C, labels);
  if (st) return st;
  const int64_t M = offsets[n_img];
  if ((st = check_offsets(offsets, n_img, M))) return st;
  if (kind != JOB_NBNN && (k < 1 || (int64_t)k + 1 > N)) return ORACLE_ERR_K;
  if (kind == JOB_LNBNN_COARSE && m < k + 1) return ORACLE_ERR_K;
  if (kind == JOB_NBNN) {
    char *has = (char *)calloc((size_t)C, 1);
    if (!has) return ORACLE_ERR_NOMEM;
    for (int64_t j = 0; j < N; ++j) has[labels[j]] = 1;
    for (int32_t c = 0; c < C; ++c)
      if (!has[c]) st = ORACLE_ERR_EMPTY_CLASS;
    free(has);
    if (st) return st;
  }
  int64_t *img_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
  if (!img_of) return ORACLE_ERR_NOMEM;
  for (int64_t i = 0; i < n_img; ++i)
    for (int64_t r = offsets[i]; r < offsets[i + 1]; ++r) img_of[r] = i;

  job_t J;
  memset(&J, 0, sizeof J);
  J.kind = kind;
  J.ref = ref;
  J.labels = labels;
  J.N = N;
  J.C = C;
  J.q = q;
  J.M = M;
  J.k = k;
  J.m = m;
  J.mt = mt;
  J.img_of = img_of;
  J.n_img = n_img;
  if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  const size_t per = (size_t)(n_img * C);
  J.partial = (int64_t *)calloc(per * (size_t)nthreads + 1, sizeof(int64_t));
  if (!J.partial) {
    free(img_of);
    return ORACLE_ERR_NOMEM;
  }
  st = run(&J, nthreads);
  if (st == ORACLE_OK) {
    memset(totals, 0, sizeof(int64_t) * per);
    for (int t = 0; t < nthreads; ++t)
      for (size_t e = 0; e < per; ++e) totals[e] += J.partial[(size_t)t * per + e];
    for (int64_t i = 0; i < n_img; ++i) classes[i] = argmin_lowest(totals + i * C, C);
  }
  free(J.partial);
  free(img_of);
  return st;
}

/* ------------------------------------------------------------- public API */

/* The metric of a row stride (128: appearance only; 130: appearance and
 * location) and location weight w >= 0; 0 if invalid. */
static int make_metric(int32_t stride, int64_t w, metric_t *mt) {
  if (!(stride == ORACLE_D || stride == ORACLE_D + ORACLE_LOC) || w < 0 || (stride == ORACLE_D && w != 0)) return 0;
  mt->stride = stride;
  mt->w = w;
  return 1;
}

/* Full matrix of squared distances, out[i*N + j] = ||q_i - r_j||^2 (tiny inputs). */
int oracle_sqdist_matrix_w(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int32_t stride,
                           int64_t w, int64_t *out) {
  metric_t mt;
  if (N < 0 || M < 0 || !make_metric(stride, w, &mt)) return ORACLE_ERR_ARG;
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) out[i * N + j] = sqdist(q + i * mt.stride, ref + j * mt.stride, &mt);
  return ORACLE_OK;
}

/* NN(q_i, kk) for every query: dist/idx [M*kk], ascending by (dist, idx). */
int oracle_knn_w(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int32_t kk, int32_t stride,
                 int64_t w, int64_t *dist, int64_t *idx, int nthreads) {
  if (N < 1 || M < 0 || kk < 1 || (int64_t)kk > N) return ORACLE_ERR_K;
  job_t J;
  memset(&J, 0, sizeof J);
  if (!make_metric(stride, w, &J.mt)) return ORACLE_ERR_ARG;
  J.kind = JOB_KNN;
  J.ref = ref;
  J.N = N;
  J.q = q;
  J.M = M;
  J.k = kk;
  J.out_d = dist;
  J.out_j = idx;
  return run(&J, nthreads);
}

/* NN_C(q_i) for every query and class: out [M*C]; INT64_MAX for empty classes. */
int oracle_class_min_w(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C, const uint8_t *q,
                       int64_t M, int32_t stride, int64_t w, int64_t *out, int nthreads) {
  int st = check_ref(N, C, labels);
  if (st) return st;
  job_t J;
  memset(&J, 0, sizeof J);
  if (!make_metric(stride, w, &J.mt)) return ORACLE_ERR_ARG;
  J.kind = JOB_CLASS_MIN;
  J.ref = ref;
  J.labels = labels;
  J.N = N;
  J.C = C;
  J.q = q;
  J.M = M;
  J.out_d = out;
  return run(&J, nthreads);
}

/* Alg. 2 (LocalNBNN): totals [n_img*C] int64, classes [n_img] int32. */
int oracle_lnbnn_w(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C, const uint8_t *q,
                   const int64_t *offsets, int64_t n_img, int32_t k, int32_t stride, int64_t w, int64_t *totals,
                   int32_t *classes, int nthreads) {
  metric_t mt;
  if (!make_metric(stride, w, &mt)) return ORACLE_ERR_ARG;
  return classify(JOB_LNBNN, ref, labels, N, C, q, offsets, n_img, k, 0, totals, classes, nthreads, mt);
}

/* Local NBNN totals by the closed form sum_i min(0, NN_C(d_i) - dist_B(d_i)). */
int oracle_lnbnn_closed_form_w(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                               const uint8_t *q, const int64_t *offsets, int64_t n_img, int32_t k, int32_t stride,
                               int64_t w, int64_t *totals, int32_t *classes, int nthreads) {
  metric_t mt;
  if (!make_metric(stride, w, &mt)) return ORACLE_ERR_ARG;
  return classify(JOB_CLOSED, ref, labels, N, C, q, offsets, n_img, k, 0, totals, classes, nthreads, mt);
}

/* Alg. 1 (original NBNN): totals [n_img*C] int64, classes [n_img] int32. */
int oracle_nbnn_w(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C, const uint8_t *q,
                  const int64_t *offsets, int64_t n_img, int32_t stride, int64_t w, int64_t *totals,
                  int32_t *classes, int nthreads) {
  metric_t mt;
  if (!make_metric(stride, w, &mt)) return ORACLE_ERR_ARG;
  return classify(JOB_NBNN, ref, labels, N, C, q, offsets, n_img, 0, 0, totals, classes, nthreads, mt);
}

/* The same on 128-byte descriptors (appearance only). */
int oracle_sqdist_matrix(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int64_t *out) {
  return oracle_sqdist_matrix_w(ref, N, q, M, ORACLE_D, 0, out);
}

int oracle_knn(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int32_t kk,
               int64_t *dist, int64_t *idx, int nthreads) {
  return oracle_knn_w(ref, N, q, M, kk, ORACLE_D, 0, dist, idx, nthreads);
}

int oracle_class_min(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                     const uint8_t *q, int64_t M, int64_t *out, int nthreads) {
  return oracle_class_min_w(ref, labels, N, C, q, M, ORACLE_D, 0, out, nthreads);
}

int oracle_lnbnn(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                 const uint8_t *q, const int64_t *offsets, int64_t n_img, int32_t k,
                 int64_t *totals, int32_t *classes, int nthreads) {
  return oracle_lnbnn_w(ref, labels, N, C, q, offsets, n_img, k, ORACLE_D, 0, totals, classes, nthreads);
}

int oracle_lnbnn_closed_form(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                             const uint8_t *q, const int64_t *offsets, int64_t n_img, int32_t k,
                             int64_t *totals, int32_t *classes, int nthreads) {
  return oracle_lnbnn_closed_form_w(ref, labels, N, C, q, offsets, n_img, k, ORACLE_D, 0, totals, classes,
                                    nthreads);
}

int oracle_nbnn(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                const uint8_t *q, const int64_t *offsets, int64_t n_img, int64_t *totals,
                int32_t *classes, int nthreads) {
  return oracle_nbnn_w(ref, labels, N, C, q, offsets, n_img, ORACLE_D, 0, totals, classes, nthreads);
}

/* E4M3 rounding of each x[i] (|x[i]| <= 448), for the pins. */
int oracle_e4m3_round(const int32_t *x, int64_t n, int32_t *out) {
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] < -448 || x[i] > 448) return ORACLE_ERR_ARG;
    out[i] = e4m3_round(x[i]);
  }
  return ORACLE_OK;
}

/* Full matrix of coarse values, out[i*N + j] = coarse(q_i, r_j) (tiny inputs). */
int oracle_coarse_matrix(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int64_t *out) {
  if (N < 0 || M < 0) return ORACLE_ERR_ARG;
  fill_rounded_shifted();
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) out[i * N + j] = coarse(q + i * ORACLE_D, ref + j * ORACLE_D);
  return ORACLE_OK;
}

/* kk nearest by the coarse shortlist of m and exact rerank: dist/idx [M*kk]. */
int oracle_knn_coarse(const uint8_t *ref, int64_t N, const uint8_t *q, int64_t M, int32_t kk, int32_t m,
                      int64_t *dist, int64_t *idx, int nthreads) {
  if (N < 1 || M < 0 || kk < 1 || (int64_t)kk > N || m < kk) return ORACLE_ERR_K;
  fill_rounded_shifted();
  job_t J;
  memset(&J, 0, sizeof J);
  J.kind = JOB_KNN_COARSE;
  J.mt = plain_metric;
  J.ref = ref;
  J.N = N;
  J.q = q;
  J.M = M;
  J.k = kk;
  J.m = m;
  J.out_d = dist;
  J.out_j = idx;
  return run(&J, nthreads);
}

/* Alg. 2 on the neighbours of the coarse shortlist (m >= k + 1). */
int oracle_lnbnn_coarse(const uint8_t *ref, const int32_t *labels, int64_t N, int32_t C,
                        const uint8_t *q, const int64_t *offsets, int64_t n_img, int32_t k, int32_t m,
                        int64_t *totals, int32_t *classes, int nthreads) {
  fill_rounded_shifted();
  return classify(JOB_LNBNN_COARSE, ref, labels, N, C, q, offsets, n_img, k, m, totals, classes, nthreads,
                  plain_metric);
}
