/*
 * ktau_oracle.c -- CPU oracle for exact Kendall tau-b (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load this
 * file's library. It shares no code, header or table with the CUDA library; the product path
 * never calls it.
 *
 * Everything here is plain, slow and written from the paper (arXiv 1704.03767):
 *   ko_pair_definition : the definition of concordance (Sec. 1) counted directly over all
 *                        n(n-1)/2 sample pairs in the sign form of Algorithm 1, extended with
 *                        the tie counts n_1, n_2, n_3 of Table 1.  O(n^2).
 *   ko_pair_knight     : Knight's sort-based method with exact ties, Sec. 3.2 Steps 1-5; Step 3
 *                        is a recursive merge sort by v that counts its exchanges (strict
 *                        comparison, equal v taken from the lower half, as Algorithm 2 requires).
 *   ko_tau_b           : Eq. 3.
 *   ko_F / ko_job_id / ko_job_coord_formula / ko_job_coord : Eq. 4-10 (diagonal included).
 *   ko_rank            : the rank transform of Sec. 3 (stable argsort, dense rank, tie pairs).
 *   ko_allpairs        : Sec. 4.2-4.3: q x q tiles over the upper triangle, tile ids mapped back
 *                        with Eq. 13-14; the requested pair range is cut into equal contiguous
 *                        slices, one per thread (static distribution).
 *   ko_rect            : every query row against every database row (Sec. 1 query search).
 * Inputs are FP64 (the caller converts float32/int32 exactly). Counts are int64.
 * Parity pins: hand-worked examples, scipy's tau-b, identities, brute force between the two
 * independent pair counters, exhaustive bijection round trips (see tests/).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t nc, nd, n1, n2, n3;
} ko_counts;

/* Sign of a difference written as comparisons, as calc_sign in Algorithm 1. */
static int ko_sign_cmp(double a, double b) { return (a > b) - (a < b); }

/* Definition (Sec. 1, Table 1): over every sample pair a < b,
 *   s = sign(u_a - u_b) * sign(v_a - v_b); concordant if s > 0, discordant if s < 0;
 *   n_1 counts pairs tied in u, n_2 tied in v, n_3 tied in both. */
void ko_pair_definition(const double* u, const double* v, int64_t n, ko_counts* c) {
  int64_t nc = 0, nd = 0, n1 = 0, n2 = 0, n3 = 0;
  for (int64_t a = 0; a < n; ++a) {
    for (int64_t b = a + 1; b < n; ++b) {
      int su = ko_sign_cmp(u[a], u[b]);
      int sv = ko_sign_cmp(v[a], v[b]);
      int s = su * sv;
      nc += (s > 0);
      nd += (s < 0);
      n1 += (su == 0);
      n2 += (sv == 0);
      n3 += (su == 0 && sv == 0);
    }
  }
  c->nc = nc;
  c->nd = nd;
  c->n1 = n1;
  c->n2 = n2;
  c->n3 = n3;
}

/* ---- Knight's method, Sec. 3.2 ---- */
typedef struct {
  double u, v;
} ko_joint;

static int ko_joint_cmp(const void* pa, const void* pb) {
  const ko_joint* a = (const ko_joint*)pa;
  const ko_joint* b = (const ko_joint*)pb;
  if (a->u < b->u) return -1;
  if (a->u > b->u) return 1;
  if (a->v < b->v) return -1;
  if (a->v > b->v) return 1;
  return 0;
}

/* Step 3 (Sec. 3.2): the list, already in (u, v) order, is put in v order by merge sort, and the
 * exchanges that sort performs are counted; that count is n_d.
 *
 * Written as a recursive top-down merge sort over x[lo, hi): sort each half, then fill the
 * scratch span t[lo, hi) front to back, each time choosing the smaller head. An element chosen
 * from the upper half jumps over every element still waiting in the lower half. Each of those
 * came earlier in the (u, v) order and has a strictly larger v, so its u is strictly smaller:
 * each jump is one discordant pair. On equal v the lower-half element is chosen first, so a tie
 * in v is never counted (the pair is tied, not discordant). On return x[lo, hi) is in v order. */
static int64_t ko_sort_count(ko_joint* x, ko_joint* t, int64_t lo, int64_t hi) {
  if (hi - lo < 2) return 0;
  const int64_t half = lo + (hi - lo) / 2;
  int64_t swaps = ko_sort_count(x, t, lo, half) + ko_sort_count(x, t, half, hi);
  int64_t a = lo, b = half;
  for (int64_t k = lo; k < hi; ++k) {
    const int lower_done = (a == half);
    const int upper_done = (b == hi);
    if (!upper_done && (lower_done || x[b].v < x[a].v)) {
      swaps += half - a; /* elements of the lower half still waiting */
      t[k] = x[b];
      ++b;
    } else {
      t[k] = x[a];
      ++a;
    }
  }
  memcpy(x + lo, t + lo, (size_t)(hi - lo) * sizeof(ko_joint));
  return swaps;
}

/* Sum over runs of equal keys of t(t-1)/2, for a list already sorted so equal keys are adjacent. */
static int64_t ko_tie_pairs_u(const ko_joint* x, int64_t n) {
  int64_t total = 0, run = 1;
  for (int64_t i = 1; i <= n; ++i) {
    if (i < n && x[i].u == x[i - 1].u) {
      ++run;
    } else {
      total += run * (run - 1) / 2;
      run = 1;
    }
  }
  return total;
}
static int64_t ko_tie_pairs_uv(const ko_joint* x, int64_t n) {
  int64_t total = 0, run = 1;
  for (int64_t i = 1; i <= n; ++i) {
    if (i < n && x[i].u == x[i - 1].u && x[i].v == x[i - 1].v) {
      ++run;
    } else {
      total += run * (run - 1) / 2;
      run = 1;
    }
  }
  return total;
}
static int64_t ko_tie_pairs_v(const ko_joint* x, int64_t n) {
  int64_t total = 0, run = 1;
  for (int64_t i = 1; i <= n; ++i) {
    if (i < n && x[i].v == x[i - 1].v) {
      ++run;
    } else {
      total += run * (run - 1) / 2;
      run = 1;
    }
  }
  return total;
}

/* Steps 1-5 of Sec. 3.2 for one pair. `work` holds 2n ko_joint. */
static void ko_pair_knight_work(const double* u, const double* v, int64_t n, ko_counts* c,
                                ko_joint* work) {
  ko_joint* pairs = work;
  ko_joint* buffer = work + n;
  for (int64_t i = 0; i < n; ++i) {
    pairs[i].u = u[i];
    pairs[i].v = v[i];
  }
  /* Step 1: sort joint variables by u, then by v. */
  qsort(pairs, (size_t)n, sizeof(ko_joint), ko_joint_cmp);
  /* Step 2: n_1 (ties in u) and n_3 (joint ties). */
  int64_t n1 = ko_tie_pairs_u(pairs, n);
  int64_t n3 = ko_tie_pairs_uv(pairs, n);
  /* Step 3: discordant pairs while re-sorting by v. */
  int64_t nd = ko_sort_count(pairs, buffer, 0, n);
  /* Step 4: n_2 (ties in v) on the list now sorted by v. */
  int64_t n2 = ko_tie_pairs_v(pairs, n);
  /* Step 5: n_c - n_d = n_0 - n_1 - n_2 + n_3 - 2 n_d. */
  int64_t n0 = n * (n - 1) / 2;
  int64_t S = n0 - n1 - n2 + n3 - 2 * nd;
  c->nc = S + nd;
  c->nd = nd;
  c->n1 = n1;
  c->n2 = n2;
  c->n3 = n3;
}

int ko_pair_knight(const double* u, const double* v, int64_t n, ko_counts* c) {
  ko_joint* work = (ko_joint*)malloc((size_t)(2 * n > 0 ? 2 * n : 1) * sizeof(ko_joint));
  if (!work) return -1;
  ko_pair_knight_work(u, v, n, c, work);
  free(work);
  return 0;
}

/* Eq. 3. NaN when a variable is constant (the denominator vanishes). */
double ko_tau_b(int64_t S, int64_t n1, int64_t n2, int64_t n) {
  int64_t n0 = n * (n - 1) / 2;
  int64_t du = n0 - n1, dv = n0 - n2;
  if (du == 0 || dv == 0) return NAN;
  return (double)S / sqrt((double)du * (double)dv);
}

/* ---- Bijection between job id and (y, x), Sec. 4.1 (diagonal included) ---- */

/* Eq. 5: number of upper-triangle cells before row y of an m x m job matrix. */
int64_t ko_F(int64_t m, int64_t y) { return y * (2 * m - y + 1) / 2; }

/* Eq. 4. */
int64_t ko_job_id(int64_t m, int64_t y, int64_t x) { return ko_F(m, y) + x - y; }

/* Eq. 9-10 exactly as printed: y = ceil(m - 0.5 - sqrt(m^2 + m + 0.25 - 2(J+1))), x = J + y - F(y),
 * evaluated in FP64. */
void ko_job_coord_formula(int64_t m, int64_t J, int64_t* y, int64_t* x) {
  double md = (double)m;
  double z = md - 0.5 - sqrt(md * md + md + 0.25 - 2.0 * ((double)J + 1.0));
  int64_t yy = (int64_t)ceil(z);
  *y = yy;
  *x = J + yy - ko_F(m, yy);
}

/* Eq. 9-10 followed by an integer check of the defining inequalities F(y) <= J < F(y+1)
 * (Eq. 6), stepping y by one where FP64 rounding of the square root moved the ceiling. */
void ko_job_coord(int64_t m, int64_t J, int64_t* y, int64_t* x) {
  int64_t yy, xx;
  ko_job_coord_formula(m, J, &yy, &xx);
  if (yy < 0) yy = 0;
  if (yy > m - 1) yy = m - 1;
  while (yy > 0 && ko_F(m, yy) > J) --yy;
  while (yy < m - 1 && ko_F(m, yy + 1) <= J) ++yy;
  *y = yy;
  *x = J + yy - ko_F(m, yy);
}

/* ---- Rank transform, Sec. 3 ---- */

/* Stable merge sort of indices by value (ties keep index order). */
static void ko_argsort_stable(const double* x, int64_t n, int64_t* idx, int64_t* tmp) {
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  for (int64_t s = 1; s < n; s *= 2) {
    for (int64_t l = 0; l < n; l += 2 * s) {
      int64_t mid = l + s < n ? l + s : n;
      int64_t r = l + 2 * s < n ? l + 2 * s : n;
      int64_t a = l, b = mid, p = l;
      while (a < mid && b < r) {
        if (x[idx[b]] < x[idx[a]])
          tmp[p++] = idx[b++];
        else
          tmp[p++] = idx[a++];
      }
      while (a < mid) tmp[p++] = idx[a++];
      while (b < r) tmp[p++] = idx[b++];
    }
    memcpy(idx, tmp, (size_t)n * sizeof(int64_t));
  }
}

/* perm[k] = index of the k-th smallest value (stable), rank[i] = number of distinct values
 * smaller than x[i], *T = sum over groups of equal values of t(t-1)/2. Returns -1 on
 * allocation failure. */
int ko_rank(const double* x, int64_t n, int64_t* perm, int64_t* rank, int64_t* T) {
  int64_t* tmp = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!tmp) return -1;
  ko_argsort_stable(x, n, perm, tmp);
  free(tmp);
  int64_t d = 0, run = 1, ties = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0) {
      if (x[perm[k]] == x[perm[k - 1]]) {
        ++run;
      } else {
        ties += run * (run - 1) / 2;
        run = 1;
        ++d;
      }
    }
    rank[perm[k]] = d;
  }
  ties += run * (run - 1) / 2;
  *T = ties;
  return 0;
}

/* ---- All pairs, Sec. 4.2-4.3 ---- */

typedef struct {
  const double* X;
  int64_t m, n, ld, q, w;
  uint64_t p_lo, p_hi; /* this thread's slice of the requested range */
  int64_t tile_begin, tile_end;
  uint64_t p_begin;    /* start of the requested range (outputs are indexed from it) */
  int method;          /* 0 = definition, 1 = Knight */
  int64_t *S, *n3, *nd, *n1, *n2;
  double* tau;
  int status;
} ko_job;

static void* ko_allpairs_worker(void* arg) {
  ko_job* jb = (ko_job*)arg;
  ko_joint* work = (ko_joint*)malloc((size_t)(2 * jb->n) * sizeof(ko_joint));
  if (!work) {
    jb->status = -1;
    return NULL;
  }
  const int64_t m = jb->m;
  for (int64_t t = jb->tile_begin; t < jb->tile_end; ++t) {
    int64_t yq, xq;
    ko_job_coord(jb->w, t, &yq, &xq); /* Eq. 13-14 on the w x w tile matrix */
    for (int64_t y = yq * jb->q; y < (yq + 1) * jb->q && y < m; ++y) {
      for (int64_t x = xq * jb->q; x < (xq + 1) * jb->q && x < m; ++x) {
        if (x <= y) continue; /* strict upper triangle: the diagonal is not a pair */
        uint64_t p = (uint64_t)(y * (2 * m - y - 1) / 2 + (x - y - 1));
        if (p < jb->p_lo || p >= jb->p_hi) continue; /* another thread's pair */
        const double* u = jb->X + y * jb->ld;
        const double* v = jb->X + x * jb->ld;
        ko_counts c;
        if (jb->method == 0)
          ko_pair_definition(u, v, jb->n, &c);
        else
          ko_pair_knight_work(u, v, jb->n, &c, work);
        uint64_t k = p - jb->p_begin;
        int64_t S = c.nc - c.nd;
        if (jb->S) jb->S[k] = S;
        if (jb->n3) jb->n3[k] = c.n3;
        if (jb->nd) jb->nd[k] = c.nd;
        if (jb->n1) jb->n1[k] = c.n1;
        if (jb->n2) jb->n2[k] = c.n2;
        if (jb->tau) jb->tau[k] = ko_tau_b(S, c.n1, c.n2, jb->n);
      }
    }
  }
  free(work);
  return NULL;
}

/* Row of the pair with packed index p: the strict upper triangle of an m x m matrix is the
 * diagonal-included triangle of an (m-1) x (m-1) matrix (pair (y, x) <-> cell (y, x-1)), so
 * Eq. 9-10 with the Eq. 6 check on m-1 gives y. */
static int64_t ko_pair_row(int64_t m, uint64_t p) {
  int64_t y, x1;
  ko_job_coord(m - 1, (int64_t)p, &y, &x1);
  return y;
}

/* Every pair (y < x) of the m x n matrix X (row stride ld) whose packed index
 * p = y(2m-y-1)/2 + (x-y-1) lies in [p_begin, p_end); outputs are indexed by p - p_begin and
 * any may be NULL. q is the tile side (Sec. 4.2) and `threads` the number of worker threads.
 * The requested range is cut into `threads` contiguous slices of equal pair counts (a static
 * distribution, Sec. 4.3.2 and 4.4). A thread walks, in tile-id order (Eq. 13-14), the tiles
 * of the tile rows its slice touches, and counts only the pairs of its own slice, so every
 * thread does the same share of the requested work whatever part of the triangle it lies in. */
int ko_allpairs(const double* X, int64_t m, int64_t n, int64_t ld, int method, int64_t q,
                int threads, uint64_t p_begin, uint64_t p_end, int64_t* S, int64_t* n3,
                int64_t* nd, int64_t* n1, int64_t* n2, double* tau) {
  if (q < 1) q = 8;
  if (threads < 1) threads = 1;
  if (m < 2 || p_end <= p_begin) return 0;
  const int64_t w = (m + q - 1) / q;
  const uint64_t span = p_end - p_begin;
  ko_job* jobs = (ko_job*)calloc((size_t)threads, sizeof(ko_job));
  pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
  char* started = (char*)calloc((size_t)threads, 1);
  if (!jobs || !tids || !started) {
    free(jobs);
    free(tids);
    free(started);
    return -1;
  }
  for (int t = 0; t < threads; ++t) {
    ko_job* jb = &jobs[t];
    jb->X = X;
    jb->m = m;
    jb->n = n;
    jb->ld = ld;
    jb->q = q;
    jb->w = w;
    jb->p_lo = p_begin + span * (uint64_t)t / (uint64_t)threads;
    jb->p_hi = p_begin + span * (uint64_t)(t + 1) / (uint64_t)threads;
    if (jb->p_lo < jb->p_hi) {
      /* tile rows from the first to the last pair row of the slice, whole rows of tiles */
      const int64_t yq_first = ko_pair_row(m, jb->p_lo) / q;
      const int64_t yq_last = ko_pair_row(m, jb->p_hi - 1) / q;
      jb->tile_begin = ko_job_id(w, yq_first, yq_first);
      jb->tile_end = ko_job_id(w, yq_last, w - 1) + 1;
    }
    jb->p_begin = p_begin;
    jb->method = method;
    jb->S = S;
    jb->n3 = n3;
    jb->nd = nd;
    jb->n1 = n1;
    jb->n2 = n2;
    jb->tau = tau;
  }
  for (int t = 0; t < threads; ++t) {
    if (threads > 1 && pthread_create(&tids[t], NULL, ko_allpairs_worker, &jobs[t]) == 0)
      started[t] = 1;
    else
      ko_allpairs_worker(&jobs[t]);
  }
  int status = 0;
  for (int t = 0; t < threads; ++t)
    if (started[t]) pthread_join(tids[t], NULL);
  for (int t = 0; t < threads; ++t)
    if (jobs[t].status) status = -1;
  free(jobs);
  free(tids);
  free(started);
  return status;
}

/* Query search (Sec. 1): every row of Q (b x n) against every row of D (mdb x n), Knight
 * counting. Outputs are [b][mdb] row-major; any may be NULL. */
int ko_rect(const double* Q, int64_t b, int64_t ldq, const double* D, int64_t mdb, int64_t ldd,
            int64_t n, int64_t* S, int64_t* n3, int64_t* n1, int64_t* n2, double* tau) {
  ko_joint* work = (ko_joint*)malloc((size_t)(2 * n) * sizeof(ko_joint));
  if (!work) return -1;
  for (int64_t i = 0; i < b; ++i) {
    for (int64_t j = 0; j < mdb; ++j) {
      ko_counts c;
      ko_pair_knight_work(Q + i * ldq, D + j * ldd, n, &c, work);
      int64_t k = i * mdb + j;
      int64_t s = c.nc - c.nd;
      if (S) S[k] = s;
      if (n3) n3[k] = c.n3;
      if (n1) n1[k] = c.n1;
      if (n2) n2[k] = c.n2;
      if (tau) tau[k] = ko_tau_b(s, c.n1, c.n2, n);
    }
  }
  free(work);
  return 0;
}
