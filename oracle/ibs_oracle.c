/*
 * Plain CPU oracle for all-pairs identity-by-state (IBS) counts.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the CPU-baseline
 * leg of the benchmark can compare the GPU library against an obviously
 * correct reading of the paper.  It shares no code, header or table with the
 * CUDA library.
 *
 * Source of the definition: "Second-generation PLINK" (Chang et al.),
 * section "Improvements in PLINK 1.9 / Bitwise parallelism", the per-marker
 * identity-by-state loop of PLINK 1.07:
 *   for every sample pair (i, j), for every marker k:
 *     1. if i_k or j_k is a missing call, skip the marker;
 *     2. if i_k equals j_k, count IBS2;
 *     3. otherwise, if both bits of the 2-bit codes differ, count IBS0;
 *     4. otherwise count IBS1.
 * The count of markers that were not skipped is N (= IBS0 + IBS1 + IBS2).
 *
 * Genotype codes are the PLINK 1 binary 2-bit values ("Bitwise parallelism":
 * packed 2-bit elements, 4 per byte), read as the integer
 * (byte >> 2*(s % 4)) & 3 for sample s:
 *   0 = homozygous A1, 1 = missing, 2 = heterozygous, 3 = homozygous A2.
 * The input buffer is variant-major: row k holds ceil(n/4) bytes, sample s in
 * byte s/4.  Bits of a row's last byte that belong to no sample are ignored.
 *
 * Derived distance (the paper prints IBS similarity; its complement is used):
 *   dist = (IBS1 + 2*IBS0) / (2*N) in IEEE double, one rounded division,
 *   and NaN when N == 0.
 *
 * The pair loop is deliberately the plain definition: one byte per genotype,
 * one comparison per marker, no blocking.  Threads split the rows i only; each
 * output element is produced by exactly the same sequence of operations
 * whatever the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_MISSING 1

/* Unpack a variant-major packed matrix into one byte per genotype, sample-major:
 * G[s * m + k] = code of sample s at marker k. */
int oracle_unpack(const uint8_t* packed, int64_t n, int64_t m, uint8_t* G) {
  if (n <= 0 || m <= 0 || !packed || !G) return 1;
  const int64_t row_bytes = (n + 3) / 4;
  for (int64_t k = 0; k < m; ++k) {
    const uint8_t* row = packed + k * row_bytes;
    for (int64_t s = 0; s < n; ++s) {
      const uint8_t byte = row[s / 4];
      const int shift = (int)(2 * (s % 4));
      G[s * m + k] = (uint8_t)((byte >> shift) & 3u);
    }
  }
  return 0;
}

/* Unpack selected samples over a window of markers [var_begin, var_begin +
 * var_len) of a variant-major packed matrix with n samples:
 * G[r * var_len + k] = code of sample sel[r] at marker var_begin + k. */
int oracle_unpack_subset(const uint8_t* packed, int64_t n, int64_t m,
                         const int64_t* sel, int64_t n_sel,
                         int64_t var_begin, int64_t var_len, uint8_t* G) {
  if (!packed || !sel || !G || n <= 0 || m <= 0 || n_sel <= 0 || var_len <= 0) return 1;
  if (var_begin < 0 || var_begin + var_len > m) return 1;
  const int64_t row_bytes = (n + 3) / 4;
  for (int64_t r = 0; r < n_sel; ++r) {
    const int64_t s = sel[r];
    if (s < 0 || s >= n) return 1;
    for (int64_t k = 0; k < var_len; ++k) {
      const uint8_t byte = packed[(var_begin + k) * row_bytes + s / 4];
      G[r * var_len + k] = (uint8_t)((byte >> (2 * (s % 4))) & 3u);
    }
  }
  return 0;
}

/* The per-marker rule for one pair of unpacked genotype rows. */
static void oracle_pair(const uint8_t* gi, const uint8_t* gj, int64_t m, int32_t out[4]) {
  int64_t ibs0 = 0, ibs1 = 0, ibs2 = 0, nn = 0;
  for (int64_t k = 0; k < m; ++k) {
    const uint8_t a = gi[k];
    const uint8_t b = gj[k];
    if (a == ORACLE_MISSING || b == ORACLE_MISSING) continue; /* step 1 */
    nn += 1;
    if (a == b) {
      ibs2 += 1;                       /* step 2 */
    } else if ((a ^ b) == 3) {
      ibs0 += 1;                       /* step 3: both bits differ */
    } else {
      ibs1 += 1;                       /* step 4 */
    }
  }
  out[0] = (int32_t)ibs0;
  out[1] = (int32_t)ibs1;
  out[2] = (int32_t)ibs2;
  out[3] = (int32_t)nn;
}

static double oracle_dist(const int32_t c[4]) {
  if (c[3] == 0) return NAN;
  return (double)(c[1] + 2 * (int64_t)c[0]) / (2.0 * (double)c[3]);
}

typedef struct {
  const uint8_t* GA;      /* rows side, sample-major [*][m] */
  const uint8_t* GB;      /* columns side, sample-major [*][m] */
  int64_t m;
  const int64_t* rows;    /* row indices into GA */
  int64_t n_rows;
  const int64_t* cols;    /* column indices into GB */
  int64_t n_cols;
  int32_t* out_counts;    /* [n_rows][n_cols][4] */
  double* out_dist;       /* [n_rows][n_cols] or NULL */
  int64_t next;           /* next row to take (guarded by lock) */
  pthread_mutex_t lock;
} oracle_job;

static void* oracle_worker(void* arg) {
  oracle_job* job = (oracle_job*)arg;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    const int64_t r = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (r >= job->n_rows) break;
    const uint8_t* gi = job->GA + job->rows[r] * job->m;
    for (int64_t c = 0; c < job->n_cols; ++c) {
      const uint8_t* gj = job->GB + job->cols[c] * job->m;
      int32_t* o = job->out_counts + (r * job->n_cols + c) * 4;
      oracle_pair(gi, gj, job->m, o);
      if (job->out_dist) job->out_dist[r * job->n_cols + c] = oracle_dist(o);
    }
  }
  return NULL;
}

/* Counts for every (row, column) combination of two lists of samples, which
 * may come from two different unpacked matrices with the same markers (a query
 * set against a panel) or from the same one (the all-pairs matrix).
 * threads <= 0 means one thread per online core.  Returns the thread count
 * used, or -1 on bad arguments. */
int oracle_ibs_block(const uint8_t* GA, const uint8_t* GB, int64_t m,
                     const int64_t* rows, int64_t n_rows,
                     const int64_t* cols, int64_t n_cols,
                     int32_t* out_counts, double* out_dist, int threads) {
  if (!GA || !GB || !rows || !cols || !out_counts || m <= 0 || n_rows < 0 || n_cols < 0) return -1;
  if (threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    threads = c > 0 ? (int)c : 1;
  }
  if (threads > 1024) threads = 1024;
  if (n_rows < threads) threads = n_rows > 0 ? (int)n_rows : 1;
  oracle_job job;
  job.GA = GA; job.GB = GB; job.m = m;
  job.rows = rows; job.n_rows = n_rows; job.cols = cols; job.n_cols = n_cols;
  job.out_counts = out_counts; job.out_dist = out_dist; job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  if (threads == 1) {
    oracle_worker(&job);
  } else {
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    for (int t = 0; t < threads; ++t) {
      if (pthread_create(&tids[t], NULL, oracle_worker, &job) == 0) started++;
      else break;
    }
    if (started == 0) oracle_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
    if (started > 0) threads = started; else threads = 1;
  }
  pthread_mutex_destroy(&job.lock);
  return threads;
}

/* Full upper triangle including the diagonal, row-major over i <= j:
 * pair (i, j) sits at index i*n - i*(i-1)/2 + (j - i).  Rows are handed to
 * threads one at a time; row i visits j = i .. n-1 in order. */
typedef struct {
  const uint8_t* G;
  int64_t n, m;
  int32_t* out_counts;
  double* out_dist;
  int64_t next;
  pthread_mutex_t lock;
} oracle_tri_job;

static void* oracle_tri_worker(void* arg) {
  oracle_tri_job* job = (oracle_tri_job*)arg;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    const int64_t i = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (i >= job->n) break;
    const int64_t base = i * job->n - i * (i - 1) / 2;
    const uint8_t* gi = job->G + i * job->m;
    for (int64_t j = i; j < job->n; ++j) {
      int32_t* o = job->out_counts + (base + j - i) * 4;
      oracle_pair(gi, job->G + j * job->m, job->m, o);
      if (job->out_dist) job->out_dist[base + j - i] = oracle_dist(o);
    }
  }
  return NULL;
}

int oracle_ibs_triangle(const uint8_t* G, int64_t n, int64_t m,
                        int32_t* out_counts, double* out_dist, int threads) {
  if (!G || n <= 0 || m <= 0 || !out_counts) return -1;
  if (threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    threads = c > 0 ? (int)c : 1;
  }
  if (threads > 1024) threads = 1024;
  if (n < threads) threads = (int)n;
  oracle_tri_job job;
  job.G = G; job.n = n; job.m = m; job.out_counts = out_counts; job.out_dist = out_dist; job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  int started = 0;
  if (threads > 1) {
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) {
      if (pthread_create(&tids[t], NULL, oracle_tri_worker, &job) == 0) started++;
      else break;
    }
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
  }
  if (started == 0) { oracle_tri_worker(&job); started = 1; }
  pthread_mutex_destroy(&job.lock);
  return started;
}

/* ------------------------------------------------------------------------
 * Linkage disequilibrium: the correlation coefficient r between two markers
 * (paper, "Improvements in PLINK 1.9 / Bitwise parallelism", the example of
 * r with missing data).  For markers x and y and samples i:
 *   x_i = -1 for a homozygous minor call, 0 for a heterozygous or missing call,
 *         +1 for a homozygous major call (y likewise);
 *   S_xy = the samples where neither x nor y is missing;
 *   r = (|S_xy|^-1 sum_{i in S} x_i y_i - xbar ybar)
 *       / sqrt((x2bar - xbar^2) (y2bar - ybar^2)),
 * with xbar, x2bar, ybar, y2bar the means of x, x^2, y, y^2 over S_xy.
 * Multiplying numerator and denominator by |S_xy|^2 gives the same value from
 * integer sums, which is what is computed here (exactly, then one square root
 * and one division in double):
 *   r = (N Sxy - Sx Sy) / sqrt((N Sxx - Sx^2) (N Syy - Sy^2)),  N = |S_xy|.
 * Readings where the paper is silent:
 *   - major allele: A1 is major when its frequency among the marker's
 *     non-missing calls is at least 1/2, i.e. when #hom A1 >= #hom A2 (ties
 *     orient to A1);
 *   - r is NaN when N = 0 or either variance term is 0.
 * Output: pairs (a, b) with 1 <= b - a <= window, at r_out[a * window + (b - a - 1)]
 * (and |S_xy| at n_out, which may be NULL); slots with b >= m hold NaN and 0.
 * G is sample-major, one byte per genotype: G[s * m + k].  Threads split the
 * markers a only.
 */
typedef struct {
  const uint8_t* G;
  int64_t n, m, window;
  const int8_t* major_a1;  /* per marker: 1 when A1 is the major allele */
  double* r_out;
  int32_t* n_out;
  int64_t next;
  pthread_mutex_t lock;
} oracle_ld_job;

/* x value of one call of marker k: +1 homozygous major, -1 homozygous minor, 0 otherwise. */
static int oracle_ld_value(uint8_t code, int major_a1) {
  if (code == 0) return major_a1 ? 1 : -1; /* homozygous A1 */
  if (code == 3) return major_a1 ? -1 : 1; /* homozygous A2 */
  return 0;                                /* heterozygous (missing calls are skipped) */
}

static void* oracle_ld_worker(void* arg) {
  oracle_ld_job* job = (oracle_ld_job*)arg;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    const int64_t a = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (a >= job->m) break;
    for (int64_t d = 0; d < job->window; ++d) {
      const int64_t b = a + 1 + d, slot = a * job->window + d;
      if (b >= job->m) {
        job->r_out[slot] = NAN;
        if (job->n_out) job->n_out[slot] = 0;
        continue;
      }
      int64_t N = 0, Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
      for (int64_t s = 0; s < job->n; ++s) {
        const uint8_t ca = job->G[s * job->m + a], cb = job->G[s * job->m + b];
        if (ca == ORACLE_MISSING || cb == ORACLE_MISSING) continue;
        const int x = oracle_ld_value(ca, job->major_a1[a]), y = oracle_ld_value(cb, job->major_a1[b]);
        N += 1;
        Sx += x;
        Sy += y;
        Sxx += x * x;
        Syy += y * y;
        Sxy += x * y;
      }
      const int64_t vx = N * Sxx - Sx * Sx, vy = N * Syy - Sy * Sy;
      job->r_out[slot] = (N == 0 || vx == 0 || vy == 0)
                             ? NAN
                             : (double)(N * Sxy - Sx * Sy) / sqrt((double)vx * (double)vy);
      if (job->n_out) job->n_out[slot] = (int32_t)N;
    }
  }
  return NULL;
}

int oracle_ld_r(const uint8_t* G, int64_t n, int64_t m, int64_t window, double* r_out, int32_t* n_out,
                int threads) {
  if (!G || n <= 0 || m <= 0 || window <= 0 || !r_out) return -1;
  int8_t* major_a1 = (int8_t*)malloc((size_t)m);
  if (!major_a1) return -1;
  for (int64_t k = 0; k < m; ++k) {
    int64_t hom_a1 = 0, hom_a2 = 0;
    for (int64_t s = 0; s < n; ++s) {
      const uint8_t c = G[s * m + k];
      hom_a1 += c == 0;
      hom_a2 += c == 3;
    }
    major_a1[k] = hom_a1 >= hom_a2 ? 1 : 0;
  }
  if (threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    threads = c > 0 ? (int)c : 1;
  }
  if (threads > 1024) threads = 1024;
  if (m < threads) threads = (int)m;
  oracle_ld_job job;
  job.G = G; job.n = n; job.m = m; job.window = window; job.major_a1 = major_a1;
  job.r_out = r_out; job.n_out = n_out; job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  int started = 0;
  if (threads > 1) {
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) {
      if (pthread_create(&tids[t], NULL, oracle_ld_worker, &job) == 0) started++;
      else break;
    }
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
  }
  if (started == 0) { oracle_ld_worker(&job); started = 1; }
  pthread_mutex_destroy(&job.lock);
  free(major_a1);
  return started;
}

/* ------------------------------------------------------------------------
 * Complete-linkage clustering of the samples under a distance matrix (paper,
 * "Identity-by-state matrices, complete linkage clustering": PLINK's
 * --cluster runs complete linkage on the IBS matrix), in the textbook greedy
 * form: start from n singleton clusters; at every step merge the two active
 * clusters at the smallest complete-linkage distance
 *   D(A, B) = max over a in A, b in B of d(a, b),
 * maintained by D(A u B, C) = max(D(A, C), D(B, C)).
 * Readings where the paper is silent:
 *   - the input is the distance (IBS1 + 2 IBS0) / (2N) as the library writes
 *     it: the upper triangle including the diagonal, row-major, diagonal
 *     ignored; NaN (no common non-missing marker) counts as +infinity;
 *   - ties: a cluster is represented by its smallest member; among equal
 *     distances the pair with the smallest (representative of A,
 *     representative of B), A's representative below B's, merges first;
 *   - output Z[n-1][4] = (id1, id2, height, size), id1 < id2, with singletons
 *     numbered 0..n-1 and the cluster formed at step s numbered n + s (the
 *     convention of scipy's linkage).
 * O(n^3): the whole active triangle is searched at every step.
 */
int oracle_complete_linkage(const double* tri, int64_t n, double* Z) {
  if (!tri || n <= 0 || !Z) return -1;
  if (n == 1) return 0;
  double* D = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  int64_t* id = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* size = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  char* active = (char*)malloc((size_t)n);
  if (!D || !id || !size || !active) {
    free(D); free(id); free(size); free(active);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = i; j < n; ++j) {
      double d = tri[i * n - i * (i - 1) / 2 + (j - i)];
      if (d != d) d = INFINITY;
      D[i * n + j] = d;
      D[j * n + i] = d;
    }
    id[i] = i;
    size[i] = 1;
    active[i] = 1;
  }
  for (int64_t step = 0; step < n - 1; ++step) {
    int64_t bi = -1, bj = -1;
    double best = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (!active[i]) continue;
      for (int64_t j = i + 1; j < n; ++j) {
        if (!active[j]) continue;
        const double d = D[i * n + j];
        if (bi < 0 || d < best) { /* strict: the first (smallest i, then j) minimum wins */
          best = d;
          bi = i;
          bj = j;
        }
      }
    }
    const int64_t a = id[bi] < id[bj] ? id[bi] : id[bj], b = id[bi] < id[bj] ? id[bj] : id[bi];
    Z[step * 4 + 0] = (double)a;
    Z[step * 4 + 1] = (double)b;
    Z[step * 4 + 2] = best;
    Z[step * 4 + 3] = (double)(size[bi] + size[bj]);
    for (int64_t k = 0; k < n; ++k) {
      if (!active[k] || k == bi || k == bj) continue;
      const double d = D[bi * n + k] > D[bj * n + k] ? D[bi * n + k] : D[bj * n + k];
      D[bi * n + k] = d;
      D[k * n + bi] = d;
    }
    active[bj] = 0;
    id[bi] = n + step;
    size[bi] += size[bj];
  }
  free(D); free(id); free(size); free(active);
  return 0;
}

/* ------------------------------------------------------------------------
 * Genomic relationship matrix (paper, "Other noteworthy algorithms / Partial
 * sum lookup": the GCTA relationship matrix as a weighted sum over markers of
 * seven per-marker cases).  For marker i, with p the frequency of the counted
 * allele over the marker's non-missing calls and x its count in a call (2 hom
 * A1, 1 het, 0 hom A2), a pair of samples with both calls present adds
 *   (x_j - 2p)(x_k - 2p) / (2p(1 - p)),
 * and a pair with a missing call adds nothing and is left out of the pair's
 * denominator ("subtract 1 from the final denominator").  So
 *   A_jk = (sum of the increments) / (number of markers where both are present).
 * Readings where the paper is silent or garbled:
 *   - the counted allele: A1.  The paper's table counts the major allele while
 *     naming q the minor allele frequency; the value does not depend on the
 *     choice, since counting the other allele negates both factors;
 *   - markers with p = 0 or 1 (monomorphic, or without calls) would divide by
 *     zero and are left out of both the sums and the denominators;
 *   - A_jk = NaN when no marker is left for the pair.
 * The algorithm follows the paper's first draft: per marker, a table of the
 * increments of the six cases without a missing call, then one lookup and one
 * addition per pair and marker (in double).
 * Output: upper triangle with diagonal, row-major over j <= k (the IBS layout).
 */
typedef struct {
  const uint8_t* G;
  int64_t n, m;
  const double* table; /* per marker 16 entries: [code_j * 4 + code_k], 0 where a call is missing */
  const char* used;    /* per marker: 1 when polymorphic */
  const int64_t* rows; /* NULL: the whole upper triangle; else these rows, every column */
  int64_t n_rows;
  double* out;
  int64_t next;
  pthread_mutex_t lock;
} oracle_grm_job;

/* A_jk: the pair's increments summed over the used markers where both calls
 * are present, divided by their number. */
static double oracle_grm_pair(const oracle_grm_job* job, int64_t j, int64_t k) {
  const int64_t m = job->m;
  double sum = 0.0;
  int64_t cnt = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (!job->used[i]) continue;
    const uint8_t gj = job->G[j * m + i], gk = job->G[k * m + i];
    if (gj == ORACLE_MISSING || gk == ORACLE_MISSING) continue;
    sum += job->table[i * 16 + gj * 4 + gk];
    cnt += 1;
  }
  return cnt == 0 ? NAN : sum / (double)cnt;
}

static void* oracle_grm_worker(void* arg) {
  oracle_grm_job* job = (oracle_grm_job*)arg;
  const int64_t n = job->n;
  const int64_t units = job->rows ? job->n_rows : n;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    const int64_t u = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (u >= units) break;
    if (job->rows) {
      const int64_t j = job->rows[u];
      for (int64_t k = 0; k < n; ++k) job->out[u * n + k] = oracle_grm_pair(job, j, k);
    } else {
      const int64_t base = u * n - u * (u - 1) / 2;
      for (int64_t k = u; k < n; ++k) job->out[base + (k - u)] = oracle_grm_pair(job, u, k);
    }
  }
  return NULL;
}

static int oracle_grm_run(const uint8_t* G, int64_t n, int64_t m, const int64_t* rows, int64_t n_rows, double* out,
                          int threads) {
  if (!G || n <= 0 || m <= 0 || !out || (rows && n_rows <= 0)) return -1;
  for (int64_t r = 0; rows && r < n_rows; ++r)
    if (rows[r] < 0 || rows[r] >= n) return -1;
  double* table = (double*)calloc((size_t)m * 16, sizeof(double));
  char* used = (char*)calloc((size_t)m, 1);
  if (!table || !used) {
    free(table);
    free(used);
    return -1;
  }
  for (int64_t i = 0; i < m; ++i) {
    int64_t alleles = 0, calls = 0;
    for (int64_t s = 0; s < n; ++s) {
      const uint8_t c = G[s * m + i];
      if (c == ORACLE_MISSING) continue;
      calls += 1;
      alleles += c == 0 ? 2 : (c == 2 ? 1 : 0);
    }
    if (calls == 0) continue;
    const double p = (double)alleles / (2.0 * (double)calls);
    if (p <= 0.0 || p >= 1.0) continue;
    used[i] = 1;
    const double x_of[4] = {2.0, 0.0, 1.0, 0.0}; /* A1 count by code; code 1 (missing) unused */
    const double denom = 2.0 * p * (1.0 - p);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        if (a != ORACLE_MISSING && b != ORACLE_MISSING)
          table[i * 16 + a * 4 + b] = (x_of[a] - 2.0 * p) * (x_of[b] - 2.0 * p) / denom;
  }
  const int64_t units = rows ? n_rows : n;
  if (threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    threads = c > 0 ? (int)c : 1;
  }
  if (threads > 1024) threads = 1024;
  if (units < threads) threads = (int)units;
  oracle_grm_job job;
  job.G = G; job.n = n; job.m = m; job.table = table; job.used = used; job.rows = rows; job.n_rows = n_rows;
  job.out = out; job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  int started = 0;
  if (threads > 1) {
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) {
      if (pthread_create(&tids[t], NULL, oracle_grm_worker, &job) == 0) started++;
      else break;
    }
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
  }
  if (started == 0) { oracle_grm_worker(&job); started = 1; }
  pthread_mutex_destroy(&job.lock);
  free(table);
  free(used);
  return started;
}

int oracle_grm(const uint8_t* G, int64_t n, int64_t m, double* out, int threads) {
  return oracle_grm_run(G, n, m, NULL, 0, out, threads);
}

/* Rows rows[0..n_rows) of the full symmetric matrix: out[r * n + k] = A_{rows[r], k}
 * (the frequencies still come from all n samples). */
int oracle_grm_rows(const uint8_t* G, int64_t n, int64_t m, const int64_t* rows, int64_t n_rows, double* out,
                    int threads) {
  return oracle_grm_run(G, n, m, rows, n_rows, out, threads);
}
