/*
 * Seeded synthetic genotype generator writing PLINK 1 binary (.bed) rows.
 *
 * This module only draws inputs; it holds none of the identity-by-state
 * arithmetic, and both the GPU library's tests and the CPU oracle's tests take
 * their inputs from it.
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator, written
 * here from its published definition.  Every genotype is a pure function of
 * (seed, global variant index, global sample id), so any subset of samples or
 * window of variants can be generated alone and in any thread order.
 *
 * Genotype model (Hardy-Weinberg): two independent allele draws with A2
 * frequency p of the sample's subpopulation; dosage 0/1/2 -> code 0 (hom A1),
 * 2 (het), 3 (hom A2).  An offspring takes one allele of its parent's
 * genotype (chosen uniformly) and draws the other from its subpopulation.  A
 * duplicate copies its source and, at a rate `dup_discord` of variants,
 * switches to one of the two other genotypes.  Missingness (code 1) is applied
 * last, independently per genotype, at the variant's missing rate.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct { uint32_t v[4]; } synth_u4;

static inline void synth_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds. */
static synth_u4 synth_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    synth_mulhilo(0xD2511F53u, c0, &hi0, &lo0);
    synth_mulhilo(0xCD9E8D57u, c2, &hi1, &lo1);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  synth_u4 out = {{c0, c1, c2, c3}};
  return out;
}

enum { SYNTH_BASE = 0, SYNTH_OFFSPRING = 1, SYNTH_DUPLICATE = 2 };
enum { STREAM_GENO = 0, STREAM_EXTRA = 1, STREAM_PAD = 2 };

static inline synth_u4 synth_draw(uint64_t seed, int64_t variant, int64_t gid, uint32_t stream) {
  return synth_philox((uint32_t)variant, (uint32_t)((uint64_t)variant >> 32) ^ (stream << 24),
                      (uint32_t)gid, (uint32_t)((uint64_t)gid >> 32),
                      (uint32_t)seed, (uint32_t)(seed >> 32));
}

static inline uint64_t synth_threshold(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return (uint64_t)1 << 32;
  return (uint64_t)(p * 4294967296.0);
}

/* Dosage (count of A2 alleles) of a base sample before missingness. */
static inline int synth_base_dosage(uint64_t seed, int64_t variant, int64_t gid, uint64_t thr) {
  const synth_u4 u = synth_draw(seed, variant, gid, STREAM_GENO);
  return (int)((uint64_t)u.v[0] < thr) + (int)((uint64_t)u.v[1] < thr);
}

typedef struct {
  int64_t m, var_offset, n;
  uint64_t seed;
  const double* p_pop;
  int32_t n_pop;
  const double* miss_rate;
  const int64_t* gid;
  const int32_t* pop;
  const int32_t* kind;
  const int64_t* src_gid;
  const int32_t* src_pop;
  uint64_t dup_thr;
  int pad_garbage;
  uint8_t* out;
  int64_t next;
  pthread_mutex_t lock;
} synth_job;

static const uint8_t kCode[3] = {0u, 2u, 3u};

static void synth_row(const synth_job* job, int64_t k) {
  const int64_t row_bytes = (job->n + 3) / 4;
  uint8_t* row = job->out + k * row_bytes;
  memset(row, 0, (size_t)row_bytes);
  const int64_t variant = job->var_offset + k;
  const uint64_t miss_thr = synth_threshold(job->miss_rate[k]);
  for (int64_t s = 0; s < job->n; ++s) {
    const int32_t pop = job->pop[s];
    const uint64_t thr = synth_threshold(job->p_pop[(int64_t)pop * job->m + k]);
    const synth_u4 u = synth_draw(job->seed, variant, job->gid[s], STREAM_GENO);
    int dosage;
    if (job->kind[s] == SYNTH_OFFSPRING) {
      const uint64_t pthr = synth_threshold(job->p_pop[(int64_t)job->src_pop[s] * job->m + k]);
      const int dp = synth_base_dosage(job->seed, variant, job->src_gid[s], pthr);
      const synth_u4 e = synth_draw(job->seed, variant, job->gid[s], STREAM_EXTRA);
      const int transmitted = dp == 0 ? 0 : (dp == 2 ? 1 : (int)(e.v[0] & 1u));
      dosage = transmitted + (int)((uint64_t)u.v[1] < thr);
    } else if (job->kind[s] == SYNTH_DUPLICATE) {
      const uint64_t pthr = synth_threshold(job->p_pop[(int64_t)job->src_pop[s] * job->m + k]);
      dosage = synth_base_dosage(job->seed, variant, job->src_gid[s], pthr);
      const synth_u4 e = synth_draw(job->seed, variant, job->gid[s], STREAM_EXTRA);
      if ((uint64_t)e.v[0] < job->dup_thr) dosage = (dosage + 1 + (int)(e.v[1] & 1u)) % 3;
    } else {
      dosage = (int)((uint64_t)u.v[0] < thr) + (int)((uint64_t)u.v[1] < thr);
    }
    uint8_t code = kCode[dosage];
    if ((uint64_t)u.v[2] < miss_thr) code = 1u;
    row[s / 4] |= (uint8_t)(code << (2 * (s % 4)));
  }
  if (job->pad_garbage && (job->n % 4) != 0) {
    const synth_u4 g = synth_draw(job->seed, variant, -1, STREAM_PAD);
    const int used_bits = (int)(2 * (job->n % 4));
    row[row_bytes - 1] |= (uint8_t)((g.v[0] & 0xFFu) & (0xFFu << used_bits));
  }
}

static void* synth_worker(void* arg) {
  synth_job* job = (synth_job*)arg;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    const int64_t k0 = job->next;
    job->next += 64;
    pthread_mutex_unlock(&job->lock);
    if (k0 >= job->m) break;
    const int64_t k1 = k0 + 64 < job->m ? k0 + 64 : job->m;
    for (int64_t k = k0; k < k1; ++k) synth_row(job, k);
  }
  return NULL;
}

/* Fill out[m][ceil(n/4)] with the genotypes of samples (gid, pop, kind,
 * src_gid, src_pop) at variants var_offset .. var_offset + m - 1.  p_pop is
 * [n_pop][m] (A2 frequency per subpopulation and variant), miss_rate is [m].
 * With pad_garbage set, the unused bits of each row's last byte get random
 * values.  Returns 0, or 1 on bad arguments. */
int synth_bed(int64_t m, uint64_t seed, int64_t var_offset,
              const double* p_pop, int32_t n_pop, const double* miss_rate,
              int64_t n, const int64_t* gid, const int32_t* pop, const int32_t* kind,
              const int64_t* src_gid, const int32_t* src_pop,
              double dup_discord, int pad_garbage, uint8_t* out, int threads) {
  if (m <= 0 || n <= 0 || !p_pop || !miss_rate || !gid || !pop || !kind || !src_gid || !src_pop || !out) return 1;
  for (int64_t s = 0; s < n; ++s) {
    if (pop[s] < 0 || pop[s] >= n_pop || src_pop[s] < 0 || src_pop[s] >= n_pop) return 1;
  }
  if (threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    threads = c > 0 ? (int)c : 1;
  }
  synth_job job;
  job.m = m; job.var_offset = var_offset; job.n = n; job.seed = seed;
  job.p_pop = p_pop; job.n_pop = n_pop; job.miss_rate = miss_rate;
  job.gid = gid; job.pop = pop; job.kind = kind; job.src_gid = src_gid; job.src_pop = src_pop;
  job.dup_thr = synth_threshold(dup_discord); job.pad_garbage = pad_garbage; job.out = out; job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  int started = 0;
  if (threads > 1) {
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) {
      if (pthread_create(&tids[t], NULL, synth_worker, &job) == 0) started++;
      else break;
    }
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
  }
  if (started == 0) synth_worker(&job);
  pthread_mutex_destroy(&job.lock);
  return 0;
}

/* The raw Philox4x32-10 block for one counter and key, exported so tests can
 * check the generator against the published known-answer vectors. */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const synth_u4 u = synth_philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  memcpy(out, u.v, sizeof(u.v));
}
