/*
 * libibs: all-pairs identity-by-state (IBS) counts over PLINK 1 binary
 * genotype matrices on one GB300 GPU (sm_103a).
 *
 * The operation (paper "Second-generation PLINK", section "Improvements in
 * PLINK 1.9 / Bitwise parallelism"): for every sample pair (i, j) and every
 * marker k, skip k when either call is missing; otherwise count IBS2 when the
 * 2-bit codes are equal, IBS0 when both bits differ and IBS1 otherwise.
 * N = IBS0 + IBS1 + IBS2 is the number of jointly non-missing markers.  The
 * paper's replacement evaluates the same counts with XOR, a missing-call mask
 * and a population count over blocks of markers.
 *
 * This library's default form counts on the tensor cores instead (tcgen05,
 * sm_103a).  Per sample and marker it writes four indicator values: V = 1 for
 * a present call, U = +1 homozygous / -1 heterozygous, Q = 1 hom A2,
 * R = 1 hom A1 (all 0 when missing).  Then N = V V^T, IBS0 = Q R^T + R Q^T,
 * IBS1 = (N - U U^T) / 2 and IBS2 = N - IBS0 - IBS1.  The products are
 * E2M1 (kind::mxf4, unit scale factors) or E4M3 (kind::f8f6f4) matrix
 * products accumulated in FP32; every term is an integer well below 2^24, so
 * the counts are exact.  The paper's own scheme (XOR / mask / POPC on
 * sample-major bit planes, LOP3 and POPC in registers) is kept as the
 * integer form, selected with IBS_KERNEL_PLAIN or IBS_KERNEL_CSA; both forms
 * give identical counts.
 *
 * Input layout (every entry point): a variant-major packed matrix, row k =
 * ceil(n/4) bytes, sample s in bits 2*(s%4) (low) and 2*(s%4)+1 (high) of
 * byte s/4, code = (byte >> 2*(s%4)) & 3 with 0 = hom A1, 1 = missing,
 * 2 = het, 3 = hom A2 (the .bed payload without its 3-byte magic header).
 * Padding bits of a row's last byte are ignored.
 *
 * Outputs: counts are int32 quadruples {IBS0, IBS1, IBS2, N}; the distance is
 * (IBS1 + 2*IBS0) / (2*N) in IEEE double (NaN when N == 0), the complement of
 * the IBS similarity printed by the paper's `--distance ibs`.  The all-pairs
 * layout is the upper triangle including the diagonal, row-major over i <= j:
 * pair (i, j) is element i*n - i*(i-1)/2 + (j - i) of P = n*(n+1)/2; with
 * IBS_OUT_SQUARE it is the full [n][n] matrix (both halves written).
 *
 * Conventions.  Every call returns an ibs_status and never throws; on a
 * non-OK return the outputs are undefined and ibs_last_error() (thread-local)
 * says why.  All input and output buffers are caller-owned; the library owns
 * its context, its bit-plane workspace, work lists, the resident panel and
 * the serving engine, all freed by ibs_shutdown.  Work is enqueued on the
 * caller's CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) and the call returns after enqueue unless stated otherwise.  There
 * is no CPU fallback: without a usable sm_103a device the calls fail with
 * IBS_ECUDA.
 */
#ifndef IBS_H_
#define IBS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibs_ctx ibs_ctx; /* opaque, library-owned */

typedef enum {
  IBS_OK = 0,
  IBS_EINVAL = 1,     /* bad argument: null pointer, size out of range, misaligned output */
  IBS_ENOMEM = 2,     /* device allocation failed or the workspace limit would be exceeded */
  IBS_ECUDA = 3,      /* a CUDA runtime call failed (message in ibs_last_error) */
  IBS_ETIMEOUT = 4,   /* a bounded device-side wait or ibs_wait timed out */
  IBS_EBUSY = 5,      /* admission refused: no slot or not enough free device memory yet */
  IBS_ECANCELLED = 6, /* the request was cancelled by ibs_shutdown */
  IBS_ESTATE = 7      /* call not valid in the context's current state */
} ibs_status;

/* ibs_config.flags */
#define IBS_OUT_SQUARE 0x1 /* write the full [n][n] matrix instead of the upper triangle */
#define IBS_NO_DIST 0x2    /* do not compute distances (out_dist may be NULL anyway) */
#define IBS_KERNEL_PLAIN 0x10 /* pair loop variant: one POPC per count and 32-marker word */
#define IBS_KERNEL_CSA 0x20   /* pair loop variant: carry-save reduction of 3 words before POPC */
#define IBS_TIMING 0x40       /* record CUDA events around each kernel of ibs_compute (ibs_kernel_times) */
#define IBS_KERNEL_TC 0x80    /* ibs_compute: tensor-core pair counts (tcgen05 indicator GEMMs, exact) */
#define IBS_TC_FP8 0x100      /* tensor-core form with E4M3 operands (kind::f8f6f4, 32 markers per MMA) */
#define IBS_TC_FP4 0x200      /* tensor-core form with E2M1 operands (kind::mxf4, unit scales, 64 markers per MMA);
                                 neither flag: the library default, E2M1 (environment IBS_TC_FORMAT=fp8|fp4
                                 overrides) */

typedef struct {
  int device;                      /* CUDA device ordinal */
  size_t workspace_bytes;          /* upper bound for library-owned device memory; 0 = no bound */
  int flags;                       /* OR of IBS_OUT_SQUARE, IBS_NO_DIST, IBS_KERNEL_PLAIN, IBS_KERNEL_CSA,
                                      IBS_KERNEL_TC, IBS_TC_FP8, IBS_TC_FP4, IBS_TIMING; no kernel flag =
                                      the tensor-core form (IBS_KERNEL_TC) with E2M1 operands */
  const char* autotune_cache_path; /* JSON file for the batched-launch tuner; NULL = in-memory only */
} ibs_config;

/* Create a context on cfg->device (NULL cfg = device 0, defaults).  Allocates
 * only the small control block; workspaces grow on demand up to
 * cfg->workspace_bytes.  (No paper passage: the context is this library's
 * handle for its device workspaces, the batched-launch tuner and the serving
 * engine.)  IBS_EINVAL for a bad device ordinal or for IBS_TC_FP8 together
 * with IBS_TC_FP4; IBS_ECUDA when the device is not an sm_103a GPU or cannot
 * be used. */
ibs_status ibs_init(const ibs_config* cfg, ibs_ctx** out_ctx);

/* Plain all-pairs IBS of one cohort (paper: the IBS matrix of
 * "Bitwise parallelism"; "Performance comparisons", IBS matrix rows).
 *   packed      DEVICE uint8 [n_variants][ceil(n_samples/4)], read-only.
 *   n_samples   1 .. 2^31-1; n_variants 1 .. 2^31-1.
 *   out_counts  DEVICE int32 [P][4] (P = n(n+1)/2, or n*n with IBS_OUT_SQUARE), 16-byte aligned.
 *   out_dist    DEVICE double [P] (8-byte aligned) or NULL.
 *   stream      cudaStream_t or NULL.
 * Transposes the matrix into library-owned sample-major bit planes, then runs
 * the triangular pair-count kernel with the fused count/distance epilogue;
 * which pair kernel a shape gets is given by ibs_compute_kernel. */
ibs_status ibs_compute(ibs_ctx* ctx, const uint8_t* packed, int64_t n_samples, int64_t n_variants,
                       int32_t* out_counts, double* out_dist, void* stream);

/* ibs_compute with the caller's buffer sizes in bytes, checked before any
 * work: packed_bytes >= n_variants * ceil(n_samples/4), counts_bytes >= P * 16
 * and, when out_dist is used, dist_bytes >= P * 8 (P = n(n+1)/2, or n*n with
 * IBS_OUT_SQUARE); a smaller buffer is refused with IBS_EINVAL and nothing is
 * enqueued.  Otherwise identical to ibs_compute. */
ibs_status ibs_compute_sz(ibs_ctx* ctx, const uint8_t* packed, size_t packed_bytes, int64_t n_samples,
                          int64_t n_variants, int32_t* out_counts, size_t counts_bytes, double* out_dist,
                          size_t dist_bytes, void* stream);

/* Allocation-free variant of ibs_compute (the paper has no counterpart; it
 * exists for callers that may not allocate device memory when they call in:
 * code running during CUDA graph capture, applications whose memory pool owns
 * the whole device, services that allocate only at start-up).  Takes no
 * context and calls no cudaMalloc/cudaFree: the bit-plane scratch is a fixed
 * 64 MiB array in the library's device image, held by every GPU that loads
 * the library until the process exits.  Arguments, layout and results are
 * those of ibs_compute (upper triangle, out_dist optional), on the CURRENT
 * device.  Inputs whose planes exceed the scratch, i.e. when
 * ceil(n/64) * ceil(ceil(m/32)/12) * 12288 > 64 MiB (for example n = 4096 with
 * m > 32,640), are rejected with IBS_EINVAL.  Small triangles split the
 * marker axis as ibs_compute does when their partial counts (16 bytes per
 * pair) fit in the scratch beside the planes; otherwise they run unsplit.  The
 * first call on a device looks
 * up the scratch address (cudaGetSymbolAddress); make it before any stream
 * capture.  All calls share the one scratch array: calls whose work overlaps
 * on the GPU (different streams, or threads) race and give undefined results;
 * serialise them.  packed, out_counts and out_dist must be device (or
 * managed) memory of the current device; anything else is refused with
 * IBS_EINVAL before any work is enqueued.  A bounded device wait that expires
 * is reported by ibs_noalloc_status, not by this call. */
ibs_status ibs_compute_noalloc(const uint8_t* packed, int64_t n_samples, int64_t n_variants, int32_t* out_counts,
                               double* out_dist, void* stream);

/* Outcome of the ibs_compute_noalloc calls enqueued on `stream` (the paper has
 * no counterpart; it completes the allocation-free entry point above).  Waits
 * for the stream, then reads the fixed device status word that every
 * ibs_compute_noalloc call clears and its kernels set: IBS_OK, or
 * IBS_ETIMEOUT when a bounded device wait expired in the last such call (its
 * outputs are then undefined).  Allocates nothing; uses the current device. */
ibs_status ibs_noalloc_status(void* stream);

/* Wait for all work enqueued on `stream` and report device-side errors of
 * this context's kernels since the last call: IBS_ETIMEOUT when a bounded
 * device wait expired (the kernel stopped early; outputs undefined), IBS_EINVAL
 * when a batched subset held an out-of-range sample index (that sample was
 * treated as all-missing).  Clears the device status word. */
ibs_status ibs_synchronize(ibs_ctx* ctx, void* stream);

/* One cohort subset of a pool for ibs_compute_batch: samples sample_idx[0..n)
 * (DEVICE int64, each in [0, pool_n), may be in any order; output row r is
 * sample_idx[r]) over the variant window [var_begin, var_begin + var_len). */
typedef struct {
  const int64_t* sample_idx; /* DEVICE */
  int64_t n;
  int64_t var_begin;
  int64_t var_len;
  int32_t* out_counts;       /* DEVICE int32 [n(n+1)/2][4] (upper triangle) */
  double* out_dist;          /* DEVICE double [n(n+1)/2] or NULL */
} ibs_subset;

/* Batched all-pairs IBS of many subsets of one pool (paper "Multicore and
 * cluster parallelism": independent pieces of sample x sample matrices).
 * Tensor-core form (the default, as ibs_compute): each subset's samples and
 * variant window are gathered from the pool straight into operand planes, in
 * four stages (about 10/30/30/30% of the comparisons, subsets by decreasing
 * variant count); the gathers of later stages run on a second stream while the
 * pair work of earlier stages runs.  Pair work, by split policy:
 *   0  one persistent launch per stage over (subset, tile) items;
 *   1  the same, the marker axis of large subsets split into K ranges that add
 *      into a partial triangle (finalised at the end);
 *   2  one persistent launch per subset over ibs_compute's own work list
 *      (a subset with fewer tiles than SMs, and the tiles of a final partial
 *      wave, split over K; their tiles finalised at the end); subsets whose
 *      windows reach the two-SM size (see ibs_compute_kernel) run the two-SM
 *      kernel;
 *   3  one two-SM persistent launch over every subset's two-SM work list,
 *      concatenated, with the gather fused: a concurrent gather kernel fills
 *      the operand planes unit by unit and per-subset readiness counters hold
 *      each item's copies until its planes are written;
 *   4  as 3, with the gather units taken by the pair launch's own epilogue
 *      warps between items (one launch after a short head start);
 *   5  policy 2's launches, gathered without gather stages: the epilogue
 *      warps of each two-SM launch gather the planes of the subsets after
 *      it (through the next two-SM subset) while its items' MMAs run; a
 *      subset that no earlier launch gathered gets a gather launch of its
 *      own.
 * Policies 3 to 5 need E2M1 operands and the two-SM kernel; they are tuner
 * candidates only then.  The tuner also tries policy 2 with the two-SM
 * kernel from 2,048 or 4,096 chunks on, or for no subset (the tile shape per
 * window size class; ibs_batch_plan_info reports the choice).
 * POPC form (IBS_KERNEL_PLAIN / IBS_KERNEL_CSA): one gather-transpose launch
 * and one persistent launch over all subsets (policies 0 and 1).  The launch
 * sequence is captured into a CUDA graph per batch shape and replayed; the
 * policy (and, for POPC, the kernel variant) is chosen by timing the
 * candidates on the first call of a shape, or fixed by the environment
 * variable IBS_BATCH_POLICY=0|1|2|3|4|5.  pool_packed is DEVICE
 * [pool_m][ceil(pool_n/4)].  Results are bit-identical to ibs_compute on each
 * subset alone. */
ibs_status ibs_compute_batch(ibs_ctx* ctx, const uint8_t* pool_packed, int64_t pool_n, int64_t pool_m,
                             const ibs_subset* subsets, int n_subsets, void* stream);

/* Serving (no paper passage: the serving workload of this library, a
 * resident reference panel queried by batches of new samples; the counts and
 * distances are the paper's, as for ibs_compute).  ibs_panel_load copies a
 * reference panel (DEVICE or HOST packed
 * [n_variants][ceil(n_panel/4)]) into library-owned resident bit planes and
 * starts the serving engine: a host thread that admits requests by free
 * device memory and slot count and advances all admitted requests together,
 * one panel chunk per step (continuous batching).  Blocks until the planes
 * are built.  Replaces any previous panel (pending requests are cancelled). */
ibs_status ibs_panel_load(ibs_ctx* ctx, const uint8_t* panel_packed, int64_t n_panel, int64_t n_variants);

/* Submit q query samples (no paper passage: serving workload, as above; the
 * counts are the paper's pair counts of each query against each panel
 * sample) (HOST or DEVICE packed [n_variants][ceil(q/4)],
 * copied before return) for counts against every panel sample plus the k
 * nearest panel samples by distance.  Non-blocking; returns a request id.
 *   out_counts    HOST or DEVICE int32 [q][n_panel][4], or NULL.
 *   out_topk_idx  HOST or DEVICE int32 [q][k]; out_topk_dist double [q][k].
 * Output buffers must be device memory or pinned (page-locked) host memory.
 * Ranking: ascending distance, ties by ascending panel index, N == 0 (NaN)
 * last, padded with (-1, NaN) when k > n_panel.  1 <= q <= 4096, 0 <= k <= 64.
 * Returns IBS_EBUSY when the request can never fit the memory budget.
 * Thread-safe. */
ibs_status ibs_query(ibs_ctx* ctx, const uint8_t* query_packed, int64_t n_query, int k,
                     int32_t* out_counts, int32_t* out_topk_idx, double* out_topk_dist, uint64_t* req_id);

/* The unbatched serving path, for comparison with the engine: one request,
 * one launch sequence (query transpose, all query x panel tiles, top-k, copies
 * back) on a private stream, returning when the outputs are written.  Same
 * arguments and results as ibs_query + ibs_wait.  Output buffers must be
 * device memory or pinned host memory (as for ibs_query). */
ibs_status ibs_query_sync(ibs_ctx* ctx, const uint8_t* query_packed, int64_t n_query, int k, int32_t* out_counts,
                          int32_t* out_topk_idx, double* out_topk_dist);

/* Wait until request req_id has written its outputs (timeout_ms < 0 = no
 * limit; no paper passage: serving workload, as above).  Returns IBS_OK, IBS_ETIMEOUT, IBS_ECANCELLED or the request's
 * error.  A request id can be waited on successfully once.  Thread-safe. */
ibs_status ibs_wait(ibs_ctx* ctx, uint64_t req_id, int64_t timeout_ms);

/* Non-blocking completion check (no paper passage: serving workload, as
 * above): IBS_OK when done, IBS_EBUSY while pending, IBS_EINVAL for an
 * unknown id, IBS_ESTATE when no panel is loaded. */
ibs_status ibs_poll(ibs_ctx* ctx, uint64_t req_id);

/* Serving-engine counters: completed requests, steps run, peak in-flight query rows. */
typedef struct {
  uint64_t requests_done;
  uint64_t steps;
  uint64_t peak_rows;
  uint64_t rejected;
} ibs_serve_stats;
ibs_status ibs_serve_stats_get(ibs_ctx* ctx, ibs_serve_stats* out);

/* Stop the engine, fail pending requests with IBS_ECANCELLED, free all
 * library-owned memory and the context.  Idempotent for NULL. */
ibs_status ibs_shutdown(ibs_ctx* ctx);

/* Thread-local message for the last non-OK status returned on this thread. */
const char* ibs_last_error(void);

/* Measure the sustained per-SM throughput of the integer instructions the pair
 * loop issues (POPC, LOP3, IADD3) with an all-SM microbenchmark on the
 * context's device: out[0..2] = operations per clock per SM for POPC, LOP3,
 * IADD3; out[3] = SM clock in MHz seen during the run; out[4] = SM count.
 * Synchronous.  Used to derive the integer-pipe roofline. */
ibs_status ibs_probe_int_pipes(ibs_ctx* ctx, double out[5]);

/* Measure the sustained tensor-core rate of the MMA kinds the tensor-core
 * form issues, with an all-SM microbenchmark on the context's device (back-to-
 * back 128 x 128 MMAs from shared-memory tiles): out[0] = E4M3
 * (kind::f8f6f4, K = 32), out[1] = E2M1 (kind::mxf4 with unit scale factors,
 * K = 64), in TFLOP/s.  Synchronous. */
ibs_status ibs_probe_mma(ibs_ctx* ctx, double out[2]);

/* The largest cached batched-launch plan: out[0] = kernel mode (0 plain,
 * 1 carry-save 2 CTAs/SM, 2 carry-save 1 CTA/SM, 3 tensor core E4M3, 4 tensor
 * core E2M1), out[1] = split policy, out[2] = work items, out[3] = grid,
 * out[4] = the two-SM size class of policies 2 and 5 in chunks (subsets of
 * at least that many chunks run the two-SM kernel; 2^40 = none; chosen by
 * the tuner among 1,024, 2,048, 4,096 and none for policy 2). */
ibs_status ibs_batch_plan_info(ibs_ctx* ctx, int64_t out[5]);

/* With IBS_TIMING: wait for the recorded events and return the summed device
 * time in ms of each kernel of all ibs_compute calls since the last query:
 * out[0] = bit-plane transpose, out[1] = pair-count kernel, out[2] = split-K
 * finalisation, out[3] = number of calls.  Resets the sums. */
ibs_status ibs_kernel_times(ibs_ctx* ctx, double out[4]);

/* Complete-linkage clustering of the samples under the IBS distance (paper,
 * "Identity-by-state matrices, complete linkage clustering": PLINK's
 * --cluster merges by complete linkage on the IBS matrix).  Greedy
 * agglomeration: the two active clusters at the smallest complete-linkage
 * distance (the largest distance between their members) merge first; ties go
 * to the smallest (representative, representative) pair, a cluster being
 * represented by its smallest member; NaN distances count as +infinity.
 * dist: DEVICE double [n(n+1)/2], the upper triangle with diagonal as
 * ibs_compute writes it (diagonal ignored).  out_linkage: DEVICE double
 * [n-1][4], rows (id1, id2, height, size) with id1 < id2, singletons 0..n-1 and
 * the cluster formed at step s numbered n + s (scipy's linkage convention).
 * Merge heights are input distances, exactly.  1 <= n <= 131072 (the working
 * matrix holds n*n doubles in library workspace).  Asynchronous on `stream`. */
ibs_status ibs_cluster_complete(ibs_ctx* ctx, const double* dist, int64_t n_samples, double* out_linkage,
                                void* stream);

/* Linkage disequilibrium between markers (paper, "Improvements in PLINK 1.9 /
 * Bitwise parallelism", the example of the correlation coefficient r with
 * missing calls).  For markers a < b <= a + window:
 *   x = +1 homozygous major, -1 homozygous minor, 0 heterozygous or missing;
 *   S_ab = samples where neither call is missing, N = |S_ab|;
 *   r = (N Sxy - Sx Sy) / sqrt((N Sxx - Sx^2) (N Syy - Sy^2)), sums over S_ab
 * (the paper's mean form multiplied through by N^2).  The major allele of a
 * marker is A1 when #hom A1 >= #hom A2 over its calls.  r is NaN when N = 0 or
 * either variance term is 0.  The sums are exact (tensor-core indicator
 * products); r is within 1e-12 relative of the exactly rounded value.
 * packed: DEVICE uint8 [n_variants][ceil(n_samples/4)] (.bed layout, as for
 * ibs_compute).  out_r: DEVICE double [n_variants][window], pair (a, a+1+d) at
 * out_r[a * window + d]; slots with a+1+d >= n_variants hold NaN.  out_n
 * (optional, DEVICE int32, same shape) receives N, 0 past the last marker.
 * 1 <= n_samples < 2^24, window >= 1.  Asynchronous on `stream`. */
ibs_status ibs_ld_r(ibs_ctx* ctx, const uint8_t* packed, int64_t n_samples, int64_t n_variants, int64_t window,
                    double* out_r, int32_t* out_n, void* stream);

/* GCTA genomic relationship matrix of the samples (paper, "Partial sum
 * lookup", the weighted-distance example).  Per marker, p = frequency of A1
 * over the marker's non-missing calls, x = number of A1 copies in a call;
 * markers with p = 0 or p = 1 are left out.  For samples j <= k:
 *   A_jk = (1 / N_jk) * sum over markers where both calls are present of
 *          (x_j - 2p)(x_k - 2p) / (2p(1 - p)),
 * N_jk = the number of such markers (the diagonal uses the same formula with
 * j = k).  A_jk is NaN when N_jk = 0.
 * packed: DEVICE uint8 [n_variants][ceil(n_samples/4)] (.bed layout, as for
 * ibs_compute).  out_grm: DEVICE double [n(n+1)/2], the upper triangle with
 * diagonal in ibs_compute's order (pair (j, k), j <= k, at
 * j*n - j*(j-1)/2 + (k - j)).
 * Precision: the standardised values z = (x - 2p) / sqrt(2p(1-p)) are formed
 * in FP64 and carried as FP16 pairs hi + lo; the products run on the tensor
 * cores in FP32, restarted every 128 markers and summed across segments
 * without rounding loss (float-float).  With S = sum over the shared markers
 * of |z_j z_k|, the result is within (3 + 24) * 2^-22 * S / N_jk
 * + 2^-25 * sum(|z_j| + |z_k|) / N_jk of the exact value, for any number of
 * markers (3 * 2^-22 from the FP16 split, 24 MMA accumulations per segment
 * at 2^-22 each); N_jk is exact.
 * 1 <= n_samples <= 8388480, 1 <= n_variants < 2^24.  Workspace: 10 KiB per
 * (128 samples, 16 markers) of library memory.  Asynchronous on `stream`. */
ibs_status ibs_grm(ibs_ctx* ctx, const uint8_t* packed, int64_t n_samples, int64_t n_variants, double* out_grm,
                   void* stream);

/* The kernels this context's ibs_compute uses: out[0] = pair kernel family
 * (0 POPC plain, 1 POPC carry-save, 2 tensor core), out[1] = tensor-core
 * operand format (0 E4M3, 1 E2M1), out[2] = SMs of the device, out[3] = device. */
ibs_status ibs_kernel_info(ibs_ctx* ctx, int64_t out[4]);

/* The pair kernel ibs_compute runs on this context for an n_samples x
 * n_variants matrix, written to *out: 0 POPC plain, 1 POPC carry-save,
 * 2 tensor core with one persistent CTA per SM, 3 tensor core with the
 * two-SM kernel (clusters of two CTAs, tcgen05 cta_group::2), 4 tensor core
 * with one CTA per tile (square output).  The two-SM kernel runs for E2M1
 * operands, triangle output and 129 or more samples when the matrix has at
 * least 65,536 variants (1,024 chunks of 64), where it is the faster one;
 * IBS_TC_PAIR=1 in the environment selects it for every size, IBS_TC_PAIR=0
 * never.  Host only, no device work; IBS_EINVAL for sizes ibs_compute
 * refuses or out == NULL. */
ibs_status ibs_compute_kernel(ibs_ctx* ctx, int64_t n_samples, int64_t n_variants, int64_t* out);

/* Counters of the last ibs_compute / ibs_compute_batch on this context:
 * out[0] = kernel launches enqueued, out[1] = pair tiles, out[2] = K splits. */
ibs_status ibs_last_launch_info(ibs_ctx* ctx, int64_t out[3]);

/* Testing hook of the failure handling (the paper has no counterpart).
 * Sets the bound, in ns, of every pipeline wait (operand stages, work queue,
 * accumulator hand-over) inside the persistent pair kernels that ibs_compute
 * launches on this context for triangle output; ns = 0 restores the default
 * of 2 s.  A wait that runs out sets the context's device status word and
 * the kernel winds down: it stops issuing work, waits (with the default
 * bound) for the copies and MMAs it already issued, frees its tensor memory
 * and returns, so the next ibs_synchronize reports IBS_ETIMEOUT (outputs of
 * that call undefined) and the context stays usable.  0 <= ns <= 2e9, else
 * IBS_EINVAL. */
ibs_status ibs_test_set_wait_limit(ibs_ctx* ctx, int64_t ns);

#ifdef __cplusplus
}
#endif

#endif /* IBS_H_ */
