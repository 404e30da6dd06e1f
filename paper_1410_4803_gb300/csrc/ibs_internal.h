// Host-side declarations shared by the libibs translation units (not part of
// the public C ABI, which is include/ibs.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace ibs {

// Geometry of a bit-plane buffer (see ibs_device.cuh for the memory order).
struct PlaneGeom {
  int64_t n = 0;         // samples
  int64_t m = 0;         // markers
  int64_t n_blocks = 0;  // ceil(n / 64)
  int64_t n_chunks = 0;  // ceil(ceil(m / 32) / 12)
  size_t bytes() const { return (size_t)n_blocks * (size_t)n_chunks * 12u * 64u * 4u * 4u; }
  static PlaneGeom make(int64_t n, int64_t m) {
    PlaneGeom g;
    g.n = n;
    g.m = m;
    g.n_blocks = (n + 63) / 64;
    const int64_t words = (m + 31) / 32;
    g.n_chunks = (words + 11) / 12;
    return g;
  }
};

// Source of a gather-transpose: rows var_begin .. var_begin+m-1 of a packed
// matrix with row_bytes bytes per row; sample r of the output is sample
// sel[r] of the source (sel == nullptr: sample r).
struct BedSource {
  const uint8_t* packed = nullptr;
  int64_t row_bytes = 0;
  int64_t var_begin = 0;
  const int64_t* sel = nullptr;
  int64_t n_src = 0;     // samples in the source (bound for sel entries)
};

// One subset of a batched launch, as the device sees it.
struct SubsetDev {
  const uint32_t* planes;  // this subset's bit planes
  int64_t n;
  int64_t n_blocks;
  int64_t n_chunks;
  int32_t* out_counts;
  double* out_dist;
  int32_t* partial;        // split-K accumulation, triangle [P][4], or nullptr
  int64_t pad;
};

// A (subset, tile, K-range) work item of the persistent batched kernel.
struct WorkItem {
  int32_t subset;
  int32_t I, J;
  int32_t c0, c1;
  int32_t split;  // 1 when the tile is split over K (accumulate into partial)
};

// A work item of the two-SM pair kernel: two tiles (I0, J) and (I1, J) that
// share their column block J, one per CTA of the pair (I1 < 0: the second CTA
// has no tile and stores nothing), over chunks c0 .. c1-1.
struct PairItem {
  int32_t I0, I1, J;
  int32_t c0, c1;
  int32_t split;   // 1 when the tiles are split over K (accumulate into partial)
  int32_t subset;  // batched launches: the subset the tiles belong to (0 for one matrix)
  int32_t pad;
};

// Per-subset plane-build job for the batched gather-transpose.
struct PlaneJob {
  BedSource src;
  int64_t m;             // markers in the window
  int64_t n;             // samples
  uint32_t* planes;
  int64_t n_blocks;
  int64_t n_chunks;
  int64_t cta_begin;     // first CTA index of this job in the flattened grid
  int64_t groups;        // ceil(n_blocks / 2)
};

// Serving: one query-block x panel-block work item of a step.  The 64 rows of
// a query block may belong to different requests, so each row carries its
// own output row ([n_panel][4] int32).
struct CrossItem {
  const uint32_t* qplanes;  // query block planes base (block already applied)
  int32_t* const* row_out;  // 64 output row pointers of this block (entries >= q_rows unused)
  int32_t q_rows;           // valid query rows in the block (<= 64)
  int32_t pb;               // panel block
};

// Serving: source of one dense step row (a row of some request's planes).
struct RowSrc {
  const uint32_t* planes;   // the request's bit planes
  int64_t row;              // row within the request
};

// Kernel launchers (ibs_planes.cu / ibs_pairs.cu / ibs_misc.cu).
cudaError_t launch_planes(const BedSource& src, int64_t n, int64_t m, const PlaneGeom& g, uint32_t* planes,
                          int* status, cudaStream_t st);
cudaError_t launch_planes_batch(const PlaneJob* jobs_dev, int n_jobs, int64_t total_ctas, int* status,
                                cudaStream_t st);

int tri_splits_for(int64_t tiles, int64_t n_chunks, int num_sms);
cudaError_t launch_tri(int mode, const uint32_t* planes, const PlaneGeom& g, int splits, int32_t* out_counts,
                       double* out_dist, int32_t* partial, bool square, int* status, int num_sms,
                       cudaStream_t st);
cudaError_t launch_finalize(const int32_t* partial, int64_t n, int32_t* out_counts, double* out_dist,
                            bool square, cudaStream_t st);
cudaError_t launch_batch(int mode, const SubsetDev* subsets, const WorkItem* items, int64_t n_items,
                         int* counter, int* status, int grid, cudaStream_t st);
cudaError_t launch_finalize_batch(const SubsetDev* subsets, const int32_t* subset_ids, int n_split_subsets,
                                  int64_t max_pairs, cudaStream_t st);
cudaError_t launch_cross(int mode, const uint32_t* panel_planes, int64_t n_panel, int64_t panel_blocks,
                         int64_t n_chunks, const CrossItem* items, int64_t n_items, int* status,
                         cudaStream_t st);
cudaError_t launch_gather_rows(const RowSrc* rows, int64_t n_rows, int64_t n_chunks, uint32_t* dst,
                               cudaStream_t st);
// Top-k of many query rows in one launch (rows of any requests, 1 <= k <= 64
// each): counts [n_panel][4] of the row -> out_idx [k], out_dist [k].
struct TopkRow {
  const int32_t* counts;
  int32_t* out_idx;
  double* out_dist;
  int32_t k;
  int32_t pad;
};
cudaError_t launch_topk_rows(const TopkRow* rows, int64_t n_rows, int64_t n_panel, cudaStream_t st);
cudaError_t launch_topk(const int32_t* counts, int64_t q, int64_t n_panel, int k, int32_t* out_idx,
                        double* out_dist, cudaStream_t st);
int pair_kernel_ctas_per_sm(int mode);

// Gather-transpose of one subset straight into tensor-core operand planes:
// samples sel[0..n) of the source pool over markers var_begin .. var_begin+m-1.
struct TcGatherJob {
  BedSource src;          // pool rows, sample index list, pool size
  int64_t m, n;           // markers in the window, samples
  uint8_t* tc;            // operand planes of the subset
  int64_t nb, nc;         // 128-sample blocks, chunks
};

// Tensor-core form (ibs_tc.cu): indicator planes and tcgen05 pair tiles, in
// one of two operand formats.
constexpr int kTcFp8 = 0;  // E4M3, kind::f8f6f4, 32 markers per chunk
constexpr int kTcFp4 = 1;  // E2M1, kind::mxf4 with unit scale factors, 64 markers per chunk
int tc_default_format();   // IBS_TC_FORMAT=fp4|fp8, else the built-in default
size_t tc_planes_bytes(int64_t n, int64_t m, int fmt);
int tc_splits_for(int64_t tiles, int64_t n_chunks, int num_sms);
int64_t tc_tiles(int64_t n);
int64_t tc_chunks(int64_t m, int fmt);
int64_t tc_max_chunks(int fmt);  // longest K range of one accumulation (2^21 markers)
cudaError_t launch_tc_planes(const uint8_t* packed, int64_t n, int64_t m, uint8_t* planes, int fmt,
                             cudaStream_t st);
cudaError_t launch_tc_pairs(const uint8_t* planes, int64_t n, int64_t m, int fmt, int splits, int32_t* out_counts,
                            double* out_dist, int32_t* partial, bool square, int* status, const int2* tile_list,
                            cudaStream_t st);
void tc_tile_order(int64_t T, int G, std::vector<int2>& out);
int64_t tc_gather_ctas(int64_t n, int64_t nc);  // CTAs of one job of the gather launch
// map_dev[c] = {job, sample block, chunk group, -} of gather CTA c; chunk groups
// hold tc_gather_chunks() chunks.
cudaError_t launch_tc_gather(const TcGatherJob* jobs_dev, const int4* map_dev, int64_t total_ctas, int fmt,
                             int* status, cudaStream_t st);
int tc_gather_chunks();
// Batched tensor-core pairs: SubsetDev.planes holds operand planes, n_blocks and
// n_chunks count 128-sample blocks and chunks, and WorkItem tiles and K ranges
// are in those units.
cudaError_t launch_tc_batch(const SubsetDev* subs, const WorkItem* items, int64_t n_items, int grid, int fmt,
                            int64_t max_chunks, int* counter, int* status, cudaStream_t st);
// One matrix through the persistent kernel (ibs_compute): work list, launch,
// and the finalisation of the split tiles.
void tc_single_items(int64_t n, int64_t m, int fmt, int num_sms, int group, std::vector<WorkItem>& items,
                     std::vector<int2>& split_tiles);
// wait_ns bounds each of the kernel's pipeline waits (the drains of work
// already in flight keep the default bound): the library default, or a test's
// shorter limit (ibs_test_set_wait_limit).
cudaError_t launch_tc_single(const SubsetDev& sd, const WorkItem* items, int64_t n_items, int grid, int fmt,
                             int* counter, int* status, unsigned long long wait_ns, cudaStream_t st);
// Two-SM form of the same (tcgen05 cta_group::2, E2M1 only): clusters of two
// CTAs, each pair item two tiles sharing their column block.  tc_pair_clusters
// is the number of clusters the launch runs (0 when the kernel cannot run);
// tc_pair_usable says whether it runs for an n x m matrix (E2M1; two or more
// blocks; within its tensor map's coordinate range; tc_pair_mode: 1 always,
// -1 never, 0 for items of at least 1,024 chunks, from IBS_TC_PAIR).
int tc_pair_mode();
int tc_pair_clusters(int64_t chunks_per_item);
// K-lockstep of the pair kernel's full waves (the default; IBS_TC_PAIR_SYNC=
// seg,lag or off): the items [0, n_items) come in waves of one item per cluster, all
// of equal length; the copy warp of every CTA counts each seg-chunk segment
// it starts in ctr[wave * n_seg + segment] and, before segment s, waits
// (bounded) until every CTA of its wave has started segment s - lag, so the
// clusters of a wave stream nearly the same chunks at the same time.
struct PairSync {
  int* ctr = nullptr;
  int32_t n_seg = 0, seg = 0, lag = 0;
  int64_t n_items = 0;
};
// The lockstep setting from the environment ({seg, lag}, seg a multiple of
// the ring's chunks per stage; {0, 0} = off).
int2 tc_pair_sync_setting(int64_t chunks_per_item);
bool tc_pair_usable(int64_t n, int64_t m, int fmt);
void tc_pair_items(int64_t n, int64_t m, int fmt, int n_clusters, int group, std::vector<PairItem>& items,
                   std::vector<int2>& split_tiles);
cudaError_t launch_tc_pair(const SubsetDev& sd, const PairItem* items, int64_t n_items, int* status,
                           unsigned long long wait_ns, cudaStream_t st, const PairSync& sync = PairSync{});
// Pair items {I0, I1, J} of a T x T block triangle in the grouped order
// (bands of `group` block rows, rounded up to even).
void tc_pair_order(int64_t T, int group, std::vector<int4>& order);
// Batched subsets through the pair kernel in one launch, the gather fused in
// (PairBatchWork in ibs_tc.cu): the subsets' planes share one buffer of
// block_chunks 16 KiB block-chunks (SubsetDev::pad = a subset's first),
// units {job, sample block, chunk group, subset} are gathered by the
// epilogue warps, ready/need count them per subset, max_chunks is the
// longest item (it picks the ring).
struct PairBatchArgs {
  const SubsetDev* subs;
  const PairItem* items;
  int64_t n_items;
  const TcGatherJob* jobs;
  const int4* units;
  int64_t n_units;
  int* unit_counter;
  int* ready;
  const int* need;
  const void* planes;
  int64_t block_chunks;
  int64_t max_chunks;
  PairSync sync;  // K-lockstep of the launch's whole waves (policy 2), or off
};
cudaError_t launch_tc_pair_batch(const PairBatchArgs& a, int* status, unsigned long long wait_ns, cudaStream_t st);
// Gather units of a PairBatchArgs list by `ctas` persistent CTAs (run beside
// the pair launch on another stream; both claim from unit_counter).
cudaError_t launch_tc_gather_units(const TcGatherJob* jobs, const int4* units, int64_t n_units, int* unit_counter,
                                   int* ready, int fmt, int ctas, int* status, cudaStream_t st);
cudaError_t launch_tc_finalize_tiles(const int2* tiles, int64_t n_tiles, const int32_t* partial, int64_t n,
                                     int32_t* out_counts, double* out_dist, cudaStream_t st);
// Batch form: tiles {subset, I, J, -}, outputs from the subsets' descriptors.
cudaError_t launch_tc_finalize_batch_tiles(const SubsetDev* subs, const int4* tiles, int64_t n_tiles,
                                           cudaStream_t st);
// Serving, tensor-core form: CrossItem.qplanes points at a 128-row query block
// of operand planes, row_out has 128 entries, pb is a 128-sample panel block.
cudaError_t launch_tc_cross(const uint8_t* panel, int64_t n_panel, int64_t n_chunks, const CrossItem* items,
                            int64_t n_items, int grid, int fmt, int* counter, int* status, cudaStream_t st);
cudaError_t launch_tc_gather_rows(const RowSrc* rows, int64_t n_rows, int64_t n_chunks, uint8_t* dst,
                                  cudaStream_t st);
// Serving on the two-SM kernel (PairCrossWork in ibs_tc.cu): items {I0, I1,
// J, 0, n_chunks} pair two 128-row blocks of the dense query planes qplanes
// (q_blocks_cap blocks allocated) with panel block J; step row r (< n_rows)
// writes its counts through row_out[r].  tc_pair_cross_usable: whether the
// kernel runs for a panel of n_panel samples and n_chunks chunks (the
// two-SM rule of tc_pair_usable).
bool tc_pair_cross_usable(int64_t n_panel, int64_t n_chunks, int fmt);
cudaError_t launch_tc_pair_cross(const uint8_t* panel, int64_t n_panel, int64_t n_chunks, const uint8_t* qplanes,
                                 int64_t q_blocks_cap, int32_t* const* row_out, int64_t n_rows, const PairItem* items,
                                 int64_t n_items, int* status, cudaStream_t st, const PairSync& sync = PairSync{});
int tc_block_samples();  // 128
// LD correlation (ibs_ld.cu): operand planes of the markers (128-marker
// blocks, 64-sample chunks, planes X, V, H), the band's work items and the
// launch sequence (operand builder with per-marker allele balance, persistent
// tensor-core kernel, fill of the slots past the last marker).
size_t ld_planes_bytes(int64_t n, int64_t m);
void ld_items(int64_t m, int64_t window, std::vector<int2>& items);
cudaError_t launch_ld(const uint8_t* packed, int64_t n, int64_t m, int64_t window, uint8_t* planes, int32_t* diff,
                      const int2* items, int64_t n_items, int* counter, double* out_r, int32_t* out_n,
                      int* status, int num_sms, cudaStream_t st);

// Genomic relationship matrix (ibs_grm.cu): per-marker frequency table and
// FP16 hi/lo/V' operand planes (128-sample blocks, 16-marker chunks) in one
// workspace of grm_planes_bytes(n, m); the work list (grouped triangle tile
// order, the tiles of a final partial wave split over the marker axis into
// parts whose sums a finalisation pass adds); the launch sequence
// (frequencies, operand builder, persistent kernel, finalisation).
struct GrmItem {
  int32_t I, J;    // tile: row block, column block (I <= J)
  int32_t c0, c1;  // chunk range (c0 a multiple of the 128-marker segment)
  int32_t part;    // part slot of a split tile's piece, -1 for a whole tile
  int32_t pad[3];
};
size_t grm_planes_bytes(int64_t n, int64_t m);
void grm_items(int64_t n, int64_t m, int num_sms, std::vector<GrmItem>& items, std::vector<int4>& splits,
               int64_t& parts);
cudaError_t launch_grm(const uint8_t* packed, int64_t n, int64_t m, double* out, uint8_t* work, const GrmItem* items,
                       int64_t n_items, const int4* splits, int64_t n_splits, double* part_num, float* part_cnt,
                       int* counter, int* status, int num_sms, cudaStream_t st);

// Complete-linkage clustering (ibs_cluster.cu) of n samples under a distance
// triangle (ibs_compute's layout), into Z [n-1][4] on the device; `work` holds
// cluster_workspace_bytes(n).
size_t cluster_workspace_bytes(int64_t n);
cudaError_t launch_cluster_complete(const double* tri, int64_t n, double* Z, void* work, int num_sms,
                                    cudaStream_t st);

// MMA-rate probe: out[0] = E4M3 (kind::f8f6f4), out[1] = E2M1 (kind::mxf4)
// TFLOP/s of 128 x 128 MMAs from shared memory, all SMs.
cudaError_t probe_tc_mma(int device, int num_sms, int* status_dev, double out[2]);
size_t pair_kernel_smem_bytes();

// Integer-pipe microbenchmark (ibs_probe.cu).
cudaError_t probe_int_pipes(int device, double out[5]);

}  // namespace ibs
