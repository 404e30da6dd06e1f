// Library context and host utilities shared by ibs_api.cu and ibs_serve.cu.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ibs.h"
#include "ibs_internal.h"

namespace ibs {

ibs_status fail(ibs_status st, const char* fmt, ...);
void clear_error();

#define IBS_CUDA_TRY(call)                                                                        \
  do {                                                                                            \
    cudaError_t _e = (call);                                                                      \
    if (_e != cudaSuccess) return ::ibs::fail(IBS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

class ServeEngine;

// Cached launch plan of one batch shape: device descriptor arrays at fixed
// addresses plus the captured graph.
struct BatchPlan {
  std::vector<int64_t> shape_key;
  DevBuf planes, partial, subsets, jobs, items, split_ids, counter;
  DevBuf tc_planes, tc_jobs;            // tensor-core modes: operand planes and their gather jobs
  // Tensor-core modes: the subsets run in stages (contiguous groups of the
  // cost-sorted subset order); the gather of stage g+1 runs on `side` while the
  // pair kernel of stage g runs.
  std::vector<int64_t> order;           // subset processing order
  std::vector<int64_t> stage_item_off, stage_job_off, stage_ctas;  // per stage (+1 end entry for offsets)
  std::vector<int64_t> stage_max_chunks;  // longest item of a stage, in chunks (picks the ring depth)
  // split policy 2 (tensor-core modes): one launch per subset over its own
  // work list (the single-matrix list: small subsets and tail waves split over
  // K); q_item_off / q_chunks per position of `order`, split tiles
  // {subset, I, J, -} finalised after the last launch
  std::vector<int64_t> q_item_off, q_chunks;
  // gather CTA map {job, sample block, chunk group, -} per stage (offsets into
  // it per stage), ordered by pool variant; rebuilt when the windows change
  DevBuf gather_map;
  std::vector<int64_t> stage_map_off, map_key;
  DevBuf split_tiles;
  int64_t n_split_tiles = 0;
  // split policy 3 (E2M1): every subset's pair items in one launch of the
  // two-SM kernel, the gather fused in (gather units, per-subset readiness)
  DevBuf pitems, units, unit_counter, ready, need;
  int64_t n_pitems = 0, n_units = 0, pair_max_chunks = 0, tc_block_chunks = 0;
  // split policy 2: subsets that ibs_compute would run on the two-SM kernel
  // take its pair work list (q_pair_off/q_pair_n into pitems, -1 = one-SM)
  std::vector<int64_t> q_pair_off, q_pair_n;
  // ... and their K-lockstep: items in whole waves per position (0 = none),
  // one counter buffer for the largest, zeroed before each launch
  std::vector<int64_t> q_pair_sync;
  // split policy 5: gather units per position of `order` (offsets into units)
  std::vector<int64_t> q_unit_off;
  DevBuf pair_sync;
  size_t pair_sync_bytes = 0;
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> stage_ev;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;  // policy 3: the side stream's gather
  int64_t n_items = 0, total_ctas = 0, max_split_pairs = 0, tc_ctas = 0;
  int n_split = 0;
  int mode = 0, split_policy = 0, grid = 0;
  // policies 2 and 5: subsets of at least this many chunks (and that the
  // two-SM kernel takes) run on it, the rest on the one-SM kernel; tuned
  int64_t pair_min_chunks = 1024;
  std::vector<int64_t> plane_offsets;   // bytes into planes
  std::vector<int64_t> tc_offsets;      // bytes into tc_planes (mode 3)
  std::vector<int64_t> partial_offsets; // bytes into partial, -1 if not split
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t tiles = 0;
};

struct TuneEntry {
  int mode = -1;
  int64_t pair_min = 1024;  // the tuned two-SM size class (chunks) of policies 2 and 5
  int split_policy = 0;
  double ms = 0;
};

}  // namespace ibs

struct ibs_ctx {
  int device = 0;
  int flags = 0;
  size_t ws_limit = 0;
  std::string tune_path;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  int default_mode = 1;
  bool default_tc = true;         // ibs_compute uses the tensor-core form unless told otherwise

  std::mutex mu;                  // guards memory accounting
  size_t owned_bytes = 0;

  ibs::DevBuf planes, partial;
  ibs::DevBuf tile_list;          // tensor-core grouped tile order, for tile_list_T tiles per side
  int64_t tile_list_T = -1;
  ibs::DevBuf cluster_work;  // complete-linkage working matrix and row minima
  // LD correlation: operand planes, per-marker allele balance, band items of the last (m, window)
  ibs::DevBuf ld_planes, ld_diff, ld_items, ld_counter;
  std::vector<int64_t> ld_key;
  int64_t ld_n_items = 0;
  // GCTA relationship matrix: operand planes and frequency table; work list,
  // split tiles and their part sums for the last (n, m)
  ibs::DevBuf grm_work, grm_items, grm_splits, grm_part, grm_counter;
  std::vector<int64_t> grm_key;
  int64_t grm_n_items = 0, grm_n_splits = 0, grm_parts = 0;
  // persistent tensor-core work list of the last (n, m, format, SMs, group)
  std::vector<int64_t> single_key;
  ibs::DevBuf single_items, single_split, single_counter, single_sync;
  int64_t single_n_items = 0, single_n_split = 0;
  int64_t single_n_sync = 0;  // pair items in full waves of equal length (the K-lockstep's items)
  int single_clusters = 0;
  bool single_pair = false;  // single_items holds PairItem (two-SM kernel), else WorkItem
  int* status_host = nullptr;     // mapped pinned status word
  int* status_dev = nullptr;
  // device-side bound of the pipeline waits of ibs_compute's persistent pair
  // kernels, in ns (0 = the library default, 2 s); tests set it shorter
  // through ibs_test_set_wait_limit to exercise the timeout path
  unsigned long long wait_ns = 0;

  int64_t last_info[3] = {0, 0, 0};

  // IBS_TIMING: events around each kernel of ibs_compute, summed by ibs_kernel_times.
  struct TimingRec {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int n = 0;
  };
  std::vector<TimingRec> timing_used, timing_free;

  std::map<std::vector<int64_t>, std::unique_ptr<ibs::BatchPlan>> plans;
  std::map<std::string, ibs::TuneEntry> tune;

  std::shared_ptr<ibs::ServeEngine> serve;  // guarded by mu
};

namespace ibs {

ibs_status ensure_buf(ibs_ctx* ctx, DevBuf& b, size_t need);
void free_buf(ibs_ctx* ctx, DevBuf& b);
bool reserve_bytes(ibs_ctx* ctx, size_t bytes);
void release_bytes(ibs_ctx* ctx, size_t bytes);
int pick_mode(const ibs_ctx* ctx);
// The pair kernels a context uses (flags, else the library defaults): the
// tensor-core form or a POPC kernel, the tensor-core operand format, the
// POPC variant.
bool ctx_use_tc(const ibs_ctx* ctx);
int ctx_tc_format(const ibs_ctx* ctx);
int ctx_popc_mode(const ibs_ctx* ctx);

// Serving engine (ibs_serve.cu).
ibs_status serve_panel_load(ibs_ctx* ctx, const uint8_t* panel, int64_t n_panel, int64_t m);
ibs_status serve_query(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi, double* od,
                       uint64_t* id);
ibs_status serve_query_sync(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi,
                            double* od);
ibs_status serve_wait(ibs_ctx* ctx, uint64_t id, int64_t timeout_ms);
ibs_status serve_poll(ibs_ctx* ctx, uint64_t id);
ibs_status serve_stats(ibs_ctx* ctx, ibs_serve_stats* out);
void serve_stop(ibs_ctx* ctx);
std::shared_ptr<ServeEngine> engine_of(ibs_ctx* ctx);

}  // namespace ibs
