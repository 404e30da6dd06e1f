// libibs C ABI: context, validation, workspaces, the plain all-pairs path and
// the batched persistent path (work list, CUDA graph, autotuner).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <fstream>
#include <sstream>

#include "ibs_ctx.h"
#include "ibs_device.cuh"

namespace ibs {

namespace {
thread_local std::string g_last_error;
}

ibs_status fail(ibs_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

void clear_error() { g_last_error.clear(); }

const char* last_error_cstr() { return g_last_error.c_str(); }

bool reserve_bytes(ibs_ctx* ctx, size_t bytes) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->ws_limit && ctx->owned_bytes + bytes > ctx->ws_limit) return false;
  ctx->owned_bytes += bytes;
  return true;
}

void release_bytes(ibs_ctx* ctx, size_t bytes) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->owned_bytes = bytes > ctx->owned_bytes ? 0 : ctx->owned_bytes - bytes;
}

ibs_status ensure_buf(ibs_ctx* ctx, DevBuf& b, size_t need) {
  if (need == 0) need = 16;
  if (b.cap >= need) return IBS_OK;
  if (b.p) {
    cudaFree(b.p);  // synchronises the device, so no launch still uses it
    release_bytes(ctx, b.cap);
    b.p = nullptr;
    b.cap = 0;
  }
  if (!reserve_bytes(ctx, need))
    return fail(IBS_ENOMEM, "workspace limit %zu bytes would be exceeded (need %zu more)", ctx->ws_limit, need);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    release_bytes(ctx, need);
    cudaGetLastError();
    return fail(IBS_ENOMEM, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
  }
  b.p = p;
  b.cap = need;
  return IBS_OK;
}

void free_buf(ibs_ctx* ctx, DevBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    release_bytes(ctx, b.cap);
  }
  b.p = nullptr;
  b.cap = 0;
}

int pick_mode(const ibs_ctx* ctx) { return ctx->default_mode; }

}  // namespace ibs

using namespace ibs;

namespace {

constexpr int kFlagPlain = 0x10;  // force the plain kernel (one POPC per count and word)
constexpr int kFlagCsa = 0x20;    // force the carry-save kernel

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ibs_status check_ctx(ibs_ctx* ctx) {
  if (!ctx) return fail(IBS_EINVAL, "context is NULL");
  return IBS_OK;
}

constexpr int kFlagTc = 0x80;     // tensor-core (tcgen05 indicator GEMM) pair counts
constexpr int kFlagTcFp8 = 0x100;  // tensor-core operands in E4M3
constexpr int kFlagTcFp4 = 0x200;  // tensor-core operands in E2M1 (block-scaled MMA, unit scales)

// The tensor-core form is the default for ibs_compute; IBS_KERNEL_PLAIN or
// IBS_KERNEL_CSA select the bit-plane POPC kernels instead.
bool use_tc(const ibs_ctx* ctx) {
  if (ctx->flags & kFlagTc) return true;
  if (ctx->flags & (kFlagPlain | kFlagCsa)) return false;
  return ctx->default_tc;
}

int tc_format_for(const ibs_ctx* ctx) {
  if (ctx->flags & kFlagTcFp4) return kTcFp4;
  if (ctx->flags & kFlagTcFp8) return kTcFp8;
  return tc_default_format();
}

int mode_for(const ibs_ctx* ctx) {
  if (ctx->flags & kFlagPlain) return 0;
  if (ctx->flags & kFlagCsa) return 1;
  return ctx->default_mode;
}

}  // namespace

namespace ibs {
bool ctx_use_tc(const ibs_ctx* ctx) { return use_tc(ctx); }
int ctx_tc_format(const ibs_ctx* ctx) { return tc_format_for(ctx); }
int ctx_popc_mode(const ibs_ctx* ctx) { return mode_for(ctx); }
}  // namespace ibs

extern "C" {

const char* ibs_last_error(void) { return ibs::last_error_cstr(); }

ibs_status ibs_init(const ibs_config* cfg, ibs_ctx** out_ctx) {
  clear_error();
  if (!out_ctx) return fail(IBS_EINVAL, "out_ctx is NULL");
  *out_ctx = nullptr;
  ibs_config c{};
  if (cfg) c = *cfg;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(IBS_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
  }
  if (c.device < 0 || c.device >= ndev) return fail(IBS_EINVAL, "device %d out of range [0, %d)", c.device, ndev);
  if ((c.flags & kFlagTcFp8) && (c.flags & kFlagTcFp4)) return fail(IBS_EINVAL, "IBS_TC_FP8 and IBS_TC_FP4 both set");
  DeviceGuard g(c.device);
  cudaDeviceProp prop;
  IBS_CUDA_TRY(cudaGetDeviceProperties(&prop, c.device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(IBS_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a only", c.device, prop.major,
                prop.minor);
  auto* ctx = new ibs_ctx();
  ctx->device = c.device;
  ctx->flags = c.flags;
  ctx->ws_limit = c.workspace_bytes;
  if (c.autotune_cache_path) ctx->tune_path = c.autotune_cache_path;
  ctx->num_sms = prop.multiProcessorCount;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  const char* tcenv = getenv("IBS_DEFAULT_KERNEL");
  ctx->default_tc = !(tcenv && strcmp(tcenv, "popc") == 0);
  const char* env = getenv("IBS_PAIR_MODE");
  if (env && env[0] >= '0' && env[0] <= '2' && env[1] == 0) ctx->default_mode = env[0] - '0';
  e = cudaHostAlloc(reinterpret_cast<void**>(&ctx->status_host), sizeof(int), cudaHostAllocMapped);
  if (e != cudaSuccess) {
    delete ctx;
    return fail(IBS_ECUDA, "cudaHostAlloc(status) failed: %s", cudaGetErrorString(e));
  }
  *ctx->status_host = 0;
  e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->status_dev), ctx->status_host, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(ctx->status_host);
    delete ctx;
    return fail(IBS_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
  }
  // Load the autotune cache.
  if (!ctx->tune_path.empty()) {
    std::ifstream f(ctx->tune_path);
    std::string line;
    while (std::getline(f, line)) {
      char key[512];
      TuneEntry t;
      long long pm = 1024;
      const int got = sscanf(line.c_str(),
                             "{\"key\": \"%511[^\"]\", \"mode\": %d, \"split\": %d, \"ms\": %lf, \"pair_min\": %lld}", key,
                             &t.mode, &t.split_policy, &t.ms, &pm);
      if (got >= 4) {  // entries written before the size class was tuned lack pair_min
        t.pair_min = pm;
        ctx->tune[key] = t;
      }
    }
  }
  *out_ctx = ctx;
  return IBS_OK;
}

// IBS_TC_TILE_KERNEL set: the tensor-core form runs one CTA per tile (or tile
// piece) instead of the persistent kernels.
static bool tc_tile_kernel_forced() {
  static const bool v = getenv("IBS_TC_TILE_KERNEL") != nullptr;
  return v;
}

ibs_status ibs_compute(ibs_ctx* ctx, const uint8_t* packed, int64_t n, int64_t m, int32_t* out_counts,
                       double* out_dist, void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!packed || !out_counts) return fail(IBS_EINVAL, "packed and out_counts must be non-NULL");
  if (n < 1 || n > 2147483647LL) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 2^31)", (long long)n);
  if (m < 1 || m > 2147483647LL) return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^31)", (long long)m);
  if (reinterpret_cast<uintptr_t>(out_counts) % 16) return fail(IBS_EINVAL, "out_counts must be 16-byte aligned");
  if (out_dist && reinterpret_cast<uintptr_t>(out_dist) % 8) return fail(IBS_EINVAL, "out_dist must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(packed) || !is_device_ptr(out_counts) || (out_dist && !is_device_ptr(out_dist)))
    return fail(IBS_EINVAL, "packed, out_counts and out_dist must be device memory");
  if (ctx->flags & IBS_NO_DIST) out_dist = nullptr;
  const bool square = (ctx->flags & IBS_OUT_SQUARE) != 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool tc = use_tc(ctx);
  const int fmt = tc_format_for(ctx);
  // Tensor-core form, triangle output: the persistent kernel over a work list
  // (tail wave split over K).  Square output, or IBS_TC_TILE_KERNEL set: one
  // CTA per tile (or tile piece).
  const bool persistent = tc && !square && !tc_tile_kernel_forced();
  static const int group = [] {
    const char* e = getenv("IBS_TC_GROUP");
    const int v = e ? atoi(e) : 16;
    return v >= 1 && v <= 1024 ? v : 16;
  }();
  const PlaneGeom geo = PlaneGeom::make(n, m);
  if (ibs_status s = ensure_buf(ctx, ctx->planes, tc ? tc_planes_bytes(n, m, fmt) : geo.bytes())) return s;
  const int64_t tiles = tc ? tc_tiles(n) : geo.n_blocks * (geo.n_blocks + 1) / 2;
  int splits = 1;
  if (persistent) {
    // the two-SM kernel where it applies (E2M1, at least two blocks, items of
    // at least 1,024 chunks unless IBS_TC_PAIR says otherwise); its work list
    // depends on how many clusters of two fit at once
    const int pair_clusters = tc_pair_usable(n, m, fmt) ? tc_pair_clusters(tc_chunks(m, fmt)) : 0;
    const std::vector<int64_t> key = {n, m, fmt, ctx->num_sms, group, pair_clusters};
    if (ctx->single_key != key) {
      std::vector<WorkItem> items;
      std::vector<PairItem> pitems;
      std::vector<int2> split_tiles;
      if (pair_clusters > 0)
        tc_pair_items(n, m, fmt, pair_clusters, group, pitems, split_tiles);
      else
        tc_single_items(n, m, fmt, ctx->num_sms, group, items, split_tiles);
      const void* src = pair_clusters > 0 ? static_cast<const void*>(pitems.data()) : items.data();
      const size_t bytes = pair_clusters > 0 ? pitems.size() * sizeof(PairItem) : items.size() * sizeof(WorkItem);
      if (ibs_status s = ensure_buf(ctx, ctx->single_items, bytes)) return s;
      if (ibs_status s = ensure_buf(ctx, ctx->single_split, std::max<size_t>(1, split_tiles.size()) * sizeof(int2)))
        return s;
      if (ibs_status s = ensure_buf(ctx, ctx->single_counter, 256)) return s;
      // pageable sources: the copies are staged before return
      IBS_CUDA_TRY(cudaMemcpyAsync(ctx->single_items.p, src, bytes, cudaMemcpyHostToDevice, st));
      ctx->single_pair = pair_clusters > 0;
      if (!split_tiles.empty())
        IBS_CUDA_TRY(cudaMemcpyAsync(ctx->single_split.p, split_tiles.data(), split_tiles.size() * sizeof(int2),
                                     cudaMemcpyHostToDevice, st));
      ctx->single_n_items = (int64_t)(pair_clusters > 0 ? pitems.size() : items.size());
      // leading unsplit pair items, in whole waves of one item per cluster
      int64_t whole = 0;
      while (whole < (int64_t)pitems.size() && pitems[whole].split == 0) ++whole;
      ctx->single_clusters = pair_clusters;
      ctx->single_n_sync = pair_clusters > 0 ? whole / pair_clusters * pair_clusters : 0;
      ctx->single_n_split = (int64_t)split_tiles.size();
      ctx->single_key = key;
    }
    splits = ctx->single_n_split > 0 ? 2 : 1;  // > 1: partial counts and a finalisation pass
  } else if (tc) {
    const int64_t nc = tc_chunks(m, fmt);
    splits = (int)std::max<int64_t>(tc_splits_for(tiles, nc, ctx->num_sms),
                                    (nc + tc_max_chunks(fmt) - 1) / tc_max_chunks(fmt));
  } else {
    splits = tri_splits_for(tiles, geo.n_chunks, ctx->num_sms);
  }
  const int64_t P = n * (n + 1) / 2;
  if (splits > 1) {
    if (ibs_status s = ensure_buf(ctx, ctx->partial, (size_t)P * 16)) return s;
    IBS_CUDA_TRY(cudaMemsetAsync(ctx->partial.p, 0, (size_t)P * 16, st));
  }
  BedSource src;
  src.packed = packed;
  src.row_bytes = (n + 3) / 4;
  src.n_src = n;
  const bool timing = (ctx->flags & IBS_TIMING) != 0;
  ibs_ctx::TimingRec rec;
  if (timing) {
    if (!ctx->timing_free.empty()) {
      rec = ctx->timing_free.back();
      ctx->timing_free.pop_back();
    } else {
      for (auto& e : rec.ev) IBS_CUDA_TRY(cudaEventCreate(&e));
    }
    rec.n = splits > 1 ? 4 : 3;
    IBS_CUDA_TRY(cudaEventRecord(rec.ev[0], st));
  }
  if (persistent) {
    IBS_CUDA_TRY(launch_tc_planes(packed, n, m, static_cast<uint8_t*>(ctx->planes.p), fmt, st));
    if (timing) IBS_CUDA_TRY(cudaEventRecord(rec.ev[1], st));
    SubsetDev sd;
    sd.planes = static_cast<const uint32_t*>(ctx->planes.p);
    sd.n = n;
    sd.n_blocks = (n + 127) / 128;
    sd.n_chunks = tc_chunks(m, fmt);
    sd.out_counts = out_counts;
    sd.out_dist = out_dist;
    sd.partial = splits > 1 ? static_cast<int32_t*>(ctx->partial.p) : nullptr;
    sd.pad = 0;
    const unsigned long long wait_ns = ctx->wait_ns > 0 ? ctx->wait_ns : kWaitLimitNs;
    if (ctx->single_pair) {
      PairSync sync;
      const int2 ss = tc_pair_sync_setting(sd.n_chunks);
      if (ss.x > 0 && ctx->single_n_sync > 0) {
        sync.seg = ss.x;
        sync.lag = ss.y;
        sync.n_seg = (int32_t)((sd.n_chunks + ss.x - 1) / ss.x);
        sync.n_items = ctx->single_n_sync;
        const size_t bytes = (size_t)(ctx->single_n_sync / ctx->single_clusters) * sync.n_seg * sizeof(int);
        if (ibs_status s = ensure_buf(ctx, ctx->single_sync, bytes)) return s;
        IBS_CUDA_TRY(cudaMemsetAsync(ctx->single_sync.p, 0, bytes, st));
        sync.ctr = static_cast<int*>(ctx->single_sync.p);
      }
      IBS_CUDA_TRY(launch_tc_pair(sd, static_cast<const PairItem*>(ctx->single_items.p), ctx->single_n_items,
                                  ctx->status_dev, wait_ns, st, sync));
    } else {
      const int grid = (int)std::min<int64_t>(ctx->num_sms, ctx->single_n_items);
      IBS_CUDA_TRY(launch_tc_single(sd, static_cast<const WorkItem*>(ctx->single_items.p), ctx->single_n_items,
                                    grid, fmt, static_cast<int*>(ctx->single_counter.p), ctx->status_dev, wait_ns,
                                    st));
    }
  } else if (tc) {
    const int64_t T = (n + 127) / 128;
    if (ctx->tile_list_T != T) {
      std::vector<int2> order;
      tc_tile_order(T, group, order);
      if (ibs_status s = ensure_buf(ctx, ctx->tile_list, order.size() * sizeof(int2))) return s;
      // pageable source: the copy is staged before return
      IBS_CUDA_TRY(cudaMemcpyAsync(ctx->tile_list.p, order.data(), order.size() * sizeof(int2),
                                   cudaMemcpyHostToDevice, st));
      ctx->tile_list_T = T;
    }
    IBS_CUDA_TRY(launch_tc_planes(packed, n, m, static_cast<uint8_t*>(ctx->planes.p), fmt, st));
    if (timing) IBS_CUDA_TRY(cudaEventRecord(rec.ev[1], st));
    IBS_CUDA_TRY(launch_tc_pairs(static_cast<const uint8_t*>(ctx->planes.p), n, m, fmt, splits, out_counts, out_dist,
                                 static_cast<int32_t*>(ctx->partial.p), square, ctx->status_dev,
                                 static_cast<const int2*>(ctx->tile_list.p), st));
  } else {
    IBS_CUDA_TRY(launch_planes(src, n, m, geo, static_cast<uint32_t*>(ctx->planes.p), ctx->status_dev, st));
    if (timing) IBS_CUDA_TRY(cudaEventRecord(rec.ev[1], st));
    IBS_CUDA_TRY(launch_tri(mode_for(ctx), static_cast<const uint32_t*>(ctx->planes.p), geo, splits, out_counts,
                            out_dist, static_cast<int32_t*>(ctx->partial.p), square, ctx->status_dev, ctx->num_sms,
                            st));
  }
  if (timing) IBS_CUDA_TRY(cudaEventRecord(rec.ev[2], st));
  if (splits > 1) {
    if (persistent)
      IBS_CUDA_TRY(launch_tc_finalize_tiles(static_cast<const int2*>(ctx->single_split.p), ctx->single_n_split,
                                            static_cast<const int32_t*>(ctx->partial.p), n, out_counts, out_dist,
                                            st));
    else
      IBS_CUDA_TRY(launch_finalize(static_cast<const int32_t*>(ctx->partial.p), n, out_counts, out_dist, square, st));
  }
  if (timing) {
    if (splits > 1) IBS_CUDA_TRY(cudaEventRecord(rec.ev[3], st));
    ctx->timing_used.push_back(rec);
  }
  ctx->last_info[0] = splits > 1 ? 3 : 2;
  ctx->last_info[1] = tiles;
  ctx->last_info[2] = splits;
  return IBS_OK;
}

ibs_status ibs_synchronize(ibs_ctx* ctx, void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  DeviceGuard g(ctx->device);
  IBS_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  const int st = __atomic_exchange_n(ctx->status_host, 0, __ATOMIC_SEQ_CST);
  if (st == kDevTimeout) return fail(IBS_ETIMEOUT, "a bounded device wait timed out");
  if (st == IBS_EINVAL) return fail(IBS_EINVAL, "a sample index was out of range (treated as missing)");
  if (st != 0) return fail((ibs_status)st, "device status %d", st);
  return IBS_OK;
}

ibs_status ibs_kernel_times(ibs_ctx* ctx, double out[4]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  DeviceGuard g(ctx->device);
  for (int i = 0; i < 4; ++i) out[i] = 0;
  for (auto& r : ctx->timing_used) {
    IBS_CUDA_TRY(cudaEventSynchronize(r.ev[r.n - 1]));
    float ms = 0;
    IBS_CUDA_TRY(cudaEventElapsedTime(&ms, r.ev[0], r.ev[1]));
    out[0] += ms;
    IBS_CUDA_TRY(cudaEventElapsedTime(&ms, r.ev[1], r.ev[2]));
    out[1] += ms;
    if (r.n == 4) {
      IBS_CUDA_TRY(cudaEventElapsedTime(&ms, r.ev[2], r.ev[3]));
      out[2] += ms;
    }
    out[3] += 1;
    ctx->timing_free.push_back(r);
  }
  ctx->timing_used.clear();
  return IBS_OK;
}

ibs_status ibs_last_launch_info(ibs_ctx* ctx, int64_t out[3]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  for (int i = 0; i < 3; ++i) out[i] = ctx->last_info[i];
  return IBS_OK;
}

ibs_status ibs_probe_mma(ibs_ctx* ctx, double out[2]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  DeviceGuard g(ctx->device);
  IBS_CUDA_TRY(probe_tc_mma(ctx->device, ctx->num_sms, ctx->status_dev, out));
  if (__atomic_exchange_n(ctx->status_host, 0, __ATOMIC_SEQ_CST) == kDevTimeout)
    return fail(IBS_ETIMEOUT, "the MMA probe's bounded wait timed out");
  return IBS_OK;
}

ibs_status ibs_probe_int_pipes(ibs_ctx* ctx, double out[5]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  DeviceGuard g(ctx->device);
  IBS_CUDA_TRY(probe_int_pipes(ctx->device, out));
  return IBS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched path.
namespace {

struct SubsetShape {
  int64_t n, m;
  PlaneGeom g;
};

// Batched modes: 0 = plain POPC, 1 = carry-save POPC (2 CTAs/SM), 2 = carry-save
// (1 CTA/SM), 3 + fmt = tensor core (indicator GEMMs, 128-sample tiles) with
// operand format fmt (kTcFp8 / kTcFp4).
constexpr int kBatchModeTc = 3;
bool is_tc_mode(int mode) { return mode >= kBatchModeTc; }
int tc_fmt_of(int mode) { return mode - kBatchModeTc; }
constexpr int kTcBatchGroup = 16;  // tile rows per band of the grouped order

// Tile grid of one subset in the units of the pair kernel of `mode`: blocks
// per side and K chunks.
struct ItemGeom {
  int64_t T, nc;
};
ItemGeom item_geom(const SubsetShape& s, int mode) {
  if (is_tc_mode(mode)) return {(s.n + 127) / 128, tc_chunks(s.m, tc_fmt_of(mode))};
  return {s.g.n_blocks, s.g.n_chunks};
}

// Build the work list for a batch: every (subset, tile) item, K-split for
// subsets whose tiles would be too large relative to one CTA's fair share
// (split_policy 1), sorted by descending cost (longest processing time first).
// Tensor-core split_policy 2: each subset's own single-matrix list (its final
// partial wave, or all of it when it has fewer tiles than CTAs, split over K;
// the split tiles go to split_tiles_out), for one launch per subset.
void build_items(const std::vector<SubsetShape>& shapes, int mode, int split_policy, int grid,
                 std::vector<WorkItem>& items, std::vector<int>& subset_split, int64_t& tiles_total,
                 std::vector<int64_t>* order_out = nullptr, std::vector<int64_t>* item_off_out = nullptr,
                 std::vector<int4>* split_tiles_out = nullptr) {
  items.clear();
  subset_split.assign(shapes.size(), 1);
  double total = 0;
  tiles_total = 0;
  for (const auto& s : shapes) {
    const ItemGeom ig = item_geom(s, mode);
    total += (double)(ig.T * (ig.T + 1) / 2) * (double)ig.nc;
    tiles_total += ig.T * (ig.T + 1) / 2;
  }
  const double share = total / std::max(1, grid);
  for (size_t k = 0; k < shapes.size(); ++k) {
    const ItemGeom ig = item_geom(shapes[k], mode);
    if (split_policy == 1) {
      const double item = (double)ig.nc;
      // aim for items no larger than a quarter of a CTA's fair share
      int pieces = (int)std::ceil(item / std::max(1.0, share / 4.0));
      pieces = std::max(1, std::min<int>(pieces, (int)std::min<int64_t>(ig.nc, 64)));
      subset_split[k] = pieces;
    }
    if (is_tc_mode(mode)) {  // exact FP32 accumulation: at most 2^21 markers per item
      const int64_t maxc = tc_max_chunks(tc_fmt_of(mode));
      subset_split[k] = std::max<int>(subset_split[k], (int)((ig.nc + maxc - 1) / maxc));
    }
  }
  if (is_tc_mode(mode)) {
    // Claimed in list order by whichever CTA is free: subsets by decreasing
    // tile cost, each subset's tiles in the grouped order, so the CTAs
    // running at one time share row and column blocks through L2.
    std::vector<size_t> order(shapes.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      return item_geom(shapes[a], mode).nc > item_geom(shapes[b], mode).nc;
    });
    std::vector<int2> tiles;
    if (order_out) order_out->assign(order.begin(), order.end());
    if (item_off_out) item_off_out->clear();
    if (split_tiles_out) split_tiles_out->clear();
    for (size_t k : order) {
      const ItemGeom ig = item_geom(shapes[k], mode);
      if (item_off_out) item_off_out->push_back((int64_t)items.size());
      if (split_policy == 2 || split_policy == 5) {
        std::vector<WorkItem> own;
        std::vector<int2> own_split;
        tc_single_items(shapes[k].n, shapes[k].m, tc_fmt_of(mode), grid, kTcBatchGroup, own, own_split);
        for (WorkItem w : own) {
          w.subset = (int32_t)k;
          items.push_back(w);
        }
        subset_split[k] = own_split.empty() ? 1 : 2;
        if (split_tiles_out)
          for (const int2& t : own_split) split_tiles_out->push_back(make_int4((int)k, t.x, t.y, 0));
        continue;
      }
      const int pieces = subset_split[k];
      tc_tile_order(ig.T, kTcBatchGroup, tiles);
      for (const int2& t : tiles)
        for (int p = 0; p < pieces; ++p) {
          WorkItem w{};
          w.subset = (int32_t)k;
          w.I = t.x;
          w.J = t.y;
          w.c0 = (int32_t)(ig.nc * p / pieces);
          w.c1 = (int32_t)(ig.nc * (p + 1) / pieces);
          w.split = pieces > 1 ? 1 : 0;
          items.push_back(w);
        }
    }
    if (item_off_out) item_off_out->push_back((int64_t)items.size());
    return;
  }
  for (size_t k = 0; k < shapes.size(); ++k) {
    const ItemGeom ig = item_geom(shapes[k], mode);
    const int pieces = subset_split[k];
    for (int64_t I = 0; I < ig.T; ++I)
      for (int64_t J = I; J < ig.T; ++J)
        for (int p = 0; p < pieces; ++p) {
          WorkItem w{};
          w.subset = (int32_t)k;
          w.I = (int32_t)I;
          w.J = (int32_t)J;
          w.c0 = (int32_t)(ig.nc * p / pieces);
          w.c1 = (int32_t)(ig.nc * (p + 1) / pieces);
          w.split = pieces > 1 ? 1 : 0;
          items.push_back(w);
        }
  }
  std::stable_sort(items.begin(), items.end(), [](const WorkItem& a, const WorkItem& b) {
    const int64_t ca = (int64_t)(a.c1 - a.c0) * (a.I == a.J ? 1 : 2);
    const int64_t cb = (int64_t)(b.c1 - b.c0) * (b.I == b.J ? 1 : 2);
    return ca > cb;
  });
}

std::string tune_key(const ibs_ctx* ctx, const std::vector<SubsetShape>& shapes) {
  // bucket: subsets count, log2 of total pair-words, log2 of the largest subset's n
  double total = 0;
  int64_t nmax = 0;
  for (const auto& s : shapes) {
    total += (double)s.n * (double)s.n * 0.5 * (double)s.m;
    nmax = std::max(nmax, s.n);
  }
  std::ostringstream o;
  o << "sms" << ctx->num_sms << "_s" << shapes.size() << "_w" << (int)std::log2(std::max(1.0, total)) << "_n"
    << (int)std::log2((double)std::max<int64_t>(1, nmax));
  return o.str();
}

ibs_status plan_build(ibs_ctx* ctx, BatchPlan& plan, const std::vector<SubsetShape>& shapes, int mode,
                      int split_policy, int64_t pair_min = 1024) {
  plan.mode = mode;
  plan.split_policy = split_policy;
  plan.pair_min_chunks = pair_min;
  const bool tc = is_tc_mode(mode);
  plan.grid = ctx->num_sms * (tc ? 1 : pair_kernel_ctas_per_sm(mode));
  std::vector<WorkItem> items;
  std::vector<int> split;
  std::vector<int64_t> subset_item_off;
  std::vector<int4> split_tiles;
  build_items(shapes, mode, split_policy, plan.grid, items, split, plan.tiles, &plan.order, &subset_item_off,
              &split_tiles);
  plan.q_item_off = subset_item_off;
  plan.q_chunks.clear();
  for (int64_t q : plan.order) plan.q_chunks.push_back(item_geom(shapes[(size_t)q], mode).nc);
  plan.q_pair_off.assign(plan.order.size(), -1);
  plan.q_pair_n.assign(plan.order.size(), 0);
  plan.q_pair_sync.assign(plan.order.size(), 0);
  plan.pair_sync_bytes = 0;
  plan.n_pitems = 0;
  plan.pair_max_chunks = 0;
  std::vector<PairItem> p2_items;
  if (tc && split_policy >= 2) {
    // Policy 2: each subset on the kernel ibs_compute picks for its shape:
    // the two-SM kernel over its own pair work list (tail wave split over K)
    // where it applies, else its one-SM items built above.  Policies 3, 4:
    // every subset's own pair work list, concatenated in processing order
    // for one launch; a subset's tail pieces keep the clusters on that
    // subset's blocks together, as its own launch would.  Before the partial
    // buffers are sized: a pair list may split tiles the one-SM list does not.
    std::vector<PairItem> own;
    std::vector<int2> own_split;
    for (size_t q = 0; q < plan.order.size(); ++q) {
      const size_t k = (size_t)plan.order[q];
      if ((split_policy == 2 || split_policy == 5) &&
          (!tc_pair_usable(shapes[k].n, shapes[k].m, tc_fmt_of(mode)) ||
           (tc_pair_mode() == 0 && item_geom(shapes[k], mode).nc < pair_min)))
        continue;  // this subset's size class runs on the one-SM kernel
      const ItemGeom ig = item_geom(shapes[k], mode);
      tc_pair_items(shapes[k].n, shapes[k].m, tc_fmt_of(mode), tc_pair_clusters(ig.nc), kTcBatchGroup, own,
                    own_split);
      plan.q_pair_off[q] = (int64_t)p2_items.size();
      plan.q_pair_n[q] = (int64_t)own.size();
      {
        // its own launch (policy 2) keeps its leading whole waves in K-lockstep
        const int C = tc_pair_clusters(ig.nc);
        const int2 ss = tc_pair_sync_setting(ig.nc);
        int64_t whole = 0;
        while (whole < (int64_t)own.size() && own[(size_t)whole].split == 0) ++whole;
        if ((split_policy == 2 || split_policy == 5) && ss.x > 0 && C > 0 && whole >= C) {
          plan.q_pair_sync[q] = whole / C * C;
          plan.pair_sync_bytes = std::max(plan.pair_sync_bytes,
                                          (size_t)(whole / C) * (size_t)((ig.nc + ss.x - 1) / ss.x) * sizeof(int));
        }
      }
      plan.pair_max_chunks = std::max(plan.pair_max_chunks, ig.nc);
      for (PairItem w : own) {
        w.subset = (int32_t)k;
        p2_items.push_back(w);
      }
      // this subset's split tiles are the pair list's, not the one-SM list's
      split_tiles.erase(std::remove_if(split_tiles.begin(), split_tiles.end(),
                                       [&](const int4& t) { return t.x == (int)k; }),
                        split_tiles.end());
      for (const int2& t : own_split) split_tiles.push_back(make_int4((int)k, t.x, t.y, 0));
      split[k] = own_split.empty() ? 1 : 2;
    }
    plan.n_pitems = (int64_t)p2_items.size();
    plan.n_units = 0;
  }
  plan.n_split_tiles = (int64_t)split_tiles.size();
  plan.n_items = (int64_t)items.size();
  if (plan.grid > plan.n_items) plan.grid = (int)std::max<int64_t>(1, plan.n_items);
  // planes and partial offsets
  size_t pb = 0, qb = 0;
  plan.plane_offsets.resize(shapes.size());
  plan.partial_offsets.assign(shapes.size(), -1);
  std::vector<int32_t> split_ids;
  plan.max_split_pairs = 0;
  for (size_t k = 0; k < shapes.size(); ++k) {
    plan.plane_offsets[k] = (int64_t)pb;
    pb += (shapes[k].g.bytes() + 255) / 256 * 256;
    if (split[k] > 1) {
      const int64_t P = shapes[k].n * (shapes[k].n + 1) / 2;
      plan.partial_offsets[k] = (int64_t)qb;
      qb += ((size_t)P * 16 + 255) / 256 * 256;
      split_ids.push_back((int32_t)k);
      plan.max_split_pairs = std::max(plan.max_split_pairs, P);
    }
  }
  plan.n_split = (int)split_ids.size();
  plan.total_ctas = 0;
  for (const auto& s : shapes) plan.total_ctas += s.g.n_chunks * ((s.g.n_blocks + 1) / 2);
  if (tc) {
    // the tensor-core form gathers straight into operand planes: no bit planes
    // (each subset's planes start on a 16 KiB block-chunk boundary, so that
    // one tensor map over the whole buffer addresses every subset)
    size_t tb = 0;
    plan.tc_offsets.resize(shapes.size());
    plan.tc_ctas = 0;
    constexpr size_t kBc = 16384;
    for (size_t k = 0; k < shapes.size(); ++k) {
      plan.tc_offsets[k] = (int64_t)tb;
      tb += (tc_planes_bytes(shapes[k].n, shapes[k].m, tc_fmt_of(mode)) + kBc - 1) / kBc * kBc;
      plan.tc_ctas += tc_gather_ctas(shapes[k].n, item_geom(shapes[k], mode).nc);
    }
    plan.tc_block_chunks = (int64_t)(tb / kBc);
    if (split_policy == 2 || split_policy == 5) {
      std::vector<int32_t> zero(shapes.size(), 0);
      if (ibs_status s = ensure_buf(ctx, plan.pitems, sizeof(PairItem) * std::max<size_t>(1, p2_items.size()))) return s;
      if (plan.pair_sync_bytes > 0)
        if (ibs_status s = ensure_buf(ctx, plan.pair_sync, plan.pair_sync_bytes)) return s;
      if (ibs_status s = ensure_buf(ctx, plan.units, sizeof(int4))) return s;
      // policy 5: two unit counters per subset position (its own gather launch, and the fused gather
      // of the two-SM launch that runs it)
      if (ibs_status s = ensure_buf(ctx, plan.unit_counter, std::max<size_t>(256, 8 * (plan.order.size() + 1))))
        return s;
      if (ibs_status s = ensure_buf(ctx, plan.ready, sizeof(int32_t) * shapes.size())) return s;
      if (ibs_status s = ensure_buf(ctx, plan.need, sizeof(int32_t) * shapes.size())) return s;
      if (!p2_items.empty())
        IBS_CUDA_TRY(
            cudaMemcpy(plan.pitems.p, p2_items.data(), sizeof(PairItem) * p2_items.size(), cudaMemcpyHostToDevice));
      IBS_CUDA_TRY(cudaMemcpy(plan.need.p, zero.data(), sizeof(int32_t) * zero.size(), cudaMemcpyHostToDevice));
      IBS_CUDA_TRY(cudaMemcpy(plan.ready.p, zero.data(), sizeof(int32_t) * zero.size(), cudaMemcpyHostToDevice));
    }
    if (split_policy == 5) {
      // Policy 5: policy 2's launches; the gather units of every subset in
      // processing order (q_unit_off per position), taken by the epilogue
      // warps of the two-SM launch before them, or by a gather launch of
      // their own.  No copy waits on readiness (need stays zero): stream
      // order has every subset gathered before its launch.
      std::vector<int4> units;
      plan.q_unit_off.assign(1, 0);
      for (size_t q = 0; q < plan.order.size(); ++q) {
        const size_t k = (size_t)plan.order[q];
        const ItemGeom ig = item_geom(shapes[k], mode);
        const int64_t groups = (ig.nc + tc_gather_chunks() - 1) / tc_gather_chunks();
        for (int64_t cg = 0; cg < groups; ++cg)
          for (int64_t bl = 0; bl < ig.T; ++bl) units.push_back(make_int4((int)q, (int)bl, (int)cg, (int)k));
        plan.q_unit_off.push_back((int64_t)units.size());
      }
      plan.n_units = (int64_t)units.size();
      if (plan.n_units > 2147483647LL) return fail(IBS_EINVAL, "batch too large for the fused gather");
      if (ibs_status s = ensure_buf(ctx, plan.units, sizeof(int4) * std::max<size_t>(1, units.size()))) return s;
      IBS_CUDA_TRY(cudaMemcpy(plan.units.p, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice));
    }
    if (split_policy == 3 || split_policy == 4) {
      // One launch of the two-SM kernel over the concatenated pair lists
      // (above), and the gather units of the subsets in the same order for
      // its epilogue warps and the side stream's gather CTAs.
      std::vector<PairItem>& pitems = p2_items;
      std::vector<int4> units;
      std::vector<int32_t> need(shapes.size(), 0);
      for (size_t q = 0; q < plan.order.size(); ++q) {
        const size_t k = (size_t)plan.order[q];
        const ItemGeom ig = item_geom(shapes[k], mode);
        const int64_t groups = (ig.nc + tc_gather_chunks() - 1) / tc_gather_chunks();
        for (int64_t cg = 0; cg < groups; ++cg)
          for (int64_t bl = 0; bl < ig.T; ++bl) units.push_back(make_int4((int)q, (int)bl, (int)cg, (int)k));
        need[k] = (int32_t)(groups * ig.T);
      }
      plan.n_split_tiles = (int64_t)split_tiles.size();
      plan.n_pitems = (int64_t)pitems.size();
      plan.n_units = (int64_t)units.size();
      if (plan.n_units > 2147483647LL) return fail(IBS_EINVAL, "batch too large for the fused gather");
      if (ibs_status s = ensure_buf(ctx, plan.pitems, sizeof(PairItem) * std::max<size_t>(1, pitems.size()))) return s;
      if (ibs_status s = ensure_buf(ctx, plan.units, sizeof(int4) * std::max<size_t>(1, units.size()))) return s;
      if (ibs_status s = ensure_buf(ctx, plan.unit_counter, 256)) return s;
      if (ibs_status s = ensure_buf(ctx, plan.ready, sizeof(int32_t) * shapes.size())) return s;
      if (ibs_status s = ensure_buf(ctx, plan.need, sizeof(int32_t) * shapes.size())) return s;
      IBS_CUDA_TRY(cudaMemcpy(plan.pitems.p, pitems.data(), sizeof(PairItem) * pitems.size(), cudaMemcpyHostToDevice));
      IBS_CUDA_TRY(cudaMemcpy(plan.units.p, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice));
      IBS_CUDA_TRY(cudaMemcpy(plan.need.p, need.data(), sizeof(int32_t) * need.size(), cudaMemcpyHostToDevice));
    }
    if (plan.tc_ctas > 2147483647LL) return fail(IBS_EINVAL, "batch too large for one gather launch");
    // Stages: about 10% of the comparisons first (its gather is the only one
    // not overlapped), then three of about 30%.
    double total = 0;
    for (const auto& sh : shapes) total += (double)sh.n * (double)sh.n * (double)sh.m;
    const double bounds[] = {0.10, 0.40, 0.70, 1.01};
    plan.stage_item_off.assign(1, 0);
    plan.stage_job_off.assign(1, 0);
    plan.stage_ctas.clear();
    plan.stage_max_chunks.clear();
    double acc = 0;
    int64_t ctas = 0, max_chunks = 0;
    int b = 0;
    for (size_t q = 0; q < plan.order.size(); ++q) {
      const SubsetShape& sh = shapes[plan.order[q]];
      acc += (double)sh.n * (double)sh.n * (double)sh.m;
      ctas += tc_gather_ctas(sh.n, item_geom(sh, mode).nc);
      max_chunks = std::max<int64_t>(max_chunks, item_geom(sh, mode).nc);
      const bool last = q + 1 == plan.order.size();
      if (last || acc >= bounds[b] * total) {
        plan.stage_item_off.push_back(subset_item_off[q + 1]);
        plan.stage_job_off.push_back((int64_t)q + 1);
        plan.stage_ctas.push_back(ctas);
        plan.stage_max_chunks.push_back(max_chunks);
        ctas = 0;
        max_chunks = 0;
        while (b < 3 && acc >= bounds[b] * total) ++b;
      }
    }
    if (split_policy == 3 || split_policy == 4) {
      IBS_CUDA_TRY(cudaStreamCreateWithFlags(&plan.side, cudaStreamNonBlocking));
      IBS_CUDA_TRY(cudaEventCreateWithFlags(&plan.fork_ev, cudaEventDisableTiming));
      IBS_CUDA_TRY(cudaEventCreateWithFlags(&plan.join_ev, cudaEventDisableTiming));
    } else if (plan.stage_ctas.size() > 1) {
      IBS_CUDA_TRY(cudaStreamCreateWithFlags(&plan.side, cudaStreamNonBlocking));
      plan.stage_ev.resize(plan.stage_ctas.size(), nullptr);
      for (auto& e : plan.stage_ev) IBS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (ibs_status s = ensure_buf(ctx, plan.tc_planes, tb)) return s;
    if (ibs_status s = ensure_buf(ctx, plan.tc_jobs, sizeof(TcGatherJob) * shapes.size())) return s;
    if (ibs_status s = ensure_buf(ctx, plan.gather_map, sizeof(int4) * std::max<int64_t>(1, plan.tc_ctas))) return s;
    plan.stage_map_off.assign(1, 0);
    for (int64_t c : plan.stage_ctas) plan.stage_map_off.push_back(plan.stage_map_off.back() + c);
    plan.map_key.clear();
    pb = 0;
  }
  if (ibs_status s = ensure_buf(ctx, plan.planes, pb)) return s;
  if (ibs_status s = ensure_buf(ctx, plan.partial, qb)) return s;
  if (ibs_status s = ensure_buf(ctx, plan.subsets, sizeof(SubsetDev) * shapes.size())) return s;
  if (ibs_status s = ensure_buf(ctx, plan.jobs, sizeof(PlaneJob) * shapes.size())) return s;
  if (ibs_status s = ensure_buf(ctx, plan.items, sizeof(WorkItem) * std::max<size_t>(1, items.size()))) return s;
  if (ibs_status s = ensure_buf(ctx, plan.split_ids, sizeof(int32_t) * std::max<size_t>(1, split_ids.size())))
    return s;
  if (ibs_status s = ensure_buf(ctx, plan.counter, 256)) return s;
  IBS_CUDA_TRY(cudaMemcpy(plan.items.p, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice));
  if (!split_tiles.empty()) {
    if (ibs_status s = ensure_buf(ctx, plan.split_tiles, sizeof(int4) * split_tiles.size())) return s;
    IBS_CUDA_TRY(cudaMemcpy(plan.split_tiles.p, split_tiles.data(), sizeof(int4) * split_tiles.size(),
                            cudaMemcpyHostToDevice));
  }
  if (!split_ids.empty())
    IBS_CUDA_TRY(cudaMemcpy(plan.split_ids.p, split_ids.data(), sizeof(int32_t) * split_ids.size(),
                            cudaMemcpyHostToDevice));
  return IBS_OK;
}

// Upload the per-call descriptors (pointers may change between calls of one shape).
ibs_status plan_upload(ibs_ctx* ctx, BatchPlan& plan, const uint8_t* pool, int64_t pool_n,
                       const ibs_subset* subs, const std::vector<SubsetShape>& shapes, cudaStream_t st) {
  const size_t k = shapes.size();
  std::vector<SubsetDev> sd(k);
  std::vector<PlaneJob> jobs(k);
  int64_t cta = 0;
  for (size_t i = 0; i < k; ++i) {
    uint32_t* planes = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(plan.planes.p) + plan.plane_offsets[i]);
    sd[i].planes = planes;
    sd[i].n = shapes[i].n;
    sd[i].n_blocks = shapes[i].g.n_blocks;
    sd[i].n_chunks = shapes[i].g.n_chunks;
    sd[i].out_counts = subs[i].out_counts;
    sd[i].out_dist = (ctx->flags & IBS_NO_DIST) ? nullptr : subs[i].out_dist;
    sd[i].partial = plan.partial_offsets[i] >= 0
                        ? reinterpret_cast<int32_t*>(static_cast<uint8_t*>(plan.partial.p) + plan.partial_offsets[i])
                        : nullptr;
    sd[i].pad = 0;
    jobs[i].src.packed = pool;
    jobs[i].src.row_bytes = (pool_n + 3) / 4;
    jobs[i].src.var_begin = subs[i].var_begin;
    jobs[i].src.sel = subs[i].sample_idx;
    jobs[i].src.n_src = pool_n;
    jobs[i].m = shapes[i].m;
    jobs[i].n = shapes[i].n;
    jobs[i].planes = planes;
    jobs[i].n_blocks = shapes[i].g.n_blocks;
    jobs[i].n_chunks = shapes[i].g.n_chunks;
    jobs[i].groups = (shapes[i].g.n_blocks + 1) / 2;
    jobs[i].cta_begin = cta;
    cta += shapes[i].g.n_chunks * jobs[i].groups;
  }
  if (is_tc_mode(plan.mode)) {
    // the pair kernel reads operand planes, in 128-sample blocks and MMA-K
    // chunks; gather jobs in processing order (the CTA map below refers to them)
    std::vector<TcGatherJob> tj(k);
    for (size_t q = 0; q < k; ++q) {
      const size_t i = (size_t)plan.order[q];
      const ItemGeom ig = item_geom(shapes[i], plan.mode);
      uint8_t* tcp = static_cast<uint8_t*>(plan.tc_planes.p) + plan.tc_offsets[i];
      sd[i].planes = reinterpret_cast<const uint32_t*>(tcp);
      sd[i].n_blocks = ig.T;
      sd[i].n_chunks = ig.nc;
      sd[i].pad = plan.tc_offsets[i] / 16384;  // first block-chunk of the subset in the shared buffer
      tj[q].src = jobs[i].src;
      tj[q].m = shapes[i].m;
      tj[q].n = shapes[i].n;
      tj[q].tc = tcp;
      tj[q].nb = ig.T;
      tj[q].nc = ig.nc;
    }
    IBS_CUDA_TRY(cudaMemcpyAsync(plan.tc_jobs.p, tj.data(), sizeof(TcGatherJob) * k, cudaMemcpyHostToDevice, st));
    // Gather CTA order within each stage: by the pool variant a CTA starts at
    // (a counting sort over chunk-group-sized buckets), then job, block.
    std::vector<int64_t> key(k);
    for (size_t i = 0; i < k; ++i) key[i] = subs[i].var_begin;
    if (plan.split_policy < 3 && plan.map_key != key) {  // policies 3-5 gather by their own unit list
      const int64_t span = (int64_t)tc_gather_chunks() * (tc_fmt_of(plan.mode) == kTcFp4 ? 64 : 32);
      int64_t vend = 0;
      for (size_t i = 0; i < k; ++i) vend = std::max<int64_t>(vend, subs[i].var_begin + shapes[i].m);
      const int64_t buckets = (vend + span - 1) / span + 1;
      std::vector<int4> map((size_t)std::max<int64_t>(1, plan.tc_ctas));
      std::vector<int64_t> count((size_t)buckets + 1);
      for (size_t g = 0; g + 1 < plan.stage_job_off.size(); ++g) {
        std::fill(count.begin(), count.end(), 0);
        auto each = [&](auto&& f) {
          for (int64_t q = plan.stage_job_off[g]; q < plan.stage_job_off[g + 1]; ++q) {
            const size_t i = (size_t)plan.order[(size_t)q];
            const ItemGeom ig = item_geom(shapes[i], plan.mode);
            const int64_t groups = (ig.nc + tc_gather_chunks() - 1) / tc_gather_chunks();
            for (int64_t cg = 0; cg < groups; ++cg) {
              const int64_t bucket = (subs[i].var_begin + cg * span) / span;
              for (int64_t bl = 0; bl < ig.T; ++bl) f(q, bl, cg, bucket);
            }
          }
        };
        each([&](int64_t, int64_t, int64_t, int64_t bucket) { ++count[(size_t)bucket + 1]; });
        for (size_t u = 1; u < count.size(); ++u) count[u] += count[u - 1];
        int4* out = map.data() + plan.stage_map_off[g];
        each([&](int64_t q, int64_t bl, int64_t cg, int64_t bucket) {
          out[count[(size_t)bucket]++] = make_int4((int)q, (int)bl, (int)cg, 0);
        });
      }
      // pageable source: the copy is staged before return
      IBS_CUDA_TRY(cudaMemcpyAsync(plan.gather_map.p, map.data(), sizeof(int4) * (size_t)plan.tc_ctas,
                                   cudaMemcpyHostToDevice, st));
      plan.map_key = key;
    }
  }
  // Pageable sources: the copy is staged before return, so the vectors may go.
  IBS_CUDA_TRY(cudaMemcpyAsync(plan.subsets.p, sd.data(), sizeof(SubsetDev) * k, cudaMemcpyHostToDevice, st));
  IBS_CUDA_TRY(cudaMemcpyAsync(plan.jobs.p, jobs.data(), sizeof(PlaneJob) * k, cudaMemcpyHostToDevice, st));
  return IBS_OK;
}

// Enqueue the batch's launches (also used under stream capture).
ibs_status plan_enqueue(ibs_ctx* ctx, BatchPlan& plan, int n_subsets, cudaStream_t st) {
  IBS_CUDA_TRY(cudaMemsetAsync(plan.counter.p, 0, sizeof(int), st));
  if (plan.n_split > 0) IBS_CUDA_TRY(cudaMemsetAsync(plan.partial.p, 0, plan.partial.cap, st));
  if (is_tc_mode(plan.mode)) {
    const int fmt = tc_fmt_of(plan.mode);
    const TcGatherJob* jobs = static_cast<const TcGatherJob*>(plan.tc_jobs.p);
    const WorkItem* items = static_cast<const WorkItem*>(plan.items.p);
    if (plan.split_policy == 5) {
      // One launch per subset, as policy 2.  The epilogue warps of each
      // two-SM launch gather the planes of the subsets after it, up to and
      // including the next two-SM subset, while its items' MMAs run; a subset
      // that no earlier launch gathered gets a gather launch first.
      const int64_t Q = (int64_t)plan.order.size();
      const int4* units = static_cast<const int4*>(plan.units.p);
      int* ctr = static_cast<int*>(plan.unit_counter.p);  // [2 q]: own gather, [2 q + 1]: fused in launch q
      IBS_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * 2 * (size_t)(Q + 1), st));
      int64_t gathered_upto = 0;  // positions [0, gathered_upto) are (being) gathered
      for (int64_t q = 0; q < Q; ++q) {
        if (gathered_upto <= q) {
          IBS_CUDA_TRY(launch_tc_gather_units(jobs, units + plan.q_unit_off[(size_t)q],
                                              plan.q_unit_off[(size_t)q + 1] - plan.q_unit_off[(size_t)q],
                                              ctr + 2 * q, static_cast<int*>(plan.ready.p), fmt, 8 * ctx->num_sms,
                                              ctx->status_dev, st));
          gathered_upto = q + 1;
        }
        if (plan.q_pair_off[(size_t)q] >= 0) {
          int64_t r = q + 1;
          while (r < Q && plan.q_pair_off[(size_t)r] < 0) ++r;
          const int64_t end = std::min<int64_t>(r + 1, Q);  // exclusive: through the next two-SM subset
          PairBatchArgs a;
          a.subs = static_cast<const SubsetDev*>(plan.subsets.p);
          a.items = static_cast<const PairItem*>(plan.pitems.p) + plan.q_pair_off[(size_t)q];
          a.n_items = plan.q_pair_n[(size_t)q];
          a.jobs = jobs;
          a.units = units + plan.q_unit_off[(size_t)gathered_upto];
          a.n_units = end > gathered_upto ? plan.q_unit_off[(size_t)end] - plan.q_unit_off[(size_t)gathered_upto] : 0;
          a.unit_counter = ctr + 2 * q + 1;
          a.ready = static_cast<int*>(plan.ready.p);
          a.need = static_cast<const int*>(plan.need.p);  // all zero: nothing to wait for
          a.planes = plan.tc_planes.p;
          a.block_chunks = plan.tc_block_chunks;
          a.max_chunks = plan.q_chunks[(size_t)q];
          if (plan.q_pair_sync[(size_t)q] > 0) {
            const int2 ss = tc_pair_sync_setting(a.max_chunks);
            a.sync.seg = ss.x;
            a.sync.lag = ss.y;
            a.sync.n_seg = (int32_t)((a.max_chunks + ss.x - 1) / ss.x);
            a.sync.n_items = plan.q_pair_sync[(size_t)q];
            a.sync.ctr = static_cast<int*>(plan.pair_sync.p);
            IBS_CUDA_TRY(cudaMemsetAsync(plan.pair_sync.p, 0,
                                         (size_t)(a.sync.n_items / tc_pair_clusters(a.max_chunks)) * a.sync.n_seg *
                                             sizeof(int),
                                         st));
          }
          IBS_CUDA_TRY(launch_tc_pair_batch(a, ctx->status_dev, kWaitLimitNs, st));
          gathered_upto = std::max(gathered_upto, end);
          continue;
        }
        const int64_t n_items = plan.q_item_off[q + 1] - plan.q_item_off[q];
        IBS_CUDA_TRY(launch_tc_batch(static_cast<const SubsetDev*>(plan.subsets.p), items + plan.q_item_off[q],
                                     n_items, (int)std::min<int64_t>(plan.grid, n_items), fmt, plan.q_chunks[q],
                                     static_cast<int*>(plan.counter.p), ctx->status_dev, st));
      }
      IBS_CUDA_TRY(launch_tc_finalize_batch_tiles(static_cast<const SubsetDev*>(plan.subsets.p),
                                                  static_cast<const int4*>(plan.split_tiles.p), plan.n_split_tiles,
                                                  st));
      return IBS_OK;
    }
    if (plan.split_policy >= 3) {
      // one launch: the two-SM kernel over every subset's pair items, its
      // epilogue warps gathering the subsets' planes from the pool as they go
      IBS_CUDA_TRY(cudaMemsetAsync(plan.unit_counter.p, 0, sizeof(int), st));
      IBS_CUDA_TRY(cudaMemsetAsync(plan.ready.p, 0, sizeof(int32_t) * (size_t)n_subsets, st));
      PairBatchArgs a;
      a.subs = static_cast<const SubsetDev*>(plan.subsets.p);
      a.items = static_cast<const PairItem*>(plan.pitems.p);
      a.n_items = plan.n_pitems;
      a.jobs = jobs;
      a.units = static_cast<const int4*>(plan.units.p);
      a.n_units = plan.n_units;
      a.unit_counter = static_cast<int*>(plan.unit_counter.p);
      a.ready = static_cast<int*>(plan.ready.p);
      a.need = static_cast<const int*>(plan.need.p);
      a.planes = plan.tc_planes.p;
      a.block_chunks = plan.tc_block_chunks;
      a.max_chunks = plan.pair_max_chunks;
      if (plan.split_policy == 4) {
        // policy 4: every unit gathered ahead, at full occupancy, then the
        // pair launch (whose gate then opens at once)
        IBS_CUDA_TRY(launch_tc_gather_units(jobs, a.units, a.n_units, a.unit_counter, a.ready, fmt,
                                            8 * ctx->num_sms, ctx->status_dev, st));
        IBS_CUDA_TRY(launch_tc_pair_batch(a, ctx->status_dev, kWaitLimitNs, st));
      } else {
        // policy 3: the pair launch first, then, on the side stream, persistent
        // gather CTAs that run beside it (two per SM fit next to a pair CTA)
        // and claim units from the same list as its epilogue warps
        IBS_CUDA_TRY(cudaEventRecord(plan.fork_ev, st));
        IBS_CUDA_TRY(launch_tc_pair_batch(a, ctx->status_dev, kWaitLimitNs, st));
        IBS_CUDA_TRY(cudaStreamWaitEvent(plan.side, plan.fork_ev, 0));
        IBS_CUDA_TRY(launch_tc_gather_units(jobs, a.units, a.n_units, a.unit_counter, a.ready, fmt,
                                            2 * ctx->num_sms, ctx->status_dev, plan.side));
        IBS_CUDA_TRY(cudaEventRecord(plan.join_ev, plan.side));
        IBS_CUDA_TRY(cudaStreamWaitEvent(st, plan.join_ev, 0));
      }
      if (plan.n_split_tiles > 0)
        IBS_CUDA_TRY(launch_tc_finalize_batch_tiles(static_cast<const SubsetDev*>(plan.subsets.p),
                                                    static_cast<const int4*>(plan.split_tiles.p), plan.n_split_tiles,
                                                    st));
      return IBS_OK;
    }
    const int G = (int)plan.stage_ctas.size();
    auto gather = [&](int g, cudaStream_t s) {
      return launch_tc_gather(jobs, static_cast<const int4*>(plan.gather_map.p) + plan.stage_map_off[g],
                              plan.stage_ctas[g], fmt, ctx->status_dev, s);
    };
    IBS_CUDA_TRY(gather(0, st));
    if (G > 1) {
      // fork: the side stream runs the later stages' gathers
      IBS_CUDA_TRY(cudaEventRecord(plan.stage_ev[0], st));
      IBS_CUDA_TRY(cudaStreamWaitEvent(plan.side, plan.stage_ev[0], 0));
    }
    for (int g = 0; g < G; ++g) {
      if (g + 1 < G) {
        IBS_CUDA_TRY(gather(g + 1, plan.side));
        IBS_CUDA_TRY(cudaEventRecord(plan.stage_ev[g + 1], plan.side));
      }
      if (g > 0) IBS_CUDA_TRY(cudaStreamWaitEvent(st, plan.stage_ev[g], 0));  // joins the side stream
      if (plan.split_policy == 2) {
        // one launch per subset of the stage, over its own work list, on the
        // kernel ibs_compute would pick for its shape
        for (int64_t q = plan.stage_job_off[g]; q < plan.stage_job_off[g + 1]; ++q) {
          if (plan.q_pair_off[(size_t)q] >= 0) {
            PairBatchArgs a;
            a.subs = static_cast<const SubsetDev*>(plan.subsets.p);
            a.items = static_cast<const PairItem*>(plan.pitems.p) + plan.q_pair_off[(size_t)q];
            a.n_items = plan.q_pair_n[(size_t)q];
            a.jobs = jobs;
            a.units = static_cast<const int4*>(plan.units.p);
            a.n_units = 0;  // gathered by the stage's gather launch
            a.unit_counter = static_cast<int*>(plan.unit_counter.p);
            a.ready = static_cast<int*>(plan.ready.p);
            a.need = static_cast<const int*>(plan.need.p);  // all zero: nothing to wait for
            a.planes = plan.tc_planes.p;
            a.block_chunks = plan.tc_block_chunks;
            a.max_chunks = plan.q_chunks[(size_t)q];
            if (plan.q_pair_sync[(size_t)q] > 0) {
              const int2 ss = tc_pair_sync_setting(a.max_chunks);
              a.sync.seg = ss.x;
              a.sync.lag = ss.y;
              a.sync.n_seg = (int32_t)((a.max_chunks + ss.x - 1) / ss.x);
              a.sync.n_items = plan.q_pair_sync[(size_t)q];
              a.sync.ctr = static_cast<int*>(plan.pair_sync.p);
              IBS_CUDA_TRY(cudaMemsetAsync(plan.pair_sync.p, 0,
                                           (size_t)(a.sync.n_items / tc_pair_clusters(a.max_chunks)) * a.sync.n_seg *
                                               sizeof(int),
                                           st));
            }
            IBS_CUDA_TRY(launch_tc_pair_batch(a, ctx->status_dev, kWaitLimitNs, st));
            continue;
          }
          const int64_t n_items = plan.q_item_off[q + 1] - plan.q_item_off[q];
          IBS_CUDA_TRY(launch_tc_batch(static_cast<const SubsetDev*>(plan.subsets.p), items + plan.q_item_off[q],
                                       n_items, (int)std::min<int64_t>(plan.grid, n_items), fmt, plan.q_chunks[q],
                                       static_cast<int*>(plan.counter.p), ctx->status_dev, st));
        }
        continue;
      }
      const int64_t n_items = plan.stage_item_off[g + 1] - plan.stage_item_off[g];
      IBS_CUDA_TRY(launch_tc_batch(static_cast<const SubsetDev*>(plan.subsets.p), items + plan.stage_item_off[g],
                                   n_items, (int)std::min<int64_t>(plan.grid, n_items), fmt, plan.stage_max_chunks[g],
                                   static_cast<int*>(plan.counter.p), ctx->status_dev, st));
    }
    if (plan.split_policy == 2) {
      IBS_CUDA_TRY(launch_tc_finalize_batch_tiles(static_cast<const SubsetDev*>(plan.subsets.p),
                                                  static_cast<const int4*>(plan.split_tiles.p), plan.n_split_tiles,
                                                  st));
      return IBS_OK;
    }
  } else {
    IBS_CUDA_TRY(launch_planes_batch(static_cast<const PlaneJob*>(plan.jobs.p), n_subsets, plan.total_ctas,
                                     ctx->status_dev, st));
    IBS_CUDA_TRY(launch_batch(plan.mode, static_cast<const SubsetDev*>(plan.subsets.p),
                              static_cast<const WorkItem*>(plan.items.p), plan.n_items,
                              static_cast<int*>(plan.counter.p), ctx->status_dev, plan.grid, st));
  }
  if (plan.n_split > 0)
    IBS_CUDA_TRY(launch_finalize_batch(static_cast<const SubsetDev*>(plan.subsets.p),
                                       static_cast<const int32_t*>(plan.split_ids.p), plan.n_split,
                                       plan.max_split_pairs, st));
  return IBS_OK;
}

void plan_free(ibs_ctx* ctx, BatchPlan& plan) {
  if (plan.side) cudaStreamSynchronize(plan.side);
  for (auto& e : plan.stage_ev)
    if (e) cudaEventDestroy(e);
  plan.stage_ev.clear();
  if (plan.fork_ev) cudaEventDestroy(plan.fork_ev);
  if (plan.join_ev) cudaEventDestroy(plan.join_ev);
  plan.fork_ev = plan.join_ev = nullptr;
  if (plan.side) cudaStreamDestroy(plan.side);
  plan.side = nullptr;
  if (plan.exec) cudaGraphExecDestroy(plan.exec);
  if (plan.graph) cudaGraphDestroy(plan.graph);
  plan.exec = nullptr;
  plan.graph = nullptr;
  for (DevBuf* b : {&plan.planes, &plan.partial, &plan.subsets, &plan.jobs, &plan.items, &plan.split_ids,
                    &plan.counter, &plan.tc_planes, &plan.tc_jobs, &plan.split_tiles, &plan.gather_map, &plan.pitems,
                    &plan.units, &plan.unit_counter, &plan.ready, &plan.need, &plan.pair_sync})
    free_buf(ctx, *b);
}

void save_tune(const ibs_ctx* ctx) {
  if (ctx->tune_path.empty()) return;
  std::ofstream f(ctx->tune_path, std::ios::trunc);
  for (const auto& kv : ctx->tune)
    f << "{\"key\": \"" << kv.first << "\", \"mode\": " << kv.second.mode << ", \"split\": " << kv.second.split_policy
      << ", \"ms\": " << kv.second.ms << ", \"pair_min\": " << kv.second.pair_min << "}\n";
}

}  // namespace

extern "C" ibs_status ibs_compute_sz(ibs_ctx* ctx, const uint8_t* packed, size_t packed_bytes, int64_t n, int64_t m,
                                     int32_t* out_counts, size_t counts_bytes, double* out_dist, size_t dist_bytes,
                                     void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (n < 1 || n > 2147483647LL) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 2^31)", (long long)n);
  if (m < 1 || m > 2147483647LL) return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^31)", (long long)m);
  using u128 = unsigned __int128;
  const u128 need_packed = (u128)m * (u128)((n + 3) / 4);
  const u128 pairs = (ctx->flags & IBS_OUT_SQUARE) ? (u128)n * (u128)n : (u128)n * (u128)(n + 1) / 2;
  if ((u128)packed_bytes < need_packed)
    return fail(IBS_EINVAL, "packed holds %zu bytes, n_variants * ceil(n_samples/4) = %llu needed", packed_bytes,
                (unsigned long long)need_packed);
  if ((u128)counts_bytes < pairs * 16)
    return fail(IBS_EINVAL, "out_counts holds %zu bytes, %llu needed", counts_bytes,
                (unsigned long long)(pairs * 16));
  if (out_dist && !(ctx->flags & IBS_NO_DIST) && (u128)dist_bytes < pairs * 8)
    return fail(IBS_EINVAL, "out_dist holds %zu bytes, %llu needed", dist_bytes, (unsigned long long)(pairs * 8));
  return ibs_compute(ctx, packed, n, m, out_counts, out_dist, stream);
}

extern "C" ibs_status ibs_compute_batch(ibs_ctx* ctx, const uint8_t* pool, int64_t pool_n, int64_t pool_m,
                                        const ibs_subset* subs, int n_subsets, void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!pool || !subs || n_subsets < 1) return fail(IBS_EINVAL, "pool, subsets must be non-NULL and n_subsets >= 1");
  if (pool_n < 1 || pool_n > 2147483647LL || pool_m < 1 || pool_m > 2147483647LL)
    return fail(IBS_EINVAL, "pool size out of range");
  if (ctx->flags & IBS_OUT_SQUARE) return fail(IBS_EINVAL, "IBS_OUT_SQUARE is not supported by the batched path");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(pool)) return fail(IBS_EINVAL, "pool_packed must be device memory");
  std::vector<SubsetShape> shapes(n_subsets);
  std::vector<int64_t> key = {pool_n, pool_m, n_subsets};
  for (int i = 0; i < n_subsets; ++i) {
    const ibs_subset& s = subs[i];
    if (!s.sample_idx || !s.out_counts) return fail(IBS_EINVAL, "subset %d: NULL sample_idx or out_counts", i);
    if (s.n < 1 || s.n > pool_n) return fail(IBS_EINVAL, "subset %d: n=%lld out of range", i, (long long)s.n);
    if (s.var_len < 1 || s.var_begin < 0 || s.var_begin + s.var_len > pool_m)
      return fail(IBS_EINVAL, "subset %d: variant window out of range", i);
    if (reinterpret_cast<uintptr_t>(s.out_counts) % 16) return fail(IBS_EINVAL, "subset %d: out_counts not 16-byte aligned", i);
    if (s.out_dist && reinterpret_cast<uintptr_t>(s.out_dist) % 8) return fail(IBS_EINVAL, "subset %d: out_dist not 8-byte aligned", i);
    if (reinterpret_cast<uintptr_t>(s.sample_idx) % 8) return fail(IBS_EINVAL, "subset %d: sample_idx not 8-byte aligned", i);
    shapes[i].n = s.n;
    shapes[i].m = s.var_len;
    shapes[i].g = PlaneGeom::make(s.n, s.var_len);
    key.push_back(s.n);
    key.push_back(s.var_len);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Kernel family: the tensor-core form unless a POPC kernel is asked for (by
  // flag, or by the context's default); within POPC, a flag fixes the mode.
  const bool tc = use_tc(ctx);
  const int forced = tc                          ? kBatchModeTc + tc_format_for(ctx)
                     : (ctx->flags & kFlagPlain) ? 0
                     : (ctx->flags & kFlagCsa)   ? 1
                                                 : -1;
  key.push_back(forced);
  key.push_back(tc ? 1 : 0);

  auto it = ctx->plans.find(key);
  if (it == ctx->plans.end()) {
    // Choose mode and split policy: cached tuning result, or measure the candidates now.
    const std::string tk = tune_key(ctx, shapes) + (tc ? "_tc" : "");
    int mode = forced >= 0 ? forced : (tc ? kBatchModeTc : ctx->default_mode), policy = 0;
    int64_t pair_min = 1024;  // the two-SM size class of policies 2 and 5
    auto te = ctx->tune.find(tk);
    // Policy 3 (one launch of the two-SM kernel, gather fused in) needs E2M1
    // operands and clusters of two.
    int64_t max_nc = 0;
    for (const auto& sh : shapes) max_nc = std::max<int64_t>(max_nc, tc_chunks(sh.m, tc_format_for(ctx)));
    const bool pair_ok = tc && tc_format_for(ctx) == kTcFp4 && tc_pair_clusters(max_nc) > 0;
    // IBS_BATCH_POLICY=0..5 fixes the split policy (2: tensor-core modes; 3-5: two-SM E2M1 only)
    const char* pe = getenv("IBS_BATCH_POLICY");
    const int fixed_policy = pe && (atoi(pe) == 0 || atoi(pe) == 1 || (atoi(pe) == 2 && tc) ||
                                    ((atoi(pe) == 3 || atoi(pe) == 4 || atoi(pe) == 5) && pair_ok))
                                 ? atoi(pe)
                                 : -1;
    if (fixed_policy >= 0) {
      policy = fixed_policy;
    } else if (te != ctx->tune.end()) {
      if (forced < 0) mode = te->second.mode;
      policy = te->second.split_policy;
      pair_min = te->second.pair_min;
    } else if (!getenv("IBS_NO_AUTOTUNE")) {
      double best = 1e30;
      // candidates: (mode, policy, size class); policy 2 of the E2M1 mode is
      // also tried with the two-SM kernel from 2,048 or 4,096 chunks on, or
      // not at all (its default is ibs_compute's rule, 1,024 chunks)
      struct Cand {
        int mode, policy;
        int64_t pair_min;
      };
      std::vector<Cand> cands;
      for (int cm = 0; cm <= kBatchModeTc + kTcFp4; ++cm) {
        if (forced >= 0 && cm != forced) continue;
        if (is_tc_mode(cm) != tc) continue;
        const bool fp4_pair = pair_ok && tc_fmt_of(cm) == kTcFp4;
        for (int cp = 0; cp < (is_tc_mode(cm) ? (fp4_pair ? 6 : 3) : 2); ++cp) {
          cands.push_back({cm, cp, 1024});
          if (cp == 2 && fp4_pair && tc_pair_mode() == 0)
            for (int64_t pm : {(int64_t)2048, (int64_t)4096, (int64_t)1 << 40}) cands.push_back({cm, cp, pm});
        }
      }
      for (const Cand& c : cands) {
        const int cm = c.mode, cp = c.policy;
        {
          BatchPlan trial;
          if (ibs_status s = plan_build(ctx, trial, shapes, cm, cp, c.pair_min)) {
            plan_free(ctx, trial);
            return s;
          }
          ibs_status s = plan_upload(ctx, trial, pool, pool_n, subs, shapes, st);
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          if (!s) s = plan_enqueue(ctx, trial, n_subsets, st);  // warm-up
          cudaEventRecord(e0, st);
          if (!s) s = plan_enqueue(ctx, trial, n_subsets, st);
          cudaEventRecord(e1, st);
          cudaError_t ce = cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          plan_free(ctx, trial);
          if (s) return s;
          if (ce != cudaSuccess) return fail(IBS_ECUDA, "autotune run failed: %s", cudaGetErrorString(ce));
          if (ms < best) {
            best = ms;
            mode = cm;
            policy = cp;
            pair_min = c.pair_min;
          }
        }
      }
      TuneEntry t;
      t.mode = mode;
      t.split_policy = policy;
      t.pair_min = pair_min;
      t.ms = best;
      ctx->tune[tk] = t;
      save_tune(ctx);
    }
    auto plan = std::make_unique<BatchPlan>();
    plan->shape_key = key;
    if (ibs_status s = plan_build(ctx, *plan, shapes, mode, policy, pair_min)) {
      plan_free(ctx, *plan);
      return s;
    }
    // Capture the launch sequence once on a private stream.
    cudaStream_t cs;
    IBS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    ibs_status s = IBS_OK;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      s = plan_enqueue(ctx, *plan, n_subsets, cs);
      cudaGraph_t graph = nullptr;
      ce = cudaStreamEndCapture(cs, &graph);
      if (!s && ce == cudaSuccess) {
        plan->graph = graph;
        ce = cudaGraphInstantiate(&plan->exec, graph, 0);
      }
    }
    cudaStreamDestroy(cs);
    if (s || ce != cudaSuccess) {
      plan_free(ctx, *plan);
      if (s) return s;
      return fail(IBS_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    }
    it = ctx->plans.emplace(key, std::move(plan)).first;
  }
  BatchPlan& plan = *it->second;
  if (ibs_status s = plan_upload(ctx, plan, pool, pool_n, subs, shapes, st)) return s;
  IBS_CUDA_TRY(cudaGraphLaunch(plan.exec, st));
  int64_t own_gathers = 0;  // policy 5: subsets no two-SM launch gathered
  if (plan.split_policy == 5) {
    int64_t upto = 0;
    for (int64_t q = 0; q < (int64_t)plan.order.size(); ++q) {
      if (upto <= q) {
        ++own_gathers;
        upto = q + 1;
      }
      if (plan.q_pair_off[(size_t)q] >= 0) {
        int64_t r = q + 1;
        while (r < (int64_t)plan.order.size() && plan.q_pair_off[(size_t)r] < 0) ++r;
        upto = std::max<int64_t>(upto, std::min<int64_t>(r + 1, (int64_t)plan.order.size()));
      }
    }
  }
  ctx->last_info[0] = !is_tc_mode(plan.mode) ? 3 + (plan.n_split > 0 ? 1 : 0)
                      : plan.split_policy == 5 ? own_gathers + n_subsets + (plan.n_split_tiles > 0 ? 1 : 0)
                      : plan.split_policy >= 3 ? 2 + (plan.n_split_tiles > 0 ? 1 : 0)
                      : plan.split_policy == 2
                          ? (int64_t)plan.stage_ctas.size() + n_subsets + (plan.n_split_tiles > 0 ? 1 : 0)
                          : 2 * (int64_t)plan.stage_ctas.size() + (plan.n_split > 0 ? 1 : 0);
  ctx->last_info[1] = plan.tiles;
  ctx->last_info[2] = plan.split_policy;
  return IBS_OK;
}

extern "C" ibs_status ibs_cluster_complete(ibs_ctx* ctx, const double* dist, int64_t n, double* out_z,
                                           void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!dist || (!out_z && n > 1)) return fail(IBS_EINVAL, "dist and out_linkage must be non-NULL");
  if (n < 1 || n > ((int64_t)1 << 17)) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 131072]", (long long)n);
  if (reinterpret_cast<uintptr_t>(dist) % 8 || (out_z && reinterpret_cast<uintptr_t>(out_z) % 8))
    return fail(IBS_EINVAL, "dist and out_linkage must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(dist) || (out_z && !is_device_ptr(out_z)))
    return fail(IBS_EINVAL, "dist and out_linkage must be device memory");
  if (n == 1) return IBS_OK;
  if (ibs_status s = ensure_buf(ctx, ctx->cluster_work, cluster_workspace_bytes(n))) return s;
  IBS_CUDA_TRY(launch_cluster_complete(dist, n, out_z, ctx->cluster_work.p, ctx->num_sms,
                                       static_cast<cudaStream_t>(stream)));
  ctx->last_info[0] = 4;
  ctx->last_info[1] = n - 1;
  ctx->last_info[2] = 1;
  return IBS_OK;
}

extern "C" ibs_status ibs_ld_r(ibs_ctx* ctx, const uint8_t* packed, int64_t n, int64_t m, int64_t window,
                               double* out_r, int32_t* out_n, void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!packed || !out_r) return fail(IBS_EINVAL, "packed and out_r must be non-NULL");
  if (n < 1 || n >= ((int64_t)1 << 24)) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 2^24)", (long long)n);
  if (m < 1 || m > 2147483647LL) return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^31)", (long long)m);
  if (window < 1 || window > 2147483647LL / 2) return fail(IBS_EINVAL, "window %lld out of range", (long long)window);
  if (reinterpret_cast<uintptr_t>(out_r) % 8) return fail(IBS_EINVAL, "out_r must be 8-byte aligned");
  if (out_n && reinterpret_cast<uintptr_t>(out_n) % 4) return fail(IBS_EINVAL, "out_n must be 4-byte aligned");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(packed) || !is_device_ptr(out_r) || (out_n && !is_device_ptr(out_n)))
    return fail(IBS_EINVAL, "packed, out_r and out_n must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ibs_status s = ensure_buf(ctx, ctx->ld_planes, ld_planes_bytes(n, m))) return s;
  if (ibs_status s = ensure_buf(ctx, ctx->ld_diff, (size_t)m * sizeof(int32_t))) return s;
  if (ibs_status s = ensure_buf(ctx, ctx->ld_counter, 256)) return s;
  const std::vector<int64_t> key = {m, window};
  if (ctx->ld_key != key) {
    std::vector<int2> items;
    ld_items(m, window, items);
    if (ibs_status s = ensure_buf(ctx, ctx->ld_items, std::max<size_t>(1, items.size()) * sizeof(int2))) return s;
    if (!items.empty())  // pageable source: the copy is staged before return
      IBS_CUDA_TRY(cudaMemcpyAsync(ctx->ld_items.p, items.data(), items.size() * sizeof(int2),
                                   cudaMemcpyHostToDevice, st));
    ctx->ld_n_items = (int64_t)items.size();
    ctx->ld_key = key;
  }
  IBS_CUDA_TRY(launch_ld(packed, n, m, window, static_cast<uint8_t*>(ctx->ld_planes.p),
                         static_cast<int32_t*>(ctx->ld_diff.p), static_cast<const int2*>(ctx->ld_items.p),
                         ctx->ld_n_items, static_cast<int*>(ctx->ld_counter.p), out_r, out_n, ctx->status_dev,
                         ctx->num_sms, st));
  ctx->last_info[0] = ctx->ld_n_items > 0 ? 3 : 2;
  ctx->last_info[1] = ctx->ld_n_items;
  ctx->last_info[2] = 1;
  return IBS_OK;
}

extern "C" ibs_status ibs_grm(ibs_ctx* ctx, const uint8_t* packed, int64_t n, int64_t m, double* out_grm,
                              void* stream) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!packed || !out_grm) return fail(IBS_EINVAL, "packed and out_grm must be non-NULL");
  if (n < 1 || n > 65535LL * 128) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 8388480]", (long long)n);
  if (m < 1 || m >= ((int64_t)1 << 24))
    return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^24)", (long long)m);
  if (reinterpret_cast<uintptr_t>(out_grm) % 8) return fail(IBS_EINVAL, "out_grm must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(packed) || !is_device_ptr(out_grm))
    return fail(IBS_EINVAL, "packed and out_grm must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ibs_status s = ensure_buf(ctx, ctx->grm_work, grm_planes_bytes(n, m))) return s;
  if (ibs_status s = ensure_buf(ctx, ctx->grm_counter, 256)) return s;
  const std::vector<int64_t> key = {n, m};
  if (ctx->grm_key != key) {
    std::vector<GrmItem> items;
    std::vector<int4> splits;
    int64_t parts = 0;
    grm_items(n, m, ctx->num_sms, items, splits, parts);
    if (ibs_status s = ensure_buf(ctx, ctx->grm_items, items.size() * sizeof(GrmItem))) return s;
    if (ibs_status s = ensure_buf(ctx, ctx->grm_splits, std::max<size_t>(1, splits.size()) * sizeof(int4))) return s;
    if (ibs_status s = ensure_buf(ctx, ctx->grm_part, std::max<int64_t>(1, parts) * 128 * 128 * 12)) return s;
    // pageable sources: the copies are staged before return
    IBS_CUDA_TRY(cudaMemcpyAsync(ctx->grm_items.p, items.data(), items.size() * sizeof(GrmItem),
                                 cudaMemcpyHostToDevice, st));
    if (!splits.empty())
      IBS_CUDA_TRY(cudaMemcpyAsync(ctx->grm_splits.p, splits.data(), splits.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, st));
    ctx->grm_n_items = (int64_t)items.size();
    ctx->grm_n_splits = (int64_t)splits.size();
    ctx->grm_parts = parts;
    ctx->grm_key = key;
  }
  double* part_num = static_cast<double*>(ctx->grm_part.p);
  float* part_cnt = reinterpret_cast<float*>(part_num + std::max<int64_t>(1, ctx->grm_parts) * 128 * 128);
  IBS_CUDA_TRY(launch_grm(packed, n, m, out_grm, static_cast<uint8_t*>(ctx->grm_work.p),
                          static_cast<const GrmItem*>(ctx->grm_items.p), ctx->grm_n_items,
                          static_cast<const int4*>(ctx->grm_splits.p), ctx->grm_n_splits, part_num, part_cnt,
                          static_cast<int*>(ctx->grm_counter.p), ctx->status_dev, ctx->num_sms, st));
  ctx->last_info[0] = ctx->grm_n_splits > 0 ? 4 : 3;  // frequencies, operands, pairs (, finalisation)
  ctx->last_info[1] = ctx->grm_n_items;
  ctx->last_info[2] = 1;
  return IBS_OK;
}

extern "C" ibs_status ibs_test_set_wait_limit(ibs_ctx* ctx, int64_t ns) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (ns < 0 || (unsigned long long)ns > kWaitLimitNs)
    return fail(IBS_EINVAL, "wait limit %lld ns out of range [0, %llu]", (long long)ns, kWaitLimitNs);
  ctx->wait_ns = (unsigned long long)ns;
  return IBS_OK;
}

extern "C" ibs_status ibs_kernel_info(ibs_ctx* ctx, int64_t out[4]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  out[0] = use_tc(ctx) ? 2 : mode_for(ctx) == 0 ? 0 : 1;
  out[1] = tc_format_for(ctx);
  out[2] = ctx->num_sms;
  out[3] = ctx->device;
  return IBS_OK;
}

extern "C" ibs_status ibs_compute_kernel(ibs_ctx* ctx, int64_t n, int64_t m, int64_t* out) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  if (n < 1 || n > 2147483647LL) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 2^31)", (long long)n);
  if (m < 1 || m > 2147483647LL) return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^31)", (long long)m);
  DeviceGuard g(ctx->device);
  if (!use_tc(ctx)) {
    *out = mode_for(ctx) == 0 ? 0 : 1;
  } else if ((ctx->flags & IBS_OUT_SQUARE) || tc_tile_kernel_forced()) {
    *out = 4;
  } else {
    *out = tc_pair_usable(n, m, tc_format_for(ctx)) ? 3 : 2;
  }
  return IBS_OK;
}

extern "C" ibs_status ibs_batch_plan_info(ibs_ctx* ctx, int64_t out[5]) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  if (ctx->plans.empty()) return fail(IBS_ESTATE, "no batch plan yet");
  // the most recently created plan is not tracked separately; report the largest
  const BatchPlan* best = nullptr;
  for (const auto& kv : ctx->plans)
    if (!best || kv.second->n_items > best->n_items) best = kv.second.get();
  out[0] = best->mode;
  out[1] = best->split_policy;
  out[2] = best->n_items;
  out[3] = best->grid;
  out[4] = best->pair_min_chunks;
  return IBS_OK;
}

extern "C" ibs_status ibs_shutdown(ibs_ctx* ctx) {
  clear_error();
  if (!ctx) return IBS_OK;
  {
    DeviceGuard g(ctx->device);
    serve_stop(ctx);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->plans) plan_free(ctx, *kv.second);
    ctx->plans.clear();
    free_buf(ctx, ctx->planes);
    free_buf(ctx, ctx->partial);
    free_buf(ctx, ctx->tile_list);
    for (DevBuf* b : {&ctx->single_items, &ctx->single_split, &ctx->single_counter, &ctx->single_sync, &ctx->ld_planes, &ctx->ld_diff,
                      &ctx->ld_items, &ctx->ld_counter, &ctx->cluster_work, &ctx->grm_work,
                      &ctx->grm_items, &ctx->grm_splits, &ctx->grm_part, &ctx->grm_counter})
      free_buf(ctx, *b);
    for (auto* v : {&ctx->timing_used, &ctx->timing_free})
      for (auto& r : *v)
        for (auto& e : r.ev)
          if (e) cudaEventDestroy(e);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
  }
  delete ctx;
  return IBS_OK;
}

// Serving entry points forward to the engine (ibs_serve.cu).
extern "C" ibs_status ibs_panel_load(ibs_ctx* ctx, const uint8_t* panel, int64_t n_panel, int64_t m) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  return serve_panel_load(ctx, panel, n_panel, m);
}

extern "C" ibs_status ibs_query(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi,
                                double* od, uint64_t* id) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  return serve_query(ctx, q, nq, k, oc, oi, od, id);
}

extern "C" ibs_status ibs_query_sync(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi,
                                     double* od) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  return serve_query_sync(ctx, q, nq, k, oc, oi, od);
}

extern "C" ibs_status ibs_wait(ibs_ctx* ctx, uint64_t id, int64_t timeout_ms) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  return serve_wait(ctx, id, timeout_ms);
}

extern "C" ibs_status ibs_poll(ibs_ctx* ctx, uint64_t id) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  return serve_poll(ctx, id);
}

extern "C" ibs_status ibs_serve_stats_get(ibs_ctx* ctx, ibs_serve_stats* out) {
  clear_error();
  if (ibs_status s = check_ctx(ctx)) return s;
  if (!out) return fail(IBS_EINVAL, "out is NULL");
  return serve_stats(ctx, out);
}
