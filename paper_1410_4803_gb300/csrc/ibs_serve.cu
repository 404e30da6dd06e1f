// Serving engine: a resident reference panel and continuous batching of
// query requests.
//
// The panel's planes stay on the device: operand planes of the tensor-core
// form (128-sample blocks), or bit planes of the POPC kernels (64-sample
// blocks), whichever the context's pair kernel is.  A host thread owns a CUDA
// stream and runs steps.  A step packs the query rows of EVERY admitted
// request densely into query blocks (a gather kernel copies each row's planes,
// and every row keeps its own output pointer) and runs them against a range
// of panel blocks.  Each panel block is therefore read once per step
// however many requests are in flight, and the items of a step are ordered
// panel-block-major so the CTAs sharing a panel block run together and hit it
// in L2.  The step length adapts to the load: with few rows in flight one step
// covers the whole panel, with many it covers about 16 waves of tiles so that
// new requests can join between steps.  A request joins at the current panel
// position and is done once it has seen every panel block; then its top-k
// kernel runs and its outputs are copied back.  Admission is FIFO, bounded by
// a row-slot limit and by a memory budget (free device memory at panel load,
// and the context's workspace limit).  Request buffers come from the
// stream-ordered memory pool, so freeing them never synchronises the device.
// At most two steps are in flight, so admission and completion are handled
// between steps while the GPU stays busy.
//
// Tensor-core form: a step with two or more query blocks runs on the two-SM
// kernel (items of two query blocks x one panel block; the faster kernel for
// panels of at least 1,024 chunks), a step of one query block on the one-SM
// kernel.  The step length is rounded so that its last wave of items is as
// full as possible.  The dense query planes are gathered again only when the
// set of admitted requests changed.  Counts bound for host memory leave the
// device step by step on a second stream (the panel columns each step wrote),
// so those copies overlap the following steps instead of trailing them.  The
// top-k of all requests that finish in a step runs as one launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "ibs_ctx.h"
#include "ibs_device.cuh"

namespace ibs {

namespace {

constexpr int kMaxQuery = 4096;     // rows per request
constexpr int kMaxK = 64;           // top-k limit of the kernel
constexpr int64_t kMaxRows = 4096;  // query rows admitted at once (slot limit)
constexpr int64_t kStepWaves = 16;  // a step aims at this many waves of (query block, panel block) tiles
constexpr int64_t kStepWavesTc = 8; // ... of the tensor-core form (a request of one query block then takes
                                    // one step over a 100,000-sample panel; two steps cost it about 3 ms)
constexpr int64_t kMinStepDiv = 32; // ... and covers at least 1/32 of the panel
constexpr size_t kMemMargin = (size_t)1 << 30;
constexpr int64_t kTcBlock = 128;          // samples per tensor-core block
constexpr size_t kTcChunkBytes = 16384;    // one (block, chunk) of operand planes

enum class RState { Pending, Active, Finishing, Done };

struct Request {
  uint64_t id = 0;
  int64_t q = 0;
  int k = 0;
  int32_t* user_counts = nullptr;
  int32_t* user_idx = nullptr;
  double* user_dist = nullptr;
  bool counts_on_dev = false, topk_on_dev = false;
  std::vector<uint8_t> host_packed;
  DevBuf packed, planes, counts, tidx, tdist;
  size_t reserved = 0;
  int64_t blocks_done = 0;  // panel blocks processed since admission
  cudaEvent_t done_ev = nullptr;  // recorded on the engine's copy stream after the request's last output
  ibs_status status = IBS_OK;
  RState state = RState::Pending;
};

enum class PtrKind { Device, PinnedHost, Pageable };

PtrKind ptr_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PtrKind::Pageable;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return PtrKind::Device;
  if (a.type == cudaMemoryTypeHost) return PtrKind::PinnedHost;
  return PtrKind::Pageable;
}

}  // namespace

// Planes geometry in the units of the engine's pair kernel.
struct Geo {
  int64_t blocks, chunks;  // sample blocks, marker chunks
  size_t bytes;            // plane bytes
};

class ServeEngine {
 public:
  ibs_ctx* ctx;
  PlaneGeom pg;          // panel sizes (pg.n, pg.m) and, for POPC, the bit-plane geometry
  bool tc = false;       // tensor-core pair kernel (else POPC)
  int fmt = 0;           // tensor-core operand format
  int64_t blk = kSB;     // samples per block: 128 (tensor core) or 64 (POPC)
  Geo pgeo{};            // the panel's geometry
  DevBuf panel_planes, counter;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> active, finishing;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  std::atomic<uint64_t> next_id{1};
  ibs_serve_stats stats{};
  int64_t cursor = 0;  // first panel block of the next step
  int grid_ctas = 0;   // persistent cross-kernel CTAs (SMs x 2)
  bool pair = false;   // two-SM kernel for steps of two or more query blocks
  int clusters = 0;    // its clusters of two CTAs
  DevBuf sync_ctr;     // the two-SM kernel's K-lockstep counters of a step
  DevBuf topk_dev[2];  // row lists of a step's finishing requests (one top-k launch)
  TopkRow* topk_host[2] = {nullptr, nullptr};
  cudaStream_t side = nullptr;  // device -> host copies of finished columns and top-k lists
  cudaEvent_t kern_ev[2] = {nullptr, nullptr}, fin_ev[2] = {nullptr, nullptr};
  uint64_t set_version = 1, gathered_version = 0;  // the admitted set; the set the step planes hold
  size_t fixed_bytes = 0;  // panel planes + step buffers
  // double-buffered item arrays (one-SM CrossItem or two-SM PairItem)
  DevBuf items_dev[2];
  uint8_t* items_host[2] = {nullptr, nullptr};
  size_t items_cap = 0;
  cudaEvent_t step_ev[2] = {nullptr, nullptr};
  int64_t step_no = 0;
  DevBuf step_planes, rows_dev[2], outs_dev[2];
  std::mutex budget_mu;
  size_t pool_budget = 0;  // bytes the requests may hold together
  size_t pool_bytes = 0;   // bytes they hold now
  RowSrc* rows_host[2] = {nullptr, nullptr};
  int32_t** outs_host[2] = {nullptr, nullptr};

  explicit ServeEngine(ibs_ctx* c) : ctx(c) {}

  Geo geo(int64_t n) const {
    if (tc) return {(n + kTcBlock - 1) / kTcBlock, tc_chunks(pg.m, fmt), tc_planes_bytes(n, pg.m, fmt)};
    const PlaneGeom g = PlaneGeom::make(n, pg.m);
    return {g.n_blocks, g.n_chunks, g.bytes()};
  }
  size_t chunk_block_bytes() const { return tc ? (size_t)kTcChunkBytes : (size_t)kChunkBytes; }

  // Planes of n samples from a packed device matrix, on stream s.
  cudaError_t build_planes(const uint8_t* packed, int64_t n, void* planes, cudaStream_t s) const {
    if (tc) return launch_tc_planes(packed, n, pg.m, static_cast<uint8_t*>(planes), fmt, s);
    BedSource src;
    src.packed = packed;
    src.row_bytes = (n + 3) / 4;
    src.n_src = n;
    return launch_planes(src, n, pg.m, PlaneGeom::make(n, pg.m), static_cast<uint32_t*>(planes), ctx->status_dev,
                         s);
  }

  cudaError_t cross(const CrossItem* items, int64_t n_items, cudaStream_t s) const {
    if (tc)
      return launch_tc_cross(static_cast<const uint8_t*>(panel_planes.p), pg.n, pgeo.chunks, items, n_items,
                             (int)std::min<int64_t>(ctx->num_sms, std::max<int64_t>(1, n_items)), fmt,
                             static_cast<int*>(counter.p), ctx->status_dev, s);
    return launch_cross(pick_mode(ctx), static_cast<const uint32_t*>(panel_planes.p), pg.n, pg.n_blocks,
                        pg.n_chunks, items, n_items, ctx->status_dev, s);
  }

  size_t mem_need(int64_t q, int k, bool counts_dev, bool topk_dev) const {
    size_t b = (size_t)pg.m * (size_t)((q + 3) / 4) + geo(q).bytes;
    if (!counts_dev) b += (size_t)q * pg.n * 16;
    if (!topk_dev) b += (size_t)q * k * 12;
    return b + 4096;
  }

  // Per-request buffers come from the device's stream-ordered memory pool
  // (cudaMallocAsync / cudaFreeAsync on the stream that uses them): no
  // device-wide synchronisation when a request's memory is returned, so the
  // step pipeline never stalls on a free.
  void release(Request& r, cudaStream_t s) {
    for (DevBuf* b : {&r.packed, &r.planes, &r.counts, &r.tidx, &r.tdist}) {
      if (b->p) cudaFreeAsync(b->p, s);
      b->p = nullptr;
      b->cap = 0;
    }
    if (r.reserved) {
      release_bytes(ctx, r.reserved);
      std::lock_guard<std::mutex> lk(budget_mu);
      pool_bytes -= r.reserved;
    }
    r.reserved = 0;
    if (r.done_ev) cudaEventDestroy(r.done_ev);
    r.done_ev = nullptr;
  }

  ibs_status alloc(DevBuf& b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return IBS_OK;
    cudaError_t e = cudaMallocAsync(&b.p, bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return IBS_ENOMEM;
    }
    b.cap = bytes;
    return IBS_OK;
  }

  // Reserve a request's bytes against the serving budget (free device memory
  // at panel load minus a margin, and the context's workspace limit).
  bool reserve_request(Request& r, size_t need) {
    {
      std::lock_guard<std::mutex> lk(budget_mu);
      if (pool_bytes + need > pool_budget) return false;
      pool_bytes += need;
    }
    if (!reserve_bytes(ctx, need)) {
      std::lock_guard<std::mutex> lk(budget_mu);
      pool_bytes -= need;
      return false;
    }
    r.reserved = need;
    return true;
  }

  // Try to admit r (engine thread).  Returns false if it must wait.
  bool admit(const std::shared_ptr<Request>& r, int64_t active_rows) {
    if (active_rows + r->q > kMaxRows && active_rows > 0) return false;
    const size_t need = mem_need(r->q, r->k, r->counts_on_dev, r->topk_on_dev);
    if (!reserve_request(*r, need)) return false;
    const size_t pk = (size_t)pg.m * (size_t)((r->q + 3) / 4);
    if (alloc(r->packed, pk, stream) || alloc(r->planes, geo(r->q).bytes, stream) ||
        (!r->counts_on_dev && alloc(r->counts, (size_t)r->q * pg.n * 16, stream)) ||
        (!r->topk_on_dev && r->k > 0 &&
         (alloc(r->tidx, (size_t)r->q * r->k * 4, stream) || alloc(r->tdist, (size_t)r->q * r->k * 8, stream)))) {
      release(*r, stream);
      return false;
    }
    cudaMemcpyAsync(r->packed.p, r->host_packed.data(), pk, cudaMemcpyHostToDevice, stream);
    build_planes(static_cast<const uint8_t*>(r->packed.p), r->q, r->planes.p, stream);
    cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
    r->blocks_done = 0;
    r->state = RState::Active;
    return true;
  }

  int32_t* counts_ptr(Request& r) { return r.counts_on_dev ? r.user_counts : static_cast<int32_t*>(r.counts.p); }

  // The request's counts columns [b0, b1) panel blocks, written by the step
  // just enqueued, to its host buffer (on the copy stream, which waits for
  // the step's kernel).
  void copy_columns(Request& r, int64_t b0, int64_t b1) {
    const int64_t c0 = b0 * blk, c1 = std::min<int64_t>(b1 * blk, pg.n);
    if (c1 <= c0) return;
    const size_t pitch = (size_t)pg.n * 16;
    cudaMemcpy2DAsync(r.user_counts + c0 * 4, pitch, static_cast<const int32_t*>(r.counts.p) + c0 * 4, pitch,
                      (size_t)(c1 - c0) * 16, (size_t)r.q, cudaMemcpyDeviceToHost, side);
  }

  // Top-k of the requests that saw their last panel block in this step (on
  // the engine stream, after the step), then their top-k lists to the host
  // and their completion events on the copy stream (after their last counts
  // columns).
  void finish(const std::vector<std::shared_ptr<Request>>& done, int slot) {
    // every row of every finishing request in one launch (at most kMaxRows
    // rows: the admitted set never holds more)
    int64_t n = 0;
    for (auto& rp : done) {
      Request& r = *rp;
      if (r.k <= 0) continue;
      int32_t* oi = r.topk_on_dev ? r.user_idx : static_cast<int32_t*>(r.tidx.p);
      double* od = r.topk_on_dev ? r.user_dist : static_cast<double*>(r.tdist.p);
      const int32_t* cnt = counts_ptr(r);
      for (int64_t row = 0; row < r.q && n < kMaxRows; ++row, ++n)
        topk_host[slot][n] = TopkRow{cnt + (size_t)row * pg.n * 4, oi + row * r.k, od + row * r.k, r.k, 0};
    }
    if (n > 0) {
      cudaMemcpyAsync(topk_dev[slot].p, topk_host[slot], (size_t)n * sizeof(TopkRow), cudaMemcpyHostToDevice, stream);
      launch_topk_rows(static_cast<const TopkRow*>(topk_dev[slot].p), n, pg.n, stream);
    }
    if (!fin_ev[slot]) cudaEventCreateWithFlags(&fin_ev[slot], cudaEventDisableTiming);
    cudaEventRecord(fin_ev[slot], stream);
    cudaStreamWaitEvent(side, fin_ev[slot], 0);
    for (auto& rp : done) {
      Request& r = *rp;
      if (!r.topk_on_dev && r.k > 0) {
        cudaMemcpyAsync(r.user_idx, r.tidx.p, (size_t)r.q * r.k * 4, cudaMemcpyDeviceToHost, side);
        cudaMemcpyAsync(r.user_dist, r.tdist.p, (size_t)r.q * r.k * 8, cudaMemcpyDeviceToHost, side);
      }
      cudaEventRecord(r.done_ev, side);
      r.state = RState::Finishing;
    }
  }

  void ensure_items(size_t n) {
    if (n <= items_cap) return;
    const size_t each = std::max(sizeof(CrossItem), sizeof(PairItem));
    for (int s = 0; s < 2; ++s) {
      if (step_ev[s]) cudaEventSynchronize(step_ev[s]);
      if (items_dev[s].p) cudaFree(items_dev[s].p);
      if (items_host[s]) cudaFreeHost(items_host[s]);
      cudaMalloc(&items_dev[s].p, n * each);
      cudaHostAlloc(reinterpret_cast<void**>(&items_host[s]), n * each, cudaHostAllocDefault);
    }
    items_cap = n;
  }

  // K-lockstep of a two-SM launch of n_items equal items (whole waves of one
  // item per cluster take part); counters zeroed on stream s.  Off (an empty
  // PairSync) when the setting is off or the counters cannot be had.
  PairSync pair_sync(int64_t n_items, DevBuf& ctr, bool library_buf, cudaStream_t s) {
    PairSync ps;
    const int2 ss = tc_pair_sync_setting(pgeo.chunks);
    const int64_t waves = n_items / std::max(1, clusters);
    if (ss.x <= 0 || waves < 1) return ps;
    const int32_t n_seg = (int32_t)((pgeo.chunks + ss.x - 1) / ss.x);
    const size_t bytes = (size_t)waves * n_seg * sizeof(int);
    if (library_buf ? ensure_buf(ctx, ctr, bytes) != IBS_OK : alloc(ctr, bytes, s) != IBS_OK) return ps;
    if (cudaMemsetAsync(ctr.p, 0, bytes, s) != cudaSuccess) return ps;
    ps.ctr = static_cast<int*>(ctr.p);
    ps.seg = ss.x;
    ps.lag = ss.y;
    ps.n_seg = n_seg;
    ps.n_items = waves * clusters;
    return ps;
  }

  // Step length in panel blocks for `units` item rows (query blocks, or query
  // block pairs on the two-SM kernel) run by C persistent CTAs or clusters:
  // about kStepWaves(Tc) waves of items, at least 1/kMinStepDiv of the panel,
  // at most all of it; among the lengths up to one more wave, the one whose
  // last wave is fullest (the items of a step all cost the same), the
  // shortest of equals.
  int64_t step_len(int64_t units, int64_t C) const {
    units = std::max<int64_t>(1, units);
    C = std::max<int64_t>(1, C);
    int64_t lo = ((tc ? kStepWavesTc : kStepWaves) * C + units - 1) / units;
    lo = std::max<int64_t>(lo, (pgeo.blocks + kMinStepDiv - 1) / kMinStepDiv);
    lo = std::min<int64_t>(lo, pgeo.blocks);
    const int64_t hi = std::min<int64_t>(pgeo.blocks, lo + (C + units - 1) / units);
    int64_t best = lo;
    double best_fill = 0.0;
    for (int64_t L = lo; L <= hi; ++L) {
      const int64_t n = units * L;
      const double fill = (double)n / (double)(((n + C - 1) / C) * C);
      if (fill > best_fill + 1e-3) {
        best_fill = fill;
        best = L;
      }
    }
    return best;
  }

  // Step-level buffers: dense query planes for kMaxRows rows and the per-row
  // source / output tables (double-buffered host staging).
  ibs_status alloc_step_buffers() {
    if (ibs_status s = ensure_buf(ctx, step_planes, geo(kMaxRows).bytes)) return s;
    if (ibs_status s = ensure_buf(ctx, counter, 256)) return s;
    for (int s = 0; s < 2; ++s) {
      if (ibs_status e = ensure_buf(ctx, topk_dev[s], kMaxRows * sizeof(TopkRow))) return e;
      if (cudaHostAlloc(reinterpret_cast<void**>(&topk_host[s]), kMaxRows * sizeof(TopkRow), cudaHostAllocDefault) !=
          cudaSuccess)
        return fail(IBS_ENOMEM, "pinned top-k tables could not be allocated");
      if (ibs_status e = ensure_buf(ctx, rows_dev[s], kMaxRows * sizeof(RowSrc))) return e;
      if (ibs_status e = ensure_buf(ctx, outs_dev[s], kMaxRows * sizeof(int32_t*))) return e;
      if (cudaHostAlloc(reinterpret_cast<void**>(&rows_host[s]), kMaxRows * sizeof(RowSrc), cudaHostAllocDefault) !=
              cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&outs_host[s]), kMaxRows * sizeof(int32_t*), cudaHostAllocDefault) !=
              cudaSuccess)
        return fail(IBS_ENOMEM, "pinned step tables could not be allocated");
    }
    return IBS_OK;
  }

  // One step: every active request's rows, packed densely into query blocks,
  // against the current panel chunk.
  void run_step() {
    const int slot = (int)(step_no & 1);
    if (step_ev[slot]) cudaEventSynchronize(step_ev[slot]);  // slot's host tables are free again
    int64_t n_rows = 0;
    for (auto& r : active)
      for (int64_t row = 0; row < r->q; ++row) {
        rows_host[slot][n_rows].planes = static_cast<const uint32_t*>(r->planes.p);
        rows_host[slot][n_rows].row = row;
        outs_host[slot][n_rows] = counts_ptr(*r) + (size_t)row * pg.n * 4;
        ++n_rows;
      }
    const int64_t qblocks = (n_rows + blk - 1) / blk;
    // Step length: few rows in flight -> one step covers the whole panel (a
    // lone request costs one launch, as on the unbatched path); many rows ->
    // shorter steps that new requests can join between.
    const bool two_sm = pair && qblocks >= 2;
    const int64_t units = two_sm ? (qblocks + 1) / 2 : qblocks;
    const int64_t len = step_len(units, two_sm ? clusters : grid_ctas);
    const size_t n_items = (size_t)units * (size_t)len;
    ensure_items(std::max<size_t>(n_items, 1));
    size_t t = 0;
    int32_t** outs_d = static_cast<int32_t**>(outs_dev[slot].p);
    if (two_sm) {
      PairItem* h = reinterpret_cast<PairItem*>(items_host[slot]);
      for (int64_t k = 0; k < len; ++k) {
        const int64_t pb = (cursor + k) % pgeo.blocks;  // wraps around the panel
        for (int64_t u = 0; u < units; ++u) {
          PairItem& it = h[t++];
          it = PairItem{};
          it.I0 = (int32_t)(2 * u);
          it.I1 = 2 * u + 1 < qblocks ? (int32_t)(2 * u + 1) : -1;
          it.J = (int32_t)pb;
          it.c0 = 0;
          it.c1 = (int32_t)pgeo.chunks;
        }
      }
    } else {
      CrossItem* h = reinterpret_cast<CrossItem*>(items_host[slot]);
      const size_t qblock_bytes = (size_t)pgeo.chunks * chunk_block_bytes();
      for (int64_t k = 0; k < len; ++k) {
        const int64_t pb = (cursor + k) % pgeo.blocks;  // wraps around the panel
        for (int64_t b = 0; b < qblocks; ++b) {
          CrossItem& it = h[t++];
          it.qplanes =
              reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(step_planes.p) + b * qblock_bytes);
          it.row_out = outs_d + b * blk;
          it.q_rows = (int32_t)std::min<int64_t>(blk, n_rows - b * blk);
          it.pb = (int32_t)pb;
        }
      }
    }
    if (t > 0) {
      if (gathered_version != set_version) {
        // the admitted set changed: pack its rows into the step planes again
        cudaMemcpyAsync(rows_dev[slot].p, rows_host[slot], n_rows * sizeof(RowSrc), cudaMemcpyHostToDevice, stream);
        if (tc)
          launch_tc_gather_rows(static_cast<const RowSrc*>(rows_dev[slot].p), n_rows, pgeo.chunks,
                                static_cast<uint8_t*>(step_planes.p), stream);
        else
          launch_gather_rows(static_cast<const RowSrc*>(rows_dev[slot].p), n_rows, pg.n_chunks,
                             static_cast<uint32_t*>(step_planes.p), stream);
        gathered_version = set_version;
      }
      cudaMemcpyAsync(outs_dev[slot].p, outs_host[slot], n_rows * sizeof(int32_t*), cudaMemcpyHostToDevice, stream);
      if (two_sm) {
        cudaMemcpyAsync(items_dev[slot].p, items_host[slot], t * sizeof(PairItem), cudaMemcpyHostToDevice, stream);
        launch_tc_pair_cross(static_cast<const uint8_t*>(panel_planes.p), pg.n, pgeo.chunks,
                             static_cast<const uint8_t*>(step_planes.p), geo(kMaxRows).blocks, outs_d, n_rows,
                             static_cast<const PairItem*>(items_dev[slot].p), (int64_t)t, ctx->status_dev, stream,
                             pair_sync((int64_t)t, sync_ctr, true, stream));
      } else {
        cudaMemcpyAsync(items_dev[slot].p, items_host[slot], t * sizeof(CrossItem), cudaMemcpyHostToDevice, stream);
        cross(static_cast<const CrossItem*>(items_dev[slot].p), (int64_t)t, stream);
      }
      // this step's panel columns of requests whose counts go to host memory
      bool any_host = false;
      for (auto& r : active) any_host |= !r->counts_on_dev && r->user_counts;
      if (any_host) {
        if (!kern_ev[slot]) cudaEventCreateWithFlags(&kern_ev[slot], cudaEventDisableTiming);
        cudaEventRecord(kern_ev[slot], stream);
        cudaStreamWaitEvent(side, kern_ev[slot], 0);
        const int64_t b0 = cursor, b1 = cursor + len;  // may wrap once
        for (auto& r : active) {
          if (r->counts_on_dev || !r->user_counts) continue;
          copy_columns(*r, b0, std::min<int64_t>(b1, pgeo.blocks));
          if (b1 > pgeo.blocks) copy_columns(*r, 0, b1 - pgeo.blocks);
        }
      }
    }
    cursor = (cursor + len) % pgeo.blocks;
    std::vector<std::shared_ptr<Request>> still, done;
    for (auto& r : active) {
      // A request joined at some cursor position and is done once it has seen
      // every panel block (blocks seen twice near the end are rewritten with
      // the same counts).
      r->blocks_done += len;
      if (r->blocks_done >= pgeo.blocks) {
        done.push_back(r);
        finishing.push_back(r);
      } else {
        still.push_back(r);
      }
    }
    if (!done.empty()) {
      finish(done, slot);
      ++set_version;
    }
    active.swap(still);
    if (!step_ev[slot]) cudaEventCreateWithFlags(&step_ev[slot], cudaEventDisableTiming);
    cudaEventRecord(step_ev[slot], stream);
    ++step_no;
    std::lock_guard<std::mutex> lk(mu);
    stats.steps++;
  }

  void check_finishing() {
    std::vector<std::shared_ptr<Request>> still;
    bool any = false;
    for (auto& r : finishing) {
      if (cudaEventQuery(r->done_ev) == cudaSuccess) {
        const int st = __atomic_load_n(ctx->status_host, __ATOMIC_SEQ_CST);
        std::lock_guard<std::mutex> lk(mu);
        r->status = st == kDevTimeout ? IBS_ETIMEOUT : IBS_OK;
        release(*r, stream);
        r->state = RState::Done;
        stats.requests_done++;
        any = true;
      } else {
        still.push_back(r);
      }
    }
    finishing.swap(still);
    if (any) cv_done.notify_all();
  }

  void loop() {
    cudaSetDevice(ctx->device);
    for (;;) {
      check_finishing();
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
        int64_t rows = 0;
        for (auto& r : active) rows += r->q;
        while (!pending.empty()) {
          auto r = pending.front();
          lk.unlock();
          const bool ok = admit(r, rows);
          lk.lock();
          if (!ok) break;
          pending.pop_front();
          active.push_back(r);
          ++set_version;
          rows += r->q;
          stats.peak_rows = std::max<uint64_t>(stats.peak_rows, (uint64_t)rows);
        }
        if (active.empty()) {
          if (finishing.empty())
            cv_work.wait(lk, [&] { return stop || !pending.empty(); });
          else
            cv_work.wait_for(lk, std::chrono::microseconds(200));
          continue;
        }
      }
      run_step();
    }
  }

  void start() { worker = std::thread([this] { loop(); }); }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (worker.joinable()) worker.join();
    cudaStreamSynchronize(stream);
    if (side) cudaStreamSynchronize(side);
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : all) {
      Request& r = *kv.second;
      if (r.state != RState::Done) {
        r.status = IBS_ECANCELLED;
        r.state = RState::Done;
      }
      release(r, stream);
    }
    pending.clear();
    active.clear();
    finishing.clear();
    cv_done.notify_all();
    for (int s = 0; s < 2; ++s) {
      if (items_dev[s].p) cudaFree(items_dev[s].p);
      if (items_host[s]) cudaFreeHost(items_host[s]);
      if (step_ev[s]) cudaEventDestroy(step_ev[s]);
      if (kern_ev[s]) cudaEventDestroy(kern_ev[s]);
      if (fin_ev[s]) cudaEventDestroy(fin_ev[s]);
      items_dev[s].p = nullptr;
      items_host[s] = nullptr;
      step_ev[s] = nullptr;
      kern_ev[s] = nullptr;
      fin_ev[s] = nullptr;
    }
    if (panel_planes.p) free_buf(ctx, panel_planes);
    free_buf(ctx, step_planes);
    free_buf(ctx, counter);
    free_buf(ctx, sync_ctr);
    for (int s = 0; s < 2; ++s) {
      free_buf(ctx, topk_dev[s]);
      if (topk_host[s]) cudaFreeHost(topk_host[s]);
      topk_host[s] = nullptr;
      free_buf(ctx, rows_dev[s]);
      free_buf(ctx, outs_dev[s]);
      if (rows_host[s]) cudaFreeHost(rows_host[s]);
      if (outs_host[s]) cudaFreeHost(outs_host[s]);
      rows_host[s] = nullptr;
      outs_host[s] = nullptr;
    }
    if (stream) cudaStreamDestroy(stream);
    if (side) cudaStreamDestroy(side);
    stream = nullptr;
    side = nullptr;
  }
};

std::shared_ptr<ServeEngine> engine_of(ibs_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return ctx->serve;
}

void serve_stop(ibs_ctx* ctx) {
  std::shared_ptr<ServeEngine> e;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    e.swap(ctx->serve);
  }
  // Waiters hold their own reference, so the engine outlives them.
  if (e) e->shutdown();
}

ibs_status serve_panel_load(ibs_ctx* ctx, const uint8_t* panel, int64_t n_panel, int64_t m) {
  if (!panel) return fail(IBS_EINVAL, "panel_packed is NULL");
  if (n_panel < 1 || n_panel > 2147483647LL || m < 1 || m > 2147483647LL)
    return fail(IBS_EINVAL, "panel size out of range");
  DeviceGuard g(ctx->device);
  serve_stop(ctx);
  auto eng = std::make_shared<ServeEngine>(ctx);
  eng->pg = PlaneGeom::make(n_panel, m);
  eng->fmt = ctx_tc_format(ctx);
  // The tensor-core form covers a panel's whole marker range in one
  // accumulation, exact up to 2^21 markers; longer panels are served by the
  // integer-pipe kernels.
  eng->tc = ctx_use_tc(ctx) && tc_chunks(m, eng->fmt) <= tc_max_chunks(eng->fmt);
  eng->blk = eng->tc ? kTcBlock : kSB;
  eng->pgeo = eng->geo(n_panel);
  IBS_CUDA_TRY(cudaStreamCreateWithFlags(&eng->stream, cudaStreamNonBlocking));
  if (cudaStreamCreateWithFlags(&eng->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(eng->stream);
    return fail(IBS_ECUDA, "copy stream could not be created");
  }
  if (ibs_status s = ensure_buf(ctx, eng->panel_planes, eng->pgeo.bytes)) {
    cudaStreamDestroy(eng->stream);
    cudaStreamDestroy(eng->side);
    return s;
  }
  const size_t bytes = (size_t)m * (size_t)((n_panel + 3) / 4);
  const uint8_t* src_dev = panel;
  void* tmp = nullptr;
  if (ptr_kind(panel) != PtrKind::Device) {
    cudaError_t e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) {
      free_buf(ctx, eng->panel_planes);
      cudaStreamDestroy(eng->stream);
      cudaStreamDestroy(eng->side);
      cudaGetLastError();
      return fail(IBS_ENOMEM, "panel staging cudaMalloc(%zu) failed", bytes);
    }
    IBS_CUDA_TRY(cudaMemcpyAsync(tmp, panel, bytes, cudaMemcpyHostToDevice, eng->stream));
    src_dev = static_cast<const uint8_t*>(tmp);
  }
  IBS_CUDA_TRY(eng->build_planes(src_dev, n_panel, eng->panel_planes.p, eng->stream));
  IBS_CUDA_TRY(cudaStreamSynchronize(eng->stream));
  if (tmp) cudaFree(tmp);
  if (ibs_status st = eng->alloc_step_buffers()) {
    eng->shutdown();
    return st;
  }
  eng->grid_ctas = eng->tc ? ctx->num_sms : ctx->num_sms * pair_kernel_ctas_per_sm(pick_mode(ctx));
  eng->pair = eng->tc && tc_pair_cross_usable(n_panel, eng->pgeo.chunks, eng->fmt);
  eng->clusters = eng->pair ? tc_pair_clusters(eng->pgeo.chunks) : 0;
  if (eng->clusters < 1) eng->pair = false;
  if (eng->pair) {
    // lockstep counters for the largest step (all 4,096 rows, every panel
    // block), so that a step never grows them while earlier steps run
    const int2 ss = tc_pair_sync_setting(eng->pgeo.chunks);
    const int64_t max_items = (eng->geo(kMaxRows).blocks + 1) / 2 * eng->pgeo.blocks;
    if (ss.x > 0) {
      const size_t bytes =
          (size_t)(max_items / eng->clusters + 1) * (size_t)((eng->pgeo.chunks + ss.x - 1) / ss.x) * sizeof(int);
      if (ibs_status st = ensure_buf(ctx, eng->sync_ctr, bytes)) {
        eng->shutdown();
        return st;
      }
    }
  }
  // Requests draw on the device's default stream-ordered pool; keep freed
  // blocks cached in it so steady-state serving does not go back to the driver.
  cudaMemPool_t mp;
  if (cudaDeviceGetDefaultMemPool(&mp, ctx->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    eng->pool_budget = free_b > kMemMargin ? free_b - kMemMargin : 0;
  }
  eng->fixed_bytes = eng->panel_planes.cap + eng->step_planes.cap + eng->counter.cap +
                     2 * (eng->rows_dev[0].cap + eng->outs_dev[0].cap);
  eng->start();
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->serve = std::move(eng);
  return IBS_OK;
}

namespace {

ibs_status validate_query(const std::shared_ptr<ServeEngine>& eng, const uint8_t* q, int64_t nq, int k, int32_t* oc,
                          int32_t* oi, double* od, bool& counts_dev, bool& topk_dev) {
  if (!eng) return fail(IBS_ESTATE, "no panel loaded (call ibs_panel_load first)");
  if (!q) return fail(IBS_EINVAL, "query_packed is NULL");
  if (nq < 1 || nq > kMaxQuery) return fail(IBS_EINVAL, "n_query %lld out of range [1, %d]", (long long)nq, kMaxQuery);
  if (k < 0 || k > kMaxK) return fail(IBS_EINVAL, "k=%d out of range [0, %d]", k, kMaxK);
  if (k > 0 && (!oi || !od)) return fail(IBS_EINVAL, "k > 0 needs out_topk_idx and out_topk_dist");
  if (oc && reinterpret_cast<uintptr_t>(oc) % 16) return fail(IBS_EINVAL, "out_counts must be 16-byte aligned");
  counts_dev = oc ? ptr_kind(oc) == PtrKind::Device : false;
  if (oc && !counts_dev && ptr_kind(oc) != PtrKind::PinnedHost)
    return fail(IBS_EINVAL, "out_counts must be device memory or pinned host memory");
  topk_dev = false;
  if (k > 0) {
    const PtrKind a = ptr_kind(oi), b = ptr_kind(od);
    if (a != b) return fail(IBS_EINVAL, "out_topk_idx and out_topk_dist must be the same kind of memory");
    if (a == PtrKind::Pageable) return fail(IBS_EINVAL, "top-k outputs must be device memory or pinned host memory");
    topk_dev = a == PtrKind::Device;
  }
  return IBS_OK;
}

std::vector<uint8_t> copy_query(const uint8_t* q, size_t bytes) {
  std::vector<uint8_t> v(bytes);
  if (ptr_kind(q) == PtrKind::Device) cudaMemcpy(v.data(), q, bytes, cudaMemcpyDeviceToHost);
  else std::memcpy(v.data(), q, bytes);
  return v;
}

}  // namespace

ibs_status serve_query(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi, double* od,
                       uint64_t* id) {
  if (!id) return fail(IBS_EINVAL, "req_id is NULL");
  DeviceGuard g(ctx->device);
  bool counts_dev = false, topk_dev = false;
  auto eng = engine_of(ctx);
  if (ibs_status s = validate_query(eng, q, nq, k, oc, oi, od, counts_dev, topk_dev)) return s;
  ServeEngine& e = *eng;
  const size_t need = e.mem_need(nq, k, counts_dev, topk_dev);
  // The engine's own buffers (panel planes, step tables) are always held, so a
  // request is refused at once when it could not fit even beside them alone.
  size_t avail = e.pool_budget;
  if (ctx->ws_limit) avail = std::min(avail, ctx->ws_limit > e.fixed_bytes ? ctx->ws_limit - e.fixed_bytes : 0);
  if (need > avail) {
    std::lock_guard<std::mutex> lk(e.mu);
    e.stats.rejected++;
    return fail(IBS_EBUSY, "request needs %zu bytes, more than the %zu bytes the serving budget leaves", need, avail);
  }
  auto r = std::make_shared<Request>();
  r->q = nq;
  r->k = k;
  r->user_counts = oc;
  r->user_idx = oi;
  r->user_dist = od;
  r->counts_on_dev = counts_dev;
  r->topk_on_dev = topk_dev;
  r->host_packed = copy_query(q, (size_t)e.pg.m * (size_t)((nq + 3) / 4));
  r->id = e.next_id.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(e.mu);
    if (e.stop) return fail(IBS_ECANCELLED, "engine is shutting down");
    e.all[r->id] = r;
    e.pending.push_back(r);
  }
  e.cv_work.notify_all();
  *id = r->id;
  return IBS_OK;
}

ibs_status serve_wait(ibs_ctx* ctx, uint64_t id, int64_t timeout_ms) {
  auto eng = engine_of(ctx);
  if (!eng) return fail(IBS_ESTATE, "no panel loaded");
  ServeEngine& e = *eng;
  std::unique_lock<std::mutex> lk(e.mu);
  auto it = e.all.find(id);
  if (it == e.all.end()) return fail(IBS_EINVAL, "unknown request id %llu", (unsigned long long)id);
  auto r = it->second;
  auto done = [&] { return r->state == RState::Done; };
  if (timeout_ms < 0) {
    e.cv_done.wait(lk, done);
  } else if (!e.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return fail(IBS_ETIMEOUT, "request %llu not done after %lld ms", (unsigned long long)id, (long long)timeout_ms);
  }
  e.all.erase(id);
  if (r->status != IBS_OK) return fail(r->status, "request %llu failed with status %d", (unsigned long long)id, r->status);
  return IBS_OK;
}

ibs_status serve_poll(ibs_ctx* ctx, uint64_t id) {
  auto eng = engine_of(ctx);
  if (!eng) return fail(IBS_ESTATE, "no panel loaded");
  ServeEngine& e = *eng;
  std::lock_guard<std::mutex> lk(e.mu);
  auto it = e.all.find(id);
  if (it == e.all.end()) return fail(IBS_EINVAL, "unknown request id");
  return it->second->state == RState::Done ? IBS_OK : IBS_EBUSY;
}

ibs_status serve_stats(ibs_ctx* ctx, ibs_serve_stats* out) {
  auto eng = engine_of(ctx);
  if (!eng) return fail(IBS_ESTATE, "no panel loaded");
  std::lock_guard<std::mutex> lk(eng->mu);
  *out = eng->stats;
  return IBS_OK;
}

// One request, one launch sequence, synchronous: the unbatched baseline.
ibs_status serve_query_sync(ibs_ctx* ctx, const uint8_t* q, int64_t nq, int k, int32_t* oc, int32_t* oi, double* od) {
  DeviceGuard g(ctx->device);
  bool counts_dev = false, topk_dev = false;
  auto eng = engine_of(ctx);
  if (ibs_status s = validate_query(eng, q, nq, k, oc, oi, od, counts_dev, topk_dev)) return s;
  ServeEngine& e = *eng;
  const PlaneGeom pg = e.pg;
  const Geo qg = e.geo(nq);
  const size_t pk = (size_t)pg.m * (size_t)((nq + 3) / 4);
  Request r;
  r.q = nq;
  r.k = k;
  ibs_status st = IBS_OK;
  cudaStream_t s;
  IBS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const size_t need = e.mem_need(nq, k, counts_dev, topk_dev);
  if (!e.reserve_request(r, need)) {
    cudaStreamDestroy(s);
    return fail(IBS_ENOMEM, "the serving memory budget is exhausted");
  }
  DevBuf counter;
  if (e.alloc(r.packed, pk, s) || e.alloc(r.planes, qg.bytes, s) || e.alloc(counter, 256, s) ||
      (!counts_dev && e.alloc(r.counts, (size_t)nq * pg.n * 16, s)) ||
      (!topk_dev && k > 0 && (e.alloc(r.tidx, (size_t)nq * k * 4, s) || e.alloc(r.tdist, (size_t)nq * k * 8, s)))) {
    if (counter.p) cudaFreeAsync(counter.p, s);
    e.release(r, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return fail(IBS_ENOMEM, "device allocation failed");
  }
  int32_t* cnt = counts_dev ? oc : static_cast<int32_t*>(r.counts.p);
  std::vector<int32_t*> outs((size_t)nq);
  for (int64_t row = 0; row < nq; ++row) outs[row] = cnt + (size_t)row * pg.n * 4;
  DevBuf outs_d;
  cudaError_t ce = cudaMallocAsync(&outs_d.p, outs.size() * sizeof(int32_t*), s);
  // the engine's kernel rule: two or more query blocks on the two-SM kernel
  const bool two_sm = e.pair && qg.blocks >= 2;
  std::vector<CrossItem> items;
  std::vector<PairItem> pitems;
  const size_t qblock_bytes = (size_t)qg.chunks * e.chunk_block_bytes();
  for (int64_t pb = 0; pb < e.pgeo.blocks; ++pb) {
    if (two_sm) {
      for (int64_t u = 0; 2 * u < qg.blocks; ++u) {
        PairItem it{};
        it.I0 = (int32_t)(2 * u);
        it.I1 = 2 * u + 1 < qg.blocks ? (int32_t)(2 * u + 1) : -1;
        it.J = (int32_t)pb;
        it.c1 = (int32_t)qg.chunks;
        pitems.push_back(it);
      }
      continue;
    }
    for (int64_t qb = 0; qb < qg.blocks; ++qb) {
      CrossItem it;
      it.qplanes = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(r.planes.p) + qb * qblock_bytes);
      it.row_out = static_cast<int32_t**>(outs_d.p) + qb * e.blk;
      it.q_rows = (int32_t)std::min<int64_t>(e.blk, nq - qb * e.blk);
      it.pb = (int32_t)pb;
      items.push_back(it);
    }
  }
  const size_t item_bytes = two_sm ? pitems.size() * sizeof(PairItem) : items.size() * sizeof(CrossItem);
  const void* item_src = two_sm ? static_cast<const void*>(pitems.data()) : static_cast<const void*>(items.data());
  DevBuf items_dev, sync_d;
  if (ce == cudaSuccess) ce = cudaMallocAsync(&items_dev.p, item_bytes, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(outs_d.p, outs.data(), outs.size() * sizeof(int32_t*), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) {
    if (ptr_kind(q) == PtrKind::Device) ce = cudaMemcpyAsync(r.packed.p, q, pk, cudaMemcpyDeviceToDevice, s);
    else ce = cudaMemcpyAsync(r.packed.p, q, pk, cudaMemcpyHostToDevice, s);
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(items_dev.p, item_src, item_bytes, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = e.build_planes(static_cast<const uint8_t*>(r.packed.p), nq, r.planes.p, s);
  if (ce == cudaSuccess) {
    if (two_sm)
      ce = launch_tc_pair_cross(static_cast<const uint8_t*>(e.panel_planes.p), pg.n, e.pgeo.chunks,
                                static_cast<const uint8_t*>(r.planes.p), qg.blocks,
                                static_cast<int32_t* const*>(outs_d.p), nq,
                                static_cast<const PairItem*>(items_dev.p), (int64_t)pitems.size(), ctx->status_dev, s,
                                e.pair_sync((int64_t)pitems.size(), sync_d, false, s));
    else if (e.tc)
      ce = launch_tc_cross(static_cast<const uint8_t*>(e.panel_planes.p), pg.n, e.pgeo.chunks,
                           static_cast<const CrossItem*>(items_dev.p), (int64_t)items.size(),
                           (int)std::min<int64_t>(ctx->num_sms, (int64_t)items.size()), e.fmt,
                           static_cast<int*>(counter.p), ctx->status_dev, s);
    else
      ce = e.cross(static_cast<const CrossItem*>(items_dev.p), (int64_t)items.size(), s);
  }
  if (ce == cudaSuccess && k > 0)
    ce = launch_topk(cnt, nq, pg.n, k, topk_dev ? oi : static_cast<int32_t*>(r.tidx.p),
                     topk_dev ? od : static_cast<double*>(r.tdist.p), s);
  if (ce == cudaSuccess && oc && !counts_dev)
    ce = cudaMemcpyAsync(oc, r.counts.p, (size_t)nq * pg.n * 16, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess && k > 0 && !topk_dev) {
    ce = cudaMemcpyAsync(oi, r.tidx.p, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(od, r.tdist.p, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, s);
  }
  if (items_dev.p) cudaFreeAsync(items_dev.p, s);
  if (sync_d.p) cudaFreeAsync(sync_d.p, s);
  if (outs_d.p) cudaFreeAsync(outs_d.p, s);
  if (counter.p) cudaFreeAsync(counter.p, s);
  e.release(r, s);
  cudaError_t se = cudaStreamSynchronize(s);
  if (ce == cudaSuccess) ce = se;
  cudaStreamDestroy(s);
  if (ce != cudaSuccess) st = fail(IBS_ECUDA, "query_sync failed: %s", cudaGetErrorString(ce));
  else if (__atomic_load_n(ctx->status_host, __ATOMIC_SEQ_CST) == kDevTimeout)
    st = fail(IBS_ETIMEOUT, "a bounded device wait timed out");
  return st;
}

}  // namespace ibs
