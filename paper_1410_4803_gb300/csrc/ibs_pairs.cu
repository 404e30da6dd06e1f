// Pair-count tile kernels: the hot loop of all-pairs IBS.
//
// Paper ("Improvements in PLINK 1.9 / Bitwise parallelism"): for every sample
// pair and every block of markers, XOR the packed genotypes, mask out markers
// with a missing call and count the set bits.  Here a CTA owns a 64 x 64 tile
// of sample pairs; its 256 threads each hold 4 x 4 pairs (rows ty + 16*i,
// columns tx + 16*j) with three int32 counters per pair in registers.  The
// marker axis is streamed in 384-marker chunks: one thread issues TMA bulk
// copies (cp.async.bulk, completion on an mbarrier) of the row block's and the
// column block's 12 KiB plane chunks into a 3-stage shared-memory ring, and
// every thread reads its 16-byte plane vectors from there.  Per pair and
// 32-marker word the update is 4 LOP3 + 3 POPC (+ adds), see ibs_device.cuh.
//
// Modes:
//   0  plain: one POPC per count per word.
//   1  carry-save: three words' masks per count are first reduced with a
//      full adder (XOR3 = sum bit, MAJ = carry bit, one LOP3 each), so three
//      words cost two POPCs instead of three: popc(a)+popc(b)+popc(c) =
//      popc(a^b^c) + 2*popc(maj(a,b,c)).  POPC issues at a quarter of the
//      LOP3 rate on this SM, so trading POPCs for LOP3s raises the ceiling.
//   2  carry-save as 1, compiled for one CTA per SM so the loop is not held to
//      128 registers (no spills, fewer warps to hide latency).
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// writes IBS_ETIMEOUT into the status word, waits (bounded) for its own
// copies still in flight and returns.
#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {

namespace {

constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr size_t kSmemBytes = (size_t)kStages * 2 * kChunkBytes + 64;

struct Acc {
  uint32_t n[4][4];
  uint32_t i0[4][4];
  uint32_t i1[4][4];
};

__device__ __forceinline__ uint4 lds128(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }

__device__ __forceinline__ void acc_zero(Acc& a) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a.n[i][j] = a.i0[i][j] = a.i1[i][j] = 0;
}

// Masks of one pair and one word: x = {V, P, Q, R} of the row sample, y of the column sample.
struct Masks {
  uint32_t v, b1, b0;
};
__device__ __forceinline__ Masks pair_masks(const uint4& x, const uint4& y) {
  Masks mk;
  mk.v = x.x & y.x;                                        // both calls present
  mk.b1 = lop3<kLutAndXor>(mk.v, x.y, y.y);                // present & exactly one het -> IBS1
  const uint32_t t = x.z & y.w;                            // Q_i & R_j
  mk.b0 = lop3<kLutAndOr>(x.w, y.z, t);                    // (R_i & Q_j) | (Q_i & R_j) -> IBS0
  return mk;
}

// Consume one chunk (kKC words) from shared memory.
template <int MODE>
__device__ __forceinline__ void consume_chunk(const uint32_t* __restrict__ srow, const uint32_t* __restrict__ scol,
                                              int tx, int ty, Acc& a) {
  if constexpr (MODE == 0) {
#pragma unroll 2
    for (int kw = 0; kw < kKC; ++kw) {
      uint4 R[4], C[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) R[i] = lds128(srow + (kw * kSB + ty + 16 * i) * kPlanes);
#pragma unroll
      for (int j = 0; j < 4; ++j) C[j] = lds128(scol + (kw * kSB + tx + 16 * j) * kPlanes);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const Masks mk = pair_masks(R[i], C[j]);
          a.n[i][j] += __popc(mk.v);
          a.i1[i][j] += __popc(mk.b1);
          a.i0[i][j] += __popc(mk.b0);
        }
    }
  } else {
    static_assert(kKC % 3 == 0, "carry-save mode needs a multiple of 3 words per chunk");
#pragma unroll 1
    for (int kw = 0; kw < kKC; kw += 3) {
      uint4 C[3][4];
#pragma unroll
      for (int w = 0; w < 3; ++w)
#pragma unroll
        for (int j = 0; j < 4; ++j) C[w][j] = lds128(scol + ((kw + w) * kSB + tx + 16 * j) * kPlanes);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint4 R[3];
#pragma unroll
        for (int w = 0; w < 3; ++w) R[w] = lds128(srow + ((kw + w) * kSB + ty + 16 * i) * kPlanes);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const Masks m0 = pair_masks(R[0], C[0][j]);
          const Masks m1 = pair_masks(R[1], C[1][j]);
          const Masks m2 = pair_masks(R[2], C[2][j]);
          const uint32_t sv = lop3<kLutXor3>(m0.v, m1.v, m2.v), cv = lop3<kLutMaj>(m0.v, m1.v, m2.v);
          const uint32_t s1 = lop3<kLutXor3>(m0.b1, m1.b1, m2.b1), c1 = lop3<kLutMaj>(m0.b1, m1.b1, m2.b1);
          const uint32_t s0 = lop3<kLutXor3>(m0.b0, m1.b0, m2.b0), c0 = lop3<kLutMaj>(m0.b0, m1.b0, m2.b0);
          a.n[i][j] += __popc(sv) + 2u * __popc(cv);
          a.i1[i][j] += __popc(s1) + 2u * __popc(c1);
          a.i0[i][j] += __popc(s0) + 2u * __popc(c0);
        }
      }
    }
  }
}

struct Pipe {
  uint32_t* stages;   // kStages x [2][kChunkWords]
  uint64_t* bars;     // kStages mbarriers
  uint32_t seq;       // chunks consumed so far by this CTA (all threads agree)
};

__device__ __forceinline__ void pipe_init(Pipe& p, uint8_t* smem) {
  p.stages = reinterpret_cast<uint32_t*>(smem);
  p.bars = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * 2 * kChunkBytes);
  p.seq = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&p.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
}

// Issue chunk c of the row and column blocks into stage s (one thread).
__device__ __forceinline__ void pipe_issue(Pipe& p, int s, const uint32_t* rowblk, const uint32_t* colblk,
                                           int64_t c) {
  uint32_t* dst = p.stages + (size_t)s * 2 * kChunkWords;
  const bool same = rowblk == colblk;
  mbar_arrive_expect_tx(&p.bars[s], same ? kChunkBytes : 2 * kChunkBytes);
  bulk_g2s(dst, rowblk + c * kChunkWords, kChunkBytes, &p.bars[s]);
  if (!same) bulk_g2s(dst + kChunkWords, colblk + c * kChunkWords, kChunkBytes, &p.bars[s]);
}

// Run the K loop of one tile over chunks [c0, c1).  Returns false (and stops
// the whole CTA consistently) if a copy did not complete within the limit.
template <int MODE>
__device__ bool run_tile(Pipe& p, const uint32_t* rowblk, const uint32_t* colblk, int64_t c0, int64_t c1, int tx,
                         int ty, Acc& a, int* status) {
  const int64_t nk = c1 - c0;
  const bool same = rowblk == colblk;
  if (threadIdx.x == 0) {
    for (int64_t k = 0; k < nk && k < kStages; ++k)
      pipe_issue(p, (int)((p.seq + k) % kStages), rowblk, colblk, c0 + k);
  }
  int64_t issued = nk < kStages ? nk : kStages;
  for (int64_t k = 0; k < nk; ++k) {
    const uint32_t g = p.seq + (uint32_t)k;
    const int s = (int)(g % kStages);
    const bool ok = mbar_wait_bounded(&p.bars[s], (g / kStages) & 1u);
    // This barrier also certifies that every thread has finished chunk k-1.
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(status, kDevTimeout);
        // Drain the copies this CTA still has in flight (bounded).
        for (int64_t r = k; r < issued; ++r) {
          const uint32_t gr = p.seq + (uint32_t)r;
          (void)mbar_wait_bounded(&p.bars[gr % kStages], (gr / kStages) & 1u);
        }
      }
      __syncthreads();
      return false;
    }
    if (k > 0 && k - 1 + kStages < nk) {
      if (threadIdx.x == 0) {
        const uint32_t gp = g - 1;
        pipe_issue(p, (int)(gp % kStages), rowblk, colblk, c0 + k - 1 + kStages);
      }
      ++issued;
    }
    const uint32_t* st = p.stages + (size_t)s * 2 * kChunkWords;
    consume_chunk<MODE>(st, same ? st : st + kChunkWords, tx, ty, a);
  }
  p.seq += (uint32_t)nk;
  __syncthreads();  // everyone done with the last stage before it is refilled
  return true;
}

// Epilogue: final counts (and distance) of one tile.
__device__ __forceinline__ void store_final(const Acc& a, int64_t I, int64_t J, int64_t n, int tx, int ty,
                                            int32_t* __restrict__ out_counts, double* __restrict__ out_dist,
                                            bool square) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = I * kSB + ty + 16 * i;
    if (gi >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = J * kSB + tx + 16 * j;
      if (gj >= n || gj < gi) continue;
      const int32_t nn = (int32_t)a.n[i][j], c0 = (int32_t)a.i0[i][j], c1 = (int32_t)a.i1[i][j];
      const int4 v = make_int4(c0, c1, nn - c0 - c1, nn);
      double d = 0.0;
      if (out_dist) d = ibs_dist(c0, c1, nn);
      if (!square) {
        const int64_t p = tri_index(gi, gj, n);
        reinterpret_cast<int4*>(out_counts)[p] = v;
        if (out_dist) out_dist[p] = d;
      } else {
        reinterpret_cast<int4*>(out_counts)[gi * n + gj] = v;
        if (out_dist) out_dist[gi * n + gj] = d;
        if (gi != gj) {
          reinterpret_cast<int4*>(out_counts)[gj * n + gi] = v;
          if (out_dist) out_dist[gj * n + gi] = d;
        }
      }
    }
  }
}

// Epilogue of a K-split tile: add the partial counts into the triangle workspace.
__device__ __forceinline__ void store_partial(const Acc& a, int64_t I, int64_t J, int64_t n, int tx, int ty,
                                              int32_t* __restrict__ partial) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = I * kSB + ty + 16 * i;
    if (gi >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = J * kSB + tx + 16 * j;
      if (gj >= n || gj < gi) continue;
      int32_t* o = partial + tri_index(gi, gj, n) * 4;
      atomicAdd(o + 0, (int)a.i0[i][j]);
      atomicAdd(o + 1, (int)a.i1[i][j]);
      atomicAdd(o + 3, (int)a.n[i][j]);
    }
  }
}

// Plain all-pairs: one CTA per (triangular tile, K split).
template <int MODE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    tri_kernel(const uint32_t* __restrict__ planes, int64_t n, int64_t n_blocks, int64_t n_chunks, int splits,
               int32_t* __restrict__ out_counts, double* __restrict__ out_dist, int32_t* __restrict__ partial,
               int square, int* status) {
  extern __shared__ __align__(128) uint8_t smem[];
  Pipe p;
  pipe_init(p, smem);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t t = blockIdx.x / splits;
  const int split = (int)(blockIdx.x % splits);
  int64_t I, J;
  tri_tile(t, n_blocks, I, J);
  const int64_t c0 = n_chunks * split / splits, c1 = n_chunks * (split + 1) / splits;
  const uint32_t* rowblk = planes + (size_t)I * n_chunks * kChunkWords;
  const uint32_t* colblk = planes + (size_t)J * n_chunks * kChunkWords;
  Acc a;
  acc_zero(a);
  if (!run_tile<MODE>(p, rowblk, colblk, c0, c1, tx, ty, a, status)) return;
  if (splits == 1) store_final(a, I, J, n, tx, ty, out_counts, out_dist, square != 0);
  else store_partial(a, I, J, n, tx, ty, partial);
}

// Batched: a persistent kernel pulling (subset, tile, K range) items.  The
// item and its subset descriptor are staged in shared memory so that none of
// their fields stays live in registers across the K loop.
template <int MODE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    batch_kernel(const SubsetDev* __restrict__ subsets, const WorkItem* __restrict__ items, int64_t n_items,
                 int* counter, int* status) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int64_t next_item;
  __shared__ WorkItem s_item;
  __shared__ SubsetDev s_sub;
  Pipe p;
  pipe_init(p, smem);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t it = atomicAdd(counter, 1);
      next_item = it;
      if (it < n_items) {
        s_item = items[it];
        s_sub = subsets[s_item.subset];
      }
    }
    __syncthreads();
    if (next_item >= n_items) break;
    const uint32_t* rowblk = s_sub.planes + (size_t)s_item.I * s_sub.n_chunks * kChunkWords;
    const uint32_t* colblk = s_sub.planes + (size_t)s_item.J * s_sub.n_chunks * kChunkWords;
    Acc a;
    acc_zero(a);
    if (!run_tile<MODE>(p, rowblk, colblk, s_item.c0, s_item.c1, tx, ty, a, status)) return;
    if (s_item.split) store_partial(a, s_item.I, s_item.J, s_sub.n, tx, ty, s_sub.partial);
    else store_final(a, s_item.I, s_item.J, s_sub.n, tx, ty, s_sub.out_counts, s_sub.out_dist, false);
    __syncthreads();  // everyone has read s_item / s_sub before thread 0 replaces them
  }
}

// Serving: query block x panel block items.  Row r of a query block writes
// its counts to row_out[r] ([n_panel][4] int32), so one block can carry the
// rows of several requests.
template <int MODE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    cross_kernel(const uint32_t* __restrict__ panel, int64_t n_panel, int64_t n_chunks,
                 const CrossItem* __restrict__ items, int64_t n_items, int* status) {
  extern __shared__ __align__(128) uint8_t smem[];
  Pipe p;
  pipe_init(p, smem);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const CrossItem w = items[it];
    const uint32_t* colblk = panel + (size_t)w.pb * n_chunks * kChunkWords;
    Acc a;
    acc_zero(a);
    if (!run_tile<MODE>(p, w.qplanes, colblk, 0, n_chunks, tx, ty, a, status)) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty + 16 * i;
      if (r >= w.q_rows) continue;
      int4* orow = reinterpret_cast<int4*>(w.row_out[r]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t gj = (int64_t)w.pb * kSB + tx + 16 * j;
        if (gj >= n_panel) continue;
        const int32_t nn = (int32_t)a.n[i][j], c0 = (int32_t)a.i0[i][j], c1 = (int32_t)a.i1[i][j];
        orow[gj] = make_int4(c0, c1, nn - c0 - c1, nn);
      }
    }
  }
}

// Serving: gather rows of several requests' bit planes into one dense block
// layout.  CTA = (chunk c, destination block b); thread = (word kw, slot s).
// Destination rows past n_rows get all-zero planes.
__global__ void __launch_bounds__(kKC * kSB)
    gather_rows_kernel(const RowSrc* __restrict__ rows, int64_t n_rows, int64_t n_chunks,
                       uint32_t* __restrict__ dst) {
  const int64_t c = blockIdx.x, b = blockIdx.y;
  const int kw = threadIdx.x / kSB, s = threadIdx.x % kSB;
  const int64_t d = b * kSB + s;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (d < n_rows) {
    const RowSrc src = rows[d];
    const int64_t sb = src.row / kSB, ss = src.row % kSB;
    v = *reinterpret_cast<const uint4*>(src.planes + (((sb * n_chunks + c) * kKC + kw) * kSB + ss) * kPlanes);
  }
  *reinterpret_cast<uint4*>(dst + (((b * n_chunks + c) * kKC + kw) * kSB + s) * kPlanes) = v;
}

// Split-K finalisation: triangle partials -> counts and distances.
__global__ void finalize_kernel(const int32_t* __restrict__ partial, int64_t n, int32_t* __restrict__ out_counts,
                                double* __restrict__ out_dist, int square) {
  const int64_t P = n * (n + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    // row i of pair p: largest i with tri_index(i, i, n) <= p
    const double b = 2.0 * (double)n + 1.0;
    int64_t i = (int64_t)((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    while (i > 0 && tri_index(i, i, n) > p) --i;
    while (i + 1 < n && tri_index(i + 1, i + 1, n) <= p) ++i;
    const int64_t j = i + (p - tri_index(i, i, n));
    const int4 q = reinterpret_cast<const int4*>(partial)[p];
    const int4 v = make_int4(q.x, q.y, q.w - q.x - q.y, q.w);
    double d = ibs_dist(q.x, q.y, q.w);
    if (!square) {
      reinterpret_cast<int4*>(out_counts)[p] = v;
      if (out_dist) out_dist[p] = d;
    } else {
      reinterpret_cast<int4*>(out_counts)[i * n + j] = v;
      if (out_dist) out_dist[i * n + j] = d;
      reinterpret_cast<int4*>(out_counts)[j * n + i] = v;
      if (out_dist) out_dist[j * n + i] = d;
    }
  }
}

// Batched split-K finalisation: blockIdx.y = index into the list of split subsets.
__global__ void finalize_batch_kernel(const SubsetDev* __restrict__ subsets, const int32_t* __restrict__ ids) {
  const SubsetDev sd = subsets[ids[blockIdx.y]];
  const int64_t n = sd.n;
  const int64_t P = n * (n + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int4 q = reinterpret_cast<const int4*>(sd.partial)[p];
    reinterpret_cast<int4*>(sd.out_counts)[p] = make_int4(q.x, q.y, q.w - q.x - q.y, q.w);
    if (sd.out_dist)
      sd.out_dist[p] = ibs_dist(q.x, q.y, q.w);
  }
}

template <typename K>
cudaError_t set_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

}  // namespace

size_t pair_kernel_smem_bytes() { return kSmemBytes; }

// Kernel variants: 0 = plain (2 CTAs/SM), 1 = carry-save (2 CTAs/SM, 128
// registers), 2 = carry-save with 1 CTA/SM (no register cap below 255).
int pair_kernel_ctas_per_sm(int mode) { return mode == 2 ? 1 : 2; }

int tri_splits_for(int64_t tiles, int64_t n_chunks, int num_sms) {
  const int64_t target = (int64_t)num_sms * 2 * 2;  // two waves of two CTAs per SM
  if (tiles >= target) return 1;
  int64_t s = (target + tiles - 1) / tiles;
  if (s > n_chunks) s = n_chunks;
  if (s > 64) s = 64;
  return s < 1 ? 1 : (int)s;
}

namespace {
template <int MODE, int MINB>
cudaError_t tri_launch(const uint32_t* planes, const PlaneGeom& g, int splits, int32_t* out_counts, double* out_dist,
                       int32_t* partial, bool square, int* status, int64_t grid, cudaStream_t st) {
  cudaError_t e = set_smem(tri_kernel<MODE, MINB>);
  if (e != cudaSuccess) return e;
  tri_kernel<MODE, MINB><<<(unsigned)grid, kThreads, kSmemBytes, st>>>(planes, g.n, g.n_blocks, g.n_chunks, splits,
                                                                       out_counts, out_dist, partial,
                                                                       square ? 1 : 0, status);
  return cudaGetLastError();
}
template <int MODE, int MINB>
cudaError_t batch_launch(const SubsetDev* subsets, const WorkItem* items, int64_t n_items, int* counter, int* status,
                         int grid, cudaStream_t st) {
  cudaError_t e = set_smem(batch_kernel<MODE, MINB>);
  if (e != cudaSuccess) return e;
  batch_kernel<MODE, MINB><<<grid, kThreads, kSmemBytes, st>>>(subsets, items, n_items, counter, status);
  return cudaGetLastError();
}
template <int MODE, int MINB>
cudaError_t cross_launch(const uint32_t* panel, int64_t n_panel, int64_t n_chunks, const CrossItem* items,
                         int64_t n_items, int* status, int64_t grid, cudaStream_t st) {
  cudaError_t e = set_smem(cross_kernel<MODE, MINB>);
  if (e != cudaSuccess) return e;
  cross_kernel<MODE, MINB><<<(unsigned)grid, kThreads, kSmemBytes, st>>>(panel, n_panel, n_chunks, items, n_items,
                                                                         status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tri(int mode, const uint32_t* planes, const PlaneGeom& g, int splits, int32_t* out_counts,
                       double* out_dist, int32_t* partial, bool square, int* status, int, cudaStream_t st) {
  const int64_t tiles = g.n_blocks * (g.n_blocks + 1) / 2;
  const int64_t grid = tiles * splits;
  if (grid > 2147483647LL) return cudaErrorInvalidValue;
  if (mode == 2) return tri_launch<1, 1>(planes, g, splits, out_counts, out_dist, partial, square, status, grid, st);
  if (mode == 1) return tri_launch<1, 2>(planes, g, splits, out_counts, out_dist, partial, square, status, grid, st);
  return tri_launch<0, 2>(planes, g, splits, out_counts, out_dist, partial, square, status, grid, st);
}

cudaError_t launch_finalize(const int32_t* partial, int64_t n, int32_t* out_counts, double* out_dist, bool square,
                            cudaStream_t st) {
  const int64_t P = n * (n + 1) / 2;
  int64_t blocks = (P + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  finalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, n, out_counts, out_dist, square ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_batch(int mode, const SubsetDev* subsets, const WorkItem* items, int64_t n_items, int* counter,
                         int* status, int grid, cudaStream_t st) {
  if (mode == 2) return batch_launch<1, 1>(subsets, items, n_items, counter, status, grid, st);
  if (mode == 1) return batch_launch<1, 2>(subsets, items, n_items, counter, status, grid, st);
  return batch_launch<0, 2>(subsets, items, n_items, counter, status, grid, st);
}

cudaError_t launch_finalize_batch(const SubsetDev* subsets, const int32_t* subset_ids, int n_split_subsets,
                                  int64_t max_pairs, cudaStream_t st) {
  if (n_split_subsets <= 0) return cudaSuccess;
  int64_t blocks = (max_pairs + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, (unsigned)n_split_subsets);
  finalize_batch_kernel<<<grid, 256, 0, st>>>(subsets, subset_ids);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const RowSrc* rows, int64_t n_rows, int64_t n_chunks, uint32_t* dst,
                               cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  const int64_t blocks = (n_rows + kSB - 1) / kSB;
  if (n_chunks > 2147483647LL || blocks > 65535) return cudaErrorInvalidValue;
  gather_rows_kernel<<<dim3((unsigned)n_chunks, (unsigned)blocks), kKC * kSB, 0, st>>>(rows, n_rows, n_chunks, dst);
  return cudaGetLastError();
}

cudaError_t launch_cross(int mode, const uint32_t* panel_planes, int64_t n_panel, int64_t, int64_t n_chunks,
                         const CrossItem* items, int64_t n_items, int* status, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (int64_t)sms * pair_kernel_ctas_per_sm(mode);
  if (grid > n_items) grid = n_items;
  if (mode == 2) return cross_launch<1, 1>(panel_planes, n_panel, n_chunks, items, n_items, status, grid, st);
  if (mode == 1) return cross_launch<1, 2>(panel_planes, n_panel, n_chunks, items, n_items, status, grid, st);
  return cross_launch<0, 2>(panel_planes, n_panel, n_chunks, items, n_items, status, grid, st);
}

}  // namespace ibs
