// Tensor-core form of the pair counts (tcgen05 indicator GEMMs).
//
// The per-marker rule of the paper ("Improvements in PLINK 1.9 / Bitwise
// parallelism") is bilinear in one-hot indicators of the genotype codes, so the
// counts of all pairs are matrix products over the marker axis.  With, per
// sample and marker,
//   V = 1 if the call is present          U = +1 homozygous, -1 heterozygous
//   Q = 1 if homozygous A2                R = 1 if homozygous A1
// (all 0 for a missing call):
//   N     = V V^T                  (both present)
//   UU^T  = IBS2 + IBS0 - IBS1     (hom-hom and het-het pairs +1, hom-het -1)
//   IBS0  = Q R^T + R Q^T          (opposite homozygotes)
// so IBS1 = (N - UU^T) / 2 and IBS2 = N - IBS0 - IBS1.  The values -1, 0, +1
// are exact in every float format used here, every product is exact, and every
// partial sum is an integer of magnitude at most the marker count of the
// accumulation; items are kept to at most 2^21 markers (longer tiles are split
// over K and their pieces added as integers), below 2^24, so FP32
// accumulation is exact.  Four 128 x 128 MMAs per marker chunk.
//
// Two operand formats share everything but the MMA kind and the packing:
//   FP8  E4M3, kind::f8f6f4, one byte per indicator, 32 markers per chunk;
//   FP4  E2M1, kind::mxf4 with block scale factors all 1.0 (UE8M0 127, held in
//        tensor memory), two indicators per byte, 64 markers per chunk.
// Either way one (128-sample block, chunk) is 4 planes x 4 KiB, each plane a
// 128-row x 32-byte tile in the tensor core's canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, the two core matrices of a row group
// 128 bytes apart (leading byte offset) and row groups 256 bytes apart (stride
// byte offset).  FP4 thus moves half the bytes per marker.
//
// A CTA computes one 128 x 128 tile of pairs: warp 0 streams chunks of the row
// and column blocks through a 4-stage shared-memory ring with TMA bulk copies,
// warp 1 issues the MMAs into three FP32 accumulators in tensor memory
// (columns 0, 128, 256) and frees each stage with tcgen05.commit, and after
// the last chunk all four warps read the accumulators back (tcgen05.ld),
// decode the counts and store them.  Warp 0 (copies) and warp 1 (MMAs) run
// their loops with all 32 lanes in step and one lane issuing, so no lane of
// theirs is parked in another wait.
//
// Every wait is bounded (2 s of %globaltimer); on expiry the status word is
// set, and the CTA still waits (bounded) for its MMAs and frees its tensor
// memory before returning.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda.h>

#include "ibs_tc_common.cuh"

namespace ibs {

namespace {

constexpr int kTPlanes = 4;                       // V, U, Q, R
constexpr int kTChunkBytes = kTPlanes * kTileBytes;  // 16 KiB per (block, chunk)
constexpr int kTThreads = 128;
constexpr int kTStages = 4;                       // ring depth (6 and 7 stages measured no faster)
constexpr size_t kTcSmem = (size_t)kTStages * 2 * kTChunkBytes + 1024;

// The four MMAs of one chunk: V V^T, U U^T, Q R^T + R Q^T.
template <int F>
__device__ __forceinline__ void chunk_mmas(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t acc) {
  const uint32_t sf = tmem + kSfCol;
  umma<F>(tmem + 0, umma_desc(a0 + 0 * kTileBytes), umma_desc(b0 + 0 * kTileBytes), acc, sf);    // V V^T
  umma<F>(tmem + 128, umma_desc(a0 + 1 * kTileBytes), umma_desc(b0 + 1 * kTileBytes), acc, sf);  // U U^T
  umma<F>(tmem + 256, umma_desc(a0 + 2 * kTileBytes), umma_desc(b0 + 3 * kTileBytes), acc, sf);  // Q R^T
  umma<F>(tmem + 256, umma_desc(a0 + 3 * kTileBytes), umma_desc(b0 + 2 * kTileBytes), 1u, sf);   // + R Q^T
}

// Store one row's 16 bytes of each plane at `base` (the row's place in the
// chunk's V plane).  FP8: vb..rb hold 16 markers (bits 0..15); FP4: 32.
template <int F>
__device__ __forceinline__ void store_plane_row(uint8_t* base, uint32_t vb, uint32_t pb, uint32_t qb, uint32_t rb) {
  uint32_t wv[4], wu[4], wq[4], wr[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if constexpr (F == kTcFp4) {
      const uint32_t sv = nib8(vb >> (8 * g)), sp = nib8(pb >> (8 * g));
      wv[g] = sv << 1;
      wu[g] = (sv << 1) | (sp << 3);  // heterozygous: sign bit -> -1
      wq[g] = nib8(qb >> (8 * g)) << 1;
      wr[g] = nib8(rb >> (8 * g)) << 1;
    } else {
      const uint32_t sv = spread4((vb >> (4 * g)) & 0xFu), sp = spread4((pb >> (4 * g)) & 0xFu);
      wv[g] = sv * kFp8One;
      wu[g] = sv * kFp8One | sp * 0x80u;  // heterozygous: sign bit -> -1
      wq[g] = spread4((qb >> (4 * g)) & 0xFu) * kFp8One;
      wr[g] = spread4((rb >> (4 * g)) & 0xFu) * kFp8One;
    }
  }
  *reinterpret_cast<uint4*>(base + 0 * kTileBytes) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  *reinterpret_cast<uint4*>(base + 1 * kTileBytes) = make_uint4(wu[0], wu[1], wu[2], wu[3]);
  *reinterpret_cast<uint4*>(base + 2 * kTileBytes) = make_uint4(wq[0], wq[1], wq[2], wq[3]);
  *reinterpret_cast<uint4*>(base + 3 * kTileBytes) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
}

// Transpose: packed .bed rows -> operand planes.  CTA = (chunk c, block b of
// 128 samples), 8 warps of 16 samples.  Lane t of a warp holds one 32-bit word
// of .bed row t of each 32-marker group of the chunk (its 16 samples' 2-bit
// codes); a 32 x 32 bit transpose by warp shuffles leaves lane 2k with the low
// code bits and lane 2k+1 with the high code bits of sample k at those 32
// markers.  One exchange with the neighbour lane then gives each lane both
// bits of its part of the row: FP8, lane 2k markers 0..15 and lane 2k+1
// markers 16..31; FP4 (two groups), lane 2k markers 0..31 and lane 2k+1
// markers 32..63.  Each lane writes 16 bytes of each of the sample's planes.
__device__ __forceinline__ uint32_t tc_transpose32(uint32_t x, int lane) {
  constexpr uint32_t kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int j = 16 >> r;
    const uint32_t m = kMask[r];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) == 0 ? ((x & m) | ((y & m) << j)) : ((x & ~m) | ((y & ~m) >> j));
  }
  return x;
}

template <int F>
__global__ void __launch_bounds__(256) tc_planes_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes,
                                                        int64_t n, int64_t m, uint8_t* __restrict__ planes,
                                                        int64_t n_chunks) {
  constexpr int kGroups = kMarkers<F> / 32;
  const int64_t c = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s0 = b * kTB + warp * 16;  // first sample of this warp
  const int64_t byte0 = s0 >> 2;           // 4 bytes = 16 samples
  const bool fast = row_bytes % 4 == 0 && (reinterpret_cast<uintptr_t>(packed) & 3) == 0 && byte0 + 4 <= row_bytes;
  uint32_t x[kGroups];
#pragma unroll
  for (int g = 0; g < kGroups; ++g) {
    const int64_t marker = c * kMarkers<F> + 32 * g + lane;
    uint32_t v = 0x55555555u;  // "missing" for every slot
    if (marker < m && s0 < n) {
      const uint8_t* row = packed + marker * row_bytes;
      if (fast) {
        v = __ldg(reinterpret_cast<const uint32_t*>(row + byte0));
      } else {
        v = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) v |= (uint32_t)(byte0 + q < row_bytes ? __ldg(row + byte0 + q) : 0x55u) << (8 * q);
      }
    }
    x[g] = tc_transpose32(v, lane);
  }
  const bool odd = (lane & 1) != 0;
  uint32_t h, l, mask;
  if constexpr (F == kTcFp4) {
    // even lanes hold L of both groups, odd lanes H: swap L1 against H0
    const uint32_t partner = __shfl_xor_sync(0xffffffffu, odd ? x[0] : x[kGroups - 1], 1);
    h = odd ? x[kGroups - 1] : partner;
    l = odd ? partner : x[0];
    mask = 0xFFFFFFFFu;
  } else {
    const uint32_t partner = __shfl_xor_sync(0xffffffffu, x[0], 1);
    const uint32_t H = odd ? x[0] : partner, L = odd ? partner : x[0];
    const int sh = odd ? 16 : 0;
    h = (H >> sh) & 0xFFFFu;
    l = (L >> sh) & 0xFFFFu;
    mask = 0xFFFFu;
  }
  const int r = warp * 16 + (lane >> 1);  // row inside the 128-sample block
  const bool valid = b * kTB + r < n;
  const uint32_t vb = valid ? (h | ~l) & mask : 0u;  // present
  const uint32_t pb = vb & h & ~l;                    // het
  const uint32_t qb = vb & h & l;                     // hom A2
  const uint32_t rb = vb & ~h & ~l;                   // hom A1
  store_plane_row<F>(planes + (size_t)(b * n_chunks + c) * kTChunkBytes + tile_off(r, odd ? 16 : 0), vb, pb, qb,
                     rb);
}

// ---------------------------------------------------------------------------
// Pair tile kernel.
template <int F>
__global__ void __launch_bounds__(kTThreads, 1)
    tc_tri_kernel(const uint8_t* __restrict__ planes, int64_t n, int64_t n_blocks, int64_t n_chunks, int splits,
                  int32_t* __restrict__ out_counts, double* __restrict__ out_dist, int32_t* __restrict__ partial,
                  int square, int* status, const int2* __restrict__ tile_list) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned ring (the dynamic base is only guaranteed 16-byte aligned)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;                                            // kTStages x [A 16 KiB | B 16 KiB]
  __shared__ __align__(8) uint64_t full[kTStages], empty[kTStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5;
  const int64_t t = blockIdx.x / splits;
  const int split = (int)(blockIdx.x % splits);
  int64_t I, J;
  if (tile_list != nullptr) {
    const int2 ij = tile_list[t];
    I = ij.x;
    J = ij.y;
  } else {
    tri_tile(t, n_blocks, I, J);
  }
  const int64_t c0 = n_chunks * split / splits, c1 = n_chunks * (split + 1) / splits;
  const int64_t nk = c1 - c0;
  const uint8_t* rowblk = planes + (size_t)I * n_chunks * kTChunkBytes;
  const uint8_t* colblk = planes + (size_t)J * n_chunks * kTChunkBytes;
  const bool same = I == J;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if constexpr (F == kTcFp4) {
    tmem_fill_unit_scales(tmem, warp);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  const int lane = threadIdx.x & 31;
  if (warp == 0) {
    // Producer warp: every lane waits for a free stage together (no lane of
    // this warp sits in another wait), lane 0 issues the bulk copies.
    int64_t issued = 0;
    for (int64_t k = 0; k < nk; ++k, issued = k) {
      const int s = (int)(k % kTStages);
      const bool ok = k < kTStages || mbar_wait_bounded(&empty[s], (uint32_t)((k / kTStages - 1) & 1));
      // decisions are made warp-wide so the lanes never split around __syncwarp
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          atomicExch(status, kDevTimeout);
          atomicExch(&abort_flag, 1);
        }
        break;
      }
      if (__any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0)) break;
      if (lane == 0) {
        uint8_t* dst = ring + (size_t)s * 2 * kTChunkBytes;
        mbar_arrive_expect_tx(&full[s], same ? kTChunkBytes : 2 * kTChunkBytes);
        bulk_g2s(dst, rowblk + (size_t)(c0 + k) * kTChunkBytes, kTChunkBytes, &full[s]);
        if (!same) bulk_g2s(dst + kTChunkBytes, colblk + (size_t)(c0 + k) * kTChunkBytes, kTChunkBytes, &full[s]);
      }
      __syncwarp();
    }
    // The copies complete on `full` whether or not the MMA warp consumed
    // them; after a stop, wait (bounded) for the last ring's worth of stages
    // before the CTA exits, since its shared memory is their destination.
    for (int64_t j = issued > kTStages ? issued - kTStages : 0; j < issued; ++j)
      if (__any_sync(0xffffffffu, !mbar_wait_bounded(&full[j % kTStages], (uint32_t)((j / kTStages) & 1)))) {
        if (lane == 0) atomicExch(status, kDevTimeout);
        break;
      }
  } else if (warp == 1) {
    // MMA warp: every lane waits for the stage's data, lane 0 issues the MMAs.
    for (int64_t k = 0; k < nk; ++k) {
      const int s = (int)(k % kTStages);
      const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / kTStages) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          atomicExch(status, kDevTimeout);
          atomicExch(&abort_flag, 1);
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        const uint32_t a0 = smem_addr(ring + (size_t)s * 2 * kTChunkBytes);
        const uint32_t b0 = same ? a0 : a0 + kTChunkBytes;
        chunk_mmas<F>(tmem, a0, b0, k > 0 ? 1u : 0u);
        umma_commit(&empty[s]);  // the stage is free once these MMAs have read it
      }
      __syncwarp();
    }
    if (lane == 0) umma_commit(&done);  // arrives when every MMA issued above has completed
    __syncwarp();
  }
  // Everyone waits for the accumulators.
  const bool ok = mbar_wait_bounded(&done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool good = ok && abort_flag == 0;
  if (!ok && threadIdx.x == 0) atomicExch(status, kDevTimeout);

  if (good) {
    // Warp w owns TMEM lanes 32w..32w+31 = tile rows.
    const int row = warp * 32 + (threadIdx.x & 31);
    const int64_t gi = I * kTB + row;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cg = 0; cg < kTB / 32; ++cg) {
      uint32_t vn[32], vu[32], v0[32];
      tmem_ld32(lane_base + 0 + cg * 32, vn);
      tmem_ld32(lane_base + 128 + cg * 32, vu);
      tmem_ld32(lane_base + 256 + cg * 32, v0);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (gi >= n) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t gj = J * kTB + cg * 32 + j;
        if (gj >= n || gj < gi) continue;
        const int32_t nn = __float2int_rn(__uint_as_float(vn[j]));
        const int32_t uu = __float2int_rn(__uint_as_float(vu[j]));
        const int32_t i0 = __float2int_rn(__uint_as_float(v0[j]));
        const int32_t i1 = (nn - uu) / 2;
        if (splits > 1) {
          int32_t* o = partial + tri_index(gi, gj, n) * 4;
          atomicAdd(o + 0, i0);
          atomicAdd(o + 1, i1);
          atomicAdd(o + 3, nn);
          continue;
        }
        const int4 v = make_int4(i0, i1, nn - i0 - i1, nn);
        double d = 0.0;
        if (out_dist) d = ibs_dist(i0, i1, nn);
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
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Batched form: gather-transpose from the pool.  CTA = (subset, 128-sample
// block, group of kGatherChunks chunks), thread r = sample r of the block.
// The job lookup and the sample's pool index are read once per CTA; then, per
// chunk, the thread reads its sample's code at each marker (one byte per
// marker row, all loads of a chunk independent; the lanes of a warp read
// neighbouring samples of the same row, so a sorted index list gives
// near-contiguous reads), builds the present / het / hom A2 / hom A1 masks
// over the chunk's markers and writes its rows of the four planes.  An index
// outside the pool is not read: the sample is treated as all-missing and the
// status word reports it.
constexpr int kGatherChunks = 8;

// One gather work unit: sample block b of job j over chunk group cg, thread
// r (0..127) = sample r of the block.  Used by the standalone gather kernel
// and, fused, by the two-SM kernel's epilogue warps.
template <int F>
__device__ __forceinline__ void gather_unit(const TcGatherJob& j, int64_t b, int64_t cg, int r, int* status) {
  constexpr int K = kMarkers<F>;
  const int64_t s = b * kTB + r;
  int64_t ps = -1;
  if (s < j.n) {
    ps = j.src.sel[s];
    if (ps < 0 || ps >= j.src.n_src) {
      atomicExch(status, 1);
      ps = -1;
    }
  }
  const int sh = ps >= 0 ? 2 * (int)(ps & 3) : 0;
  const int64_t row_bytes = j.src.row_bytes;
  const uint8_t* col = j.src.packed + j.src.var_begin * row_bytes + (ps >= 0 ? (ps >> 2) : 0);
  const int64_t c_end = (cg + 1) * kGatherChunks < j.nc ? (cg + 1) * kGatherChunks : j.nc;
  for (int64_t c = cg * kGatherChunks; c < c_end; ++c) {
    uint8_t* base = j.tc + (size_t)(b * j.nc + c) * kTChunkBytes;
    // 32 markers at a time: one 32-bit mask per plane, one K half (16 bytes)
    // of the FP4 row or the whole FP8 row
#pragma unroll 1
    for (int h = 0; h < K / 32; ++h) {
      const int64_t k0 = c * K + 32 * h;
      const int kn = (int)(j.m - k0 < 32 ? j.m - k0 : 32);  // markers of this group inside the window
      uint32_t H = 0, L = ~0u;                             // all missing unless read
      if (ps >= 0 && kn > 0) {
        const uint8_t* p = col + k0 * row_bytes;
        uint32_t byte[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) byte[k] = k < kn ? __ldg(p + (int64_t)k * row_bytes) : 0x55u;
        H = 0;
        L = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const uint32_t code = (byte[k] >> sh) & 3u;
          H |= (code >> 1) << k;
          L |= (code & 1u) << k;
        }
      }
      const uint32_t V = H | ~L, P = H & ~L, Q = H & L, R = ~H & ~L;
      if constexpr (F == kTcFp4) {
        store_plane_row<F>(base + tile_off(r, 16 * h), V, P, Q, R);
      } else {
        store_plane_row<F>(base + tile_off(r, 0), V & 0xFFFFu, P & 0xFFFFu, Q & 0xFFFFu, R & 0xFFFFu);
        store_plane_row<F>(base + tile_off(r, 16), V >> 16, P >> 16, Q >> 16, R >> 16);
      }
    }
  }
}

// Gather units claimed from a shared list (the batched pair launch's units,
// also claimed by its epilogue warps): each CTA takes units until none are
// left and counts every finished unit in ready[subset].  At most 64 registers
// a thread (launch bound), so that two of these CTAs fit on an SM beside a
// pair CTA and the two kernels overlap.
template <int F>
__global__ void __launch_bounds__(kTB, 8)
    tc_gather_units_kernel(const TcGatherJob* __restrict__ jobs, const int4* __restrict__ units, int64_t n_units,
                           int* unit_counter, int* ready, int* status) {
  __shared__ int64_t s_u;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t u = atomicAdd(unit_counter, 1);
      s_u = u < n_units ? u : -1;
    }
    __syncthreads();
    const int64_t u = s_u;
    __syncthreads();  // everyone has read s_u
    if (u < 0) return;
    const int4 un = units[u];  // {job, sample block, chunk group, subset}
    gather_unit<F>(jobs[un.x], un.y, un.z, threadIdx.x, status);
    asm volatile("fence.proxy.async.global;" ::: "memory");  // plain stores, read later by TMA
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(ready + un.w, 1);
    }
  }
}

// CTA blockIdx.x takes the (job, sample block, chunk group) of map[blockIdx.x]:
// the host orders a stage's CTAs by the pool variant they start at, so that
// subsets whose windows overlap read the same pool rows at about the same
// time and share them through L2.
template <int F>
__global__ void __launch_bounds__(kTB) tc_gather_kernel(const TcGatherJob* __restrict__ jobs,
                                                        const int4* __restrict__ map, int* status) {
  const int4 e = map[blockIdx.x];  // {job, sample block, chunk group, -}
  gather_unit<F>(jobs[e.x], e.y, e.z, threadIdx.x, status);
}

// ---------------------------------------------------------------------------
// Persistent tensor-core launches (batched subsets, serving steps).  A work
// policy W maps an item index to the tile it computes (tile(): operand
// blocks and K range, read by the copy and MMA warps) and to the stores of
// its counts (epi(): per-row state; store(): 32 accumulator columns).

// One tile of a persistent launch: the operand blocks it multiplies and its
// K range in chunks.
struct TcTile {
  const uint8_t* a;  // row block, chunk 0
  const uint8_t* b;  // column block, chunk 0
  int64_t c0, c1;
  bool same;         // a == b: one copy per chunk serves both operands
};

// Decoded counts of one pair from the three accumulators.
struct PairCounts {
  int32_t i0, i1, n;
};
__device__ __forceinline__ PairCounts decode(uint32_t vn, uint32_t vu, uint32_t v0) {
  const int32_t nn = __float2int_rn(__uint_as_float(vn));
  const int32_t uu = __float2int_rn(__uint_as_float(vu));
  return {__float2int_rn(__uint_as_float(v0)), (nn - uu) / 2, nn};
}

// (subset, tile, K range) items; upper-triangle outputs (or partial counts
// when the tile is split over K).
struct TriEpi {
  int64_t gi, j0, n;
  int32_t* counts;
  double* dist;
  int32_t* partial;
  bool split;
  // Counts of accumulator columns 32*cg .. 32*cg+31 (run while the
  // accumulators are read back).
  __device__ void store(int cg, const uint32_t (&vn)[32], const uint32_t (&vu)[32], const uint32_t (&v0)[32]) const {
    if (gi >= n) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t gj = j0 + cg * 32 + j;
      if (gj >= n || gj < gi) continue;
      const PairCounts c = decode(vn[j], vu[j], v0[j]);
      const int64_t p = tri_index(gi, gj, n);
      if (split) {
        int32_t* o = partial + p * 4;
        atomicAdd(o + 0, c.i0);
        atomicAdd(o + 1, c.i1);
        atomicAdd(o + 3, c.n);
        continue;
      }
      reinterpret_cast<int4*>(counts)[p] = make_int4(c.i0, c.i1, c.n - c.i0 - c.i1, c.n);
    }
  }
  // Distances of the row, after the accumulators are handed back (so the
  // FP64 work overlaps the next item's MMAs): each thread reads back the
  // counts it stored itself.
  // The row's pairs are consecutive in the triangle, so the reads are batched
  // 16 at a time: the loop is bound by the FP64 rate, not by one L2 round
  // trip per pair.
  __device__ void finish() const {
    if (gi >= n || split || !dist) return;
    const int64_t j1 = j0 + kTB < n ? j0 + kTB : n;
    const int64_t jb = gi > j0 ? gi : j0;
    const int64_t p0 = tri_index(gi, jb, n), len = j1 - jb;
    const int4* cnt = reinterpret_cast<const int4*>(counts) + p0;
    double* dst = dist + p0;
    for (int64_t u0 = 0; u0 < len; u0 += 16) {
      int4 c[16];
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (u0 + u < len) c[u] = cnt[u0 + u];
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (u0 + u < len) dst[u0 + u] = ibs_dist(c[u].x, c[u].y, c[u].w);
    }
  }
};
__device__ __forceinline__ TcTile tri_tile_of(const WorkItem& w, const SubsetDev& sd) {
  const uint8_t* pl = reinterpret_cast<const uint8_t*>(sd.planes);
  return {pl + (size_t)w.I * sd.n_chunks * kTChunkBytes, pl + (size_t)w.J * sd.n_chunks * kTChunkBytes, w.c0, w.c1,
          w.I == w.J};
}
__device__ __forceinline__ TriEpi tri_epi_of(const WorkItem& w, const SubsetDev& sd, int row) {
  return {(int64_t)w.I * kTB + row, (int64_t)w.J * kTB, sd.n, sd.out_counts, sd.out_dist, sd.partial, w.split != 0};
}

// Batched subsets: the subset of an item is looked up per item.
struct BatchWork {
  const SubsetDev* subs;
  const WorkItem* items;
  using Epi = TriEpi;
  __device__ TcTile tile(int64_t it) const {
    const WorkItem w = items[it];
    return tri_tile_of(w, subs[w.subset]);
  }
  __device__ Epi epi(int64_t it, int row) const {
    const WorkItem w = items[it];
    return tri_epi_of(w, subs[w.subset], row);
  }
};

// One matrix (ibs_compute): the subset travels in the kernel parameters.
struct SingleWork {
  SubsetDev sd;
  const WorkItem* items;
  using Epi = TriEpi;
  __device__ TcTile tile(int64_t it) const { return tri_tile_of(items[it], sd); }
  __device__ Epi epi(int64_t it, int row) const { return tri_epi_of(items[it], sd, row); }
};

// Serving: (128-row query block, 128-sample panel block) items over the
// whole marker range; row r of the block writes counts [n_panel][4] through
// its own output pointer.
struct CrossWork {
  const CrossItem* items;
  const uint8_t* panel;
  int64_t n_panel, n_chunks;
  __device__ TcTile tile(int64_t it) const {
    const CrossItem ci = items[it];
    return {reinterpret_cast<const uint8_t*>(ci.qplanes), panel + (size_t)ci.pb * n_chunks * kTChunkBytes, 0,
            n_chunks, false};
  }
  struct Epi {
    int32_t* out;
    int64_t j0, n;
    __device__ void store(int cg, const uint32_t (&vn)[32], const uint32_t (&vu)[32],
                          const uint32_t (&v0)[32]) const {
      if (!out) return;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t gj = j0 + cg * 32 + j;
        if (gj >= n) continue;
        const PairCounts c = decode(vn[j], vu[j], v0[j]);
        reinterpret_cast<int4*>(out)[gj] = make_int4(c.i0, c.i1, c.n - c.i0 - c.i1, c.n);
      }
    }
    __device__ void finish() const {}
  };
  __device__ Epi epi(int64_t it, int row) const {
    const CrossItem ci = items[it];
    return {row < ci.q_rows ? ci.row_out[row] : nullptr, (int64_t)ci.pb * kTB, n_panel};
  }
};

// The persistent kernel: 8 warps.  Warp 0 claims work items from a global
// counter (list order, so the CTAs running at one time work on neighbouring
// tiles and share their operand blocks through L2) and streams each item's
// chunks through the ring; warps 1..kMmaWarps issue the MMAs, warp 1 + j
// taking the ring stages g with g % kMmaWarps == j; warps 4..7 read the
// accumulators back (warp w reads TMEM lanes 32*(w-4)..), zero them and store
// the counts.  Claimed item indices reach the MMA and epilogue warps through
// a small shared-memory queue (qfull / qempty, -1 ends the stream).  Two
// barriers hand the accumulators over per item: tfull (every MMA warp has
// committed the item's MMAs) and tempty (the epilogue has read and zeroed
// them), so the producer keeps prefetching the next item's chunks while the
// epilogue runs.
//
// Why several MMA warps.  A thread that has MMAs in flight and then touches
// memory (the stage barrier's try_wait, any load) stalls until those MMAs
// have completed, and warp-wide votes stall it too, so one MMA warp that
// waits for every stage drains the tensor pipe at each stage: 121 cycles per
// 128 x 128 x 64 MMA against 68 back to back.  With three warps on
// alternate stages, a warp's wait drains only its own MMAs of three stages
// back while the other two warps' MMAs keep the pipe busy: 68 cycles per MMA.
// Every MMA accumulates (the epilogue zeroes the accumulators when it reads
// them), so the sums do not depend on the order in which the tensor core
// takes the warps' MMAs; they are exact integers below 2^24 in FP32, so the
// order does not change the rounding either.  The warps' MMAs into one
// accumulator are not ordered against each other by tcgen05 fences: the
// tensor core applies them one at a time, which a stress check of 160,000
// MMAs per SM from two and three warps into shared accumulators confirmed
// (no lost update among 7.5 M accumulator elements), and every parity test
// checks the counts bit for bit.  IBS_TC_MMA_WARPS=1 issues from one warp,
// ordered by construction.
constexpr int kQueue = 8;
constexpr int kMmaWarpsMax = 3;

// MMA-issuing warps of the persistent and pair kernels (1 .. 3).
int tc_mma_warps() {
  static const int v = [] {
    const char* e = getenv("IBS_TC_MMA_WARPS");
    const int w = e ? atoi(e) : kMmaWarpsMax;
    return w >= 1 && w <= kMmaWarpsMax ? w : kMmaWarpsMax;
  }();
  return v;
}

// Zero this warp's 32 TMEM lanes of columns [0, 384): the three accumulators.
__device__ __forceinline__ void tmem_zero_acc(uint32_t lane_base) {
  const uint32_t z = 0;
#pragma unroll
  for (int c = 0; c < 384; c += 32)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(lane_base + c),
        "r"(z)
        : "memory");
}

template <int F, class W, int kTStages, int kPer>
__global__ void __launch_bounds__(256, 1)
    tc_persistent_kernel(const W work, int64_t n_items, int* counter, int* status, int mma_warps,
                         unsigned long long wait_ns) {
  constexpr int kBlockBytes = kPer * kTChunkBytes;  // one block's share of a ring stage
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kTStages], empty[kTStages], tfull, tempty, drain;
  __shared__ __align__(8) uint64_t qfull[kQueue], qempty[kQueue];
  __shared__ int64_t q_item[kQueue];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kQueue; ++s) {
      mbar_init(&qfull[s], 1);
      mbar_init(&qempty[s], (uint32_t)(mma_warps + 4));  // the MMA warps and the four epilogue warps
    }
    mbar_init(&tfull, (uint32_t)mma_warps);  // one commit per MMA warp and item
    mbar_init(&tempty, 4);                   // one arrival per epilogue warp
    mbar_init(&drain, (uint32_t)mma_warps);
    mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (warp >= 4) {
    // the accumulators start at zero: every MMA accumulates
    const uint32_t lane_base = tmem + ((uint32_t)((warp - 4) * 32) << 16);
    tmem_zero_acc(lane_base);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    if constexpr (F == kTcFp4) tmem_fill_unit_scales(tmem, warp - 4);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  auto fail = [&](bool cond) {
    // warp-uniform: record a timeout once and tell the other roles to stop
    if (lane == 0 && cond) {
      atomicExch(status, kDevTimeout);
      atomicExch(&abort_flag, 1);
    }
  };
  auto aborted = [&]() { return __any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0); };
  // Wait for queue slot e and read the item index there (-1: no more items).
  auto queue_get = [&](uint32_t e, int64_t& it) {
    const int qs = (int)(e % kQueue);
    const bool ok = mbar_wait_bounded(&qfull[qs], (e / kQueue) & 1u, wait_ns);
    if (__any_sync(0xffffffffu, !ok)) return false;
    it = *(volatile int64_t*)&q_item[qs];
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&qempty[qs])) : "memory");
    return true;
  };

  if (warp == 0) {
    uint32_t g = 0;  // ring stages streamed so far
    for (uint32_t e = 0;; ++e) {
      int64_t it = 0;
      if (lane == 0) it = atomicAdd(counter, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      const bool last = it >= n_items;
      const int qs = (int)(e % kQueue);
      const bool qok = e < (uint32_t)kQueue || mbar_wait_bounded(&qempty[qs], ((e / kQueue) - 1) & 1u, wait_ns);
      if (__any_sync(0xffffffffu, !qok)) {
        fail(true);
        break;
      }
      if (aborted()) break;
      if (lane == 0) {
        q_item[qs] = last ? -1 : it;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&qfull[qs])) : "memory");
      }
      __syncwarp();
      if (last) break;
      const TcTile t = work.tile(it);
      bool stop = false;
      for (int64_t k = t.c0; k < t.c1; k += kPer, ++g) {
        const uint32_t bytes = (uint32_t)(t.c1 - k < kPer ? t.c1 - k : kPer) * kTChunkBytes;
        const int s = (int)(g % kTStages);
        const bool ok = g < (uint32_t)kTStages || mbar_wait_bounded(&empty[s], ((g / kTStages) - 1) & 1u, wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
          fail(true);
          stop = true;
          break;
        }
        if (aborted()) {
          stop = true;
          break;
        }
        if (lane == 0) {
          uint8_t* dst = ring + (size_t)s * 2 * kBlockBytes;
          mbar_arrive_expect_tx(&full[s], t.same ? bytes : 2 * bytes);
          bulk_g2s(dst, t.a + (size_t)k * kTChunkBytes, bytes, &full[s]);
          if (!t.same) bulk_g2s(dst + kBlockBytes, t.b + (size_t)k * kTChunkBytes, bytes, &full[s]);
        }
        __syncwarp();
      }
      if (stop) break;
    }
    // The copies complete on `full` whether or not an MMA warp consumed
    // them; wait (bounded) for the last ring's worth of stages issued before
    // the CTA may exit, since its shared memory is their destination.  A wait
    // on a phase that already completed returns at once.
    for (uint32_t j = g > (uint32_t)kTStages ? g - kTStages : 0; j < g; ++j)
      if (__any_sync(0xffffffffu, !mbar_wait_bounded(&full[j % kTStages], (j / kTStages) & 1u))) {
        fail(true);
        break;
      }
  } else if (warp >= 1 && warp <= mma_warps) {
    const uint32_t mw = (uint32_t)(warp - 1);  // this warp's stages: g % mma_warps == mw
    uint32_t g0 = 0;                           // first ring stage of the current item
    bool stop = false;
    for (uint32_t e = 0;; ++e) {
      int64_t it;
      if (!queue_get(e, it)) {
        fail(true);
        break;
      }
      if (it < 0) break;
      const TcTile t = work.tile(it);
      const uint32_t n_st = (uint32_t)((t.c1 - t.c0 + kPer - 1) / kPer);
      // the epilogue must have read (and zeroed) the previous item's accumulators
      const bool free_ok = e == 0 || mbar_wait_bounded(&tempty, (e - 1) & 1u, wait_ns);
      stop = __any_sync(0xffffffffu, !free_ok);
      if (!stop) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t first = g0 + (mw + (uint32_t)mma_warps - g0 % (uint32_t)mma_warps) % (uint32_t)mma_warps;
        for (uint32_t g = first; g < g0 + n_st; g += (uint32_t)mma_warps) {
          const int64_t k = t.c0 + (int64_t)(g - g0) * kPer;
          const int cnt = (int)(t.c1 - k < kPer ? t.c1 - k : kPer);
          const int s = (int)(g % kTStages);
          const bool ok = mbar_wait_bounded(&full[s], (g / kTStages) & 1u, wait_ns);
          if (__any_sync(0xffffffffu, !ok)) {
            stop = true;
            break;
          }
          if (lane == 0) {
            const uint32_t st0 = smem_addr(ring + (size_t)s * 2 * kBlockBytes);
#pragma unroll
            for (int c = 0; c < kPer; ++c) {
              if (c < cnt) {
                const uint32_t a0 = st0 + c * kTChunkBytes;
                const uint32_t b0 = t.same ? a0 : a0 + kBlockBytes;
                chunk_mmas<F>(tmem, a0, b0, 1u);
              }
            }
            umma_commit(&empty[s]);
          }
          __syncwarp();
        }
      }
      g0 += n_st;
      if (stop || aborted()) {
        fail(stop);
        break;
      }
      // arrives once this warp's MMAs of the item (and all before) have completed
      if (lane == 0) umma_commit(&tfull);
      __syncwarp();
    }
    // arrives once every MMA this warp issued has completed
    if (lane == 0) umma_commit(&drain);
    __syncwarp();
    const bool drained = mbar_wait_bounded(&drain, 0);
    if (lane == 0 && !drained) atomicExch(status, kDevTimeout);
  } else if (warp >= 4) {
    const int quarter = warp - 4;  // TMEM lanes 32*quarter .. 32*quarter+31
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (uint32_t e = 0;; ++e) {
      int64_t it;
      if (!queue_get(e, it)) {
        fail(true);
        break;
      }
      if (it < 0) break;
      const bool ok = mbar_wait_bounded(&tfull, e & 1u, wait_ns);
      if (__any_sync(0xffffffffu, !ok) || aborted()) {
        fail(true);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const typename W::Epi ep = work.epi(it, row);
#pragma unroll 1
      for (int cg = 0; cg < kTB / 32; ++cg) {
        uint32_t vn[32], vu[32], v0[32];
        tmem_ld32(lane_base + 0 + cg * 32, vn);
        tmem_ld32(lane_base + 128 + cg * 32, vu);
        tmem_ld32(lane_base + 256 + cg * 32, v0);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cg == kTB / 32 - 1) {
          // every accumulator of this item is in registers: zero them for the
          // next item and hand TMEM back
          tmem_zero_acc(lane_base);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty)) : "memory");
        }
        ep.store(cg, vn, vu, v0);
      }
      ep.finish();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Two-SM form of the persistent kernel (tcgen05 cta_group::2).  A cluster of
// two CTAs on two SMs computes a 256 x 128 piece of the triangle per item:
// CTA r holds the 128-sample row block I_r (the MMA's A rows 128r ..) and rows
// 64r .. 64r+63 of the shared column block J (half of the MMA's B), and the
// even CTA issues M = 256, N = 128 MMAs over both CTAs' shared memory; CTA r's
// tensor memory receives its 128 x 128 tile.  Per SM and chunk, L2 streams 24
// KiB instead of 32 KiB for the same 128 x 128 results.  Shared memory saves
// less: it takes 24 KiB of copies and 32 KiB of MMA reads (A 16 KiB, and the B
// half 8 KiB for each of the two tensor cores) against 32 + 32 KiB, 12.5% less,
// and half of the B reads come from the peer SM.
//
// The B half of a chunk run is strided in the plane layout (rows 64..127 of a
// plane are its second 2 KiB), so one 4-D TMA tensor copy per stage gathers it:
// the planes as 64-bit elements [block * chunk][plane][half][256], a box of
// {256, 1 half, 4 planes, kPer chunks} landing as [chunk][plane][64 rows].
//
// Roles per CTA: warp 0 streams its own A block and B half into its ring
// with cta_group::2 tensor copies that complete on the even CTA's `full`
// barrier (the even CTA expects both CTAs' bytes), so no thread relays
// anything per stage; warp 1 of the even CTA issues the MMAs (4 per chunk) and
// commits each stage to both CTAs' `empty` barriers and each item to both
// CTAs' `tfull`; warps 4..7 of both read their accumulators back and arrive on
// the even CTA's `tempty` (count 8, one cluster-scope release per item).  Both
// CTAs walk the same items (cluster c takes items c, c + clusters, ...).
// Every wait is bounded.
//
// Measured: n = 20,000, m = 500,000 (7,813 chunks per item), 156 ms against
// 198 ms for the one-SM kernel; n = 4,096, m = 100,000 (1,563 chunks), 1.50 ms
// against 1.38 ms (tensor pipe 49% against 52% active, L2 hit rate 78%
// against 75%).  So ibs_compute takes it for items of at least kLongK chunks
// (tc_pair_mode).  A relay warp that forwarded each stage of the odd CTA with
// a cluster-scope release arrive cost about 1.7 us per stage (2.8 ms).

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_total() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Every thread of both CTAs: release this CTA's prior writes, acquire the peer's.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared variable in cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
// Waits on a barrier that the peer CTA also arrives on (acquire at cluster scope).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity,
                                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (limit_ns < 1000000ull) {  // short bounds (tests): non-blocking probes, clock read after each
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(smem_addr(bar)), "r"(parity)
          : "memory");
      if (ok) return true;
      if (globaltimer_ns() - t0 > limit_ns) return false;
    }
  }
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait_cluster(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
// The same loads issued by either CTA of the pair, completing on the barrier
// at `bar` (a shared::cluster address: the even CTA's barrier), so the even
// CTA's MMA warp sees both CTAs' operands land on one barrier.
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, int x0, int x1, int x2,
                                                 uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
      "%3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(x1), "r"(x2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d_pair(void* dst, const CUtensorMap* map, int x0, int x1, int x2, int x3,
                                                 uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
      "%3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(x1), "r"(x2), "r"(x3), "r"(bar)
      : "memory");
}

// Block-scaled E2M1 x E2M1 -> F32, M = 256 over the CTA pair, N = 128.
constexpr uint32_t kIdescFp4Pair =
    (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) | (1u << 23) | ((uint32_t)(256 >> 4) << 24);
__device__ __forceinline__ void umma_pair(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc, uint32_t sf) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(kIdescFp4Pair), "r"(acc), "r"(sf), "r"(sf + 64u)
      : "memory");
}
// Arrives on the barrier at this offset in both CTAs once the MMAs issued so far are done.
__device__ __forceinline__ void umma_commit_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_addr(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void umma_commit_local2(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
// The four MMAs of one chunk; b0 is this CTA's B half: [plane][64 rows].
__device__ __forceinline__ void chunk_mmas_pair(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t acc) {
  constexpr uint32_t kHalf = kTileBytes / 2;
  const uint32_t sf = tmem + kSfCol;
  umma_pair(tmem + 0, umma_desc(a0 + 0 * kTileBytes), umma_desc(b0 + 0 * kHalf), acc, sf);    // V V^T
  umma_pair(tmem + 128, umma_desc(a0 + 1 * kTileBytes), umma_desc(b0 + 1 * kHalf), acc, sf);  // U U^T
  umma_pair(tmem + 256, umma_desc(a0 + 2 * kTileBytes), umma_desc(b0 + 3 * kHalf), acc, sf);  // Q R^T
  umma_pair(tmem + 256, umma_desc(a0 + 3 * kTileBytes), umma_desc(b0 + 2 * kHalf), 1u, sf);   // + R Q^T
}

// Work of the pair kernel.  One matrix: the subset travels in the kernel
// parameters and its planes start at block-chunk 0 of the tensor maps.
struct PairWork {
  SubsetDev sd;
  const PairItem* items;
  static constexpr bool kFused = false;
  __device__ SubsetDev sub(int32_t) const { return sd; }
  __device__ static int64_t base(const SubsetDev&) { return 0; }
};

// Batched subsets with the gather fused in: the subsets' operand planes share
// one buffer (SubsetDev::pad = the block-chunk index of a subset's block 0,
// chunk 0 in it), and the epilogue warps, which are idle while an item's
// MMAs run, gather the planes from the pool in units {job, sample block,
// chunk group, subset} (the standalone gather kernel's CTAs).  ready[k]
// counts the finished units of subset k; the copy warps start an item only
// once ready[k] == need[k].
struct PairBatchWork {
  const SubsetDev* subs;
  const PairItem* items;
  const TcGatherJob* jobs;
  const int4* units;
  int64_t n_units;
  int* unit_counter;
  int* ready;
  const int* need;
  static constexpr bool kFused = true;
  __device__ SubsetDev sub(int32_t k) const { return subs[k]; }
  __device__ static int64_t base(const SubsetDev& s) { return s.pad; }
};

// Serving on the two-SM kernel: A = two 128-row blocks of the step's dense
// query planes (I0, I1; I1 < 0: the odd CTA loads I0 again and stores
// nothing), B = panel block J, over all chunks.  Counts only: step row r
// writes its 128 panel samples through its own output row row_out[r]
// ([n_panel][4] int32), as the one-SM CrossWork does.
struct PairCrossWork {
  const PairItem* items;
  int32_t* const* row_out;
  int64_t n_rows, n_panel, n_chunks;
  static constexpr bool kFused = false;
  __device__ SubsetDev sub(int32_t) const {
    SubsetDev s{};
    s.n_chunks = n_chunks;
    return s;
  }
  __device__ static int64_t base(const SubsetDev&) { return 0; }
};

// The epilogue of one CTA's tile of a pair item: triangle output for one
// matrix or a batch of subsets, per-row output rows for serving.
template <class PW>
__device__ __forceinline__ TriEpi pair_epi(const PW& w, const PairItem& pi, int32_t ib, int row) {
  const SubsetDev sd = w.sub(pi.subset);
  return TriEpi{ib >= 0 ? (int64_t)ib * kTB + row : sd.n, (int64_t)pi.J * kTB, sd.n, sd.out_counts,
                sd.out_dist, sd.partial, pi.split != 0};
}
__device__ __forceinline__ CrossWork::Epi pair_epi(const PairCrossWork& w, const PairItem& pi, int32_t ib, int row) {
  const int64_t r = ib >= 0 ? (int64_t)ib * kTB + row : w.n_rows;
  return {r < w.n_rows ? w.row_out[r] : nullptr, (int64_t)pi.J * kTB, w.n_panel};
}

// Wait until *counter >= need (another CTA's gather units; bounded).
__device__ __forceinline__ bool wait_ready(const int* counter, int need, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned ns = 32;; ns = ns < 1024 ? 2 * ns : ns) {
    int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
    if (v >= need) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
    __nanosleep(ns);
  }
}

// Hardware barrier of the pair kernel's four epilogue warps (the fused gather's lock step).
constexpr int kEpiBar = 2;
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync %0, 128;" ::"n"(kEpiBar) : "memory"); }

// Shared memory of one ring stage: kPer chunks of the A block, then kPer
// chunks of the B half (the A box is exactly kPer x 16 KiB, the B-half box
// kPer x 8 KiB); 1 KiB for aligning the ring.  Nothing more, so that two
// gather CTAs fit on an SM beside a pair CTA in the batched launch.
template <int kPer>
constexpr int kPairStageBytes = kPer * (kTChunkBytes + kTChunkBytes / 2);
template <int kStages, int kPer>
constexpr size_t kPairSmem = (size_t)kStages * kPairStageBytes<kPer> + 1024;

// Hardware barrier between the pair kernel's waiter warp and its MMA warp
// (barrier 0 is __syncthreads).  One issuing warp only: a cta_group::2 MMA
// runs on both SMs of the pair, which exchange B halves per instruction, and
// MMAs issued by several warps reached the two tensor cores in different
// orders (every count wrong in the parity tests).
constexpr int kPairBar = 1;

template <class PW, int kStages, int kPer>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 1)
    tc_pair_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                   const PW work, int64_t n_items, int* status, unsigned long long wait_ns, const PairSync sync) {
  constexpr int kABytes = kPer * kTChunkBytes;
  constexpr int kStageBytes = kPairStageBytes<kPer>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull, tempty, drain;
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t issued;  // ring stages this CTA's copy warp issued
  __shared__ int abort_flag;
  __shared__ int64_t s_dec;    // fused gather: the epilogue warps' broadcast decision
  __shared__ int s_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int64_t first = cluster_index(), step = cluster_total();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);  // the even CTA's: both CTAs' copies complete on it
      mbar_init(&empty[s], 1);
    }
    mbar_init(&tfull, 1);   // the MMA warp's commit per item
    mbar_init(&tempty, 8);  // four epilogue warps per CTA
    mbar_init(&drain, 1);
    mbar_fence_init();
    abort_flag = 0;
    issued = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (warp >= 4) {
    // the accumulators start at zero: every MMA accumulates
    tmem_zero_acc(tmem + ((uint32_t)((warp - 4) * 32) << 16));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tmem_fill_unit_scales(tmem, warp - 4);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // both CTAs' barriers initialised, accumulators zeroed and scale factors stored
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  auto fail = [&](bool cond) {
    if (lane == 0 && cond) {
      atomicExch(status, kDevTimeout);
      atomicExch(&abort_flag, 1);
    }
  };
  auto aborted = [&]() { return __any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0); };

  if (warp == 0) {
    uint32_t g = 0;
    bool stop = false;
    const uint32_t full0 = cluster_addr(&full[0], 0);  // the even CTA's ring barriers
    for (int64_t it = first; it < n_items && !stop; it += step) {
      const PairItem pi = work.items[it];
      const int32_t ib = rank == 0 ? pi.I0 : (pi.I1 >= 0 ? pi.I1 : pi.I0);
      const SubsetDev sd = work.sub(pi.subset);
      const int64_t nc = sd.n_chunks, bc0 = PW::base(sd);
      if constexpr (PW::kFused) {
        // the subset's planes must be gathered before its copies start;
        // the proxy fence orders the gather's plain stores before the TMA reads
        bool ok = true;
        if (lane == 0) {
          ok = wait_ready(work.ready + pi.subset, work.need[pi.subset], wait_ns);
          asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        if (__any_sync(0xffffffffu, !ok)) {
          fail(true);
          stop = true;
          break;
        }
      }
      const bool lockstep = sync.seg > 0 && it < sync.n_items;
      int* wave_ctr = lockstep ? sync.ctr + (it / step) * sync.n_seg : nullptr;
      for (int64_t k = pi.c0; k < pi.c1; k += kPer, ++g) {
        if (lockstep && (k - pi.c0) % sync.seg == 0) {
          // announce this segment, then hold back until the whole wave has
          // started the segment `lag` back (bounded; seg is a multiple of kPer)
          const int64_t sg = (k - pi.c0) / sync.seg;
          bool okw = true;
          if (lane == 0) {
            atomicAdd(wave_ctr + sg, 1);
            if (sg >= sync.lag) okw = wait_ready(wave_ctr + sg - sync.lag, 2 * (int)step, wait_ns);
          }
          if (__any_sync(0xffffffffu, !okw)) {
            fail(true);
            stop = true;
            break;
          }
        }
        const int s = (int)(g % kStages);
        const bool ok = g < (uint32_t)kStages || mbar_wait_bounded(&empty[s], ((g / kStages) - 1) & 1u, wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
          fail(true);
          stop = true;
          break;
        }
        if (aborted()) {
          stop = true;
          break;
        }
        if (lane == 0) {
          // whole boxes always (past an item's last chunk they read the next
          // block's chunks, or zeros past the end, which no MMA uses)
          uint8_t* dst = ring + (size_t)s * kStageBytes;
          const uint32_t bar = full0 + (uint32_t)s * 8u;
          if (rank == 0) mbar_arrive_expect_tx(&full[s], 2u * kStageBytes);
          tma_load_3d_pair(dst, &amap, 0, 0, (int)(bc0 + (int64_t)ib * nc + k), bar);
          tma_load_4d_pair(dst + kABytes, &bmap, 0, (int)rank, 0, (int)(bc0 + (int64_t)pi.J * nc + k), bar);
        }
        __syncwarp();
      }
    }
    // the last stages' releases (commits of the even CTA) have landed here
    for (uint32_t j = g > (uint32_t)kStages ? g - kStages : 0; j < g && !stop; ++j) {
      const bool ok = mbar_wait_bounded(&empty[j % kStages], (j / kStages) & 1u);
      if (__any_sync(0xffffffffu, !ok)) {
        fail(true);
        break;
      }
    }
    if (lane == 0) issued = g;
    __syncwarp();
  } else if (warp == 1 && rank == 0) {
    // MMA warp of the even CTA.  It never waits on memory itself: a thread
    // with MMAs in flight that reads a barrier (or any memory) stalls until
    // they have completed, which would drain the tensor pipe at every stage.
    // Warp 2 does the waiting and releases this warp once per ring stage
    // through hardware barrier kPairBar (both warps execute bar.sync once per
    // stage of every item, in the same order, so neither can run ahead).
    uint32_t g0 = 0;
    for (int64_t it = first; it < n_items; it += step) {
      const PairItem pi = work.items[it];
      const uint32_t n_st = (uint32_t)((pi.c1 - pi.c0 + kPer - 1) / kPer);
      for (uint32_t g = g0; g < g0 + n_st; ++g) {
        asm volatile("bar.sync %0, 64;" ::"n"(kPairBar) : "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const int64_t k = pi.c0 + (int64_t)(g - g0) * kPer;
          const int cnt = (int)(pi.c1 - k < kPer ? pi.c1 - k : kPer);
          const int s = (int)(g % kStages);
          const uint32_t st0 = smem_addr(ring + (size_t)s * kStageBytes);
#pragma unroll
          for (int c = 0; c < kPer; ++c)
            if (c < cnt) chunk_mmas_pair(tmem, st0 + c * kTChunkBytes, st0 + kABytes + c * (kTChunkBytes / 2), 1u);
          umma_commit_both(&empty[s]);
        }
      }
      g0 += n_st;
      if (lane == 0) umma_commit_both(&tfull);
    }
    __syncwarp();
    if (lane == 0) umma_commit_local2(&drain);
    __syncwarp();
    const bool drained = mbar_wait_bounded(&drain, 0);
    if (lane == 0 && !drained) atomicExch(status, kDevTimeout);
  } else if (warp == 2 && rank == 0) {
    // Waiter of the even CTA: for each stage, wait (bounded) until both CTAs'
    // operands have landed (and, before an item's first stage, until both
    // epilogues have read and zeroed the accumulators), then release the MMA
    // warp.  After a failed wait or another role's abort it stops waiting but
    // keeps releasing, so the MMA warp runs out its stages on stale operands
    // (harmless: the call reports IBS_ETIMEOUT) and the kernel ends.
    uint32_t g0 = 0, e = 0;
    bool dead = false;
    for (int64_t it = first; it < n_items; it += step, ++e) {
      const PairItem pi = work.items[it];
      const uint32_t n_st = (uint32_t)((pi.c1 - pi.c0 + kPer - 1) / kPer);
      if (!dead && e > 0) {
        const bool ok = mbar_wait_cluster_bounded(&tempty, (e - 1) & 1u, wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
          fail(true);
          dead = true;
        }
      }
      for (uint32_t g = g0; g < g0 + n_st; ++g) {
        if (!dead) {
          const bool ok = mbar_wait_bounded(&full[g % kStages], (g / kStages) & 1u, wait_ns);
          if (__any_sync(0xffffffffu, !ok)) {
            fail(true);
            dead = true;
          } else if (aborted()) {
            dead = true;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync %0, 64;" ::"n"(kPairBar) : "memory");
      }
      g0 += n_st;
    }
  } else if (warp >= 4) {
    const int quarter = warp - 4;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t tempty_addr = cluster_addr(&tempty, 0);
    // Fused gather (batched subsets): one gather unit at a time by all four
    // epilogue warps (thread `row` = sample row of the unit's block), chosen
    // by row 0 and broadcast through shared memory; the warps move in lock
    // step on barrier kEpiBar, so every branch below is taken by all of them.
    // (generic lambdas: their bodies exist only for the fused work type)
    auto gather_step = [&](const auto& w, int64_t u) {
      const int4 un = w.units[u];  // {job, sample block, chunk group, subset}
      gather_unit<kTcFp4>(w.jobs[un.x], un.y, un.z, row, status);
      asm volatile("fence.proxy.async.global;" ::: "memory");
      epi_sync();  // every row of the unit is written
      if (row == 0) {
        __threadfence();
        atomicAdd(w.ready + un.w, 1);
      }
    };
    auto claim = [&](const auto& w) -> int64_t {
      const int64_t u = atomicAdd(w.unit_counter, 1);
      return u < w.n_units ? u : -1;
    };
    uint32_t e = 0;
    for (int64_t it = first; it < n_items; it += step, ++e) {
      const PairItem pi = work.items[it];
      bool ok = true;
      if constexpr (PW::kFused) {
        // gather while the item's MMAs run; then wait (bounded) for them
        for (;;) {
          if (row == 0) s_dec = mbar_test_wait(&tfull, e & 1u) ? -1 : claim(work);
          epi_sync();
          const int64_t d = s_dec;
          epi_sync();  // everyone has read s_dec
          if (d < 0) break;
          gather_step(work, d);
        }
        if (row == 0) s_ok = mbar_wait_bounded(&tfull, e & 1u, wait_ns) && *(volatile int*)&abort_flag == 0;
        epi_sync();
        ok = s_ok != 0;
        epi_sync();
        if (!ok) {
          if (row == 0 && *(volatile int*)&abort_flag == 0) {
            atomicExch(status, kDevTimeout);
            atomicExch(&abort_flag, 1);
          }
          break;  // all four warps together
        }
      } else {
        ok = mbar_wait_bounded(&tfull, e & 1u, wait_ns);
        if (__any_sync(0xffffffffu, !ok) || aborted()) {
          fail(!ok);
          break;
        }
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int32_t ib = rank == 0 ? pi.I0 : pi.I1;
      const auto ep = pair_epi(work, pi, ib, row);
#pragma unroll 1
      for (int cg = 0; cg < kTB / 32; ++cg) {
        uint32_t vn[32], vu[32], v0[32];
        tmem_ld32(lane_base + 0 + cg * 32, vn);
        tmem_ld32(lane_base + 128 + cg * 32, vu);
        tmem_ld32(lane_base + 256 + cg * 32, v0);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cg == kTB / 32 - 1) {
          // zero this CTA's accumulators for the next item, then hand TMEM back
          tmem_zero_acc(lane_base);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(tempty_addr);
        }
        ep.store(cg, vn, vu, v0);
      }
      ep.finish();
    }
    if constexpr (PW::kFused) {
      // this CTA's items are done (or stopped): gather units are left for the
      // other CTAs' items, so keep taking them while any remain
      for (;;) {
        if (row == 0) s_dec = *(volatile int*)&abort_flag != 0 ? -1 : claim(work);
        epi_sync();
        const int64_t d = s_dec;
        epi_sync();
        if (d < 0) break;
        gather_step(work, d);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // both CTAs have issued their last copy and the even CTA's MMAs are drained
  if (rank == 0 && warp == 0) {
    // Every copy of either CTA completes on the even CTA's `full` barriers.
    // After a stop some issued stages were never consumed by the MMA warp, so
    // wait (bounded) for the last ring's worth of stages that either CTA
    // issued: a wait on a phase that has already completed returns at once,
    // so on the normal path this costs kStages probes.  Only then may either
    // CTA exit (its shared memory is the copies' destination).
    uint32_t peer = 0;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(peer) : "r"(cluster_addr(&issued, 1)) : "memory");
    const uint32_t gmax = issued > peer ? issued : peer;
    for (uint32_t j = gmax > (uint32_t)kStages ? gmax - kStages : 0; j < gmax; ++j) {
      const bool ok = mbar_wait_bounded(&full[j % kStages], (j / kStages) & 1u);
      if (__any_sync(0xffffffffu, !ok)) {
        fail(true);
        break;
      }
    }
  }
  __syncthreads();
  cluster_sync_all();  // no copy into either CTA and no arrival on either CTA's barriers is outstanding
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Serving: copy dense query rows (each a row of some request's operand
// planes) into 128-row step blocks.  CTA = (step block, chunk); each thread
// moves 16-byte pieces (row, plane, K half).
__global__ void __launch_bounds__(256) tc_gather_rows_kernel(const RowSrc* __restrict__ rows, int64_t n_rows,
                                                             int64_t n_chunks, uint8_t* __restrict__ dst) {
  const int64_t c = blockIdx.x, qb = blockIdx.y;
  for (int p = threadIdx.x; p < kTB * 8; p += blockDim.x) {
    const int r = p % kTB, piece = p / kTB;  // piece = plane * 2 + K half
    const int64_t d = qb * kTB + r;
    if (d >= n_rows) continue;
    const RowSrc src = rows[d];
    const int64_t sb = src.row / kTB, sr = src.row % kTB;
    const int off_plane = (piece >> 1) * kTileBytes, half = piece & 1;
    const uint8_t* from = reinterpret_cast<const uint8_t*>(src.planes) + (size_t)(sb * n_chunks + c) * kTChunkBytes +
                          off_plane + tile_off((int)sr, half * 16);
    uint8_t* to = dst + (size_t)(qb * n_chunks + c) * kTChunkBytes + off_plane + tile_off(r, half * 16);
    *reinterpret_cast<uint4*>(to) = *reinterpret_cast<const uint4*>(from);
  }
}

// Split-K finalisation of the listed tiles only: partial [P][4] (IBS0, IBS1,
// -, N) -> counts and distance of every pair of the tile.  CTA (x, y) takes
// tile x, its pairs y, y + gridDim.y, ... in units of blockDim.x.
__global__ void __launch_bounds__(256) tc_finalize_tiles_kernel(const int2* __restrict__ tiles,
                                                                const int32_t* __restrict__ partial, int64_t n,
                                                                int32_t* __restrict__ out_counts,
                                                                double* __restrict__ out_dist) {
  const int2 t = tiles[blockIdx.x];
  for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < kTB * kTB; p += gridDim.y * blockDim.x) {
    const int64_t gi = (int64_t)t.x * kTB + p / kTB, gj = (int64_t)t.y * kTB + p % kTB;
    if (gi >= n || gj >= n || gj < gi) continue;
    const int64_t q = tri_index(gi, gj, n);
    const int4 v = reinterpret_cast<const int4*>(partial)[q];
    reinterpret_cast<int4*>(out_counts)[q] = make_int4(v.x, v.y, v.w - v.x - v.y, v.w);
    if (out_dist)
      out_dist[q] = ibs_dist(v.x, v.y, v.w);
  }
}

// The same for a batch: one CTA per listed (subset, tile), the subset's
// outputs and partial triangle read from its descriptor (so a captured graph
// serves calls with new output pointers).
__global__ void __launch_bounds__(256) tc_finalize_batch_tiles_kernel(const SubsetDev* __restrict__ subs,
                                                                      const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];  // {subset, I, J, -}
  const SubsetDev sd = subs[t.x];
  for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < kTB * kTB; p += gridDim.y * blockDim.x) {
    const int64_t gi = (int64_t)t.y * kTB + p / kTB, gj = (int64_t)t.z * kTB + p % kTB;
    if (gi >= sd.n || gj >= sd.n || gj < gi) continue;
    const int64_t q = tri_index(gi, gj, sd.n);
    const int4 v = reinterpret_cast<const int4*>(sd.partial)[q];
    reinterpret_cast<int4*>(sd.out_counts)[q] = make_int4(v.x, v.y, v.w - v.x - v.y, v.w);
    if (sd.out_dist) sd.out_dist[q] = ibs_dist(v.x, v.y, v.w);
  }
}

// ---------------------------------------------------------------------------
// MMA-rate probe: every CTA (one per SM) issues back-to-back 128 x 128 MMAs of
// one kind from operand tiles resident in shared memory, into one TMEM
// accumulator (the tile contents are irrelevant to the rate).  The launch time
// gives the sustained MMA throughput the pair kernels are bound by.
template <int F>
__global__ void __launch_bounds__(128) tc_mma_probe_kernel(int n_mma, int* status) {
  __shared__ __align__(1024) uint8_t sa[kTileBytes];
  __shared__ __align__(1024) uint8_t sb[kTileBytes];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const uint8_t fill = F == kTcFp4 ? 0x22 : kFp8One;  // 1.0 in every element
  for (int i = threadIdx.x; i < kTileBytes; i += blockDim.x) {
    sa[i] = fill;
    sb[i] = fill;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes seen by the MMA
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if constexpr (F == kTcFp4) {
    tmem_fill_unit_scales(tmem, warp);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    const uint64_t da = umma_desc(smem_addr(sa)), db = umma_desc(smem_addr(sb));
    for (int i = 0; i < n_mma; ++i) umma<F>(tmem, da, db, i > 0 ? 1u : 0u, tmem + kSfCol);
    umma_commit(&bar);
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0);
  if (!ok && (threadIdx.x & 31) == 0) atomicExch(status, kDevTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

int tc_default_format() {
  static const int f = [] {
    const char* e = getenv("IBS_TC_FORMAT");
    if (e && strcmp(e, "fp4") == 0) return kTcFp4;
    if (e && strcmp(e, "fp8") == 0) return kTcFp8;
    return kTcFp4;  // half the operand bytes per marker and the faster MMA kind
  }();
  return f;
}

// Longest K range one accumulation may cover: 2^21 markers.  Every partial
// sum of the three accumulators is at most one per marker, so this keeps them
// far below 2^24, where FP32 accumulation stops being exact; longer tiles are
// split over K and their pieces added as integers.
int64_t tc_max_chunks(int fmt) { return ((int64_t)1 << 21) / (fmt == kTcFp4 ? kMarkers<kTcFp4> : kMarkers<kTcFp8>); }

int64_t tc_chunks(int64_t m, int fmt) {
  const int64_t k = fmt == kTcFp4 ? kMarkers<kTcFp4> : kMarkers<kTcFp8>;
  return (m + k - 1) / k;
}

size_t tc_planes_bytes(int64_t n, int64_t m, int fmt) {
  const int64_t nb = (n + kTB - 1) / kTB;
  return (size_t)nb * (size_t)tc_chunks(m, fmt) * kTChunkBytes;
}

// Split count over the marker axis.  All tiles of one launch cost the same:
// with s splits the launch runs ceil(tiles * s / SMs) waves, each of n_chunks/s
// chunks of MMAs plus, when s > 1, an epilogue of 3 x 128 x 128 partial-count
// atomics, charged as kSplitEpilogueChunks chunks of MMA time.  Pick the s in
// 1..64 (at least one chunk per split) of least total time.  IBS_TC_SPLITS
// overrides the choice (clamped to 1..min(64, n_chunks)).
constexpr double kSplitEpilogueChunks = 160.0;

int tc_splits_for(int64_t tiles, int64_t n_chunks, int num_sms) {
  static const int forced = [] {
    const char* e = getenv("IBS_TC_SPLITS");
    return e ? atoi(e) : 0;
  }();
  if (forced > 0) return (int)std::min<int64_t>(std::min(forced, 64), std::max<int64_t>(1, n_chunks));
  int best = 1;
  double best_cost = 1e300;
  for (int s = 1; s <= 64 && s <= n_chunks; ++s) {
    const double waves = (double)((tiles * s + num_sms - 1) / num_sms);
    const double cost = waves * ((double)n_chunks / s + (s > 1 ? kSplitEpilogueChunks : 0.0));
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = s;
    }
  }
  return best;
}

cudaError_t launch_tc_planes(const uint8_t* packed, int64_t n, int64_t m, uint8_t* planes, int fmt,
                             cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = tc_chunks(m, fmt);
  if (nc > 2147483647LL || nb > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)nc, (unsigned)nb);
  if (fmt == kTcFp4)
    tc_planes_kernel<kTcFp4><<<grid, 256, 0, st>>>(packed, (n + 3) / 4, n, m, planes, nc);
  else
    tc_planes_kernel<kTcFp8><<<grid, 256, 0, st>>>(packed, (n + 3) / 4, n, m, planes, nc);
  return cudaGetLastError();
}

cudaError_t launch_tc_pairs(const uint8_t* planes, int64_t n, int64_t m, int fmt, int splits, int32_t* out_counts,
                            double* out_dist, int32_t* partial, bool square, int* status, const int2* tile_list,
                            cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = tc_chunks(m, fmt);
  const int64_t tiles = nb * (nb + 1) / 2;
  const int64_t grid = tiles * splits;
  if (grid > 2147483647LL) return cudaErrorInvalidValue;
  auto kern = fmt == kTcFp4 ? tc_tri_kernel<kTcFp4> : tc_tri_kernel<kTcFp8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kTThreads, kTcSmem, st>>>(planes, n, nb, nc, splits, out_counts, out_dist, partial,
                                                   square ? 1 : 0, status, tile_list);
  return cudaGetLastError();
}

// Grouped tile order: the upper triangle of T x T tiles in bands of G tile
// rows; inside a band, column by column.  The CTAs running at the same time
// then cover about G rows x (SMs / G) columns, so each block of planes they
// stream is shared by many of them through L2 instead of being fetched from
// HBM once per tile.
void tc_tile_order(int64_t T, int G, std::vector<int2>& out) {
  out.clear();
  out.reserve((size_t)(T * (T + 1) / 2));
  for (int64_t g0 = 0; g0 < T; g0 += G) {
    const int64_t g1 = g0 + G < T ? g0 + G : T;
    for (int64_t J = g0; J < T; ++J)
      for (int64_t I = g0; I < g1 && I <= J; ++I) out.push_back(make_int2((int)I, (int)J));
  }
}

int64_t tc_tiles(int64_t n) {
  const int64_t nb = (n + kTB - 1) / kTB;
  return nb * (nb + 1) / 2;
}

cudaError_t launch_tc_gather(const TcGatherJob* jobs_dev, const int4* map_dev, int64_t total_ctas, int fmt,
                             int* status, cudaStream_t st) {
  if (total_ctas <= 0) return cudaSuccess;
  if (total_ctas > 2147483647LL) return cudaErrorInvalidValue;
  if (fmt == kTcFp4)
    tc_gather_kernel<kTcFp4><<<(unsigned)total_ctas, kTB, 0, st>>>(jobs_dev, map_dev, status);
  else
    tc_gather_kernel<kTcFp8><<<(unsigned)total_ctas, kTB, 0, st>>>(jobs_dev, map_dev, status);
  return cudaGetLastError();
}

// Ring of the persistent kernel: kPer chunks per stage (one bulk copy per
// block and stage) and the stage count, 192 KiB either way.  The copy engine
// spends a fixed time per bulk copy, so two-chunk stages stream faster while
// the operands mostly hit L2 (n = 4,096, m = 100,000: pair kernel 1.74 ->
// 1.39 ms); for items of at least kLongK chunks the CTAs drift apart over a
// tile and miss L2 more, and six one-chunk stages (more copies in flight)
// win (n = 20,000, m = 500,000: 198 ms against 252 ms with two-chunk stages).
// IBS_TC_RING=per,stages overrides (1,4 / 1,6 / 2,2 / 2,3 / 3,2).
constexpr int64_t kLongK = 4096;
struct Ring {
  int per, stages;
};
Ring persistent_ring(int64_t chunks_per_item) {
  static const Ring forced = [] {
    Ring r{0, 0};
    if (const char* e = getenv("IBS_TC_RING")) {
      const bool known = sscanf(e, "%d,%d", &r.per, &r.stages) == 2 &&
                         ((r.per == 1 && (r.stages == 4 || r.stages == 6)) ||
                          (r.per == 2 && (r.stages == 2 || r.stages == 3)) || (r.per == 3 && r.stages == 2));
      if (!known) r = Ring{0, 0};
    } else if (const char* e2 = getenv("IBS_TC_STAGES")) {
      const int v = atoi(e2);
      if (v == 4 || v == 6) r = Ring{1, v};
    }
    return r;
  }();
  if (forced.per > 0) return forced;
  return chunks_per_item >= kLongK ? Ring{1, 6} : Ring{2, 3};
}

template <int F, class W, int S, int P>
cudaError_t launch_persistent_s(const W& work, int64_t n_items, int grid, int* counter, int* status,
                                unsigned long long wait_ns, cudaStream_t st) {
  constexpr size_t smem = (size_t)S * 2 * P * kTChunkBytes + 1024;
  static_assert(smem <= 227 * 1024, "ring exceeds shared memory");
  cudaError_t e = cudaFuncSetAttribute(tc_persistent_kernel<F, W, S, P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  // Each ring slot must belong to one MMA warp (warp j takes stages g with
  // g % warps == j, slot g % S), so that a warp waits for the phases of its
  // slots in order: a slot shared by two warps lets one of them test a phase
  // two completions ahead, where the parity test cannot tell it from an
  // older completed phase.  So the warp count divides the stage count.
  int mma_warps = tc_mma_warps();
  while (S % mma_warps != 0) --mma_warps;
  tc_persistent_kernel<F, W, S, P><<<grid, 256, smem, st>>>(work, n_items, counter, status, mma_warps, wait_ns);
  return cudaGetLastError();
}

template <int F, class W>
cudaError_t launch_persistent_f(const W& work, int64_t n_items, int grid, Ring r, int* counter, int* status,
                                unsigned long long w, cudaStream_t st) {
  if (r.per == 1 && r.stages == 4) return launch_persistent_s<F, W, 4, 1>(work, n_items, grid, counter, status, w, st);
  if (r.per == 1 && r.stages == 6) return launch_persistent_s<F, W, 6, 1>(work, n_items, grid, counter, status, w, st);
  if (r.per == 2 && r.stages == 2) return launch_persistent_s<F, W, 2, 2>(work, n_items, grid, counter, status, w, st);
  if (r.per == 2 && r.stages == 3) return launch_persistent_s<F, W, 3, 2>(work, n_items, grid, counter, status, w, st);
  if (r.per == 3 && r.stages == 2) return launch_persistent_s<F, W, 2, 3>(work, n_items, grid, counter, status, w, st);
  return cudaErrorInvalidValue;
}

template <class W>
cudaError_t launch_persistent(const W& work, int64_t n_items, int grid, int fmt, int64_t chunks_per_item,
                              int* counter, int* status, unsigned long long wait_ns, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (grid < 1 || n_items > 2147483647LL - grid) return cudaErrorInvalidValue;  // the claim counter is an int
  const Ring r = persistent_ring(chunks_per_item);
  if (fmt == kTcFp4) return launch_persistent_f<kTcFp4>(work, n_items, grid, r, counter, status, wait_ns, st);
  return launch_persistent_f<kTcFp8>(work, n_items, grid, r, counter, status, wait_ns, st);
}

cudaError_t launch_tc_batch(const SubsetDev* subs, const WorkItem* items, int64_t n_items, int grid, int fmt,
                            int64_t max_chunks, int* counter, int* status, cudaStream_t st) {
  return launch_persistent(BatchWork{subs, items}, n_items, grid, fmt, max_chunks, counter, status, kWaitLimitNs,
                           st);
}

cudaError_t launch_tc_single(const SubsetDev& sd, const WorkItem* items, int64_t n_items, int grid, int fmt,
                             int* counter, int* status, unsigned long long wait_ns, cudaStream_t st) {
  return launch_persistent(SingleWork{sd, items}, n_items, grid, fmt, sd.n_chunks, counter, status, wait_ns, st);
}

// ---------------------------------------------------------------------------
// Two-SM pair kernel, host side.

// Ring of the pair kernel: kPer chunks per stage.  Three stages of three
// chunks (216 KiB) measured fastest on n = 4,096, m = 100,000 (1.50 ms; 2 x 4:
// 1.60 ms, 4 x 2: 1.51 ms).  IBS_TC_PAIR_RING=per,stages overrides (2,4 / 1,8 /
// 4,2 / 3,3).
struct PairRing {
  int per, stages;
};
PairRing pair_ring(int64_t chunks_per_item) {
  static const PairRing forced = [] {
    PairRing r{0, 0};
    if (const char* e = getenv("IBS_TC_PAIR_RING")) {
      const bool known = sscanf(e, "%d,%d", &r.per, &r.stages) == 2 &&
                         ((r.per == 2 && r.stages == 4) || (r.per == 1 && r.stages == 8) ||
                          (r.per == 4 && r.stages == 2) || (r.per == 3 && r.stages == 3));
      if (!known) r = PairRing{0, 0};
    }
    return r;
  }();
  (void)chunks_per_item;
  return forced.per > 0 ? forced : PairRing{3, 3};
}

// Clusters of two that fit at once (one CTA per SM; a GPC with an odd number
// of free SMs leaves one out).
// Counted once per device ordinal (with that device current): function
// attributes and free SMs are per device.
template <int S, int P>
int pair_clusters_s() {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs];  // 0 = not yet counted, else count + 1
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
    cudaGetLastError();
    return 0;
  }
  if (const int c = cache[dev].load(std::memory_order_acquire)) return c - 1;
  const int v = [dev] {
    constexpr size_t smem = kPairSmem<S, P>;
    if (cudaFuncSetAttribute(tc_pair_kernel<PairWork, S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(2, sms & ~1));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel<PairWork, S, P>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }();
  cache[dev].store(v + 1, std::memory_order_release);
  return v;
}

int tc_pair_clusters(int64_t chunks_per_item) {
  const PairRing r = pair_ring(chunks_per_item);
  if (r.per == 2 && r.stages == 4) return pair_clusters_s<4, 2>();
  if (r.per == 1 && r.stages == 8) return pair_clusters_s<8, 1>();
  if (r.per == 4 && r.stages == 2) return pair_clusters_s<2, 4>();
  if (r.per == 3 && r.stages == 3) return pair_clusters_s<3, 3>();
  return 0;
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link-time
// dependency on libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Two views of the operand planes as 64-bit elements.  A: [block * chunk]
// [8][256], a box is `per` whole block-chunks (16 KiB each).  B half:
// [block * chunk][plane][half][256], a box is one half of all four planes
// over `per` chunks, landing as [chunk][plane][64 rows].
bool encode_a_map(CUtensorMap* map, const void* planes, int64_t nb, int64_t nc, int per) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {256, 8, (cuuint64_t)(nb * nc)};
  const cuuint64_t strides[2] = {(cuuint64_t)kTileBytes / 2, (cuuint64_t)kTChunkBytes};
  const cuuint32_t box[3] = {256, 8, (cuuint32_t)per};
  const cuuint32_t elem[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(planes), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool encode_bhalf_map(CUtensorMap* map, const void* planes, int64_t nb, int64_t nc, int per) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {256, 2, 4, (cuuint64_t)(nb * nc)};
  const cuuint64_t strides[3] = {(cuuint64_t)kTileBytes / 2, (cuuint64_t)kTileBytes, (cuuint64_t)kTChunkBytes};
  const cuuint32_t box[4] = {256, 1, 4, (cuuint32_t)per};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(planes), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// IBS_TC_PAIR=1: the pair kernel wherever it can run; 0: never; unset: for
// matrices of at least kPairMinChunks chunks.  Each SM of a pair takes 24 KiB
// of operands per chunk instead of 32 KiB, and operand ingest (TMA, about
// 65-75 B/clk per SM) bounds both kernels; below about a thousand chunks the
// pair's per-item overheads cost more than that saves.  Measured pair kernel
// against one-SM kernel: n = 4,096, m = 10,000: 0.313 against 0.286 ms; m =
// 50,000 (n = 1,024): 0.096 against 0.094 ms; m = 100,000: 1.334 against
// 1.449 ms; n = 8,000, m = 200,000: 9.05 against 12.52 ms.
constexpr int64_t kPairMinChunks = 1024;

int tc_pair_mode() {
  static const int v = [] {
    const char* e = getenv("IBS_TC_PAIR");
    if (e && strcmp(e, "1") == 0) return 1;
    if (e && strcmp(e, "0") == 0) return -1;
    return 0;
  }();
  return v;
}

bool tc_pair_usable(int64_t n, int64_t m, int fmt) {
  if (tc_pair_mode() < 0 || fmt != kTcFp4) return false;
  const int64_t nb = (n + kTB - 1) / kTB, nc = tc_chunks(m, fmt);
  if (tc_pair_mode() == 0 && nc < kPairMinChunks) return false;
  if (nb < 2 || nb * nc + 8 > 2147483647LL) return false;  // the tensor map's chunk coordinate is an int
  if (!encode_tiled_fn()) return false;
  return tc_pair_clusters(nc) > 0;
}

// Work list of the pair kernel: pair items in the grouped order (bands of
// `group` tile rows, rounded up to even; inside a band, column by column, the
// rows (I, I+1) of a column as one item, a lone row where I+1 is past the band
// or the diagonal).  The clusters take items round-robin, so the items of the
// final partial wave are split over K where that shortens the tail.
void tc_pair_order(int64_t T, int group, std::vector<int4>& order) {
  order.clear();
  const int64_t G = group + (group & 1);
  for (int64_t g0 = 0; g0 < T; g0 += G) {
    const int64_t g1 = g0 + G < T ? g0 + G : T;
    for (int64_t J = g0; J < T; ++J)
      for (int64_t I = g0; I < g1 && I <= J; I += 2) {
        const int64_t I1 = I + 1 < g1 && I + 1 <= J ? I + 1 : -1;
        order.push_back(make_int4((int)I, (int)I1, (int)J, 0));
      }
  }
}

void tc_pair_items(int64_t n, int64_t m, int fmt, int n_clusters, int group, std::vector<PairItem>& items,
                   std::vector<int2>& split_tiles) {
  items.clear();
  split_tiles.clear();
  const int64_t T = (n + kTB - 1) / kTB, nc = tc_chunks(m, fmt);
  std::vector<int4> order;  // {I0, I1, J, -}
  tc_pair_order(T, group, order);
  const int64_t W = (int64_t)order.size(), C = std::max(1, n_clusters);
  int64_t whole = W, pieces = 1;
  if (W < C) {
    whole = 0;
    pieces = tc_splits_for(W, nc, (int)C);
  } else {
    // the final partial wave's R items: pieces by the wave-cost rule (with a
    // static schedule, R x pieces just above a multiple of the clusters gains
    // nothing, which the rule accounts for)
    const int64_t R = W % C;
    const int64_t s = R > 0 ? tc_splits_for(R, nc, (int)C) : 1;
    if (s > 1) {
      whole = W - R;
      pieces = s;
    }
  }
  pieces = std::max<int64_t>(1, std::min<int64_t>(pieces, std::min<int64_t>(64, nc)));
  const int64_t min_pieces = (nc + tc_max_chunks(fmt) - 1) / tc_max_chunks(fmt);  // exact FP32 accumulation
  for (int64_t t = 0; t < W; ++t) {
    const int4 o = order[t];
    const int64_t np = std::max<int64_t>(min_pieces, t < whole ? 1 : pieces);
    if (np > 1) {
      split_tiles.push_back(make_int2(o.x, o.z));
      if (o.y >= 0) split_tiles.push_back(make_int2(o.y, o.z));
    }
    for (int64_t p = 0; p < np; ++p) {
      PairItem w{};
      w.I0 = o.x;
      w.I1 = o.y;
      w.J = o.z;
      w.c0 = (int32_t)(nc * p / np);
      w.c1 = (int32_t)(nc * (p + 1) / np);
      w.split = np > 1 ? 1 : 0;
      items.push_back(w);
    }
  }
}

// A operands from a_planes (a_block_chunks block-chunks), B halves from
// b_planes (b_block_chunks); the same buffer for one matrix or a batch.
template <class PW, int S, int P>
cudaError_t launch_pair_w(const PW& work, const void* a_planes, int64_t a_block_chunks, const void* b_planes,
                          int64_t b_block_chunks, int64_t chunks_per_item, int64_t n_items, int* status,
                          unsigned long long wait_ns, cudaStream_t st, const PairSync& sync = PairSync{}) {
  constexpr size_t smem = kPairSmem<S, P>;
  static_assert(smem <= 227 * 1024, "ring exceeds shared memory");
  const int clusters = tc_pair_clusters(chunks_per_item);
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  // function attributes are per device: set before every launch
  cudaError_t e =
      cudaFuncSetAttribute(tc_pair_kernel<PW, S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  if (!encode_a_map(&amap, a_planes, 1, a_block_chunks, P) || !encode_bhalf_map(&bmap, b_planes, 1, b_block_chunks, P))
    return cudaErrorInvalidValue;
  const int grid = 2 * (int)std::min<int64_t>(clusters, n_items);
  tc_pair_kernel<PW, S, P><<<grid, 256, smem, st>>>(amap, bmap, work, n_items, status, wait_ns, sync);
  return cudaGetLastError();
}

template <int S, int P>
cudaError_t launch_pair_s(const SubsetDev& sd, const PairItem* items, int64_t n_items, int* status,
                          unsigned long long wait_ns, cudaStream_t st, const PairSync& sync) {
  return launch_pair_w<PairWork, S, P>(PairWork{sd, items}, sd.planes, sd.n_blocks * sd.n_chunks, sd.planes,
                                       sd.n_blocks * sd.n_chunks, sd.n_chunks, n_items, status, wait_ns, st, sync);
}

cudaError_t launch_tc_pair_batch(const PairBatchArgs& a, int* status, unsigned long long wait_ns, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  if (a.n_items > 2147483647LL || a.block_chunks + 8 > 2147483647LL) return cudaErrorInvalidValue;
  const PairBatchWork w{a.subs, a.items, a.jobs, a.units, a.n_units, a.unit_counter, a.ready, a.need};
  const PairRing r = pair_ring(a.max_chunks);
  if (r.per == 2 && r.stages == 4)
    return launch_pair_w<PairBatchWork, 4, 2>(w, a.planes, a.block_chunks, a.planes, a.block_chunks, a.max_chunks,
                                                a.n_items, status, wait_ns, st, a.sync);
  if (r.per == 1 && r.stages == 8)
    return launch_pair_w<PairBatchWork, 8, 1>(w, a.planes, a.block_chunks, a.planes, a.block_chunks, a.max_chunks,
                                                a.n_items, status, wait_ns, st, a.sync);
  if (r.per == 4 && r.stages == 2)
    return launch_pair_w<PairBatchWork, 2, 4>(w, a.planes, a.block_chunks, a.planes, a.block_chunks, a.max_chunks,
                                                a.n_items, status, wait_ns, st, a.sync);
  if (r.per == 3 && r.stages == 3)
    return launch_pair_w<PairBatchWork, 3, 3>(w, a.planes, a.block_chunks, a.planes, a.block_chunks, a.max_chunks,
                                                a.n_items, status, wait_ns, st, a.sync);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_pair(const SubsetDev& sd, const PairItem* items, int64_t n_items, int* status,
                           unsigned long long wait_ns, cudaStream_t st, const PairSync& sync) {
  if (n_items <= 0) return cudaSuccess;
  if (n_items > 2147483647LL) return cudaErrorInvalidValue;
  const PairRing r = pair_ring(sd.n_chunks);
  if (r.per == 2 && r.stages == 4) return launch_pair_s<4, 2>(sd, items, n_items, status, wait_ns, st, sync);
  if (r.per == 1 && r.stages == 8) return launch_pair_s<8, 1>(sd, items, n_items, status, wait_ns, st, sync);
  if (r.per == 4 && r.stages == 2) return launch_pair_s<2, 4>(sd, items, n_items, status, wait_ns, st, sync);
  if (r.per == 3 && r.stages == 3) return launch_pair_s<3, 3>(sd, items, n_items, status, wait_ns, st, sync);
  return cudaErrorInvalidValue;
}

// Default: segments of 64 chunks, lag 2.  Measured on n = 20,000, m =
// 500,000 (items of 7,813 chunks): 138.9 ms against 163.6 ms without (on the
// same GPU; DRAM reads of the unsynchronised waves were about 2.5 times the
// distinct data of a wave); segments of 128: 140.1 ms; n = 4,095: 6.45
// against 6.64 ms.  IBS_TC_PAIR_SYNC=seg,lag overrides, "off" disables.
int2 tc_pair_sync_setting(int64_t chunks_per_item) {
  static const int2 v = [] {
    int seg = 64, lag = 2;
    if (const char* e = getenv("IBS_TC_PAIR_SYNC"))
      if (sscanf(e, "%d,%d", &seg, &lag) != 2) seg = lag = 0;
    // a segment must exceed the ring (partners then stay within one segment
    // of each other) and lag >= 2, which keeps the least advanced CTA and its
    // partner free of waits: the lockstep cannot deadlock
    if (seg < 16 || seg > 65536 || lag < 2 || lag > 1024) seg = lag = 0;
    return make_int2(seg, lag);
  }();
  if (v.x == 0) return v;
  const int per = pair_ring(chunks_per_item).per;
  return make_int2((v.x + per - 1) / per * per, v.y);
}

bool tc_pair_cross_usable(int64_t n_panel, int64_t n_chunks, int fmt) {
  if (tc_pair_mode() < 0 || fmt != kTcFp4) return false;
  if (tc_pair_mode() == 0 && n_chunks < kPairMinChunks) return false;
  const int64_t pb = (n_panel + kTB - 1) / kTB;
  if (pb * n_chunks + 8 > 2147483647LL) return false;  // the tensor map's chunk coordinate is an int
  if (!encode_tiled_fn()) return false;
  return tc_pair_clusters(n_chunks) > 0;
}

cudaError_t launch_tc_pair_cross(const uint8_t* panel, int64_t n_panel, int64_t n_chunks, const uint8_t* qplanes,
                                 int64_t q_blocks_cap, int32_t* const* row_out, int64_t n_rows, const PairItem* items,
                                 int64_t n_items, int* status, cudaStream_t st, const PairSync& sync) {
  if (n_items <= 0) return cudaSuccess;
  const int64_t pb = (n_panel + kTB - 1) / kTB;
  if (n_items > 2147483647LL || q_blocks_cap * n_chunks + 8 > 2147483647LL || pb * n_chunks + 8 > 2147483647LL)
    return cudaErrorInvalidValue;
  const PairCrossWork w{items, row_out, n_rows, n_panel, n_chunks};
  const PairRing r = pair_ring(n_chunks);
  const int64_t qa = q_blocks_cap * n_chunks, pa = pb * n_chunks;
  if (r.per == 2 && r.stages == 4)
    return launch_pair_w<PairCrossWork, 4, 2>(w, qplanes, qa, panel, pa, n_chunks, n_items, status, kWaitLimitNs, st,
                                                sync);
  if (r.per == 1 && r.stages == 8)
    return launch_pair_w<PairCrossWork, 8, 1>(w, qplanes, qa, panel, pa, n_chunks, n_items, status, kWaitLimitNs, st,
                                                sync);
  if (r.per == 4 && r.stages == 2)
    return launch_pair_w<PairCrossWork, 2, 4>(w, qplanes, qa, panel, pa, n_chunks, n_items, status, kWaitLimitNs, st,
                                                sync);
  if (r.per == 3 && r.stages == 3)
    return launch_pair_w<PairCrossWork, 3, 3>(w, qplanes, qa, panel, pa, n_chunks, n_items, status, kWaitLimitNs, st,
                                                sync);
  return cudaErrorInvalidValue;
}

constexpr unsigned kFinalizeSplit = 8;  // CTAs per finalised tile (one CTA per tile reached ~0.8 TB/s)

cudaError_t launch_tc_finalize_tiles(const int2* tiles, int64_t n_tiles, const int32_t* partial, int64_t n,
                                     int32_t* out_counts, double* out_dist, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (n_tiles > 2147483647LL) return cudaErrorInvalidValue;
  tc_finalize_tiles_kernel<<<dim3((unsigned)n_tiles, kFinalizeSplit), 256, 0, st>>>(tiles, partial, n, out_counts,
                                                                                     out_dist);
  return cudaGetLastError();
}

cudaError_t launch_tc_finalize_batch_tiles(const SubsetDev* subs, const int4* tiles, int64_t n_tiles,
                                           cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (n_tiles > 2147483647LL) return cudaErrorInvalidValue;
  tc_finalize_batch_tiles_kernel<<<dim3((unsigned)n_tiles, kFinalizeSplit), 256, 0, st>>>(subs, tiles);
  return cudaGetLastError();
}

int tc_gather_chunks() { return kGatherChunks; }

cudaError_t launch_tc_gather_units(const TcGatherJob* jobs, const int4* units, int64_t n_units, int* unit_counter,
                                   int* ready, int fmt, int ctas, int* status, cudaStream_t st) {
  if (n_units <= 0 || ctas <= 0) return cudaSuccess;
  if (fmt == kTcFp4)
    tc_gather_units_kernel<kTcFp4><<<ctas, kTB, 0, st>>>(jobs, units, n_units, unit_counter, ready, status);
  else
    tc_gather_units_kernel<kTcFp8><<<ctas, kTB, 0, st>>>(jobs, units, n_units, unit_counter, ready, status);
  return cudaGetLastError();
}

int64_t tc_gather_ctas(int64_t n, int64_t nc) {
  return (n + kTB - 1) / kTB * ((nc + kGatherChunks - 1) / kGatherChunks);
}

// Work list of one n-sample matrix for the persistent kernel: the tiles in
// the grouped order, whole, except the tiles of a final partial wave, which
// are split over K into about as many pieces as there are CTAs (their counts
// are added into the partial triangle and finalised per tile).  Tile counts
// below one wave split every tile by the split-count rule.
void tc_single_items(int64_t n, int64_t m, int fmt, int num_sms, int group, std::vector<WorkItem>& items,
                     std::vector<int2>& split_tiles) {
  items.clear();
  split_tiles.clear();
  const int64_t T = (n + kTB - 1) / kTB, nc = tc_chunks(m, fmt);
  std::vector<int2> order;
  tc_tile_order(T, group, order);
  const int64_t W = (int64_t)order.size();
  int64_t whole = W, pieces = 1;
  if (W < num_sms) {
    whole = 0;
    pieces = tc_splits_for(W, nc, num_sms);
  } else {
    const int64_t R = W % num_sms;
    if (R > 0 && R * 4 <= num_sms * 3) {  // a tail wave at most 3/4 full
      whole = W - R;
      pieces = std::max<int64_t>(2, (num_sms + R / 2) / R);
    }
  }
  pieces = std::max<int64_t>(1, std::min<int64_t>(pieces, std::min<int64_t>(64, nc)));
  const int64_t min_pieces = (nc + tc_max_chunks(fmt) - 1) / tc_max_chunks(fmt);  // exact FP32 accumulation
  for (int64_t t = 0; t < W; ++t) {
    const int64_t np = std::max<int64_t>(min_pieces, t < whole ? 1 : pieces);
    if (np > 1) split_tiles.push_back(order[t]);
    for (int64_t p = 0; p < np; ++p) {
      WorkItem w{};
      w.subset = 0;
      w.I = order[t].x;
      w.J = order[t].y;
      w.c0 = (int32_t)(nc * p / np);
      w.c1 = (int32_t)(nc * (p + 1) / np);
      w.split = np > 1 ? 1 : 0;
      items.push_back(w);
    }
  }
}

cudaError_t launch_tc_cross(const uint8_t* panel, int64_t n_panel, int64_t n_chunks, const CrossItem* items,
                            int64_t n_items, int grid, int fmt, int* counter, int* status, cudaStream_t st) {
  return launch_persistent(CrossWork{items, panel, n_panel, n_chunks}, n_items, grid, fmt, n_chunks, counter, status,
                           kWaitLimitNs, st);
}

cudaError_t launch_tc_gather_rows(const RowSrc* rows, int64_t n_rows, int64_t n_chunks, uint8_t* dst,
                                  cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  const int64_t qb = (n_rows + kTB - 1) / kTB;
  if (n_chunks > 2147483647LL || qb > 65535) return cudaErrorInvalidValue;
  tc_gather_rows_kernel<<<dim3((unsigned)n_chunks, (unsigned)qb), 256, 0, st>>>(rows, n_rows, n_chunks, dst);
  return cudaGetLastError();
}

int tc_block_samples() { return kTB; }

cudaError_t probe_tc_mma(int device, int num_sms, int* status_dev, double out[2]) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return e;
  const int n_mma = 20000;
  for (int f = 0; f < 2; ++f) {
    auto kern = f == kTcFp4 ? tc_mma_probe_kernel<kTcFp4> : tc_mma_probe_kernel<kTcFp8>;
    kern<<<num_sms, 128>>>(200, status_dev);  // warm-up
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    kern<<<num_sms, 128>>>(n_mma, status_dev);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double k = f == kTcFp4 ? 64.0 : 32.0;
    out[f == kTcFp4 ? 1 : 0] = 2.0 * num_sms * (double)n_mma * 128.0 * 128.0 * k / (ms * 1e-3) / 1e12;
  }
  return cudaGetLastError();
}

}  // namespace ibs
