// Tensor-core form of the pair counts (tcgen05, FP8 indicator GEMMs).
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
// are exact in FP8 (E4M3), every product is exact, and every partial sum is an
// integer of magnitude at most the marker count, far below 2^24, so FP32
// accumulation is exact.  Four 128 x 128 x 32 MMAs per 32 markers.
//
// Layout: one (128-sample block, 32-marker chunk) is 4 planes x 4 KiB, each
// plane a 128 x 32 byte tile in the tensor core's canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, the two core matrices of a
// row group 128 bytes apart (leading byte offset) and row groups 256 bytes
// apart (stride byte offset).  A CTA computes one 128 x 128 tile of pairs:
// warp 0 streams chunks of the row and column blocks through a 4-stage
// shared-memory ring with TMA bulk copies, warp 1 issues the MMAs into three
// FP32 accumulators in tensor memory (columns 0, 128, 256) and frees each
// stage with tcgen05.commit, and after the last chunk all four warps read the
// accumulators back (tcgen05.ld), decode the counts and store them.  Warp 0
// (copies) and warp 1 (MMAs) run their loops with all 32 lanes in step and
// one lane issuing, so no lane of theirs is parked in another wait.
//
// Every wait is bounded (2 s of %globaltimer); on expiry the status word is
// set, and the CTA still waits (bounded) for its MMAs and frees its tensor
// memory before returning.
#include <cstdlib>
#include <vector>

#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {

namespace {

constexpr int kTB = 128;                          // samples per block (tile edge)
constexpr int kTK = 32;                           // markers per chunk (one MMA K step)
constexpr int kTPlanes = 4;                       // V, U, Q, R
constexpr int kTileBytes = kTB * kTK;             // one plane of one chunk: 4 KiB
constexpr int kTChunkBytes = kTPlanes * kTileBytes;  // 16 KiB per (block, chunk)
constexpr int kTThreads = 128;
constexpr size_t tc_smem(int stages) { return (size_t)stages * 2 * kTChunkBytes + 1024; }
constexpr uint32_t kTmemCols = 512;               // 3 x 128 used
constexpr uint8_t kFp8One = 0x38, kFp8MinusOne = 0xB8;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version
  return d;                          // no swizzle
}

// E4M3 x E4M3 -> F32, K-major A and B, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Byte offset of (sample row r, marker k) inside one 128 x 32 canonical tile.
__device__ __forceinline__ int tile_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15);
}

// ---------------------------------------------------------------------------
// Transpose: packed .bed rows -> FP8 planes.  CTA = (chunk c of 32 markers,
// block b of 128 samples), 8 warps of 16 samples.  Lane t of a warp holds one
// 32-bit word of .bed row t (its 16 samples' 2-bit codes); a 32 x 32 bit
// transpose by warp shuffles leaves lane 2k with the low code bits and lane
// 2k+1 with the high code bits of sample k at the 32 markers.  After one
// exchange each lane of the pair has both words; lane 2k writes markers 0..15
// and lane 2k+1 markers 16..31 of the sample's four FP8 plane rows.  Bits
// become bytes with a multiply: (x * 0x204081) & 0x01010101 spreads 4 bits
// to 4 bytes, and a second multiply turns each 1 into the FP8 value.
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

__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }

__global__ void __launch_bounds__(256) tc_planes_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes,
                                                        int64_t n, int64_t m, uint8_t* __restrict__ planes,
                                                        int64_t n_chunks) {
  const int64_t c = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t marker = c * kTK + lane;
  const int64_t s0 = b * kTB + warp * 16;  // first sample of this warp
  const int64_t byte0 = s0 >> 2;           // 4 bytes = 16 samples
  uint32_t x = 0x55555555u;                // "missing" for every slot
  if (marker < m && s0 < n) {
    const uint8_t* row = packed + marker * row_bytes;
    if (row_bytes % 4 == 0 && (reinterpret_cast<uintptr_t>(packed) & 3) == 0 && byte0 + 4 <= row_bytes) {
      x = __ldg(reinterpret_cast<const uint32_t*>(row + byte0));
    } else {
      x = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) x |= (uint32_t)(byte0 + q < row_bytes ? __ldg(row + byte0 + q) : 0x55u) << (8 * q);
    }
  }
  x = tc_transpose32(x, lane);
  const uint32_t partner = __shfl_xor_sync(0xffffffffu, x, 1);
  const bool odd = (lane & 1) != 0;
  const uint32_t H = odd ? x : partner, L = odd ? partner : x;
  const int r = warp * 16 + (lane >> 1);  // row inside the 128-sample block
  const bool valid = b * kTB + r < n;
  // this lane's 16 markers: bits 0..15 (even lane) or 16..31 (odd lane)
  const int sh = odd ? 16 : 0;
  const uint32_t h = (H >> sh) & 0xFFFFu, l = (L >> sh) & 0xFFFFu;
  const uint32_t vb = valid ? (h | ~l) & 0xFFFFu : 0u;  // present
  const uint32_t pb = vb & h & ~l;                       // het
  const uint32_t qb = vb & h & l;                        // hom A2
  const uint32_t rb = vb & ~h & ~l;                      // hom A1
  uint32_t wv[4], wu[4], wq[4], wr[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const uint32_t sv = spread4((vb >> (4 * g)) & 0xFu), sp = spread4((pb >> (4 * g)) & 0xFu);
    wv[g] = sv * kFp8One;
    wu[g] = sv * kFp8One | sp * 0x80u;  // heterozygous: sign bit -> -1
    wq[g] = spread4((qb >> (4 * g)) & 0xFu) * kFp8One;
    wr[g] = spread4((rb >> (4 * g)) & 0xFu) * kFp8One;
  }
  uint8_t* base = planes + (size_t)(b * n_chunks + c) * kTChunkBytes + tile_off(r, odd ? 16 : 0);
  *reinterpret_cast<uint4*>(base + 0 * kTileBytes) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  *reinterpret_cast<uint4*>(base + 1 * kTileBytes) = make_uint4(wu[0], wu[1], wu[2], wu[3]);
  *reinterpret_cast<uint4*>(base + 2 * kTileBytes) = make_uint4(wq[0], wq[1], wq[2], wq[3]);
  *reinterpret_cast<uint4*>(base + 3 * kTileBytes) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
}

// ---------------------------------------------------------------------------
// Pair tile kernel (kTStages-deep ring).
template <int kTStages>
__global__ void __launch_bounds__(kTThreads, 1)
    tc_tri_kernel(const uint8_t* __restrict__ planes, int64_t n, int64_t n_blocks, int64_t n_chunks, int splits,
                  int32_t* __restrict__ out_counts, double* __restrict__ out_dist, int32_t* __restrict__ partial,
                  int square, int* status, int piece, const int2* __restrict__ tile_list) {
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

  const int lane = threadIdx.x & 31;
  if (warp == 0) {
    // Producer warp: every lane waits for a free stage together (no lane of
    // this warp sits in another wait), lane 0 issues the bulk copies.
    for (int64_t k = 0; k < nk; ++k) {
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
        // Each 16 KiB chunk goes as several smaller bulk copies, which the
        // copy engine keeps in flight together.
        for (int off = 0; off < kTChunkBytes; off += piece) {
          bulk_g2s(dst + off, rowblk + (size_t)(c0 + k) * kTChunkBytes + off, piece, &full[s]);
          if (!same)
            bulk_g2s(dst + kTChunkBytes + off, colblk + (size_t)(c0 + k) * kTChunkBytes + off, piece, &full[s]);
        }
      }
      __syncwarp();
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
        const uint32_t acc = k > 0 ? 1u : 0u;
        umma(tmem + 0, umma_desc(a0 + 0 * kTileBytes), umma_desc(b0 + 0 * kTileBytes), acc);    // V V^T
        umma(tmem + 128, umma_desc(a0 + 1 * kTileBytes), umma_desc(b0 + 1 * kTileBytes), acc);  // U U^T
        umma(tmem + 256, umma_desc(a0 + 2 * kTileBytes), umma_desc(b0 + 3 * kTileBytes), acc);  // Q R^T
        umma(tmem + 256, umma_desc(a0 + 3 * kTileBytes), umma_desc(b0 + 2 * kTileBytes), 1u);   // + R Q^T
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
        if (out_dist) d = nn == 0 ? __longlong_as_double(0x7ff8000000000000LL)
                                  : (double)(i1 + 2 * i0) / (2.0 * (double)nn);
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

}  // namespace

size_t tc_planes_bytes(int64_t n, int64_t m) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = (m + kTK - 1) / kTK;
  return (size_t)nb * (size_t)nc * kTChunkBytes;
}

// Split count over the marker axis.  All tiles of one launch cost the same,
// so the launch takes ceil(tiles * s / SMs) waves of 1/s of a tile each; pick
// the s in 1..64 (at least one chunk per split) with the fewest tile-equivalents,
// charging splits 3% for the partial-count atomics and the finalisation pass.
int tc_splits_for(int64_t tiles, int64_t n_chunks, int num_sms) {
  int best = 1;
  double best_cost = 1e300;
  for (int s = 1; s <= 64 && s <= n_chunks; ++s) {
    const double waves = (double)((tiles * s + num_sms - 1) / num_sms);
    const double cost = waves / s * (s > 1 ? 1.03 : 1.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = s;
    }
  }
  return best;
}

cudaError_t launch_tc_planes(const uint8_t* packed, int64_t n, int64_t m, uint8_t* planes, cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = (m + kTK - 1) / kTK;
  if (nc > 2147483647LL || nb > 65535) return cudaErrorInvalidValue;
  tc_planes_kernel<<<dim3((unsigned)nc, (unsigned)nb), 256, 0, st>>>(packed, (n + 3) / 4, n, m, planes, nc);
  return cudaGetLastError();
}

cudaError_t launch_tc_pairs(const uint8_t* planes, int64_t n, int64_t m, int splits, int32_t* out_counts,
                            double* out_dist, int32_t* partial, bool square, int* status, const int2* tile_list,
                            cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = (m + kTK - 1) / kTK;
  const int64_t tiles = nb * (nb + 1) / 2;
  const int64_t grid = tiles * splits;
  if (grid > 2147483647LL) return cudaErrorInvalidValue;
  static const int stages = [] {
    const char* e = getenv("IBS_TC_STAGES");
    return (e && e[0] == '6') ? 6 : 4;
  }();
  static const int piece = [] {
    const char* e = getenv("IBS_TC_PIECE");
    const int v = e ? atoi(e) : kTChunkBytes;
    return (v >= 512 && v <= kTChunkBytes && kTChunkBytes % v == 0 && v % 16 == 0) ? v : kTChunkBytes;
  }();
  cudaError_t e;
  if (stages == 6) {
    e = cudaFuncSetAttribute(tc_tri_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(6));
    if (e != cudaSuccess) return e;
    tc_tri_kernel<6><<<(unsigned)grid, kTThreads, tc_smem(6), st>>>(planes, n, nb, nc, splits, out_counts, out_dist,
                                                                   partial, square ? 1 : 0, status, piece, tile_list);
  } else {
    e = cudaFuncSetAttribute(tc_tri_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(4));
    if (e != cudaSuccess) return e;
    tc_tri_kernel<4><<<(unsigned)grid, kTThreads, tc_smem(4), st>>>(planes, n, nb, nc, splits, out_counts, out_dist,
                                                                   partial, square ? 1 : 0, status, piece, tile_list);
  }
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

int64_t tc_chunks(int64_t m) { return (m + kTK - 1) / kTK; }

}  // namespace ibs
