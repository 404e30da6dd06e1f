// Linkage disequilibrium: the correlation r of marker pairs within a window,
// on the tensor cores.
//
// The paper's example of bit population counts beyond identity-by-state
// ("Improvements in PLINK 1.9 / Bitwise parallelism") is the correlation
// coefficient r between two markers x and y with missing calls: x_i = +1 for
// a homozygous major call, -1 for a homozygous minor call, 0 for a
// heterozygous or missing call; with S_xy the samples where neither call is
// missing and N = |S_xy|, the paper's form with means over S_xy multiplied
// through by N^2 is
//   r = (N Sxy - Sx Sy) / sqrt((N Sxx - Sx^2) (N Syy - Sy^2)),
// Sx, Sxx, Sy, Syy, Sxy being sums over S_xy.  All six sums are products over
// the sample axis of per-marker indicator rows:
//   V = 1 present,  X = +1 hom A1 / -1 hom A2 / 0,  H = X^2 = 1 homozygous;
//   N = V_a V_b^T,  Sx = X_a V_b^T,  Sy = V_a X_b^T,  Sxx = H_a V_b^T,
//   Syy = V_a H_b^T,  Sxy = X_a X_b^T.
// They are computed relative to A1 and oriented afterwards:
// r_major = s_a s_b r_A1, with s = +1 when A1 is the major allele (#hom A1 >=
// #hom A2 over the marker's calls), which is the same as flipping x.
//
// Markers are the MMA rows (128 per block for A, 64 per half-block for B) and
// samples the K axis (64 per E2M1 chunk).  The variant-major .bed rows already
// have this orientation, so the operand builder only expands 2-bit codes into
// E2M1 values.  Every value is 0 or +-1 and every partial sum an integer of
// magnitude at most the sample count (kept below 2^24), so FP32 accumulation
// is exact.  The numerator and variance terms are formed in int64.  Only the
// reciprocal square root and the products are rounded, in float-float
// arithmetic on the FP32 pipe (see ld_r_value).
//
// One persistent CTA per SM, 12 warps: the copy warp claims (A block, B
// half-block) items of the band |b - a| <= window from a counter and streams
// each item's sample chunks through a ring of 3 stages x 4 chunks (one copy of
// the A block's 3 planes x 4 KiB per chunk, one of the B half-block's 3 planes
// x 2 KiB per chunk, from a second copy of the planes laid out for it); the
// MMA warp issues 6 MMAs (M = 128, N = 64, K = 64) per chunk into six FP32
// accumulators (tensor-memory columns 0, 64, ..., 320; unit scale factors at
// 384..511); warps 4..11 read the accumulators back (two warps per lane
// quarter, 32 columns each) and store r.  Every wait is bounded (2 s of
// %globaltimer), as in the IBS kernels.
#include <algorithm>
#include <vector>

#include "ibs_tc_common.cuh"

namespace ibs {

namespace {

constexpr int kLdPlanes = 3;                         // X, V, H
constexpr int kLdChunkBytes = kLdPlanes * kTileBytes;  // 12 KiB per (marker block, sample chunk)
constexpr int kLdHalfBytes = kTileBytes / 2;         // 64 rows of a plane tile
constexpr int kLdHalfChunkBytes = kLdPlanes * kLdHalfBytes;  // 6 KiB per (half-block, sample chunk)
// A ring stage holds kLdPer chunks of the A block and of the B half-block, one
// bulk copy each (the copy engine spends a fixed time per copy).
constexpr int kLdPer = 4;
constexpr int kLdStageBytes = kLdPer * (kLdChunkBytes + kLdHalfChunkBytes);  // 72 KiB
constexpr int kLdStages = 3;
constexpr size_t kLdSmem = (size_t)kLdStages * kLdStageBytes + 1024;
constexpr int kLdN = 64;                             // B rows (markers) per item
constexpr int kLdQueue = 8;
// warps 0 (copies), 1 (MMAs), 2 (the MMA warp's waits), 3 idle, 4..11 epilogue: two warps per TMEM lane
// quarter, each reading 32 of the item's 64 accumulator columns
constexpr int kLdEpiWarps = 8;
// Hardware barrier between the waiter warp (2) and the MMA warp (1); barrier
// 0 is __syncthreads.
constexpr int kLdBar = 1;
constexpr int kLdThreads = (4 + kLdEpiWarps) * 32;

// Even bits of a 64-bit word packed into 32 bits (bit 2i -> bit i).
__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

// Operand rows: CTA = (sample chunk c, marker block b), thread (row r, half):
// marker b*128 + r, samples c*64 + 32*half .. +31 (8 bytes of the .bed row).
// Writes 16 bytes of each of X, V, H (E2M1: +1 = 0x2, -1 = 0xA) twice: into
// the A layout [block][chunk][plane][128 rows] and into the B layout
// [half-block][chunk][plane][64 rows], so that an item's B operand for a run
// of chunks is one contiguous copy; adds the marker's #hom A1 - #hom A2 over
// these samples to diff.
__global__ void __launch_bounds__(256) ld_planes_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes,
                                                        int64_t n, int64_t m, uint8_t* __restrict__ planes,
                                                        uint8_t* __restrict__ planes_b, int64_t n_chunks,
                                                        int32_t* __restrict__ diff) {
  const int64_t c = blockIdx.x, b = blockIdx.y;
  const int r = threadIdx.x >> 1, half = threadIdx.x & 1;
  const int64_t k = b * kTB + r;
  const int64_t s0 = c * 64 + 32 * half;
  uint32_t a1 = 0, a2 = 0, pres = 0;
  int d = 0;
  if (k < m && s0 < n) {
    const uint8_t* row = packed + k * row_bytes + (s0 >> 2);
    const int64_t left = row_bytes - (s0 >> 2);
    uint64_t w = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) w |= (uint64_t)(q < left ? __ldg(row + q) : 0x55u) << (8 * q);
    const uint32_t lo = even_bits(w), hi = even_bits(w >> 1);  // code bit 0, code bit 1 of 32 samples
    const uint32_t valid = n - s0 >= 32 ? 0xFFFFFFFFu : ((1u << (uint32_t)(n - s0)) - 1u);
    pres = (hi | ~lo) & valid;   // code != 1
    a1 = ~hi & ~lo & valid;      // code 0, homozygous A1
    a2 = hi & lo & valid;        // code 3, homozygous A2
    d = __popc(a1) - __popc(a2);
  }
  d += __shfl_xor_sync(0xffffffffu, d, 1);  // the row's two halves (all lanes converged here)
  if (half == 0 && k < m && d != 0) atomicAdd(diff + k, d);
  uint32_t wx[4], wv[4], wh[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const uint32_t s1 = nib8(a1 >> (8 * g)), s2 = nib8(a2 >> (8 * g)), sv = nib8(pres >> (8 * g));
    wx[g] = ((s1 | s2) << 1) | (s2 << 3);
    wv[g] = sv << 1;
    wh[g] = (s1 | s2) << 1;
  }
  uint8_t* base = planes + (size_t)(b * n_chunks + c) * kLdChunkBytes + tile_off(r, 16 * half);
  *reinterpret_cast<uint4*>(base + 0 * kTileBytes) = make_uint4(wx[0], wx[1], wx[2], wx[3]);
  *reinterpret_cast<uint4*>(base + 1 * kTileBytes) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  *reinterpret_cast<uint4*>(base + 2 * kTileBytes) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
  uint8_t* bb = planes_b + (size_t)((b * 2 + (r >> 6)) * n_chunks + c) * kLdHalfChunkBytes + tile_off(r & 63, 16 * half);
  *reinterpret_cast<uint4*>(bb + 0 * kLdHalfBytes) = make_uint4(wx[0], wx[1], wx[2], wx[3]);
  *reinterpret_cast<uint4*>(bb + 1 * kLdHalfBytes) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  *reinterpret_cast<uint4*>(bb + 2 * kLdHalfBytes) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
}

// r from the six exact sums, oriented by the two markers' signs; NaN when N = 0
// or a variance term is 0.  The numerator and the variance terms are exact
// int64 values below 2^48 (N < 2^24); they are split exactly into float-float
// pairs, and r = num / sqrt(va vb) is formed in float-float arithmetic on the
// FP32 pipe (GB300 runs FP32 at 64x its FP64 rate): the product va vb, an
// rsqrtf seed (relative error near 2^-22) refined by one Newton step whose
// residual 1 - P y^2 is taken in float-float, and the product with the
// numerator.  Error: about 1.5 * 2^-44 from the Newton step plus a few 2^-46
// from the float-float operations, well under 1e-12 relative.
struct FF {
  float hi, lo;
};

// Error-free sum (Knuth): s + e == a + b.
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// x (|x| < 2^48) as an exact float-float: x = h 2^24 + l with 0 <= l < 2^24.
__device__ __forceinline__ FF ff_from_i48(long long x) {
  const long long h = x >> 24;  // floor: |h| < 2^24
  const int l = (int)(x - (h << 24));
  return ff_two_sum(__fmul_rn((float)(int)h, 16777216.0f), (float)l);
}

// a * b in float-float (products exact by FMA, cross terms added once).
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, e);
  return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

__device__ __forceinline__ double ld_r_value(int32_t N, int32_t sx, int32_t sy, int32_t sxx, int32_t syy,
                                             int32_t sxy, int sign) {
  const long long n = N;
  const long long va = n * sxx - (long long)sx * sx, vb = n * syy - (long long)sy * sy;
  if (N == 0 || va == 0 || vb == 0) return __longlong_as_double(0x7ff8000000000000LL);
  const long long num = n * sxy - (long long)sx * sy;
  const FF P = ff_mul(ff_from_i48(va), ff_from_i48(vb));
  const float y0 = rsqrtf(P.hi);
  const float q = __fmul_rn(y0, y0);
  const FF w = ff_mul(P, FF{q, __fmaf_rn(y0, y0, -q)});  // P y0^2, near 1
  const float t = __fsub_rn(__fsub_rn(1.0f, w.hi), w.lo);  // 1 - P y0^2 (the first difference is exact)
  const FF y = ff_two_sum(y0, __fmul_rn(__fmul_rn(y0, t), 0.5f));  // one Newton step
  const FF r = ff_mul(ff_from_i48(sign * num), y);
  return (double)r.hi + (double)r.lo;
}

struct LdArgs {
  const uint8_t* planes;    // A layout
  const uint8_t* planes_b;  // B layout
  int64_t n_chunks, m, window;
  const int2* items;  // (A marker block, B half-block)
  int64_t n_items;
  const int32_t* diff;
  double* out_r;
  int32_t* out_n;
  int* counter;
  int* status;
};

__global__ void __launch_bounds__(kLdThreads, 1) tc_ld_kernel(const LdArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kLdStages], empty[kLdStages], tfull, tempty, drain;
  __shared__ __align__(8) uint64_t qfull[kLdQueue], qempty[kLdQueue];
  __shared__ int64_t q_item[kLdQueue];
  __shared__ int64_t s_item[2];  // the waiter's hand-over of items to the MMA warp
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* status = args.status;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kLdStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kLdQueue; ++s) {
      mbar_init(&qfull[s], 1);
      mbar_init(&qempty[s], 1 + kLdEpiWarps);  // the waiter warp and the epilogue warps
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, kLdEpiWarps);
    mbar_init(&drain, 1);
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
  if (warp >= 4 && warp < 8) tmem_fill_unit_scales(tmem, warp - 4);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  auto fail = [&](bool cond) {
    if (lane == 0 && cond) {
      atomicExch(status, kDevTimeout);
      atomicExch(&abort_flag, 1);
    }
  };
  auto aborted = [&]() { return __any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0); };
  auto queue_get = [&](uint32_t e, int64_t& it) {
    const int qs = (int)(e % kLdQueue);
    const bool ok = mbar_wait_bounded(&qfull[qs], (e / kLdQueue) & 1u);
    if (__any_sync(0xffffffffu, !ok)) return false;
    it = *(volatile int64_t*)&q_item[qs];
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&qempty[qs])) : "memory");
    return true;
  };
  const int64_t nk = args.n_chunks;

  if (warp == 0) {
    uint32_t g = 0;
    for (uint32_t e = 0;; ++e) {
      int64_t it = 0;
      if (lane == 0) it = atomicAdd(args.counter, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      const bool last = it >= args.n_items;
      const int qs = (int)(e % kLdQueue);
      const bool qok = e < (uint32_t)kLdQueue || mbar_wait_bounded(&qempty[qs], ((e / kLdQueue) - 1) & 1u);
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
      const int2 item = args.items[it];
      const uint8_t* ablk = args.planes + (size_t)item.x * nk * kLdChunkBytes;
      const uint8_t* bblk = args.planes_b + (size_t)item.y * nk * kLdHalfChunkBytes;
      bool stop = false;
      for (int64_t k = 0; k < nk; k += kLdPer, ++g) {
        const int s = (int)(g % kLdStages);
        const bool ok = g < (uint32_t)kLdStages || mbar_wait_bounded(&empty[s], ((g / kLdStages) - 1) & 1u);
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
          uint8_t* dst = ring + (size_t)s * kLdStageBytes;
          mbar_arrive_expect_tx(&full[s], kLdStageBytes);
          bulk_g2s(dst, ablk + (size_t)k * kLdChunkBytes, kLdPer * kLdChunkBytes, &full[s]);
          bulk_g2s(dst + kLdPer * kLdChunkBytes, bblk + (size_t)k * kLdHalfChunkBytes, kLdPer * kLdHalfChunkBytes,
                   &full[s]);
        }
        __syncwarp();
      }
      if (stop) break;
    }
  } else if (warp == 1) {
    // MMA warp.  It never waits on memory itself: a thread with MMAs in flight
    // that polls a barrier or loads from memory stalls until they complete,
    // which would drain the tensor pipe at every ring stage.  Warp 2 takes the
    // items from the queue and does every wait; it hands each item over
    // through s_item and releases this warp once per stage through hardware
    // barrier kLdBar (both warps execute bar.sync once per hand-over and once
    // per stage, in the same order; every item covers all chunks).
    uint32_t g = 0;
    const uint32_t sf = tmem + kSfCol;
    for (uint32_t e = 0;; ++e) {
      asm volatile("bar.sync %0, 64;" ::"n"(kLdBar) : "memory");
      const int64_t it = *(volatile int64_t*)&s_item[e & 1u];
      if (it < 0) break;
      for (int64_t k0 = 0; k0 < nk; k0 += kLdPer, ++g) {
        asm volatile("bar.sync %0, 64;" ::"n"(kLdBar) : "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int s = (int)(g % kLdStages);
        if (lane == 0) {
          const uint32_t st0 = smem_addr(ring + (size_t)s * kLdStageBytes);
#pragma unroll
          for (int c = 0; c < kLdPer; ++c) {
            const uint32_t a0 = st0 + c * kLdChunkBytes, b0 = st0 + kLdPer * kLdChunkBytes + c * kLdHalfChunkBytes;
            const uint64_t aX = umma_desc(a0), aV = umma_desc(a0 + kTileBytes), aH = umma_desc(a0 + 2 * kTileBytes);
            const uint64_t bX = umma_desc(b0), bV = umma_desc(b0 + kLdHalfBytes),
                           bH = umma_desc(b0 + 2 * kLdHalfBytes);
            const uint32_t acc = k0 + c > 0 ? 1u : 0u;
            umma<kTcFp4, kLdN>(tmem + 0 * kLdN, aV, bV, acc, sf);  // N
            umma<kTcFp4, kLdN>(tmem + 1 * kLdN, aX, bV, acc, sf);  // Sx
            umma<kTcFp4, kLdN>(tmem + 2 * kLdN, aV, bX, acc, sf);  // Sy
            umma<kTcFp4, kLdN>(tmem + 3 * kLdN, aH, bV, acc, sf);  // Sxx
            umma<kTcFp4, kLdN>(tmem + 4 * kLdN, aV, bH, acc, sf);  // Syy
            umma<kTcFp4, kLdN>(tmem + 5 * kLdN, aX, bX, acc, sf);  // Sxy
          }
          umma_commit(&empty[s]);
        }
        __syncwarp();
      }
      if (lane == 0) umma_commit(&tfull);
      __syncwarp();
    }
    if (lane == 0) umma_commit(&drain);
    __syncwarp();
    const bool drained = mbar_wait_bounded(&drain, 0);
    if (lane == 0 && !drained) atomicExch(status, kDevTimeout);
  } else if (warp == 2) {
    // Waiter: for each item from the queue, hand it over; before its first
    // stage wait (bounded) until the epilogue has read the previous item's
    // accumulators, and before each stage until its operands have landed;
    // then release the MMA warp.  After a failed wait or another role's abort
    // it stops waiting but keeps releasing the current item's stages (the MMA
    // warp runs them out on stale operands; the call reports IBS_ETIMEOUT),
    // then hands over the end (-1).
    uint32_t g = 0;
    bool dead = false;
    for (uint32_t e = 0;; ++e) {
      int64_t it = -1;
      if (!dead && !queue_get(e, it)) {
        fail(true);
        dead = true;
      }
      if (dead) it = -1;
      if (lane == 0) s_item[e & 1u] = it;
      __syncwarp();
      asm volatile("bar.sync %0, 64;" ::"n"(kLdBar) : "memory");
      if (it < 0) break;
      for (int64_t k0 = 0; k0 < nk; k0 += kLdPer, ++g) {
        if (!dead) {
          bool ok = k0 > 0 || e == 0 || mbar_wait_bounded(&tempty, (e - 1) & 1u);
          if (ok) ok = mbar_wait_bounded(&full[(int)(g % kLdStages)], (g / kLdStages) & 1u);
          if (__any_sync(0xffffffffu, !ok)) {
            fail(true);
            dead = true;
          } else if (aborted()) {
            dead = true;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync %0, 64;" ::"n"(kLdBar) : "memory");
      }
    }
  } else if (warp >= 4) {
    const int quarter = warp & 3, colhalf = (warp - 4) >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (uint32_t e = 0;; ++e) {
      int64_t it;
      if (!queue_get(e, it)) {
        fail(true);
        break;
      }
      if (it < 0) break;
      const bool ok = mbar_wait_bounded(&tfull, e & 1u);
      if (__any_sync(0xffffffffu, !ok) || aborted()) {
        fail(true);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int2 item = args.items[it];
      const int64_t a = (int64_t)item.x * kTB + row;
      const int sa = a < args.m ? (args.diff[a] >= 0 ? 1 : -1) : 1;
#pragma unroll 1
      for (int cg = 2 * colhalf; cg < 2 * colhalf + 2; ++cg) {
        uint32_t v[6][16];
#pragma unroll
        for (int q = 0; q < 6; ++q) tmem_ld16(lane_base + q * kLdN + cg * 16, v[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cg == 2 * colhalf + 1) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty)) : "memory");
        }
        if (a >= args.m) continue;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int64_t b = (int64_t)item.y * kLdN + cg * 16 + u;
          const int64_t d = b - a - 1;
          if (d < 0 || d >= args.window || b >= args.m) continue;
          const int32_t N = __float2int_rn(__uint_as_float(v[0][u]));
          const int sb = args.diff[b] >= 0 ? 1 : -1;
          const double r = ld_r_value(N, __float2int_rn(__uint_as_float(v[1][u])),
                                      __float2int_rn(__uint_as_float(v[2][u])),
                                      __float2int_rn(__uint_as_float(v[3][u])),
                                      __float2int_rn(__uint_as_float(v[4][u])),
                                      __float2int_rn(__uint_as_float(v[5][u])), sa * sb);
          args.out_r[a * args.window + d] = r;
          if (args.out_n) args.out_n[a * args.window + d] = N;
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

// Slots whose second marker lies past the last one: r = NaN, N = 0.
__global__ void ld_fill_tail_kernel(int64_t m, int64_t window, double* __restrict__ out_r,
                                    int32_t* __restrict__ out_n) {
  const int64_t a0 = m > window ? m - window : 0;
  const int64_t total = (m - a0) * window;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = a0 + t / window, d = t % window;
    if (a + 1 + d < m) continue;
    out_r[a * window + d] = __longlong_as_double(0x7ff8000000000000LL);
    if (out_n) out_n[a * window + d] = 0;
  }
}

}  // namespace

// Sample chunks: ceil(n / 64), padded to a multiple of kLdPer with zero chunks.
static int64_t ld_chunks(int64_t n) { return ((n + 63) / 64 + kLdPer - 1) / kLdPer * kLdPer; }

size_t ld_planes_bytes(int64_t n, int64_t m) {  // A layout, then B layout
  return (size_t)((m + kTB - 1) / kTB) * (size_t)ld_chunks(n) * (kLdChunkBytes + 2 * kLdHalfChunkBytes);
}

// Items of the band: (A block I of 128 markers, B half-block j of 64 markers)
// holding at least one pair a < b <= a + window, in order of I then j.
void ld_items(int64_t m, int64_t window, std::vector<int2>& items) {
  items.clear();
  const int64_t nb = (m + kTB - 1) / kTB, nh = (m + kLdN - 1) / kLdN;
  for (int64_t I = 0; I < nb; ++I) {
    const int64_t a_min = I * kTB, a_max = std::min<int64_t>(a_min + kTB - 1, m - 1);
    const int64_t j0 = std::max<int64_t>(0, (a_min + 1) / kLdN);
    const int64_t j1 = std::min<int64_t>(nh - 1, (a_max + window) / kLdN);
    for (int64_t j = j0; j <= j1; ++j) items.push_back(make_int2((int)I, (int)j));
  }
}

cudaError_t launch_ld(const uint8_t* packed, int64_t n, int64_t m, int64_t window, uint8_t* planes, int32_t* diff,
                      const int2* items, int64_t n_items, int* counter, double* out_r, int32_t* out_n,
                      int* status, int num_sms, cudaStream_t st) {
  const int64_t nc = ld_chunks(n), nb = (m + kTB - 1) / kTB;
  if (nc > 2147483647LL || nb > 65535 || n_items > 2147483647LL - num_sms) return cudaErrorInvalidValue;
  uint8_t* planes_b = planes + (size_t)nb * nc * kLdChunkBytes;
  cudaError_t e = cudaMemsetAsync(diff, 0, (size_t)m * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  ld_planes_kernel<<<dim3((unsigned)nc, (unsigned)nb), 256, 0, st>>>(packed, (n + 3) / 4, n, m, planes, planes_b, nc,
                                                                      diff);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tc_ld_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLdSmem)) !=
      cudaSuccess)
    return e;
  LdArgs args{planes, planes_b, nc, m, window, items, n_items, diff, out_r, out_n, counter, status};
  if (n_items > 0) {
    tc_ld_kernel<<<(int)std::min<int64_t>(num_sms, n_items), kLdThreads, kLdSmem, st>>>(args);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  ld_fill_tail_kernel<<<64, 256, 0, st>>>(m, window, out_r, out_n);
  return cudaGetLastError();
}

}  // namespace ibs
