// Genomic relationship matrix (GCTA), on the tensor cores.
//
// The paper's "Partial sum lookup" section writes the GCTA relationship
// matrix as a weighted distance: per marker i, with p the frequency of the
// counted allele (A1) over the marker's non-missing calls and x its count in a
// call, a pair of samples whose calls are both present adds
//   (x_j - 2p)(x_k - 2p) / (2p(1 - p)),
// and the sum is divided by the number of markers where both calls are present
// (markers with p = 0 or 1 are left out).  With z = (x - 2p) / sqrt(2p(1 - p))
// (0 for a missing call or an unused marker) and V' = 1 where the call is
// present and the marker used, that is
//   A = (Z Z^T) / (V' V'^T),
// two products over the marker axis.  V' V'^T is exact (0/1 values, integer
// sums below 2^24 in FP32).  Z is real: each value is carried as a pair of
// FP16 numbers z = hi + lo (hi = fp16(z), lo = fp16(z - hi), about 22
// significant bits), Z Z^T ~ hi hi^T + hi lo^T + lo hi^T (the dropped lo lo^T
// is below 2^-22 of each term), accumulated by tcgen05.mma.kind::f16 in FP32.
//
// Accumulation.  An FP32 accumulator that runs over all m markers loses up to
// an ulp of its running sum per MMA, a relative error growing with m/16.  So
// the numerator restarts every kGrmSeg chunks (128 markers): the MMA warp
// alternates between two numerator banks, and the epilogue warps fold each
// finished segment into a float-float sum (the high word in tensor memory, the
// low word in registers) by an error-free two-sum, while the MMAs of the next
// segment run.  The error left is that of one segment's 3 x 8 MMA
// accumulations plus the FP16 split, independent of m.
//
// Layout: samples are the MMA rows (128 per block), markers the K axis (16 per
// FP16 chunk); a pair of chunks of one block holds hi and lo of each chunk
// (128 x 32-byte FP16 tiles) and V' of its 32 markers as one E4M3 tile, in
// the canonical K-major layout (20 KiB).  Tensor memory: numerator banks at
// columns 0 and 128, the count at 256, the float-float high words at 384.
// One persistent CTA per SM, 10 warps: warp 8 claims triangle tiles in the
// grouped order and streams both blocks' chunks through a ring of two stages
// of four chunks (one 40 KiB bulk copy per block and stage: the copy engine
// spends a fixed time per copy, measured near 340 cycles, so one chunk per
// stage ran 1.6x slower); warp 9 issues 3 kind::f16 MMAs per chunk and one
// kind::f8f6f4 MMA (the counts) per pair; warps 0..7 fold segments (warp w:
// TMEM lanes of quarter w % 4, columns 64 (w / 4) .. +63) and store A.  Every
// wait is bounded (2 s of %globaltimer).
#include <algorithm>
#include <cuda_fp16.h>
#include <vector>

#include "ibs_tc_common.cuh"

namespace ibs {

namespace {

constexpr int kGrmK = 16;                                // markers per FP16 chunk
// Operand unit: a pair of chunks (32 markers) of one 128-sample block, 20 KiB:
// hi and lo of the first chunk, hi and lo of the second (FP16, 4 KiB tiles),
// then V' for all 32 markers as one E4M3 tile (1.0 = 0x38; kind::f8f6f4 takes
// 32 markers per MMA, so the pair counts cost one MMA and 4 KiB per pair).
constexpr int kGrmPairBytes = 5 * kTileBytes;            // 20 KiB
constexpr int kGrmChunkBytes = kGrmPairBytes / 2;        // 10 KiB per chunk on average
constexpr int kGrmVpOff = 4 * kTileBytes;                // V' tile within a pair
constexpr int kGrmPad = 4;                               // chunk count padded to a multiple of this
constexpr int kGrmQueue = 8;
constexpr int kGrmSeg = 8;                               // chunks per numerator segment
static_assert(kGrmSeg % kGrmPad == 0, "a ring stage never straddles two segments");
constexpr int kGrmEpiWarps = 8;
constexpr int kGrmThreads = (kGrmEpiWarps + 3) * 32;
constexpr int kGrmCopyWarp = kGrmEpiWarps, kGrmMmaWarp = kGrmEpiWarps + 1, kGrmWaitWarp = kGrmEpiWarps + 2;
// Hardware barrier between the waiter warp and the MMA warp (barrier 0 is
// __syncthreads): both execute bar.sync once per item hand-over and once per
// ring stage, in the same order.
constexpr int kGrmBar = 1;
constexpr uint32_t kColNum = 0, kColCnt = 256, kColHi = 384;

// FP16 x FP16 -> F32 (kind::f16): D format F32 (bit 4), A and B formats F16
// (0 at bits 7 and 10), K-major A and B, N = 128 (N >> 3 at bit 17), M = 128
// (M >> 4 at bit 24).
constexpr uint32_t kIdescF16 = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdescF16), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// Per marker: the A1 frequency and, for the three called codes, hi and lo of
// z; table[i] = {hi, lo} of hom A1 (x = 2), het (x = 1), hom A2 (x = 0), then
// V' (1.0 when 0 < p < 1) and a pad, as FP16 bit patterns.  The codes are
// counted by population counts over 16 genotypes per 32-bit word (codes 0 hom
// A1, 1 missing, 2 het, 3 hom A2 in bit pairs); p and z in FP64.
__device__ __forceinline__ void count_codes(uint32_t w, uint32_t valid, int& hom1, int& het, int& miss) {
  const uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;
  hom1 += __popc(~(lo | hi) & valid);
  het += __popc(hi & ~lo & valid);
  miss += __popc(lo & ~hi & valid);
}

// A warp takes 32 consecutive markers: it counts each row with all lanes,
// lane j keeps marker j's totals, and the 32 lanes then form p and z in FP64
// side by side (GB300's FP64 rate is low, so the arithmetic is spread over
// the lanes rather than left to one).
__global__ void grm_freq_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes, int64_t n, int64_t m,
                                uint16_t* __restrict__ table) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  // rows are 16-byte aligned when the row length is (the buffer base is)
  const bool vec = (row_bytes & 15) == 0 && (reinterpret_cast<uintptr_t>(packed) & 15) == 0;
  for (int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; i0 < m; i0 += warps * 32) {
    int my_hom1 = 0, my_het = 0, my_miss = 0;
    const int rows = (int)(m - i0 < 32 ? m - i0 : 32);
    for (int j = 0; j < rows; ++j) {
      const uint8_t* row = packed + (i0 + j) * row_bytes;
      int hom1 = 0, het = 0, miss = 0;
      if (vec) {
        const uint4* r4 = reinterpret_cast<const uint4*>(row);
        for (int64_t q = lane; q < row_bytes / 16; q += 32) {
          const uint4 v = __ldg(r4 + q);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int64_t s0 = q * 64 + t * 16;  // first sample of the word
            const uint32_t valid =
                s0 + 16 <= n ? 0x55555555u : (s0 >= n ? 0u : 0x55555555u >> (2 * (s0 + 16 - n)));
            count_codes(w[t], valid, hom1, het, miss);
          }
        }
      } else {
        for (int64_t q = lane; q < row_bytes; q += 32) {
          const int64_t s0 = q * 4;
          const uint32_t valid = s0 + 4 <= n ? 0x55u : 0x55u >> (2 * (s0 + 4 - n));
          count_codes(__ldg(row + q), valid, hom1, het, miss);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        hom1 += __shfl_xor_sync(0xffffffffu, hom1, o);
        het += __shfl_xor_sync(0xffffffffu, het, o);
        miss += __shfl_xor_sync(0xffffffffu, miss, o);
      }
      if (lane == j) {
        my_hom1 = hom1;
        my_het = het;
        my_miss = miss;
      }
    }
    if (lane < rows) {
      const int64_t i = i0 + lane;
      const int64_t calls = n - my_miss;
      const double p = calls > 0 ? (double)(2 * (int64_t)my_hom1 + my_het) / (2.0 * (double)calls) : 0.0;
      const bool used = p > 0.0 && p < 1.0;
      const double sc = used ? 1.0 / sqrt(2.0 * p * (1.0 - p)) : 0.0;
      uint16_t t[8];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double z = used ? ((double)(2 - c) - 2.0 * p) * sc : 0.0;
        const __half zh = __double2half(z);
        const __half zl = __double2half(z - (double)__half2float(zh));
        t[2 * c] = __half_as_ushort(zh);
        t[2 * c + 1] = __half_as_ushort(zl);
      }
      t[6] = __half_as_ushort(__float2half(used ? 1.0f : 0.0f));
      t[7] = 0;
      *reinterpret_cast<uint4*>(table + i * 8) = make_uint4(t[0] | ((uint32_t)t[1] << 16), t[2] | ((uint32_t)t[3] << 16),
                                                            t[4] | ((uint32_t)t[5] << 16), t[6] | ((uint32_t)t[7] << 16));
    }
  }
}

// Operand rows: CTA = (marker chunk c, sample block b), thread = sample row r.
// The chunk's 16 table entries are staged in shared memory; the thread reads
// its sample's codes at the 16 markers and writes 32 bytes (16 FP16 values)
// of each of hi and lo, and its 16 bytes of the pair's E4M3 V' row.
__global__ void __launch_bounds__(128) grm_planes_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes,
                                                         int64_t n, int64_t m, const uint16_t* __restrict__ table,
                                                         uint8_t* __restrict__ planes, int64_t n_chunks) {
  __shared__ uint4 tab[kGrmK];
  const int64_t c = blockIdx.x, b = blockIdx.y;
  const int r = threadIdx.x;
  if (r < kGrmK) {
    const int64_t i = c * kGrmK + r;
    tab[r] = i < m ? __ldg(reinterpret_cast<const uint4*>(table) + i) : make_uint4(0, 0, 0, 0);
  }
  const int64_t s = b * kTB + r;
  uint32_t code[kGrmK];
#pragma unroll
  for (int k = 0; k < kGrmK; ++k) {
    const int64_t i = c * kGrmK + k;
    code[k] = s < n && i < m ? (__ldg(packed + i * row_bytes + (s >> 2)) >> (2 * (s & 3))) & 3u : 1u;
  }
  __syncthreads();
  const uint16_t* t16 = reinterpret_cast<const uint16_t*>(tab);
  uint32_t hi[kGrmK / 2], lo[kGrmK / 2], vp[kGrmK / 4];
#pragma unroll
  for (int k = 0; k < kGrmK / 2; ++k) hi[k] = lo[k] = 0;
#pragma unroll
  for (int k = 0; k < kGrmK / 4; ++k) vp[k] = 0;
#pragma unroll
  for (int k = 0; k < kGrmK; ++k) {
    if (code[k] != 1) {  // missing (and padding) stays 0
      // code 0 = hom A1 (slot 0), 2 = het (slot 1), 3 = hom A2 (slot 2)
      const uint32_t slot = code[k] == 0 ? 0u : code[k] - 1u;
      const int sh = 16 * (k & 1);
      hi[k >> 1] |= (uint32_t)t16[k * 8 + 2 * slot] << sh;
      lo[k >> 1] |= (uint32_t)t16[k * 8 + 2 * slot + 1] << sh;
      if (t16[k * 8 + 6] != 0) vp[k >> 2] |= (uint32_t)kFp8One << (8 * (k & 3));  // used marker
    }
  }
  // the pair unit of chunks (c & ~1, c | 1)
  uint8_t* unit = planes + ((size_t)b * n_chunks + (c & ~(int64_t)1)) * kGrmChunkBytes;
  uint8_t* base = unit + (c & 1) * 2 * kTileBytes;
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // K core matrices: markers 0..7 and 8..15
    *reinterpret_cast<uint4*>(base + 0 * kTileBytes + tile_off(r, 16 * h)) =
        make_uint4(hi[4 * h], hi[4 * h + 1], hi[4 * h + 2], hi[4 * h + 3]);
    *reinterpret_cast<uint4*>(base + 1 * kTileBytes + tile_off(r, 16 * h)) =
        make_uint4(lo[4 * h], lo[4 * h + 1], lo[4 * h + 2], lo[4 * h + 3]);
  }
  // E4M3 V': markers 0..15 of the pair in byte columns 0..15, 16..31 in 16..31
  *reinterpret_cast<uint4*>(unit + kGrmVpOff + tile_off(r, 16 * (int)(c & 1))) =
      make_uint4(vp[0], vp[1], vp[2], vp[3]);
}

struct GrmArgs {
  const uint8_t* planes;
  int64_t n, n_chunks;
  const GrmItem* items;
  int64_t n_items;
  double* out;       // upper triangle with diagonal
  double* part_num;  // split items: [part][128][128] numerators and counts
  float* part_cnt;
  int* counter;
  int* status;
};

// Error-free sum (Knuth's two-sum): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// x / c for an integer count c in [1, 2^24): an FP32 reciprocal seed and one
// FP64 residual step (relative error near 2^-46).
__device__ __forceinline__ double div_count(double x, float c) {
  const double r = (double)__frcp_rn(c), cd = (double)c;
  const double q = x * r;
  return fma(fma(-q, cd, x), r, q);
}

// kPer chunks per ring stage (one bulk copy per block), kStages stages.
template <int kPer, int kStages>
__global__ void __launch_bounds__(kGrmThreads, 1) tc_grm_kernel(const GrmArgs args) {
  static_assert(kGrmSeg % kPer == 0 && kGrmPad % kPer == 0 && kPer % 2 == 0, "stage size: whole chunk pairs");
  constexpr int kBlockBytes = kPer * kGrmChunkBytes;  // one block's share of a stage
  constexpr int kGrmStages = kStages;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kGrmStages], empty[kGrmStages];
  __shared__ __align__(8) uint64_t seg_full[2], seg_free[2], cnt_free, drain;
  __shared__ __align__(8) uint64_t qfull[kGrmQueue], qempty[kGrmQueue];
  __shared__ int64_t q_item[kGrmQueue];
  __shared__ int64_t s_item[2];  // the waiter's hand-over of items to the MMA warp
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* status = args.status;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGrmStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kGrmQueue; ++s) {
      mbar_init(&qfull[s], 1);
      mbar_init(&qempty[s], kGrmEpiWarps + 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&seg_full[b], 1);
      mbar_init(&seg_free[b], kGrmEpiWarps);
    }
    mbar_init(&cnt_free, kGrmEpiWarps);
    mbar_init(&drain, 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == kGrmCopyWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  auto fail = [&](bool cond) {
    if (lane == 0 && cond) {
      atomicExch(status, kDevTimeout);
      atomicExch(&abort_flag, 1);
    }
  };
  auto aborted = [&]() { return __any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0); };
  auto queue_get = [&](uint32_t e, int64_t& it) {
    const int qs = (int)(e % kGrmQueue);
    const bool ok = mbar_wait_bounded(&qfull[qs], (e / kGrmQueue) & 1u);
    if (__any_sync(0xffffffffu, !ok)) return false;
    it = *(volatile int64_t*)&q_item[qs];
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&qempty[qs])) : "memory");
    return true;
  };
  auto arrive = [&](uint64_t* bar) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
  };
  const int64_t nk = args.n_chunks;  // a multiple of kGrmPad

  if (warp == kGrmCopyWarp) {
    uint32_t g = 0;
    for (uint32_t e = 0;; ++e) {
      int64_t it = 0;
      if (lane == 0) it = atomicAdd(args.counter, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      const bool last = it >= args.n_items;
      const int qs = (int)(e % kGrmQueue);
      const bool qok = e < (uint32_t)kGrmQueue || mbar_wait_bounded(&qempty[qs], ((e / kGrmQueue) - 1) & 1u);
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
      const GrmItem t = args.items[it];
      const bool same = t.I == t.J;
      const uint8_t* ablk = args.planes + (size_t)t.I * nk * kGrmChunkBytes;
      const uint8_t* bblk = args.planes + (size_t)t.J * nk * kGrmChunkBytes;
      bool stop = false;
      for (int64_t q = t.c0 / kPer; q < t.c1 / kPer; ++q, ++g) {
        const int s = (int)(g % kGrmStages);
        const bool ok = g < (uint32_t)kGrmStages || mbar_wait_bounded(&empty[s], ((g / kGrmStages) - 1) & 1u);
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
          mbar_arrive_expect_tx(&full[s], same ? kBlockBytes : 2 * kBlockBytes);
          bulk_g2s(dst, ablk + (size_t)q * kBlockBytes, kBlockBytes, &full[s]);
          if (!same) bulk_g2s(dst + kBlockBytes, bblk + (size_t)q * kBlockBytes, kBlockBytes, &full[s]);
        }
        __syncwarp();
      }
      if (stop) break;
    }
  } else if (warp == kGrmMmaWarp) {
    // MMA warp.  It never waits on memory itself: a thread with MMAs in flight
    // that polls a barrier or loads from memory stalls until they complete,
    // which would drain the tensor pipe at every ring stage.  The waiter warp
    // takes the items from the queue and does every wait; it hands each item
    // over through s_item and releases this warp once per stage through
    // hardware barrier kGrmBar.
    uint32_t g = 0, gs = 0;
    for (uint32_t e = 0;; ++e) {
      asm volatile("bar.sync %0, 64;" ::"n"(kGrmBar) : "memory");
      const int64_t it = *(volatile int64_t*)&s_item[e & 1u];
      if (it < 0) break;
      const GrmItem t = args.items[it];
      const bool same = t.I == t.J;
      const int64_t q1 = t.c1 / kPer;
      for (int64_t q = t.c0 / kPer; q < q1; ++q, ++g) {
        const int64_t k0 = q * kPer, r0 = k0 - t.c0;  // r0: chunks into the item
        const uint32_t b = gs & 1u;
        const bool seg_end = (r0 + kPer) % kGrmSeg == 0 || q == q1 - 1;
        asm volatile("bar.sync %0, 64;" ::"n"(kGrmBar) : "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int s = (int)(g % kGrmStages);
        if (lane == 0) {
          const uint32_t st0 = smem_addr(ring + (size_t)s * 2 * kBlockBytes);
          const uint32_t num = tmem + kColNum + 128u * b;
#pragma unroll
          for (int c = 0; c < kPer; ++c) {
            const int64_t k = k0 + c - t.c0;  // chunk index within the item
            const uint32_t ua = st0 + (c >> 1) * kGrmPairBytes;  // pair unit of A
            const uint32_t ub = same ? ua : ua + kBlockBytes;
            const uint32_t a0 = ua + (c & 1) * 2 * kTileBytes, b0 = ub + (c & 1) * 2 * kTileBytes;
            const uint64_t ah = umma_desc(a0), al = umma_desc(a0 + kTileBytes);
            const uint64_t bh = umma_desc(b0), bl = umma_desc(b0 + kTileBytes);
            umma_f16(num, ah, bh, k % kGrmSeg != 0 ? 1u : 0u);  // hi hi^T (restarts every segment)
            umma_f16(num, ah, bl, 1u);                          // + hi lo^T
            umma_f16(num, al, bh, 1u);                          // + lo hi^T
            if (c & 1)  // pair counts over the pair's 32 markers
              umma<kTcFp8>(tmem + kColCnt, umma_desc(ua + kGrmVpOff), umma_desc(ub + kGrmVpOff), k > 1 ? 1u : 0u, 0u);
          }
          umma_commit(&empty[s]);
          if (seg_end) umma_commit(&seg_full[b]);
        }
        __syncwarp();
        if (seg_end) ++gs;
      }
    }
    if (lane == 0) umma_commit(&drain);
    __syncwarp();
    const bool drained = mbar_wait_bounded(&drain, 0);
    if (lane == 0 && !drained) atomicExch(status, kDevTimeout);
  } else if (warp == kGrmWaitWarp) {
    // Waiter: for each item from the queue, hand it over; then for each ring
    // stage wait (bounded) until its operands have landed and, at a segment's
    // start, until the epilogue has freed that numerator bank (the segment
    // two back) and, at a tile's start, has read the previous tile's count;
    // then release the MMA warp.  After a failed wait or another role's abort
    // it stops waiting but keeps releasing the current item's stages (the MMA
    // warp runs them out on stale operands; the call reports IBS_ETIMEOUT),
    // then hands over the end (-1).
    uint32_t g = 0, gs = 0;
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
      asm volatile("bar.sync %0, 64;" ::"n"(kGrmBar) : "memory");
      if (it < 0) break;
      const GrmItem t = args.items[it];
      const int64_t q1 = t.c1 / kPer;
      for (int64_t q = t.c0 / kPer; q < q1; ++q, ++g) {
        const int64_t k0 = q * kPer, r0 = k0 - t.c0;
        const uint32_t b = gs & 1u;
        const bool seg_end = (r0 + kPer) % kGrmSeg == 0 || q == q1 - 1;
        if (!dead) {
          bool ok = true;
          if (r0 % kGrmSeg == 0) {
            ok = gs < 2 || mbar_wait_bounded(&seg_free[b], ((gs >> 1) - 1) & 1u);
            if (ok && r0 == 0 && e > 0) ok = mbar_wait_bounded(&cnt_free, (e - 1) & 1u);
          }
          if (ok) ok = mbar_wait_bounded(&full[(int)(g % kGrmStages)], (g / kGrmStages) & 1u);
          if (__any_sync(0xffffffffu, !ok)) {
            fail(true);
            dead = true;
          } else if (aborted()) {
            dead = true;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync %0, 64;" ::"n"(kGrmBar) : "memory");
        if (seg_end) ++gs;
      }
    }
  } else if (warp < kGrmEpiWarps) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + 64u * half;
    uint32_t gs = 0;
    bool stop = false;
    for (uint32_t e = 0; !stop; ++e) {
      int64_t it;
      if (!queue_get(e, it)) {
        fail(true);
        break;
      }
      if (it < 0) break;
      const GrmItem t = args.items[it];
      const int64_t nseg = (t.c1 - t.c0 + kGrmSeg - 1) / kGrmSeg;
      float lo[64];
      for (int64_t sg = 0; sg < nseg; ++sg, ++gs) {
        const uint32_t b = gs & 1u;
        const bool ok = mbar_wait_bounded(&seg_full[b], (gs >> 1) & 1u);
        if (__any_sync(0xffffffffu, !ok) || aborted()) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int h = 0; h < 4; ++h) {  // 16 columns at a time
          uint32_t vn[16], vh[16];
          tmem_ld16(tl + kColNum + 128u * b + 16 * h, vn);
          if (sg > 0) tmem_ld16(tl + kColHi + 16 * h, vh);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (h == 3) arrive(&seg_free[b]);
          if (sg == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              vh[j] = vn[j];
              lo[16 * h + j] = 0.0f;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float err;
              vh[j] = __float_as_uint(two_sum(__uint_as_float(vh[j]), __uint_as_float(vn[j]), err));
              lo[16 * h + j] = __fadd_rn(lo[16 * h + j], err);
            }
          }
          tmem_st16(tl + kColHi + 16 * h, vh);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      if (stop) {
        fail(true);
        break;
      }
      // the item's last segment is folded: read the counts, hand the count
      // accumulator back, then divide and store (a split item stores its sums)
      const int64_t gi = (int64_t)t.I * kTB + row;
      const int64_t j0 = (int64_t)t.J * kTB + 64 * half;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t vc[16], vh[16];
        tmem_ld16(tl + kColCnt + 16 * h, vc);
        tmem_ld16(tl + kColHi + 16 * h, vh);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (h == 3) arrive(&cnt_free);
        if (t.part >= 0) {
          const size_t base = (size_t)t.part * kTB * kTB + (size_t)row * kTB + 64 * half + 16 * h;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            args.part_num[base + j] = (double)__uint_as_float(vh[j]) + (double)lo[16 * h + j];
            args.part_cnt[base + j] = __uint_as_float(vc[j]);
          }
        } else if (gi < args.n) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t gj = j0 + 16 * h + j;
            if (gj >= args.n || gj < gi) continue;
            const float cnt = __uint_as_float(vc[j]);
            const double num = (double)__uint_as_float(vh[j]) + (double)lo[16 * h + j];
            args.out[tri_index(gi, gj, args.n)] =
                cnt == 0.0f ? __longlong_as_double(0x7ff8000000000000LL) : div_count(num, cnt);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kGrmCopyWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Split items: the pieces of a tile, added in piece order (deterministic),
// divided by the count and stored.  CTA (x, y) takes split tile x, its entries
// y, y + gridDim.y, ... in units of blockDim.x.
__global__ void __launch_bounds__(256) grm_finalize_kernel(const int4* __restrict__ splits, const double* part_num,
                                                           const float* part_cnt, int64_t n, double* __restrict__ out) {
  const int4 sp = splits[blockIdx.x];  // {I, J, first part, pieces}
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < kTB * kTB; e += gridDim.y * blockDim.x) {
    const int64_t gi = (int64_t)sp.x * kTB + e / kTB, gj = (int64_t)sp.y * kTB + e % kTB;
    if (gi >= n || gj >= n || gj < gi) continue;
    double num = 0.0;
    float cnt = 0.0f;
    for (int p = 0; p < sp.w; ++p) {
      const size_t q = (size_t)(sp.z + p) * kTB * kTB + e;
      num += part_num[q];
      cnt += part_cnt[q];  // integers below 2^24: exact
    }
    out[tri_index(gi, gj, n)] = cnt == 0.0f ? __longlong_as_double(0x7ff8000000000000LL) : div_count(num, cnt);
  }
}

template <int kPer, int kStages>
cudaError_t launch_grm_pairs(const GrmArgs& args, int grid, cudaStream_t st) {
  constexpr size_t smem = (size_t)kStages * 2 * kPer * kGrmChunkBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_grm_kernel<kPer, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tc_grm_kernel<kPer, kStages><<<grid, kGrmThreads, smem, st>>>(args);
  return cudaGetLastError();
}

// Chunks per sample block: ceil(m / 16), padded to a multiple of kGrmPad with
// zero chunks (no contribution to either product).
int64_t grm_chunks(int64_t m) { return ((m + kGrmK - 1) / kGrmK + kGrmPad - 1) / kGrmPad * kGrmPad; }

}  // namespace

size_t grm_planes_bytes(int64_t n, int64_t m) {
  const int64_t nb = (n + kTB - 1) / kTB;
  return (size_t)nb * grm_chunks(m) * kGrmChunkBytes + (size_t)m * 16;
}


// Work list: the triangle's tiles in the grouped order, whole, except the
// tiles of a final wave at most 3/4 full (or every tile, when there are fewer
// tiles than SMs), which are split over the marker axis into pieces of whole
// 128-marker segments; each piece's sums go to a part slot of their own.
void grm_items(int64_t n, int64_t m, int num_sms, std::vector<GrmItem>& items, std::vector<int4>& splits,
               int64_t& parts) {
  std::vector<int2> order;
  tc_tile_order((n + kTB - 1) / kTB, 16, order);
  const int64_t W = (int64_t)order.size(), nc = grm_chunks(m), nsegs = (nc + kGrmSeg - 1) / kGrmSeg;
  int64_t whole = W, pieces = 1;
  if (W < num_sms) {
    whole = 0;
    pieces = (num_sms + W - 1) / W;
  } else {
    const int64_t R = W % num_sms;
    if (R > 0 && R * 4 <= (int64_t)num_sms * 3) {
      whole = W - R;
      pieces = std::max<int64_t>(2, (num_sms + R / 2) / R);
    }
  }
  pieces = std::max<int64_t>(1, std::min<int64_t>(pieces, std::min<int64_t>(nsegs, 16)));
  items.clear();
  splits.clear();
  parts = 0;
  for (int64_t t = 0; t < W; ++t) {
    const int np = t < whole ? 1 : (int)pieces;
    if (np > 1) splits.push_back(make_int4(order[t].x, order[t].y, (int)parts, np));
    for (int p = 0; p < np; ++p) {
      GrmItem w{};
      w.I = order[t].x;
      w.J = order[t].y;
      w.c0 = (int32_t)(nsegs * p / np * kGrmSeg);
      w.c1 = p + 1 == np ? (int32_t)nc : (int32_t)(nsegs * (p + 1) / np * kGrmSeg);
      w.part = np > 1 ? (int32_t)(parts + p) : -1;
      items.push_back(w);
    }
    if (np > 1) parts += np;
  }
}

cudaError_t launch_grm(const uint8_t* packed, int64_t n, int64_t m, double* out, uint8_t* work, const GrmItem* items,
                       int64_t n_items, const int4* splits, int64_t n_splits, double* part_num, float* part_cnt,
                       int* counter, int* status, int num_sms, cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = grm_chunks(m);
  if (nc > 2147483647LL || nb > 65535 || n_items < 1 || n_items > 2147483647LL - num_sms ||
      n_splits > 2147483647LL)
    return cudaErrorInvalidValue;
  uint8_t* planes = work;
  uint16_t* table = reinterpret_cast<uint16_t*>(planes + (size_t)nb * nc * kGrmChunkBytes);
  const int64_t row_bytes = (n + 3) / 4;
  const int64_t freq_warps = (m + 31) / 32;
  grm_freq_kernel<<<(unsigned)std::min<int64_t>((freq_warps + 7) / 8, (int64_t)num_sms * 8), 256, 0, st>>>(
      packed, row_bytes, n, m, table);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grm_planes_kernel<<<dim3((unsigned)nc, (unsigned)nb), 128, 0, st>>>(packed, row_bytes, n, m, table, planes, nc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  const GrmArgs args{planes, n, nc, items, n_items, out, part_num, part_cnt, counter, status};
  const int grid = (int)std::min<int64_t>(num_sms, n_items);
  if ((e = launch_grm_pairs<4, 2>(args, grid, st)) != cudaSuccess) return e;
  if (n_splits > 0) {
    grm_finalize_kernel<<<dim3((unsigned)n_splits, 8), 256, 0, st>>>(splits, part_num, part_cnt, n, out);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace ibs
