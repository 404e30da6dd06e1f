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
// chunk); one (block, chunk) holds three 128 x 32-byte tiles, hi, lo and V',
// in the canonical K-major layout (12 KiB).  Tensor memory: numerator banks at
// columns 0 and 128, the count at 256, the float-float high words at 384.
// One persistent CTA per SM, 10 warps: warp 8 claims triangle tiles in the
// grouped order and streams both blocks' chunks through a ring of two stages
// of four chunks (one 48 KiB bulk copy per block and stage: the copy engine
// spends a fixed time per copy, measured near 340 cycles, so one chunk per
// stage ran 1.6x slower); warp 9 issues 4 MMAs per chunk; warps 0..7 fold
// segments (warp w: TMEM lanes of quarter w % 4, columns 64 (w / 4) .. +63) and
// store A.  Every wait is bounded (2 s of %globaltimer).
#include <algorithm>
#include <cuda_fp16.h>
#include <vector>

#include "ibs_tc_common.cuh"

namespace ibs {

namespace {

constexpr int kGrmK = 16;                                // markers per FP16 chunk
constexpr int kGrmPlanes = 3;                            // hi, lo, V'
constexpr int kGrmChunkBytes = kGrmPlanes * kTileBytes;  // 12 KiB
constexpr int kGrmPad = 4;                               // chunk count padded to a multiple of this
constexpr int kGrmQueue = 8;
constexpr int kGrmSeg = 8;                               // chunks per numerator segment
static_assert(kGrmSeg % kGrmPad == 0, "a ring stage never straddles two segments");
constexpr int kGrmEpiWarps = 8;
constexpr int kGrmThreads = (kGrmEpiWarps + 2) * 32;
constexpr int kGrmCopyWarp = kGrmEpiWarps, kGrmMmaWarp = kGrmEpiWarps + 1;
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
// V' (1.0 when 0 < p < 1) and a pad, as FP16 bit patterns.  One warp per
// marker row; the codes are counted by population counts over 16 genotypes
// per 32-bit word (codes 0 hom A1, 1 missing, 2 het, 3 hom A2 in bit pairs);
// p and z in FP64.
__device__ __forceinline__ void count_codes(uint32_t w, uint32_t valid, int& hom1, int& het, int& miss) {
  const uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;
  hom1 += __popc(~(lo | hi) & valid);
  het += __popc(hi & ~lo & valid);
  miss += __popc(lo & ~hi & valid);
}

__global__ void grm_freq_kernel(const uint8_t* __restrict__ packed, int64_t row_bytes, int64_t n, int64_t m,
                                uint16_t* __restrict__ table) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  // rows are 16-byte aligned when the row length is (the buffer base is)
  const bool vec = (row_bytes & 15) == 0 && (reinterpret_cast<uintptr_t>(packed) & 15) == 0;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < m; i += warps) {
    const uint8_t* row = packed + i * row_bytes;
    int hom1 = 0, het = 0, miss = 0;
    if (vec) {
      const uint4* r4 = reinterpret_cast<const uint4*>(row);
      for (int64_t q = lane; q < row_bytes / 16; q += 32) {
        const uint4 v = __ldg(r4 + q);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t s0 = q * 64 + t * 16;  // first sample of the word
          const uint32_t valid = s0 + 16 <= n ? 0x55555555u : (s0 >= n ? 0u : 0x55555555u >> (2 * (s0 + 16 - n)));
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
    if (lane == 0) {
      const int64_t calls = n - miss;
      const double p = calls > 0 ? (double)(2 * (int64_t)hom1 + het) / (2.0 * (double)calls) : 0.0;
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
// of each of hi, lo and V'.
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
  uint32_t hi[kGrmK / 2], lo[kGrmK / 2], vp[kGrmK / 2];
#pragma unroll
  for (int k = 0; k < kGrmK / 2; ++k) hi[k] = lo[k] = vp[k] = 0;
#pragma unroll
  for (int k = 0; k < kGrmK; ++k) {
    if (code[k] != 1) {  // missing (and padding) stays 0
      // code 0 = hom A1 (slot 0), 2 = het (slot 1), 3 = hom A2 (slot 2)
      const uint32_t slot = code[k] == 0 ? 0u : code[k] - 1u;
      const int sh = 16 * (k & 1);
      hi[k >> 1] |= (uint32_t)t16[k * 8 + 2 * slot] << sh;
      lo[k >> 1] |= (uint32_t)t16[k * 8 + 2 * slot + 1] << sh;
      vp[k >> 1] |= (uint32_t)t16[k * 8 + 6] << sh;
    }
  }
  uint8_t* base = planes + (size_t)(b * n_chunks + c) * kGrmChunkBytes;
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // K core matrices: markers 0..7 and 8..15
    *reinterpret_cast<uint4*>(base + 0 * kTileBytes + tile_off(r, 16 * h)) =
        make_uint4(hi[4 * h], hi[4 * h + 1], hi[4 * h + 2], hi[4 * h + 3]);
    *reinterpret_cast<uint4*>(base + 1 * kTileBytes + tile_off(r, 16 * h)) =
        make_uint4(lo[4 * h], lo[4 * h + 1], lo[4 * h + 2], lo[4 * h + 3]);
    *reinterpret_cast<uint4*>(base + 2 * kTileBytes + tile_off(r, 16 * h)) =
        make_uint4(vp[4 * h], vp[4 * h + 1], vp[4 * h + 2], vp[4 * h + 3]);
  }
}

struct GrmArgs {
  const uint8_t* planes;
  int64_t n, n_chunks;
  const int2* tiles;
  int64_t n_tiles;
  double* out;  // upper triangle with diagonal
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
  static_assert(kGrmSeg % kPer == 0 && kGrmPad % kPer == 0, "stage size");
  constexpr int kBlockBytes = kPer * kGrmChunkBytes;  // one block's share of a stage
  constexpr int kGrmStages = kStages;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kGrmStages], empty[kGrmStages];
  __shared__ __align__(8) uint64_t seg_full[2], seg_free[2], cnt_free, drain;
  __shared__ __align__(8) uint64_t qfull[kGrmQueue], qempty[kGrmQueue];
  __shared__ int64_t q_item[kGrmQueue];
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
  const int64_t nq = nk / kPer;
  const int64_t nseg = (nk + kGrmSeg - 1) / kGrmSeg;

  if (warp == kGrmCopyWarp) {
    uint32_t g = 0;
    for (uint32_t e = 0;; ++e) {
      int64_t it = 0;
      if (lane == 0) it = atomicAdd(args.counter, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      const bool last = it >= args.n_tiles;
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
      const int2 t = args.tiles[it];
      const bool same = t.x == t.y;
      const uint8_t* ablk = args.planes + (size_t)t.x * nk * kGrmChunkBytes;
      const uint8_t* bblk = args.planes + (size_t)t.y * nk * kGrmChunkBytes;
      bool stop = false;
      for (int64_t q = 0; q < nq; ++q, ++g) {
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
    uint32_t g = 0, gs = 0;
    bool stop = false;
    for (uint32_t e = 0; !stop; ++e) {
      int64_t it;
      if (!queue_get(e, it)) {
        fail(true);
        break;
      }
      if (it < 0) break;
      const int2 t = args.tiles[it];
      const bool same = t.x == t.y;
      for (int64_t q = 0; q < nq && !stop; ++q, ++g) {
        const int64_t k0 = q * kPer;
        const uint32_t b = gs & 1u;
        const bool seg_end = (k0 + kPer) % kGrmSeg == 0 || q == nq - 1;
        if (k0 % kGrmSeg == 0) {
          // the numerator bank is free once the epilogue has read the segment
          // two back; the previous tile's count must be read before the first
          // count MMA of this one
          bool ok = gs < 2 || mbar_wait_bounded(&seg_free[b], ((gs >> 1) - 1) & 1u);
          if (ok && k0 == 0 && e > 0) ok = mbar_wait_bounded(&cnt_free, (e - 1) & 1u);
          if (__any_sync(0xffffffffu, !ok)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int s = (int)(g % kGrmStages);
        const bool ok = mbar_wait_bounded(&full[s], (g / kGrmStages) & 1u);
        if (__any_sync(0xffffffffu, !ok)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const uint32_t st0 = smem_addr(ring + (size_t)s * 2 * kBlockBytes);
          const uint32_t num = tmem + kColNum + 128u * b;
#pragma unroll
          for (int c = 0; c < kPer; ++c) {
            const int64_t k = k0 + c;
            const uint32_t a0 = st0 + c * kGrmChunkBytes;
            const uint32_t b0 = same ? a0 : a0 + kBlockBytes;
            const uint64_t ah = umma_desc(a0), al = umma_desc(a0 + kTileBytes), av = umma_desc(a0 + 2 * kTileBytes);
            const uint64_t bh = umma_desc(b0), bl = umma_desc(b0 + kTileBytes), bv = umma_desc(b0 + 2 * kTileBytes);
            umma_f16(num, ah, bh, k % kGrmSeg != 0 ? 1u : 0u);  // hi hi^T
            umma_f16(num, ah, bl, 1u);                          // + hi lo^T
            umma_f16(num, al, bh, 1u);                          // + lo hi^T
            umma_f16(tmem + kColCnt, av, bv, k > 0 ? 1u : 0u);  // pair counts
          }
          umma_commit(&empty[s]);
          if (seg_end) umma_commit(&seg_full[b]);
        }
        __syncwarp();
        if (seg_end) ++gs;
      }
      if (stop || aborted()) {
        fail(stop);
        break;
      }
    }
    if (lane == 0) umma_commit(&drain);
    __syncwarp();
    const bool drained = mbar_wait_bounded(&drain, 0);
    if (lane == 0 && !drained) atomicExch(status, kDevTimeout);
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
      // the tile's last segment is folded: read the counts, hand the count
      // accumulator back, divide and store
      const int2 t = args.tiles[it];
      const int64_t gi = (int64_t)t.x * kTB + row;
      const int64_t j0 = (int64_t)t.y * kTB + 64 * half;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t vc[16], vh[16];
        tmem_ld16(tl + kColCnt + 16 * h, vc);
        tmem_ld16(tl + kColHi + 16 * h, vh);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (h == 3) arrive(&cnt_free);
        if (gi < args.n) {
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

}  // namespace

// Chunks per sample block: ceil(m / 16), padded to a multiple of kGrmPad with
// zero chunks (no contribution to either product).
static int64_t grm_chunks(int64_t m) { return ((m + kGrmK - 1) / kGrmK + kGrmPad - 1) / kGrmPad * kGrmPad; }

size_t grm_planes_bytes(int64_t n, int64_t m) {
  const int64_t nb = (n + kTB - 1) / kTB;
  return (size_t)nb * grm_chunks(m) * kGrmChunkBytes + (size_t)m * 16;
}

void grm_tiles(int64_t n, std::vector<int2>& out) { tc_tile_order((n + kTB - 1) / kTB, 16, out); }

template <int kPer, int kStages>
static cudaError_t launch_grm_pairs(const GrmArgs& args, int grid, cudaStream_t st) {
  constexpr size_t smem = (size_t)kStages * 2 * kPer * kGrmChunkBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_grm_kernel<kPer, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tc_grm_kernel<kPer, kStages><<<grid, kGrmThreads, smem, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_grm(const uint8_t* packed, int64_t n, int64_t m, double* out, uint8_t* work, const int2* tiles,
                       int64_t n_tiles, int* counter, int* status, int num_sms, cudaStream_t st) {
  const int64_t nb = (n + kTB - 1) / kTB, nc = grm_chunks(m);
  if (nc > 2147483647LL || nb > 65535 || n_tiles < 1 || n_tiles > 2147483647LL - num_sms)
    return cudaErrorInvalidValue;
  uint8_t* planes = work;
  uint16_t* table = reinterpret_cast<uint16_t*>(planes + (size_t)nb * nc * kGrmChunkBytes);
  const int64_t row_bytes = (n + 3) / 4;
  grm_freq_kernel<<<num_sms * 4, 256, 0, st>>>(packed, row_bytes, n, m, table);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grm_planes_kernel<<<dim3((unsigned)nc, (unsigned)nb), 128, 0, st>>>(packed, row_bytes, n, m, table, planes, nc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  const GrmArgs args{planes, n, nc, tiles, n_tiles, out, counter, status};
  const int grid = (int)std::min<int64_t>(num_sms, n_tiles);
  return launch_grm_pairs<4, 2>(args, grid, st);
}

}  // namespace ibs
