// Device-side building blocks shared by the libibs kernels: the bit-plane
// format, the TMA bulk-copy pipeline with bounded mbarrier waits, and the
// per-pair LOP3/POPC update.
//
// Bit-plane format.  For each sample and each 32-marker word, four one-bit-per
// -marker planes (bit t of word w is marker 32*w + t):
//   V = call present (code != 1)      P = heterozygous (code 2)
//   Q = homozygous A2 (code 3)        R = homozygous A1 (code 0)
// Missing calls, markers past the end and samples past the end have all four
// bits clear.  For a pair (i, j) and one word:
//   v    = Vi & Vj                    -> N    += popc(v)
//   ibs1 = v & (Pi ^ Pj)              -> IBS1 += popc(ibs1)   (hom vs het)
//   ibs0 = (Qi & Rj) | (Ri & Qj)      -> IBS0 += popc(ibs0)   (opposite homozygotes)
// and IBS2 = N - IBS0 - IBS1.  This is the paper's "XOR, mask out missing
// calls, count set bits" step ("Improvements in PLINK 1.9 / Bitwise
// parallelism") on a one-hot encoding of the 2-bit code: the XOR of the raw
// code bits decides IBS0 (both bits differ) against IBS1 (one bit differs),
// and with one-hot planes each of the two decisions is a single LOP3.
//
// Memory order of the planes (uint32):
//   planes[block b][chunk c][word kw][sample s][plane p]
// with 64-sample blocks, 12-word chunks (384 markers) and p in {V, P, Q, R}.
// One (block, chunk) is a contiguous 12 KiB piece, which a single TMA bulk
// copy moves to shared memory; inside it, the four planes of one sample-word
// are one 16-byte vector.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ibs {

constexpr int kSB = 64;                             // samples per plane block (= pair-tile edge)
constexpr int kKC = 12;                             // 32-bit words per chunk
constexpr int kPlanes = 4;                          // V, P, Q, R
constexpr int kChunkWords = kKC * kSB * kPlanes;    // uint32 per (block, chunk)
constexpr int kChunkBytes = kChunkWords * 4;        // 12 KiB
constexpr int kMarkersPerChunk = kKC * 32;          // 384

// Status word values written by kernels (match ibs_status).
constexpr int kDevTimeout = 4;

// Bounded waits: give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// One non-blocking probe of the barrier phase with the given parity.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// One non-blocking test of the barrier phase with the given parity (try_wait
// may block in hardware until the phase completes).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase; returns false after limit_ns (default kWaitLimitNs)
// without completion.  Bounds under 1 ms (the test hook's) probe with the
// non-blocking test and read the clock after every probe, so the bound holds
// even where one blocking probe would have outlasted it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (limit_ns < 1000000ull) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
      if (mbar_test_wait(bar, parity)) return true;
      if (globaltimer_ns() - t0 > limit_ns) return false;
    }
  }
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// TMA bulk copy global -> shared, completion counted on the mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}
// LUT operands: a = 0xF0, b = 0xCC, c = 0xAA.
constexpr int kLutAndXor = 0x60;  // a & (b ^ c)
constexpr int kLutAndOr = 0xEA;   // (a & b) | c
constexpr int kLutXor3 = 0x96;    // a ^ b ^ c
constexpr int kLutMaj = 0xE8;     // majority(a, b, c)

// IBS distance (IBS1 + 2 IBS0) / (2N) in FP64, NaN when N = 0.  FP64
// division is slow on this part, so the quotient is seeded in FP32 and
// corrected once in FP64 (a Newton-Raphson step in residual form,
// q1 = q0 + (a - q0 b) r0 with r0 ~ 1/b): the seed is within ~2^-22 of a/b and
// r0 within 2^-24 of 1/b, so q1 is within ~2^-46 (about 1.1e-14) relative of
// the exact quotient, well inside the 1e-12 bound.  Every kernel that writes a
// distance uses this function, so all paths give identical doubles for
// identical counts.
__device__ __forceinline__ double ibs_dist(int32_t i0, int32_t i1, int32_t n) {
  if (n == 0) return __longlong_as_double(0x7ff8000000000000LL);
  const long long ai = (long long)i1 + 2 * (long long)i0, bi = 2 * (long long)n;
  const double a = (double)ai, b = (double)bi;
  const float r0 = __frcp_rn((float)bi);
  const double q0 = (double)((float)ai * r0);
  return fma(fma(-q0, b, a), (double)r0, q0);
}

// Triangle index of pair (i, j), i <= j.
__host__ __device__ __forceinline__ int64_t tri_index(int64_t i, int64_t j, int64_t n) {
  return i * n - i * (i - 1) / 2 + (j - i);
}

// Tile (I, J), I <= J, of linear index t in a row-major upper triangle of T x T tiles.
__device__ __forceinline__ void tri_tile(int64_t t, int64_t T, int64_t& I, int64_t& J) {
  const double b = 2.0 * (double)T + 1.0;
  int64_t i = (int64_t)((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (i < 0) i = 0;
  if (i > T - 1) i = T - 1;
  auto start = [T](int64_t r) { return r * T - r * (r - 1) / 2; };
  while (i > 0 && start(i) > t) --i;
  while (i + 1 < T && start(i + 1) <= t) ++i;
  I = i;
  J = i + (t - start(i));
}

}  // namespace ibs
