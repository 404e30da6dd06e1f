/*
 * Device-side twin of synth_bed.c: the same seeded genotypes, written by a
 * CUDA kernel straight into device memory (for the large benchmark and test
 * workloads, where the CPU generator would take tens of seconds).
 *
 * This file only draws inputs; it holds none of the identity-by-state
 * arithmetic.  Every genotype is the same pure function of (seed, global
 * variant index, global sample id) as in synth_bed.c: Philox4x32-10 (Salmon,
 * Moraes, Dror and Shaw, SC 2011), written here from its published
 * definition, and the same Hardy-Weinberg, offspring, duplicate and
 * missingness rules.  The per-variant probabilities arrive as 32-bit
 * fixed-point thresholds (floor(p * 2^32), 0 for p <= 0, 2^32 for p >= 1),
 * computed once on the host, so the kernel is integer-only and its bytes
 * equal the C generator's on any machine.  A test compares the two.
 */
#include <cstdint>
#include <cuda_runtime.h>

namespace {

struct U4 {
  uint32_t v[4];
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{{c0, c1, c2, c3}};
}

enum { kBase = 0, kOffspring = 1, kDuplicate = 2 };
enum { kStreamGeno = 0, kStreamExtra = 1, kStreamPad = 2 };

__device__ __forceinline__ U4 draw(uint64_t seed, int64_t variant, int64_t gid, uint32_t stream) {
  return philox4x32_10((uint32_t)variant, (uint32_t)((uint64_t)variant >> 32) ^ (stream << 24), (uint32_t)gid,
                       (uint32_t)((uint64_t)gid >> 32), (uint32_t)seed, (uint32_t)(seed >> 32));
}

struct Job {
  int64_t m, var_offset, n, row_bytes;
  uint64_t seed, dup_thr;
  const uint64_t* thr_pop;  // [n_pop][m]
  const uint64_t* miss_thr; // [m]
  const int64_t* gid;
  const int32_t* pop;
  const int32_t* kind;
  const int64_t* src_gid;
  const int32_t* src_pop;
  int pad_garbage;
  uint8_t* out;
};

// Thread = one output byte (4 samples) of one variant row.
__global__ void __launch_bounds__(256) synth_bed_kernel(const Job j) {
  const int64_t byte = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
  if (byte >= j.row_bytes || k >= j.m) return;
  const int64_t variant = j.var_offset + k;
  const uint64_t miss_thr = j.miss_thr[k];
  uint32_t packed = 0;
  for (int q = 0; q < 4; ++q) {
    const int64_t s = byte * 4 + q;
    if (s >= j.n) break;
    const uint64_t thr = j.thr_pop[(int64_t)j.pop[s] * j.m + k];
    const U4 u = draw(j.seed, variant, j.gid[s], kStreamGeno);
    int dosage;
    if (j.kind[s] == kOffspring) {
      const uint64_t pthr = j.thr_pop[(int64_t)j.src_pop[s] * j.m + k];
      const U4 b = draw(j.seed, variant, j.src_gid[s], kStreamGeno);
      const int dp = (int)((uint64_t)b.v[0] < pthr) + (int)((uint64_t)b.v[1] < pthr);
      const U4 e = draw(j.seed, variant, j.gid[s], kStreamExtra);
      const int transmitted = dp == 0 ? 0 : (dp == 2 ? 1 : (int)(e.v[0] & 1u));
      dosage = transmitted + (int)((uint64_t)u.v[1] < thr);
    } else if (j.kind[s] == kDuplicate) {
      const uint64_t pthr = j.thr_pop[(int64_t)j.src_pop[s] * j.m + k];
      const U4 b = draw(j.seed, variant, j.src_gid[s], kStreamGeno);
      dosage = (int)((uint64_t)b.v[0] < pthr) + (int)((uint64_t)b.v[1] < pthr);
      const U4 e = draw(j.seed, variant, j.gid[s], kStreamExtra);
      if ((uint64_t)e.v[0] < j.dup_thr) dosage = (dosage + 1 + (int)(e.v[1] & 1u)) % 3;
    } else {
      dosage = (int)((uint64_t)u.v[0] < thr) + (int)((uint64_t)u.v[1] < thr);
    }
    uint32_t code = dosage == 0 ? 0u : (dosage == 1 ? 2u : 3u);
    if ((uint64_t)u.v[2] < miss_thr) code = 1u;
    packed |= code << (2 * q);
  }
  if (j.pad_garbage && (j.n % 4) != 0 && byte == j.row_bytes - 1) {
    const U4 g = draw(j.seed, variant, -1, kStreamPad);
    const int used_bits = (int)(2 * (j.n % 4));
    packed |= (g.v[0] & 0xFFu) & (0xFFu << used_bits);
  }
  j.out[k * j.row_bytes + byte] = (uint8_t)packed;
}

}  // namespace

/* Fill out[m][ceil(n/4)] (DEVICE) with the genotypes synth_bed() writes for the
 * same arguments, except that the probabilities come as thresholds: thr_pop
 * [n_pop][m] and miss_thr [m] (DEVICE uint64, floor(p * 2^32) clamped to
 * [0, 2^32]), dup_thr likewise.  Sample descriptors are DEVICE arrays.
 * Enqueued on `stream`.  Returns 0, 1 on bad arguments, 2 on a launch error. */
extern "C" int synth_bed_gpu(int64_t m, uint64_t seed, int64_t var_offset, const uint64_t* thr_pop, int32_t n_pop,
                             const uint64_t* miss_thr, int64_t n, const int64_t* gid, const int32_t* pop,
                             const int32_t* kind, const int64_t* src_gid, const int32_t* src_pop, uint64_t dup_thr,
                             int pad_garbage, uint8_t* out, void* stream) {
  if (m <= 0 || n <= 0 || n_pop <= 0 || !thr_pop || !miss_thr || !gid || !pop || !kind || !src_gid || !src_pop ||
      !out)
    return 1;
  Job j;
  j.m = m;
  j.var_offset = var_offset;
  j.n = n;
  j.row_bytes = (n + 3) / 4;
  j.seed = seed;
  j.dup_thr = dup_thr;
  j.thr_pop = thr_pop;
  j.miss_thr = miss_thr;
  j.gid = gid;
  j.pop = pop;
  j.kind = kind;
  j.src_gid = src_gid;
  j.src_pop = src_pop;
  j.pad_garbage = pad_garbage;
  j.out = out;
  const int64_t gx = (j.row_bytes + 255) / 256;
  const int64_t gy = m < 65535 ? m : 65535;
  const int64_t gz = (m + gy - 1) / gy;
  if (gx > 2147483647LL || gz > 65535) return 1;
  synth_bed_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), 256, 0, static_cast<cudaStream_t>(stream)>>>(j);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
