// Transpose of variant-major packed genotypes (.bed rows) into sample-major
// one-hot bit planes (V, P, Q, R per 32-marker word; see ibs_device.cuh).
//
// The paper processes the packed 2-bit data many genotypes at a time with bit
// arithmetic ("Improvements in PLINK 1.9 / Bitwise parallelism"); the GPU form
// regroups it so that each 32-bit word holds one sample's calls at 32
// consecutive markers.  A warp owns 32 markers (one per lane, so one .bed row
// per lane) and turns each sample's column of 2-bit codes into two 32-bit
// words with two warp ballots (high bit, low bit); the lane whose index
// matches the sample then derives the four planes and stores them as one
// 16-byte vector.  The kernel is bound by HBM: it reads the 2-bit input once
// and writes 16 bytes per sample-word.
#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {

namespace {

constexpr int kGroup = 128;  // samples per CTA (two plane blocks)

struct JobView {
  BedSource src;
  int64_t m, n;
  uint32_t* planes;
  int64_t n_blocks, n_chunks;
  int* status;
};

// CTA (chunk c, sample group g): warp kw handles word kw of the chunk.
__device__ __forceinline__ void planes_body(const JobView& jv, int64_t c, int64_t g, int64_t* sel_s) {
  const int kw = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t s_base = g * kGroup;
  if (jv.src.sel != nullptr) {
    for (int t = threadIdx.x; t < kGroup; t += blockDim.x) {
      const int64_t s = s_base + t;
      int64_t ps = s < jv.n ? jv.src.sel[s] : -1;
      if (s < jv.n && (ps < 0 || ps >= jv.src.n_src)) {
        // Out-of-range index: read nothing, report it, treat the sample as missing.
        atomicExch(jv.status, 1);
        ps = -1;
      }
      sel_s[t] = ps;
    }
    __syncthreads();
  }
  const int64_t marker = (c * kKC + kw) * 32 + lane;
  const bool marker_ok = marker < jv.m;
  const uint8_t* row = jv.src.packed + (jv.src.var_begin + (marker_ok ? marker : 0)) * jv.src.row_bytes;

  for (int base = 0; base < kGroup; base += 32) {
    uint32_t myH = 0, myL = 0;
    if (jv.src.sel == nullptr) {
      // Contiguous samples: one byte holds four of them.
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        const int64_t s0 = s_base + base + q;
        uint32_t byte = 0x55u;  // "missing" in all four slots
        if (marker_ok && s0 < jv.n) byte = __ldg(row + (s0 >> 2));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          uint32_t code = (byte >> (2 * t)) & 3u;
          if (s0 + t >= jv.n) code = 1u;
          const uint32_t h = __ballot_sync(0xffffffffu, code >> 1);
          const uint32_t l = __ballot_sync(0xffffffffu, code & 1u);
          if (lane == q + t) {
            myH = h;
            myL = l;
          }
        }
      }
    } else {
      // Gathered samples: each one reads its own byte.
#pragma unroll 4
      for (int q = 0; q < 32; ++q) {
        const int64_t ps = sel_s[base + q];
        uint32_t code = 1u;
        if (marker_ok && ps >= 0) code = (__ldg(row + (ps >> 2)) >> (2 * (ps & 3))) & 3u;
        const uint32_t h = __ballot_sync(0xffffffffu, code >> 1);
        const uint32_t l = __ballot_sync(0xffffffffu, code & 1u);
        if (lane == q) {
          myH = h;
          myL = l;
        }
      }
    }
    // Codes: 0 = 00 hom A1, 1 = 01 missing, 2 = 10 het, 3 = 11 hom A2.
    const uint32_t V = myH | ~myL;
    const uint32_t P = myH & ~myL;
    const uint32_t Q = myH & myL;
    const uint32_t R = ~myH & ~myL;
    const int64_t s_local = base + lane;            // 0..127
    const int64_t b = g * 2 + (s_local >> 6);
    if (b < jv.n_blocks) {
      const int64_t off = (((b * jv.n_chunks + c) * kKC + kw) * kSB + (s_local & 63)) * kPlanes;
      *reinterpret_cast<uint4*>(jv.planes + off) = make_uint4(V, P, Q, R);
    }
  }
}

__global__ void __launch_bounds__(kKC * 32) planes_kernel(JobView jv) {
  __shared__ int64_t sel_s[kGroup];
  planes_body(jv, blockIdx.x, blockIdx.y, sel_s);
}

// Contiguous samples with 16-byte aligned rows: each lane reads 64 bytes of
// its .bed row (256 samples) with four 16-byte loads, so a warp moves whole
// 32-byte sectors with few instructions, and the CTA covers 4 plane blocks of
// one chunk.
constexpr int kWideGroup = 256;

__global__ void __launch_bounds__(kKC * 32, 2) planes_wide_kernel(JobView jv) {
  const int kw = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x, g = blockIdx.y;
  const int64_t s_base = g * kWideGroup;
  const int64_t marker = (c * kKC + kw) * 32 + lane;
  const bool marker_ok = marker < jv.m;
  const uint8_t* row = jv.src.packed + (jv.src.var_begin + (marker_ok ? marker : 0)) * jv.src.row_bytes;
  const int64_t byte0 = s_base >> 2;  // first byte of this group in the row
  uint32_t d[kWideGroup / 16];
#pragma unroll
  for (int v = 0; v < kWideGroup / 64; ++v) {
    uint4 x = make_uint4(0x55555555u, 0x55555555u, 0x55555555u, 0x55555555u);  // "missing"
    if (marker_ok && byte0 + 16 * v < jv.src.row_bytes) x = __ldg(reinterpret_cast<const uint4*>(row + byte0 + 16 * v));
    d[4 * v + 0] = x.x;
    d[4 * v + 1] = x.y;
    d[4 * v + 2] = x.z;
    d[4 * v + 3] = x.w;
  }
#pragma unroll
  for (int r = 0; r < kWideGroup / 32; ++r) {
    uint32_t myH = 0, myL = 0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int s = 32 * r + t;  // sample within the group
      uint32_t code = (d[s >> 4] >> (2 * (s & 15))) & 3u;
      if (s_base + s >= jv.n) code = 1u;
      const uint32_t h = __ballot_sync(0xffffffffu, code >> 1);
      const uint32_t l = __ballot_sync(0xffffffffu, code & 1u);
      if (lane == t) {
        myH = h;
        myL = l;
      }
    }
    const uint32_t V = myH | ~myL;
    const uint32_t P = myH & ~myL;
    const uint32_t Q = myH & myL;
    const uint32_t R = ~myH & ~myL;
    const int64_t s_local = 32 * r + lane;
    const int64_t b = g * (kWideGroup / kSB) + (s_local >> 6);
    if (b < jv.n_blocks) {
      const int64_t off = (((b * jv.n_chunks + c) * kKC + kw) * kSB + (s_local & 63)) * kPlanes;
      *reinterpret_cast<uint4*>(jv.planes + off) = make_uint4(V, P, Q, R);
    }
  }
}

// Batched: one flattened grid over all jobs; each CTA finds its job by
// binary search on cta_begin.
__global__ void __launch_bounds__(kKC * 32) planes_batch_kernel(const PlaneJob* __restrict__ jobs, int n_jobs,
                                                                int* status) {
  __shared__ int64_t sel_s[kGroup];
  const int64_t cta = blockIdx.x;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].cta_begin <= cta) lo = mid;
    else hi = mid - 1;
  }
  const PlaneJob& j = jobs[lo];
  const int64_t local = cta - j.cta_begin;
  JobView jv;
  jv.src = j.src;
  jv.m = j.m;
  jv.n = j.n;
  jv.planes = j.planes;
  jv.n_blocks = j.n_blocks;
  jv.n_chunks = j.n_chunks;
  jv.status = status;
  planes_body(jv, local / j.groups, local % j.groups, sel_s);
}

}  // namespace

cudaError_t launch_planes(const BedSource& src, int64_t n, int64_t m, const PlaneGeom& g, uint32_t* planes,
                          int* status, cudaStream_t st) {
  JobView jv;
  jv.src = src;
  jv.m = m;
  jv.n = n;
  jv.planes = planes;
  jv.n_blocks = g.n_blocks;
  jv.n_chunks = g.n_chunks;
  jv.status = status;
  const bool wide = src.sel == nullptr && src.row_bytes % 16 == 0 &&
                    reinterpret_cast<uintptr_t>(src.packed) % 16 == 0;
  const int64_t per = wide ? kWideGroup / kSB : 2;
  const int64_t groups = (g.n_blocks + per - 1) / per;
  if (g.n_chunks > 2147483647LL || groups > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)g.n_chunks, (unsigned)groups);
  if (wide) planes_wide_kernel<<<grid, kKC * 32, 0, st>>>(jv);
  else planes_kernel<<<grid, kKC * 32, 0, st>>>(jv);
  return cudaGetLastError();
}

cudaError_t launch_planes_batch(const PlaneJob* jobs_dev, int n_jobs, int64_t total_ctas, int* status,
                                cudaStream_t st) {
  if (total_ctas <= 0) return cudaSuccess;
  if (total_ctas > 2147483647LL) return cudaErrorInvalidValue;
  planes_batch_kernel<<<(unsigned)total_ctas, kKC * 32, 0, st>>>(jobs_dev, n_jobs, status);
  return cudaGetLastError();
}

}  // namespace ibs
