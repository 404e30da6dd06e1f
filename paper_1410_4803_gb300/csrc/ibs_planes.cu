// Transpose of variant-major packed genotypes (.bed rows) into sample-major
// one-hot bit planes (V, P, Q, R per 32-marker word; see ibs_device.cuh).
//
// The paper processes the packed 2-bit data many genotypes at a time with bit
// arithmetic ("Improvements in PLINK 1.9 / Bitwise parallelism"); the GPU form
// regroups it so that each 32-bit word holds one sample's calls at 32
// consecutive markers.  A warp owns 32 markers (one per lane, so one .bed row
// per lane).  For contiguous samples a 32 x 32 bit transpose by warp shuffles
// turns 16 samples' packed codes into their low-bit and high-bit words at
// once; for gathered samples (a sample index list) each sample's column is
// built with two warp ballots.  The four planes of a sample-word are stored as
// one 16-byte vector.  The kernel reads the 2-bit input once and writes 16
// bytes per sample-word.
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

// Ballot form, used for gathered samples (a sample index list): CTA (chunk c,
// sample group g of 128), warp kw handles word kw of the chunk.
__device__ __forceinline__ void planes_body(const JobView& jv, int64_t c, int64_t g, int64_t* sel_s) {
  const int kw = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t s_base = g * kGroup;
  {
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
    {
      // Each gathered sample reads its own byte; two ballots give its H and L words.
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

// Contiguous samples: a 32 x 32 bit transpose by warp shuffles.  Lane t
// holds one 32-bit word of .bed row t (16 samples x 2 bits); five rounds of
// __shfl_xor_sync swap ever smaller off-diagonal bit blocks between lane
// pairs, after which lane 2k holds the low code bits (L) and lane 2k+1 the
// high code bits (H) of sample k at the warp's 32 markers.  One exchange with
// the neighbour lane gives each lane both words; the even lane stores (V, P)
// and the odd lane (Q, R) of the sample's 16-byte plane vector.  This costs
// about 30 instructions per 16 samples x 32 markers, a quarter of the ballot
// form.  The CTA covers 256 samples (4 plane blocks) of one chunk.
constexpr int kShflGroup = 256;

__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
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

__global__ void __launch_bounds__(kKC * 32) planes_shfl_kernel(JobView jv) {
  const int kw = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x, g = blockIdx.y;
  const int64_t s_base = g * kShflGroup;
  const int64_t marker = (c * kKC + kw) * 32 + lane;
  const bool marker_ok = marker < jv.m;
  const int64_t rb = jv.src.row_bytes;
  const uint8_t* row = jv.src.packed + (jv.src.var_begin + (marker_ok ? marker : 0)) * rb;
  const int64_t byte0 = s_base >> 2;  // first byte of the group in the row
  constexpr uint32_t kMissing = 0x55555555u;
  uint32_t d[kShflGroup / 16];
  const uintptr_t base = reinterpret_cast<uintptr_t>(jv.src.packed);
  if (rb % 16 == 0 && base % 16 == 0) {
#pragma unroll
    for (int v = 0; v < kShflGroup / 64; ++v) {
      uint4 x = make_uint4(kMissing, kMissing, kMissing, kMissing);
      if (marker_ok && byte0 + 16 * v < rb) x = __ldg(reinterpret_cast<const uint4*>(row + byte0 + 16 * v));
      d[4 * v + 0] = x.x;
      d[4 * v + 1] = x.y;
      d[4 * v + 2] = x.z;
      d[4 * v + 3] = x.w;
    }
  } else if (rb % 4 == 0 && base % 4 == 0) {
#pragma unroll
    for (int w = 0; w < kShflGroup / 16; ++w)
      d[w] = (marker_ok && byte0 + 4 * w < rb) ? __ldg(reinterpret_cast<const uint32_t*>(row + byte0 + 4 * w))
                                              : kMissing;
  } else {
#pragma unroll
    for (int w = 0; w < kShflGroup / 16; ++w) {
      uint32_t x = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t at = byte0 + 4 * w + b;
        const uint32_t byte = (marker_ok && at < rb) ? (uint32_t)__ldg(row + at) : 0x55u;
        x |= byte << (8 * b);
      }
      d[w] = x;
    }
  }
  const int k = lane >> 1;          // sample within a 16-sample word
  const bool odd = (lane & 1) != 0;
#pragma unroll
  for (int w = 0; w < kShflGroup / 16; ++w) {
    const uint32_t x = warp_transpose32(d[w], lane);
    const uint32_t partner = __shfl_xor_sync(0xffffffffu, x, 1);
    const uint32_t H = odd ? x : partner;
    const uint32_t L = odd ? partner : x;
    const int64_t s_local = 16 * w + k;  // 0..255
    const int64_t s = s_base + s_local;
    uint2 out;
    if (s >= jv.n) {
      out = make_uint2(0u, 0u);
    } else if (!odd) {
      out = make_uint2(H | ~L, H & ~L);   // V (present), P (het)
    } else {
      out = make_uint2(H & L, ~H & ~L);   // Q (hom A2), R (hom A1)
    }
    const int64_t b = g * (kShflGroup / kSB) + (s_local >> 6);
    if (b < jv.n_blocks) {
      const int64_t off = (((b * jv.n_chunks + c) * kKC + kw) * kSB + (s_local & 63)) * kPlanes + (odd ? 2 : 0);
      *reinterpret_cast<uint2*>(jv.planes + off) = out;
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
  const bool contiguous = src.sel == nullptr;
  const int64_t per = contiguous ? kShflGroup / kSB : 2;
  const int64_t groups = (g.n_blocks + per - 1) / per;
  if (g.n_chunks > 2147483647LL || groups > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)g.n_chunks, (unsigned)groups);
  if (contiguous) planes_shfl_kernel<<<grid, kKC * 32, 0, st>>>(jv);
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
