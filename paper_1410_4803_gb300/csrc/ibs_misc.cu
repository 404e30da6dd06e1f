// Serving-side helper kernels (top-k nearest panel samples) and the
// integer-pipe microbenchmark used to derive the pair loop's roofline.
#include <cstdio>

#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {

namespace {

// ---------------------------------------------------------------------------
// Top-k by distance.  Key = IEEE bits of the non-negative double distance
// (monotone as unsigned), NaN (N == 0) mapped above +inf, padding above NaN;
// ties are broken by ascending panel index.
constexpr int kTopkMax = 64;
constexpr int kTopkThreads = 256;
constexpr uint64_t kNanKey = 0x7FF8000000000000ull;
constexpr uint64_t kPadKey = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ bool key_less(uint64_t ka, int ia, uint64_t kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// One row's k nearest panel samples (one CTA of kTopkThreads threads):
// counts c[n_panel] -> out_idx[k], out_dist[k].
__device__ __forceinline__ void topk_row(const int4* __restrict__ c, int64_t n_panel, int k,
                                         int32_t* __restrict__ out_idx, double* __restrict__ out_dist) {
  uint64_t key[kTopkMax];
  int idx[kTopkMax];
#pragma unroll
  for (int r = 0; r < kTopkMax; ++r) {
    key[r] = kPadKey;
    idx[r] = 0x7FFFFFFF;
  }
  // Local pass: each thread keeps its k best in ascending order.  It visits
  // indices in increasing order, so a strict comparison keeps the lower index
  // among equal keys.
  for (int64_t e = threadIdx.x; e < n_panel; e += kTopkThreads) {
    const int4 q = c[e];
    uint64_t kk;
    if (q.w == 0) {
      kk = kNanKey;
    } else {
      // Cheap exact reject once the list is full of finite keys: the two
      // integer-to-FP32 conversions and the FP32 division are each correctly
      // rounded, so the FP32 quotient f is within 3 * 2^-24 (relative) of the
      // rational r.  If f > t (1 + 2^-20), with t the list's k-th key, then
      // r > t, and the double key (r rounded, a monotone map) is >= t: it
      // would not be inserted (strict comparison below).  Only the others pay
      // the FP64 division.
      const uint64_t last = key[k - 1];
      if (last < kNanKey) {
        const float f = __fdiv_rn((float)(q.y + 2 * q.x), (float)(2 * q.w));
        if ((double)f > __longlong_as_double((long long)last) * (1.0 + 0x1p-20)) continue;
      }
      const double d = (double)(q.y + 2 * q.x) / (2.0 * (double)q.w);
      kk = (uint64_t)__double_as_longlong(d);
    }
    if (kk < key[k - 1]) {
      int pos = k - 1;
#pragma unroll 1
      while (pos > 0 && kk < key[pos - 1]) {
        key[pos] = key[pos - 1];
        idx[pos] = idx[pos - 1];
        --pos;
      }
      key[pos] = kk;
      idx[pos] = (int)e;
    }
  }
  // Merge: k rounds of a block-wide argmin over each thread's list head.
  __shared__ uint64_t wk[kTopkThreads / 32];
  __shared__ int wi[kTopkThreads / 32];
  __shared__ int wt[kTopkThreads / 32];
  __shared__ int winner;
  int head = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < k; ++r) {
    uint64_t hk = kPadKey;
    int hi = 0x7FFFFFFF;
    // head < k always holds for the owner of unconsumed entries
    for (int t = 0; t < kTopkMax; ++t)
      if (t == head) {
        hk = key[t];
        hi = idx[t];
      }
    int ht = threadIdx.x;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t ok = __shfl_down_sync(0xffffffffu, hk, off);
      const int oi = __shfl_down_sync(0xffffffffu, hi, off);
      const int ot = __shfl_down_sync(0xffffffffu, ht, off);
      if (key_less(ok, oi, hk, hi)) {
        hk = ok;
        hi = oi;
        ht = ot;
      }
    }
    if (lane == 0) {
      wk[warp] = hk;
      wi[warp] = hi;
      wt[warp] = ht;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t bk = wk[0];
      int bi = wi[0], bt = wt[0];
      for (int w = 1; w < kTopkThreads / 32; ++w)
        if (key_less(wk[w], wi[w], bk, bi)) {
          bk = wk[w];
          bi = wi[w];
          bt = wt[w];
        }
      const bool pad = bk == kPadKey;
      out_idx[r] = pad ? -1 : bi;
      out_dist[r] =
          (pad || bk == kNanKey) ? __longlong_as_double(0x7ff8000000000000LL) : __longlong_as_double((long long)bk);
      winner = pad ? -1 : bt;
    }
    __syncthreads();
    if (threadIdx.x == winner) ++head;
    __syncthreads();
  }
}

// One request: row r of counts [q][n_panel] -> out_idx/out_dist [q][k].
__global__ void __launch_bounds__(kTopkThreads)
    topk_kernel(const int32_t* __restrict__ counts, int64_t n_panel, int k, int32_t* __restrict__ out_idx,
                double* __restrict__ out_dist) {
  const int64_t row = blockIdx.x;
  topk_row(reinterpret_cast<const int4*>(counts) + row * n_panel, n_panel, k, out_idx + row * k,
           out_dist + row * k);
}

// Many requests in one launch: CTA r takes row list entry r.
__global__ void __launch_bounds__(kTopkThreads) topk_rows_kernel(const TopkRow* __restrict__ rows, int64_t n_panel) {
  const TopkRow t = rows[blockIdx.x];
  topk_row(reinterpret_cast<const int4*>(t.counts), n_panel, t.k, t.out_idx, t.out_dist);
}

// ---------------------------------------------------------------------------
// Integer-pipe microbenchmark: 8 independent dependency chains per thread.
template <int OP>
__global__ void __launch_bounds__(256) pipe_kernel(uint32_t* out, int iters, uint32_t seed,
                                                   unsigned long long* clk, unsigned long long* ns) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = seed * (threadIdx.x + 1) + i * 0x9E3779B9u + blockIdx.x;
    b[i] = a[i] * 0x85EBCA6Bu + 7u;
  }
  const unsigned long long c0 = clock64();
  const unsigned long long g0 = globaltimer_ns();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (OP == 0) {
          uint32_t d;
          asm volatile("popc.b32 %0, %1;" : "=r"(d) : "r"(a[i]));
          a[i] = d;
        } else if (OP == 1) {
          a[i] = lop3<kLutXor3>(a[i], b[i], a[(i + 1) & 7]);
        } else {
          a[i] = a[i] + b[i] + a[(i + 3) & 7];
        }
      }
    }
  }
  const unsigned long long g1 = globaltimer_ns();
  const unsigned long long c1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i] * (i + 1);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) {
    clk[blockIdx.x] = c1 - c0;
    ns[blockIdx.x] = g1 - g0;
  }
}

template <int OP>
cudaError_t run_probe(int sms, uint32_t* out, unsigned long long* clk, unsigned long long* ns, double* per_clk,
                      double* mhz) {
  const int blocks = sms * 4, threads = 256, iters = 2048;
  pipe_kernel<OP><<<blocks, threads>>>(out, 8, 1u, clk, ns);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  pipe_kernel<OP><<<blocks, threads>>>(out, iters, 1u, clk, ns);
  cudaEventRecord(e1);
  e = cudaDeviceSynchronize();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  unsigned long long* hc = new unsigned long long[blocks];
  unsigned long long* hn = new unsigned long long[blocks];
  cudaMemcpy(hc, clk, sizeof(unsigned long long) * blocks, cudaMemcpyDeviceToHost);
  cudaMemcpy(hn, ns, sizeof(unsigned long long) * blocks, cudaMemcpyDeviceToHost);
  double sc = 0, sn = 0;
  for (int i = 0; i < blocks; ++i) {
    sc += (double)hc[i];
    sn += (double)hn[i];
  }
  delete[] hc;
  delete[] hn;
  const double ghz = sc / sn;  // cycles per ns
  const double ops = 64.0 * iters * (double)blocks * threads;
  *per_clk = ops / ((double)ms * 1e6 * ghz * sms);
  *mhz = ghz * 1e3;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_topk(const int32_t* counts, int64_t q, int64_t n_panel, int k, int32_t* out_idx, double* out_dist,
                        cudaStream_t st) {
  if (q <= 0 || k <= 0) return cudaSuccess;
  if (k > kTopkMax || q > 2147483647LL) return cudaErrorInvalidValue;
  topk_kernel<<<(unsigned)q, kTopkThreads, 0, st>>>(counts, n_panel, k, out_idx, out_dist);
  return cudaGetLastError();
}

cudaError_t launch_topk_rows(const TopkRow* rows, int64_t n_rows, int64_t n_panel, cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  if (n_rows > 2147483647LL) return cudaErrorInvalidValue;
  topk_rows_kernel<<<(unsigned)n_rows, kTopkThreads, 0, st>>>(rows, n_panel);
  return cudaGetLastError();
}

cudaError_t probe_int_pipes(int device, double out[5]) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  uint32_t* buf = nullptr;
  unsigned long long *clk = nullptr, *ns = nullptr;
  const int blocks = sms * 4;
  if ((e = cudaMalloc(&buf, sizeof(uint32_t) * blocks * 256)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&clk, sizeof(unsigned long long) * blocks)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ns, sizeof(unsigned long long) * blocks)) != cudaSuccess) return e;
  double mhz[3] = {0, 0, 0};
  if (e == cudaSuccess) e = run_probe<0>(sms, buf, clk, ns, &out[0], &mhz[0]);
  if (e == cudaSuccess) e = run_probe<1>(sms, buf, clk, ns, &out[1], &mhz[1]);
  if (e == cudaSuccess) e = run_probe<2>(sms, buf, clk, ns, &out[2], &mhz[2]);
  out[3] = (mhz[0] + mhz[1] + mhz[2]) / 3.0;
  out[4] = sms;
  cudaFree(buf);
  cudaFree(clk);
  cudaFree(ns);
  return e;
}

}  // namespace ibs
