// Complete-linkage clustering of the samples under the IBS distance matrix.
//
// The paper's identity-by-state section ("Identity-by-state matrices, complete
// linkage clustering") runs complete linkage on the IBS matrix and brings the
// clustering from O(n^3) down to O(n^2 log n).  The same merges come from the
// textbook greedy rule: merge the two active clusters at the smallest
// complete-linkage distance D(A, B) = max over members, maintained by
// D(A u B, C) = max(D(A, C), D(B, C)).  Ties: a cluster is represented by its
// smallest member, and among equal distances the smallest (representative A,
// representative B) pair merges first; NaN distances (no common non-missing
// marker) count as +infinity.
//
// Here every active row i keeps its minimum (D[i][j], j) over active j > i,
// compared lexicographically.  Each step is then O(n) parallel work:
//   1. the global minimum over the row minima, (value, row), lexicographic;
//   2. the merged row and column become the elementwise max of the two;
//   3. only the rows whose minimum pointed at one of the two merged clusters,
//      and the merged row itself, rescan their row.  A distance to the merged
//      cluster only grows, so no other row's minimum can change.
// The steps form one persistent CTA of 1,024 threads (32 warps); phases are
// separated by block barriers, which also order the memory updates.  Up to
// 12,000 samples the row minima and activity flags sit in shared memory.
// The working matrix is square and symmetric in HBM (8 bytes per entry).
#include <cstdint>

#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {

namespace {

constexpr int kClThreads = 1024;

// Triangle (upper, with diagonal, as ibs_compute writes it) -> square, NaN -> +inf.
__global__ void cl_init_kernel(const double* __restrict__ tri, int64_t n, double* __restrict__ D) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    const int64_t a = i < j ? i : j, b = i < j ? j : i;
    double d = tri[a * n - a * (a - 1) / 2 + (b - a)];
    if (d != d) d = __longlong_as_double(0x7ff0000000000000LL);
    D[t] = d;
  }
}

// Row minimum of row r over active columns j > r, (value, column) lexicographic,
// by one warp; column -1 when the row has no active column to its right.
__device__ __forceinline__ void row_min_warp(const double* __restrict__ D, const uint8_t* __restrict__ active,
                                             int64_t n, int64_t r, double& v_out, int32_t& j_out) {
  const int lane = threadIdx.x & 31;
  double v = 0;
  int32_t j = -1;
  for (int64_t c = r + 1 + lane; c < n; c += 32) {
    if (!active[c]) continue;
    const double d = D[r * n + c];
    if (j < 0 || d < v) {  // columns visited in increasing order per lane
      v = d;
      j = (int32_t)c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int32_t oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (oj >= 0 && (j < 0 || ov < v || (ov == v && oj < j))) {
      v = ov;
      j = oj;
    }
  }
  v_out = v;
  j_out = j;
}

__global__ void cl_rowmin_kernel(const double* __restrict__ D, const uint8_t* __restrict__ active, int64_t n,
                                 double* __restrict__ rmin_v, int32_t* __restrict__ rmin_j) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); r < n; r += warps) {
    double v;
    int32_t j;
    row_min_warp(D, active, n, r, v, j);
    if ((threadIdx.x & 31) == 0) {
      rmin_v[r] = v;
      rmin_j[r] = j;
    }
  }
}

struct ClArgs {
  double* D;
  int64_t n;
  double* rmin_v;
  int32_t* rmin_j;
  uint8_t* active;
  int32_t* id;
  int32_t* size;
  double* Z;  // [n-1][4]
};

// Row minima and activity flags live in shared memory when they fit (13 bytes
// per sample, up to kClSmemRows samples), so that the per-step argmin and the
// rescan checks touch no global memory.
constexpr int64_t kClSmemRows = 12000;
constexpr size_t cl_smem_bytes(int64_t n) { return n <= kClSmemRows ? (size_t)n * 13 + 16 : 0; }

__global__ void __launch_bounds__(kClThreads, 1) cl_main_kernel(ClArgs a) {
  extern __shared__ __align__(16) uint8_t cl_smem[];
  __shared__ double s_v[kClThreads / 32];
  __shared__ int32_t s_i[kClThreads / 32];
  __shared__ int64_t s_bi, s_bj;
  const int64_t n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (n <= kClSmemRows) {
    double* sv = reinterpret_cast<double*>(cl_smem);
    int32_t* sj = reinterpret_cast<int32_t*>(cl_smem + (size_t)n * 8);
    uint8_t* sa = cl_smem + (size_t)n * 12;
    for (int64_t r = threadIdx.x; r < n; r += kClThreads) {
      sv[r] = a.rmin_v[r];
      sj[r] = a.rmin_j[r];
      sa[r] = a.active[r];
    }
    __syncthreads();
    a.rmin_v = sv;
    a.rmin_j = sj;
    a.active = sa;
  }
  for (int64_t step = 0; step + 1 < n; ++step) {
    // 1. global minimum over the row minima: (value, row) lexicographic
    double v = 0;
    int32_t bi = -1;
    for (int64_t r = threadIdx.x; r < n; r += kClThreads) {
      if (!a.active[r] || a.rmin_j[r] < 0) continue;
      const double d = a.rmin_v[r];
      if (bi < 0 || d < v) {
        v = d;
        bi = (int32_t)r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || ov < v || (ov == v && oi < bi))) {
        v = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_v[warp] = v;
      s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bv = 0;
      int32_t b = -1;
      for (int w = 0; w < kClThreads / 32; ++w) {
        const int32_t oi = s_i[w];
        if (oi >= 0 && (b < 0 || s_v[w] < bv || (s_v[w] == bv && oi < b))) {
          bv = s_v[w];
          b = oi;
        }
      }
      const int64_t j = a.rmin_j[b];
      s_bi = b;
      s_bj = j;
      const int32_t ia = a.id[b], ib = a.id[j];
      double* z = a.Z + step * 4;
      z[0] = (double)(ia < ib ? ia : ib);
      z[1] = (double)(ia < ib ? ib : ia);
      z[2] = bv;
      z[3] = (double)(a.size[b] + a.size[j]);
    }
    __syncthreads();
    const int64_t i0 = s_bi, j0 = s_bj;
    // 2. the merged cluster's distances: elementwise max of the two rows
    for (int64_t k = threadIdx.x; k < n; k += kClThreads) {
      if (!a.active[k] || k == i0 || k == j0) continue;
      const double di = a.D[i0 * n + k], dj = a.D[j0 * n + k];
      const double d = di > dj ? di : dj;
      a.D[i0 * n + k] = d;
      a.D[k * n + i0] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.active[j0] = 0;
      a.id[i0] = (int32_t)(n + step);
      a.size[i0] += a.size[j0];
    }
    __syncthreads();
    // 3. rows whose minimum pointed at either merged cluster, and the merged
    // row: each warp checks 32 rows at a time and rescans the flagged ones
    for (int64_t base = (int64_t)warp * 32; base < n; base += kClThreads) {
      const int64_t r = base + lane;
      bool redo = false;
      if (r < n && a.active[r]) {
        const int32_t rj = a.rmin_j[r];
        redo = r == i0 || (r < i0 && rj == i0) || (r < j0 && rj == j0);
      }
      unsigned flagged = __ballot_sync(0xffffffffu, redo);
      while (flagged) {
        const int l = __ffs(flagged) - 1;
        flagged &= flagged - 1;
        const int64_t rr = base + l;
        double rv;
        int32_t nj;
        row_min_warp(a.D, a.active, n, rr, rv, nj);
        if (lane == 0) {
          a.rmin_v[rr] = rv;
          a.rmin_j[rr] = nj;
        }
      }
    }
    __syncthreads();
  }
}

__global__ void cl_state_init_kernel(int64_t n, uint8_t* active, int32_t* id, int32_t* size) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    active[i] = 1;
    id[i] = (int32_t)i;
    size[i] = 1;
  }
}

}  // namespace

size_t cluster_workspace_bytes(int64_t n) {
  return (size_t)n * (size_t)n * 8 + (size_t)n * (8 + 4 + 4 + 4 + 1) + 4096;
}

cudaError_t launch_cluster_complete(const double* tri, int64_t n, double* Z, void* work, int num_sms,
                                    cudaStream_t st) {
  if (n <= 1) return cudaSuccess;
  uint8_t* w = static_cast<uint8_t*>(work);
  double* D = reinterpret_cast<double*>(w);
  w += (size_t)n * n * 8;
  double* rmin_v = reinterpret_cast<double*>(w);
  w += (size_t)n * 8;
  int32_t* rmin_j = reinterpret_cast<int32_t*>(w);
  w += (size_t)n * 4;
  int32_t* id = reinterpret_cast<int32_t*>(w);
  w += (size_t)n * 4;
  int32_t* size = reinterpret_cast<int32_t*>(w);
  w += (size_t)n * 4;
  uint8_t* active = w;
  const int grid = num_sms * 8;
  cl_init_kernel<<<grid, 256, 0, st>>>(tri, n, D);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cl_state_init_kernel<<<grid, 256, 0, st>>>(n, active, id, size);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cl_rowmin_kernel<<<grid, 256, 0, st>>>(D, active, n, rmin_v, rmin_j);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ClArgs args{D, n, rmin_v, rmin_j, active, id, size, Z};
  const size_t smem = cl_smem_bytes(n);
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(cl_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return e;
  cl_main_kernel<<<1, kClThreads, smem, st>>>(args);
  return cudaGetLastError();
}

}  // namespace ibs
