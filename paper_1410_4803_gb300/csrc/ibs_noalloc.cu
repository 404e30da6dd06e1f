// ibs_compute_noalloc: the plain all-pairs computation for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// result: code running while a CUDA graph is being captured, applications
// whose memory pool owns every byte of the device and forbids side
// allocations, real-time services that allocate only at start-up, and
// plug-ins hosted by a process that controls the allocator.  For them this
// entry point keeps its bit-plane scratch in a fixed array that is part of
// the library's device image, so a call only enqueues kernels.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes.  Each
// GPU that loads this library holds that memory until the process exits.  In
// host code the array's name is only a host-side stand-in, never a device
// address, so the entry point looks the address up with cudaGetSymbolAddress
// once per device (with that device current) and passes it to the kernels.
#include <mutex>

#include "ibs_ctx.h"
#include "ibs_device.cuh"

namespace ibs {
namespace {

// Bit-plane scratch of the allocation-free entry point: 64 MiB.
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) uint32_t g_noalloc_planes[kNoAllocScratchBytes / sizeof(uint32_t)];
// Status word of the kernels' bounded waits (cleared before every call).
static __device__ __align__(16) int g_noalloc_status[4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
bool g_ready[kMaxDevices] = {};
uint32_t* g_planes_addr[kMaxDevices] = {};
int* g_status_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: resolve the arrays' device addresses.
ibs_status setup_device(int dev) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_ready[dev]) return IBS_OK;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_planes);
  if (e != cudaSuccess) return fail(IBS_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
  g_planes_addr[dev] = static_cast<uint32_t*>(p);
  e = cudaGetSymbolAddress(&p, g_noalloc_status);
  if (e != cudaSuccess) return fail(IBS_ECUDA, "cudaGetSymbolAddress(status) failed: %s", cudaGetErrorString(e));
  g_status_addr[dev] = static_cast<int*>(p);
  e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(IBS_ECUDA, "cudaDeviceGetAttribute failed: %s", cudaGetErrorString(e));
  g_ready[dev] = true;
  return IBS_OK;
}

// True when p is device (or managed) memory that device `dev` can use as a
// kernel operand.  cudaPointerGetAttributes is not a stream operation, so the
// check is also valid while a stream is being captured.
bool device_ptr_on(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace ibs

using namespace ibs;

extern "C" ibs_status ibs_compute_noalloc(const uint8_t* packed, int64_t n, int64_t m, int32_t* out_counts,
                                          double* out_dist, void* stream) {
  clear_error();
  if (!packed || !out_counts) return fail(IBS_EINVAL, "packed and out_counts must be non-NULL");
  if (n < 1 || n > 2147483647LL) return fail(IBS_EINVAL, "n_samples %lld out of range [1, 2^31)", (long long)n);
  if (m < 1 || m > 2147483647LL) return fail(IBS_EINVAL, "n_variants %lld out of range [1, 2^31)", (long long)m);
  if (reinterpret_cast<uintptr_t>(out_counts) % 16) return fail(IBS_EINVAL, "out_counts must be 16-byte aligned");
  if (out_dist && reinterpret_cast<uintptr_t>(out_dist) % 8) return fail(IBS_EINVAL, "out_dist must be 8-byte aligned");
  const PlaneGeom geo = PlaneGeom::make(n, m);
  if (geo.bytes() > kNoAllocScratchBytes)
    return fail(IBS_EINVAL,
                "n_samples=%lld x n_variants=%lld needs %zu bytes of bit-plane scratch; the allocation-free entry "
                "point has %zu (use ibs_compute for larger inputs)",
                (long long)n, (long long)m, geo.bytes(), kNoAllocScratchBytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(IBS_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(IBS_EINVAL, "device ordinal %d not supported", dev);
  if (!device_ptr_on(packed, dev) || !device_ptr_on(out_counts, dev) || (out_dist && !device_ptr_on(out_dist, dev)))
    return fail(IBS_EINVAL, "packed, out_counts and out_dist must be device memory of the current device (%d)", dev);
  if (ibs_status s = setup_device(dev)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The status word must start at zero; the planes are fully rewritten by the transpose.
  IBS_CUDA_TRY(cudaMemsetAsync(g_status_addr[dev], 0, sizeof(int) * 4, st));
  BedSource src;
  src.packed = packed;
  src.row_bytes = (n + 3) / 4;
  src.n_src = n;
  IBS_CUDA_TRY(launch_planes(src, n, m, geo, g_planes_addr[dev], g_status_addr[dev], st));
  // Small triangles (fewer tiles than two waves) split the marker axis as
  // ibs_compute does; their partial counts ([P][4] int32, zeroed here) sit in
  // the same scratch after the planes when both fit, else one split runs.
  const int64_t tiles = geo.n_blocks * (geo.n_blocks + 1) / 2;
  int splits = tri_splits_for(tiles, geo.n_chunks, g_sms[dev]);
  const size_t planes_bytes = (geo.bytes() + 255) / 256 * 256;
  const size_t partial_bytes = (size_t)(n * (n + 1) / 2) * 16;
  if (splits > 1 && planes_bytes + partial_bytes > kNoAllocScratchBytes) splits = 1;
  int32_t* partial =
      splits > 1 ? reinterpret_cast<int32_t*>(reinterpret_cast<uint8_t*>(g_planes_addr[dev]) + planes_bytes) : nullptr;
  if (partial) IBS_CUDA_TRY(cudaMemsetAsync(partial, 0, partial_bytes, st));
  IBS_CUDA_TRY(launch_tri(1, g_planes_addr[dev], geo, splits, out_counts, out_dist, partial, false,
                          g_status_addr[dev], g_sms[dev], st));
  if (partial) IBS_CUDA_TRY(launch_finalize(partial, n, out_counts, out_dist, false, st));
  return IBS_OK;
}

extern "C" ibs_status ibs_noalloc_status(void* stream) {
  clear_error();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(IBS_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(IBS_EINVAL, "device ordinal %d not supported", dev);
  if (ibs_status s = setup_device(dev)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IBS_CUDA_TRY(cudaStreamSynchronize(st));
  int word = 0;
  // a 4-byte read from the fixed status array: no allocation, staged by the runtime
  IBS_CUDA_TRY(cudaMemcpy(&word, g_status_addr[dev], sizeof(int), cudaMemcpyDeviceToHost));
  if (word == kDevTimeout)
    return fail(IBS_ETIMEOUT, "a bounded device wait of ibs_compute_noalloc expired; its outputs are undefined");
  if (word != 0) return fail(IBS_ECUDA, "device status word %d", word);
  return IBS_OK;
}
