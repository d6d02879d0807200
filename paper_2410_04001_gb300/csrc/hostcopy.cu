// Copies between page-locked host memory and device memory by a kernel that reads and
// writes through the unified address space.  For the few hundred KB of a batch (the
// collocation points and s of one SPInProp step) a grid of 16-byte loads over the
// chip-to-chip link to the host takes about half the time of a copy-engine transfer, and
// the copy is one more kernel on the caller's stream (it is captured into a CUDA graph
// with the step like any launch).  Host bytes are read with ld.global.cv, so a value the
// host wrote after an earlier read of the same line is fetched again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lrnr_internal.cuh"

namespace lrnr {
namespace {

constexpr int HC_THREADS = 256;

// Bytes [0, head) and [head + 16 n16, head + 16 n16 + tail) one at a time, the
// 16-byte-aligned middle as uint4: every index below is within its range.
__global__ void __launch_bounds__(HC_THREADS) k_copy_pinned(const unsigned char *__restrict__ src,
                                                            unsigned char *__restrict__ dst, size_t head,
                                                            size_t n16, size_t tail) {
  const size_t tid = (size_t)blockIdx.x * HC_THREADS + threadIdx.x;
  const size_t nth = (size_t)gridDim.x * HC_THREADS;
  const uint4 *s16 = reinterpret_cast<const uint4 *>(src + head);
  uint4 *d16 = reinterpret_cast<uint4 *>(dst + head);
  for (size_t i = tid; i < n16; i += nth) d16[i] = __ldcv(s16 + i);
  for (size_t i = tid; i < head; i += nth) dst[i] = __ldcv(src + i);
  const size_t t0 = head + 16 * n16;
  for (size_t i = tid; i < tail; i += nth) dst[t0 + i] = __ldcv(src + t0 + i);
}

// The address a kernel on the current device uses for `p`: itself for device or managed
// memory of this device, the mapped address for page-locked host memory; nullptr for
// pageable host memory, another device's memory or an unknown pointer.
const void *kernel_address(const void *p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  switch (a.type) {
    case cudaMemoryTypeHost: return a.devicePointer;
    case cudaMemoryTypeDevice: return a.device == dev ? p : nullptr;
    case cudaMemoryTypeManaged: return p;
    default: return nullptr;
  }
}

}  // namespace
}  // namespace lrnr

using namespace lrnr;

extern "C" lrnr_status lrnr_copy_pinned(void *dst, const void *src, size_t bytes, void *stream) {
  if (bytes == 0) return LRNR_OK;
  if (!dst || !src) return LRNR_EINVAL;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LRNR_ECUDA;
  const unsigned char *s = static_cast<const unsigned char *>(kernel_address(src, dev));
  unsigned char *d = static_cast<unsigned char *>(const_cast<void *>(kernel_address(dst, dev)));
  if (!s || !d) return LRNR_EINVAL;
  const uintptr_t sa = reinterpret_cast<uintptr_t>(s), da = reinterpret_cast<uintptr_t>(d);
  if ((sa < da && da - sa < bytes) || (da < sa && sa - da < bytes)) return LRNR_EINVAL;   // overlap
  size_t head = bytes, n16 = 0, tail = 0;
  if ((sa & 15) == (da & 15)) {
    head = std::min(bytes, (size_t)((16 - (sa & 15)) & 15));
    n16 = (bytes - head) / 16;
    tail = bytes - head - 16 * n16;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t work = std::max(n16, std::max(head, tail));
  const int blocks = (int)std::min<size_t>((work + HC_THREADS - 1) / HC_THREADS, (size_t)4 * sms);
  k_copy_pinned<<<std::max(blocks, 1), HC_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(s, d, head, n16,
                                                                                         tail);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRNR_OK : LRNR_ECUDA;
}
