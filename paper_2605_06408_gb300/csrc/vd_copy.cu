// vd_copy.cu -- transfers between device memory and page-locked host memory
// by the SMs (vd_copy of include/vd.h).
//
// On the GB300's Grace host every page-locked host buffer is reachable from
// a kernel through the same pointer, over NVLink-C2C. A grid of SM threads
// moving 16-byte vectors reaches the link's rate at once, whereas the copy
// engine, idle during a long build, starts its next transfer far slower.
#include <cuda_runtime.h>

#include <algorithm>

#include "vd_internal.cuh"

namespace vd {
namespace {

// 16-byte vectors over [0, n16), then the tail bytes; src and dst share
// their alignment modulo 16 and start at a 16-byte boundary here.
__global__ void copy16_kernel(const int4* __restrict__ src, int4* __restrict__ dst, size_t n16,
                              const unsigned char* __restrict__ tsrc, unsigned char* __restrict__ tdst, int tail) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < tail) tdst[threadIdx.x] = tsrc[threadIdx.x];
}

// Bytes, for the head before the first 16-byte boundary and for pointers
// whose alignments differ.
__global__ void copy1_kernel(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// 4-byte words, for pointers that share their alignment modulo 4 only.
__global__ void copy4_kernel(const unsigned* __restrict__ src, unsigned* __restrict__ dst, size_t n4) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) dst[i] = src[i];
}

// The address a kernel uses for p, or nullptr if the GPU cannot reach it.
const void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return p;
    case cudaMemoryTypeHost:
      if (a.devicePointer == nullptr || a.hostPointer == nullptr) return nullptr;
      // the same offset into the page-locked allocation
      return (const char*)a.devicePointer + ((const char*)p - (const char*)a.hostPointer);
    default:
      return nullptr;
  }
}

}  // namespace
}  // namespace vd

extern "C" int vd_copy(void* dst, const void* src, int64_t bytes, void* stream) {
  using namespace vd;
  if (bytes < 0) return VD_ERR_INVALID_ARG;
  if (bytes == 0) return VD_OK;
  if (dst == nullptr || src == nullptr) return VD_ERR_INVALID_ARG;
  const unsigned char* s = (const unsigned char*)device_view(src);
  unsigned char* d = (unsigned char*)device_view(dst);
  if (s == nullptr || d == nullptr) return VD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return VD_ERR_CUDA;
  const int threads = 256;
  const size_t n = (size_t)bytes;
  auto blocks_for = [&](size_t items) {
    const size_t b = (items + threads - 1) / threads;
    return (int)std::max((size_t)1, std::min(b, (size_t)sms * 8));
  };
  // each launch reports its own error (an earlier error of the caller's is
  // neither reported nor cleared)
  cudaError_t err = cudaSuccess;
  auto bytes1 = [&](const unsigned char* a, unsigned char* b, size_t m, int grid) {
    if (m == 0 || err != cudaSuccess) return;
    void* args[] = {(void*)&a, (void*)&b, (void*)&m};
    err = cudaLaunchKernel((const void*)copy1_kernel, dim3(grid), dim3(grid == 1 ? 32 : threads), args, 0, st);
  };
  if ((((uintptr_t)s ^ (uintptr_t)d) & 15u) == 0) {
    const size_t head = std::min(n, (size_t)((16u - ((uintptr_t)s & 15u)) & 15u));
    bytes1(s, d, head, 1);
    const size_t body = n - head;
    size_t n16 = body >> 4;
    int tail = (int)(body & 15u);
    if ((n16 || tail) && err == cudaSuccess) {
      const int4* a = (const int4*)(s + head);
      int4* b = (int4*)(d + head);
      const unsigned char* ta = s + head + 16 * n16;
      unsigned char* tb = d + head + 16 * n16;
      void* args[] = {(void*)&a, (void*)&b, (void*)&n16, (void*)&ta, (void*)&tb, (void*)&tail};
      err = cudaLaunchKernel((const void*)copy16_kernel, dim3(blocks_for(n16)), dim3(threads), args, 0, st);
    }
  } else if ((((uintptr_t)s ^ (uintptr_t)d) & 3u) == 0) {
    const size_t head = std::min(n, (size_t)((4u - ((uintptr_t)s & 3u)) & 3u));
    bytes1(s, d, head, 1);
    const size_t body = n - head;
    size_t n4 = body >> 2;
    if (n4 && err == cudaSuccess) {
      const unsigned* a = (const unsigned*)(s + head);
      unsigned* b = (unsigned*)(d + head);
      void* args[] = {(void*)&a, (void*)&b, (void*)&n4};
      err = cudaLaunchKernel((const void*)copy4_kernel, dim3(blocks_for(n4)), dim3(threads), args, 0, st);
    }
    bytes1(s + head + 4 * n4, d + head + 4 * n4, body & 3u, 1);
  } else {
    bytes1(s, d, n, blocks_for(n));
  }
  return err == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}
