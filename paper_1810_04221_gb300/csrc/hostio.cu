// hostio.cu -- moving a caller's host arrays in and out of the device for amg_setup and
// amg_pcg_solve (and cwm_copy).
//
// Page-locked host memory is read and written by SM kernels through its device mapping
// (over the GPU's link to host memory), not by the copy engines: on GB300 the copy-engine
// transfer of the 745 MB of a Q1 elasticity 64^3 input ran at 212 GB/s but stalled about
// every 0.46 s for 40-70 ms, while the same transfer by SM loads from the mapped pinned
// buffer ran at 211 GB/s with no stall in 160 timed copies (spaced like the steps of a
// solve, and back to back).  Pageable host memory goes through cudaMemcpyAsync, which
// stages it (the call then waits for the copy); device memory is copied device to device.
#include "common.cuh"

namespace cwm {

namespace {

constexpr int kCopyBlock = 512;

// dst[i] = src[i] for i < n elements of T (16-, 8-, 4- or 1-byte words), grid-stride.
template <class T>
__global__ void __launch_bounds__(kCopyBlock) k_copy(const T *__restrict__ src, T *__restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <class T>
amg_status launch_copy(const void *src, void *dst, long long n, cudaStream_t s) {
  if (n <= 0) return AMG_OK;
  // four resident blocks of 512 threads per SM kept the link busy (2 to 8 measured equal)
  k_copy<T><<<grid_for(n, kCopyBlock, num_sms() * 4), kCopyBlock, 0, s>>>((const T *)src, (T *)dst, n);
  CWM_LAUNCH();
  return AMG_OK;
}

// Copies with the widest word that both addresses and the size allow.
amg_status kernel_copy(const void *src, void *dst, size_t bytes, cudaStream_t s) {
  const uintptr_t a = (uintptr_t)src | (uintptr_t)dst | (uintptr_t)bytes;
  if ((a & 15) == 0) return launch_copy<int4>(src, dst, (long long)(bytes / 16), s);
  if ((a & 7) == 0) return launch_copy<unsigned long long>(src, dst, (long long)(bytes / 8), s);
  if ((a & 3) == 0) return launch_copy<unsigned>(src, dst, (long long)(bytes / 4), s);
  return launch_copy<unsigned char>(src, dst, (long long)bytes, s);
}

}  // namespace

MemKind mem_kind(const void *p, void **dev_alias) {
  cudaPointerAttributes at;
  if (dev_alias) *dev_alias = nullptr;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return MemKind::kPageable;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return MemKind::kDevice;
    case cudaMemoryTypeHost:
      if (!at.devicePointer || !at.hostPointer) return MemKind::kPageable;
      // the device address of byte p (device and host addresses of the mapping differ by a
      // constant; with unified addressing they coincide)
      if (dev_alias) *dev_alias = (char *)at.devicePointer + ((const char *)p - (const char *)at.hostPointer);
      return MemKind::kPinned;
    default:
      return MemKind::kPageable;
  }
}

amg_status copy_in(void *d_dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return AMG_OK;
  void *alias = nullptr;
  switch (mem_kind(src, &alias)) {
    case MemKind::kDevice:
      CWM_CUDA(cudaMemcpyAsync(d_dst, src, bytes, cudaMemcpyDeviceToDevice, s));
      return AMG_OK;
    case MemKind::kPinned:
      return kernel_copy(alias, d_dst, bytes, s);
    default:
      CWM_CUDA(cudaMemcpyAsync(d_dst, src, bytes, cudaMemcpyDefault, s));
      return AMG_OK;
  }
}

amg_status copy_out(void *dst, const void *d_src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return AMG_OK;
  void *alias = nullptr;
  switch (mem_kind(dst, &alias)) {
    case MemKind::kDevice:
      CWM_CUDA(cudaMemcpyAsync(dst, d_src, bytes, cudaMemcpyDeviceToDevice, s));
      return AMG_OK;
    case MemKind::kPinned:
      return kernel_copy(d_src, alias, bytes, s);
    default:
      CWM_CUDA(cudaMemcpyAsync(dst, d_src, bytes, cudaMemcpyDefault, s));
      return AMG_OK;
  }
}

}  // namespace cwm

extern "C" amg_status cwm_copy(void *dst, const void *src, int64_t bytes, void *stream) {
  using namespace cwm;
  if (bytes < 0 || (bytes > 0 && (!dst || !src))) {
    set_error("cwm_copy: NULL pointer or negative size");
    return AMG_ERR_INVALID_ARG;
  }
  if (bytes == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const MemKind kd = mem_kind(dst, nullptr), ks = mem_kind(src, nullptr);
  if (kd == MemKind::kDevice) return copy_in(dst, src, (size_t)bytes, s);
  if (ks == MemKind::kDevice) return copy_out(dst, src, (size_t)bytes, s);
  set_error("cwm_copy: neither pointer is device memory");
  return AMG_ERR_INVALID_ARG;
}
