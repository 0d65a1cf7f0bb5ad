// noalloc.cu -- Suitor matching for callers that cannot allocate device memory.
//
// The matching kernels need 16 bytes of scratch per vertex (the packed suitor keys) and
// one error word.  cwm_suitor_match takes that scratch from the stream-ordered pool; this
// variant takes it from the file-scope array below instead, so a call makes no device
// allocation and frees nothing.  The array is sized for kNoAllocMaxVertices vertices and
// is held by every GPU that loads this library until the process exits.
#include "coarsen.cuh"

namespace cwm {
namespace {

constexpr int kNoAllocMaxVertices = 1 << 20;                       // 1,048,576 vertices
constexpr size_t kKeyBytes = (size_t)kNoAllocMaxVertices * 16;     // 16 MiB of suitor keys
constexpr size_t kScratchBytes = kKeyBytes + 256;                  // + the error word

// In host code this name is only a stand-in for the symbol, never a device address; the
// address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_suitor_scratch[kScratchBytes];

// The scratch array's device address on the current device, looked up on every call (a
// host-side table lookup that allocates nothing): an address kept from an earlier call
// would be stale after the host application resets the device (cudaDeviceReset), and a
// kernel given it would fault.
amg_status scratch_address(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_suitor_scratch);
  if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_suitor_scratch)", __FILE__, __LINE__);
  *out = p;
  return AMG_OK;
}

}  // namespace
}  // namespace cwm

extern "C" amg_status cwm_suitor_match_noalloc(int n, int64_t nnz, const int32_t *d_row_ptr,
                                               const int32_t *d_col, const double *d_w, int32_t *d_mate,
                                               void *stream) {
  using namespace cwm;
  if (n < 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX || (n > 0 && (!d_row_ptr || !d_mate)) ||
      (nnz > 0 && (!d_col || !d_w))) {
    set_error("cwm_suitor_match_noalloc: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxVertices) {
    set_error("cwm_suitor_match_noalloc: n = %d exceeds the fixed scratch capacity of %d vertices "
              "(use cwm_suitor_match)", n, kNoAllocMaxVertices);
    return AMG_ERR_UNSUPPORTED;
  }
  if (n == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  void *base = nullptr;
  CWM_TRY(scratch_address(&base));
  int *d_err = reinterpret_cast<int *>(static_cast<unsigned char *>(base) + kKeyBytes);
  // the array keeps the previous call's contents: the error word is cleared here, and
  // suitor_match clears the first n keys itself before the proposals start
  CWM_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  CWM_TRY(suitor_match(n, nnz, d_row_ptr, d_col, d_w, base, d_mate, nnz + n + 1024, d_err, s));
  int h_err = 0;
  CWM_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  return status_from_device_bits(h_err, "cwm_suitor_match_noalloc");
}
