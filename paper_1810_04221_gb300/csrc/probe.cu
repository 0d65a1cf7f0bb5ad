// probe.cu -- measured FP64 issue rates of the GPU the library runs on: the denominators
// against which the FP64-bound kernels (the edge weights with their IEEE divisions, the
// binary64 SpMV of the FCG) are reported.  Not a step of the method.
#include "common.cuh"

namespace cwm {
namespace {

constexpr int kProbeChains = 8;   // independent chains per thread
constexpr int kProbeSteps = 512;  // operations per chain
constexpr int kProbeBlock = 256;

// Every thread runs kProbeChains independent FMA chains of kProbeSteps steps; the result is
// stored only if it takes a value it cannot reach, so the chains are not optimised away.
__global__ void __launch_bounds__(kProbeBlock) k_probe_dfma(double seed, double *sink) {
  double a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.999999, k = 1e-7;
  for (int s = 0; s < kProbeSteps; ++s) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], m, k);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) t += a[c];
  if (t == -1.0) *sink = t;
}

// Same with correctly rounded divisions a <- (a + k) / m.
__global__ void __launch_bounds__(kProbeBlock) k_probe_ddiv(double seed, double *sink) {
  double a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 1.000001;
  for (int s = 0; s < kProbeSteps / 8; ++s) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = __ddiv_rn(a[c], m);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) t += a[c];
  if (t == -1.0) *sink = t;
}

template <class K>
amg_status time_kernel(K kernel, int grid, double *sink, cudaStream_t s, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CWM_CUDA(cudaEventCreate(&e0));
  CWM_CUDA(cudaEventCreate(&e1));
  kernel<<<grid, kProbeBlock, 0, s>>>(1.0, sink);  // warm-up
  CWM_LAUNCH();
  cudaEventRecord(e0, s);
  for (int r = 0; r < 5; ++r) kernel<<<grid, kProbeBlock, 0, s>>>(1.0 + r, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "probe timing", __FILE__, __LINE__);
  *ms = t / 5.f;
  return AMG_OK;
}

}  // namespace
}  // namespace cwm

extern "C" amg_status cwm_fp64_rates(double *fma_per_s, double *div_per_s, void *stream) {
  using namespace cwm;
  if (!fma_per_s || !div_per_s) {
    set_error("cwm_fp64_rates: NULL output");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<double> sink;
  CWM_TRY(sink.alloc(1, s));
  const int grid = num_sms() * 8;
  const double threads = (double)grid * kProbeBlock * kProbeChains;
  float ms = 0.f;
  CWM_TRY(time_kernel(k_probe_dfma, grid, sink.get(), s, &ms));
  *fma_per_s = threads * kProbeSteps / (ms * 1e-3);
  CWM_TRY(time_kernel(k_probe_ddiv, grid, sink.get(), s, &ms));
  *div_per_s = threads * (kProbeSteps / 8) / (ms * 1e-3);
  CWM_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
}
