// probe.cu -- measured FP64 issue rates of the GPU the library runs on: the denominators
// against which the FP64-bound kernels (the edge weights, the binary64 SpMV of the FCG) are
// reported; and the self-check of the integer-pipe quotient of the edge weights against the
// hardware division.  Not steps of the method.
#include "common.cuh"
#include "divint.cuh"

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

// splitmix64 (Steele, Lea and Flood, 2014): the operand bits of check i are a function of
// (seed, i) alone.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double make_f64(unsigned long long sign, int biased_exp, unsigned long long frac) {
  return __longlong_as_double((long long)((sign << 63) | ((unsigned long long)biased_exp << 52) |
                                          (frac & ((1ull << 52) - 1ull))));
}

// Operand pair i, by class i % 8: raw 64-bit patterns (zeros, subnormals, infinities, NaNs
// and every exponent); exponents within 40 of each other; x = RN(y q) with y, q in [1, 2)
// (quotients next to a binary64 value, so near rounding boundaries); y a power of two;
// mx = my; significands of all ones or a single low bit; quotient exponents at the edges of
// the normal range (and just outside it).
__device__ void div_check_pair(unsigned long long seed, long long i, double *x, double *y) {
  const unsigned long long h1 = mix64(seed ^ (2ull * (unsigned long long)i)),
                           h2 = mix64(seed ^ (2ull * (unsigned long long)i + 1ull)), h3 = mix64(h1 ^ h2);
  const int cls = (int)(i & 7);
  if (cls == 0) {
    *x = __longlong_as_double((long long)h1);
    *y = __longlong_as_double((long long)h2);
  } else if (cls == 1) {
    *x = make_f64(h3 & 1, 1023 + (int)((h3 >> 8) % 81) - 40, h1);
    *y = make_f64((h3 >> 1) & 1, 1023 + (int)((h3 >> 20) % 81) - 40, h2);
  } else if (cls == 2) {
    const double yy = make_f64(0, 1023, h1), qq = make_f64(0, 1023, h2);
    *x = __dmul_rn(yy, qq);
    *y = yy;
  } else if (cls == 3) {
    *x = make_f64(h3 & 1, 1 + (int)((h1 >> 53) % 2046), h2);
    *y = make_f64(0, 1 + (int)((h3 >> 11) % 2046), 0);
  } else if (cls == 4) {
    *x = make_f64(0, 1 + (int)((h3 >> 11) % 2046), h1);
    *y = make_f64(h3 & 1, 1 + (int)((h3 >> 30) % 2046), h1);
  } else if (cls == 5) {
    const unsigned long long ones = (1ull << 52) - 1ull;
    *x = make_f64(0, 1000 + (int)(h3 % 47), (h1 & 1) ? ones : (1ull << (h1 >> 58) % 52));
    *y = make_f64(0, 1000 + (int)((h3 >> 8) % 47), (h2 & 1) ? ones : h2 >> 12);
  } else if (cls == 6) {
    // ex - ey + 1023 near 1 (subnormal quotients just below) and near 2046 (overflow above)
    const int ey = 1 + (int)(h3 % 2046);
    const int ex = (h3 >> 32) & 1 ? ey - 1022 + (int)((h3 >> 40) % 5) - 2 : ey + 1022 + (int)((h3 >> 40) % 5) - 2;
    *x = make_f64(0, ex < 1 ? 1 : (ex > 2046 ? 2046 : ex), h1);
    *y = make_f64(0, ey, h2);
  } else {
    *x = make_f64(h3 & 1, 1023 + (int)((h3 >> 8) % 21) - 10, h1);
    *y = make_f64(0, 1023 + (int)((h3 >> 20) % 21) - 10, h2);
  }
}

__global__ void k_div_check(long long n, unsigned long long seed, unsigned long long *count,
                            unsigned long long *first) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double x, y;
    div_check_pair(seed, i, &x, &y);
    if (__double_as_longlong(__ddiv_rn(x, y)) != __double_as_longlong(div_rn_int(x, y))) {
      atomicAdd(count, 1ull);
      atomicMin(first, (unsigned long long)i);
    }
  }
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

extern "C" amg_status cwm_div_check(long long n, unsigned long long seed, long long *mismatches, long long *first,
                                    void *stream) {
  using namespace cwm;
  if (!mismatches || !first || n < 0) {
    set_error("cwm_div_check: NULL output or negative count");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<unsigned long long> buf;
  CWM_TRY(buf.alloc(2, s));
  const unsigned long long init[2] = {0ull, ~0ull};
  CWM_CUDA(cudaMemcpyAsync(buf.get(), init, sizeof(init), cudaMemcpyHostToDevice, s));
  if (n > 0) {
    k_div_check<<<num_sms() * 8, 256, 0, s>>>(n, seed, buf.get(), buf.get() + 1);
    CWM_LAUNCH();
  }
  unsigned long long out[2] = {0ull, 0ull};
  CWM_CUDA(cudaMemcpyAsync(out, buf.get(), sizeof(out), cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  *mismatches = (long long)out[0];
  *first = out[0] ? (long long)out[1] : -1;
  return AMG_OK;
}
