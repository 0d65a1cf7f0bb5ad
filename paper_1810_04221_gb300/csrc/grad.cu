// grad.cu -- the sampled outer product used by the backward pass of a solve x = A^{-1} b:
// for a loss L(x), dL/dA = -lambda x^T with lambda = A^{-1} dL/dx (A symmetric), needed only
// on the stored pattern of A.  This is a streaming kernel: one pass over the CSR pattern with
// gathers of x (row-block layout as the SpMV kernels).
#include "common.cuh"

namespace cwm {
namespace {

constexpr int kOB = 256;
constexpr int kOE = 8;
constexpr int kOC = kOB * kOE;

// out[k] = alpha * (lambda_i * x_j) for stored slot k = (i, j)
__global__ void __launch_bounds__(kOB) k_pattern_outer(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const double *__restrict__ lambda,
                                                       const double *__restrict__ x, double alpha,
                                                       double *__restrict__ out) {
  __shared__ int s_rp[kOB + 1];
  __shared__ double s_l[kOB];
  __shared__ unsigned char s_row[kOC];
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * kOB;
  const int nrows = min(kOB, n - r0);
  for (int i = t; i <= nrows; i += kOB) s_rp[i] = rp[r0 + i];
  if (t < nrows) s_l[t] = lambda[r0 + t];
  __syncthreads();
  const int rs = s_rp[0], re = s_rp[nrows];
  const int my_s = t < nrows ? s_rp[t] : 0, my_e = t < nrows ? s_rp[t + 1] : 0;
  for (int c0 = rs; c0 < re; c0 += kOC) {
    const int cend = min(c0 + kOC, re);
    for (int k = max(my_s, c0); k < min(my_e, cend); ++k) s_row[k - c0] = (unsigned char)t;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kOE; ++e) {
      const int k = c0 + e * kOB + t;
      if (k < cend) {
        const int j = __ldcs(ci + k);
        const double li = s_l[s_row[k - c0]];
        __stcs(out + k, alpha * (li * __ldg(x + j)));
      }
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace cwm

extern "C" amg_status cwm_pattern_outer(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                                        const double *d_lambda, const double *d_x, double alpha, double *d_out,
                                        void *stream) {
  using namespace cwm;
  if (n < 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX || (n > 0 && (!d_row_ptr || !d_lambda || !d_x)) ||
      (nnz > 0 && (!d_col || !d_out))) {
    set_error("cwm_pattern_outer: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  if (n == 0 || nnz == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CWM_TRACE("pattern_outer", 4.0 * (n + 1) + 12.0 * nnz + 16.0 * n, s);
  k_pattern_outer<<<(n + kOB - 1) / kOB, kOB, 0, s>>>(n, d_row_ptr, d_col, d_lambda, d_x, alpha, d_out);
  CWM_LAUNCH();
  return AMG_OK;
}
