// fcg.cuh -- device helpers of the fused flexible-CG reductions (Sec. 3.2, Algorithm 3):
// block sums with few FP64 instructions, the last-block ticket, and the turning of every
// block's partial sums into the FCG scalars.  Shared by the CSR kernels (solve.cu) and the
// 3x3-block kernels (block3.cu).
#pragma once

#include "solve.cuh"

namespace cwm {

constexpr int kRedBlock = 256;  // block size the reductions below assume

// Block sums of up to three values per thread with few FP64 instructions (blockDim ==
// kRedBlock): the values go to shared memory, then warp w folds value w (kRedBlock / 32
// sequential adds per lane and five shuffle steps).  GB300 retires FP64 adds as whole-warp
// instructions at a low rate, so this beats a shuffle tree in every warp.  Results valid in
// every thread.
template <int NV>
__device__ __forceinline__ void block_sums(const double (&in)[NV], double (&out)[NV]) {
  __shared__ double s_in[NV][kRedBlock];
  __shared__ double s_out[NV];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < NV; ++v) s_in[v][threadIdx.x] = in[v];
  __syncthreads();
  if (w < NV) {
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < kRedBlock / 32; ++k) a += s_in[w][lane * (kRedBlock / 32) + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s_out[w] = a;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = s_out[v];
  __syncthreads();
}

// The block that finishes last (atomic ticket after a fence) reduces every block's partial
// sums in block order -- a fixed order, so the result does not depend on scheduling -- and
// resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(unsigned *tick) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(tick, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Sum of part[stride * i + c] over i = threadIdx.x, threadIdx.x + blockDim.x, ... < nb, in
// that order; the L2 loads of four iterations are issued before their adds (this runs on
// the critical path, in the last block, after every other block has finished).
template <int STRIDE, int C>
__device__ __forceinline__ double strided_sum(int nb, const double *part) {
  double a = 0.0;
  int i = threadIdx.x;
  const int bd = blockDim.x;
  for (; i + 3 * bd < nb; i += 4 * bd) {
    const double t0 = __ldcg(part + STRIDE * i + C), t1 = __ldcg(part + STRIDE * (i + bd) + C);
    const double t2 = __ldcg(part + STRIDE * (i + 2 * bd) + C), t3 = __ldcg(part + STRIDE * (i + 3 * bd) + C);
    a += t0;
    a += t1;
    a += t2;
    a += t3;
  }
  for (; i < nb; i += bd) a += __ldcg(part + STRIDE * i + C);
  return a;
}

__device__ __forceinline__ void fcg_scalars_from(int nb, const double *part, double *scal, int first) {
  double a = strided_sum<3, 0>(nb, part), b = strided_sum<3, 1>(nb, part), g = strided_sum<3, 2>(nb, part);
  {
    const double in3[3] = {a, b, g};
    double o3[3];
    block_sums<3>(in3, o3);
    a = o3[0];
    b = o3[1];
    g = o3[2];
  }
  if (threadIdx.x == 0) {
    double rho, coef;
    if (first) {
      rho = b;
      coef = 0.0;
      g = 0.0;
    } else {
      const double rp = scal[kRhoPrev];
      rho = b - g * g / rp;
      coef = g / rp;
    }
    scal[kAlpha] = a;
    scal[kBeta] = b;
    scal[kGamma] = g;
    scal[kRho] = rho;
    scal[kCoef] = coef;
    scal[kStep] = a / rho;
    scal[kRhoPrev] = rho;
    if (!(rho > 0.0) || !isfinite(rho) || !isfinite(a)) scal[kFlags] = 1.0;
  }
}

// The end of every SpMV + dots kernel: block sums of the three partial dot products into
// part[3 * block], and the last block's turning of all of them into the FCG scalars.
__device__ __forceinline__ void fcg_dots_finish(double sa, double sb, double sg, double *part, double *scal,
                                                unsigned *tick, int first) {
  const double in3[3] = {sa, sb, sg};
  double t3[3];
  block_sums<3>(in3, t3);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = t3[0];
    part[3 * blockIdx.x + 1] = t3[1];
    part[3 * blockIdx.x + 2] = t3[2];
  }
  if (last_block(tick)) {
    fcg_scalars_from(gridDim.x, part, scal, first);
    if (threadIdx.x == 0) *tick = 0u;
  }
}

}  // namespace cwm
