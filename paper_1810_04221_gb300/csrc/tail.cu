// tail.cu -- the coarse end of the V-cycle (Sec. 2.1, Algorithm 1) in one launch.
//
// Levels with few rows leave most of the GPU idle and their kernels are dominated by launch
// latency.  From the first level with at most kTailMaxRows rows down to the coarsest, the
// V-cycle runs here as one cooperative kernel: each step (smoothing sweep, residual,
// restriction, coarsest solve, prolongation) is a grid-stride loop over rows, and the steps
// are separated by a grid barrier.  The barrier's wait is bounded: a block that waits too
// long sets kErrTimeout and moves on, so a fault shows up as an error status, never a hang.
// Vectors written inside the kernel are read with ld.global.cg (L2), never through L1.
#include "solve.cuh"

namespace cwm {

namespace {

__device__ __forceinline__ void grid_barrier(unsigned *bar, int *err, unsigned spin_cap) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (++spins > spin_cap) {
          atomicOr(err, kErrTimeout);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <class V>
__device__ __forceinline__ V row_dot(const TailLevel<V> &L, int i, const V *x) {
  V acc = V(0);
  for (int k = L.rp[i]; k < L.rp[i + 1]; ++k) acc = fma(L.val[k], __ldcg(x + L.ci[k]), acc);
  return acc;
}

// One pre- and one post-sweep (the default cycle): each level costs two barriers.
//   down: bc[I] = sum_{m in I} p_m (b_m - sum_k a_mk x_k) with x = D^{-1} b formed on the fly;
//   up:   x_i = y_i + dinv_i (b_i - sum_k a_ik y_k) with y = D^{-1} b + P x_c formed on the fly.
template <class V>
__device__ __forceinline__ void tail_fused_11(const TailArgs<V> &A, const V *b0, V *x0, unsigned *bar, int *err,
                                              long long tid, long long nth) {
  // A lives in global memory: the level table is read through the cache, not copied
  for (int l = 0; l < A.nlev - 1; ++l) {
    const TailLevel<V> &L = A.lev[l];
    const TailLevel<V> &C = A.lev[l + 1];
    const V *b = l == 0 ? b0 : L.b;
    for (long long I = tid; I < C.n; I += nth) {
      V acc = V(0);
      for (int q = L.mptr[I]; q < L.mptr[I + 1]; ++q) {
        const int m = L.mlist[q];
        V dot = V(0);
        for (int k = L.rp[m]; k < L.rp[m + 1]; ++k) {
          const int j = L.ci[k];
          dot = fma(L.val[k], L.dinv[j] * __ldcg(b + j), dot);
        }
        acc += L.p[m] * (__ldcg(b + m) - dot);
      }
      C.b[I] = acc;
    }
    grid_barrier(bar, err, A.spin_cap);
  }
  {
    const TailLevel<V> &L = A.lev[A.nlev - 1];
    const V *b = A.nlev == 1 ? b0 : L.b;
    V *x = A.nlev == 1 ? x0 : L.x;
    if (L.dense) {
      const int lane = threadIdx.x & 31;
      const long long warp = tid >> 5, nwarps = nth >> 5;
      for (long long i = warp; i < L.n; i += nwarps) {
        const V *row = L.dense + i * L.n;
        V acc = V(0);
        for (int c = lane; c < L.n; c += 32) acc = fma(row[c], __ldcg(b + c), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = acc;
      }
      grid_barrier(bar, err, A.spin_cap);
    } else {
      const V *cur = nullptr;
      const int sweeps = A.coarse_sweeps;
      for (int s = 0; s < (sweeps > 0 ? sweeps : 1); ++s) {
        V *dst = s == sweeps - 1 || sweeps <= 0 ? x : (cur == L.t1 ? L.t2 : L.t1);
        for (long long i = tid; i < L.n; i += nth) {
          const V bi = __ldcg(b + i);
          dst[i] = sweeps <= 0 ? V(0)
                   : s == 0    ? L.dinv[i] * bi
                               : __ldcg(cur + i) + L.dinv[i] * (bi - row_dot(L, (int)i, cur));
        }
        grid_barrier(bar, err, A.spin_cap);
        cur = dst;
      }
    }
  }
  for (int l = A.nlev - 2; l >= 0; --l) {
    const TailLevel<V> &L = A.lev[l];
    const TailLevel<V> &C = A.lev[l + 1];
    const V *b = l == 0 ? b0 : L.b;
    V *xout = l == 0 ? x0 : L.x;
    for (long long i = tid; i < L.n; i += nth) {
      V dot = V(0);
      for (int k = L.rp[i]; k < L.rp[i + 1]; ++k) {
        const int j = L.ci[k];
        const V yj = fma(L.p[j], __ldcg(C.x + L.agg[j]), L.dinv[j] * __ldcg(b + j));
        dot = fma(L.val[k], yj, dot);
      }
      const V bi = __ldcg(b + i);
      const V yi = fma(L.p[i], __ldcg(C.x + L.agg[i]), L.dinv[i] * bi);
      xout[i] = yi + L.dinv[i] * (bi - dot);
    }
    grid_barrier(bar, err, A.spin_cap);
  }
}

template <class V>
__global__ void __launch_bounds__(256) k_vcycle_tail(const TailArgs<V> *__restrict__ Ap, const V *b0, V *x0,
                                                    unsigned *bar, int *err) {
  const TailArgs<V> &A = *Ap;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  if (A.pre == 1 && A.post == 1) {
    tail_fused_11(A, b0, x0, bar, err, tid, nth);
    return;
  }
  const V *xs_of[kTailMaxLevels];
  // ---- down: pre-smoothing, residual, restriction
  for (int l = 0; l < A.nlev - 1; ++l) {
    const TailLevel<V> &L = A.lev[l];
    const TailLevel<V> &C = A.lev[l + 1];
    const V *b = l == 0 ? b0 : L.b;
    const V *xs = nullptr;
    for (int s = 0; s < A.pre; ++s) {
      V *dst = (xs == L.t1) ? L.t2 : L.t1;
      for (long long i = tid; i < L.n; i += nth) {
        const V bi = __ldcg(b + i);
        dst[i] = s == 0 ? L.dinv[i] * bi : __ldcg(xs + i) + L.dinv[i] * (bi - row_dot(L, (int)i, xs));
      }
      grid_barrier(bar, err, A.spin_cap);
      xs = dst;
    }
    V *rt = (xs == L.t1) ? L.t2 : L.t1;
    for (long long i = tid; i < L.n; i += nth) rt[i] = __ldcg(b + i) - (xs ? row_dot(L, (int)i, xs) : V(0));
    grid_barrier(bar, err, A.spin_cap);
    for (long long I = tid; I < C.n; I += nth) {
      V acc = V(0);
      for (int k = L.mptr[I]; k < L.mptr[I + 1]; ++k) {
        const int m = L.mlist[k];
        acc += L.p[m] * __ldcg(rt + m);
      }
      C.b[I] = acc;
    }
    grid_barrier(bar, err, A.spin_cap);
    xs_of[l] = xs;
  }
  // ---- coarsest level: the sweeps from zero (dense operator when available)
  {
    const TailLevel<V> &L = A.lev[A.nlev - 1];
    const V *b = A.nlev == 1 ? b0 : L.b;
    V *x = A.nlev == 1 ? x0 : L.x;
    if (L.dense) {
      const int lane = threadIdx.x & 31;
      const long long warp = tid >> 5, nwarps = nth >> 5;
      for (long long i = warp; i < L.n; i += nwarps) {
        const V *row = L.dense + i * L.n;
        V acc = V(0);
        for (int c = lane; c < L.n; c += 32) acc = fma(row[c], __ldcg(b + c), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = acc;
      }
      grid_barrier(bar, err, A.spin_cap);
    } else if (A.coarse_sweeps <= 0) {
      for (long long i = tid; i < L.n; i += nth) x[i] = V(0);
      grid_barrier(bar, err, A.spin_cap);
    } else {
      const V *cur = nullptr;
      for (int s = 0; s < A.coarse_sweeps; ++s) {
        V *dst = s == A.coarse_sweeps - 1 ? x : (cur == L.t1 ? L.t2 : L.t1);
        for (long long i = tid; i < L.n; i += nth) {
          const V bi = __ldcg(b + i);
          dst[i] = s == 0 ? L.dinv[i] * bi : __ldcg(cur + i) + L.dinv[i] * (bi - row_dot(L, (int)i, cur));
        }
        grid_barrier(bar, err, A.spin_cap);
        cur = dst;
      }
    }
  }
  // ---- up: prolongation and post-smoothing
  for (int l = A.nlev - 2; l >= 0; --l) {
    const TailLevel<V> &L = A.lev[l];
    const TailLevel<V> &C = A.lev[l + 1];
    const V *b = l == 0 ? b0 : L.b;
    V *xout = l == 0 ? x0 : L.x;
    const V *xs = xs_of[l];
    V *y = (xs == L.t1) ? L.t2 : L.t1;
    for (long long i = tid; i < L.n; i += nth)
      y[i] = (xs ? __ldcg(xs + i) : V(0)) + L.p[i] * __ldcg(C.x + L.agg[i]);
    grid_barrier(bar, err, A.spin_cap);
    if (A.post <= 0) {
      for (long long i = tid; i < L.n; i += nth) xout[i] = __ldcg(y + i);
      grid_barrier(bar, err, A.spin_cap);
      continue;
    }
    const V *cur = y;
    for (int s = 0; s < A.post; ++s) {
      V *dst = s == A.post - 1 ? xout : (cur == L.t1 ? L.t2 : L.t1);
      for (long long i = tid; i < L.n; i += nth) {
        const V bi = __ldcg(b + i);
        dst[i] = __ldcg(cur + i) + L.dinv[i] * (bi - row_dot(L, (int)i, cur));
      }
      grid_barrier(bar, err, A.spin_cap);
      cur = dst;
    }
  }
}

}  // namespace

template <class V>
amg_status vcycle_tail(const TailArgs<V> &a, const TailArgs<V> *d_a, const V *b0, V *x0, unsigned *bar, int *err,
                       cudaStream_t s) {
  double bytes = 0.0;
  for (int l = 0; l < a.nlev; ++l) {
    const TailLevel<V> &L = a.lev[l];
    const double nnz = L.n ? (double)L.rp_host_nnz : 0.0;
    bytes += 4.0 * (L.n + 1) + (4.0 + sizeof(V)) * nnz * 3.0 + 10.0 * sizeof(V) * L.n;
  }
  CWM_TRACE("vcycle_tail", bytes, s);
  const int grid = a.grid > 0 ? a.grid : num_sms();
  int per_sm = 0;
  CWM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vcycle_tail<V>, 256, 0));
  if (per_sm < 1) {
    set_error("vcycle_tail: kernel cannot be resident");
    return AMG_ERR_UNSUPPORTED;
  }
  void *args[] = {(void *)&d_a, (void *)&b0, (void *)&x0, (void *)&bar, (void *)&err};
  CWM_CUDA(cudaLaunchCooperativeKernel((const void *)k_vcycle_tail<V>, dim3(grid), dim3(256), args, 0, s));
  count_launch();
  return AMG_OK;
}

template amg_status vcycle_tail<double>(const TailArgs<double> &, const TailArgs<double> *, const double *, double *,
                                        unsigned *, int *, cudaStream_t);
template amg_status vcycle_tail<float>(const TailArgs<float> &, const TailArgs<float> *, const float *, float *,
                                       unsigned *, int *, cudaStream_t);

}  // namespace cwm
