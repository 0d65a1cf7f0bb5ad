// solve.cu -- solve-phase kernels: CSR row products with a sub-warp ("miniwarp", Sec. 3.1)
// per row, the l1-Jacobi sweep (Sec. 3.2), residual + restriction by the aggregation
// prolongator, prolongation, the one-block coarsest solve, and the fused FCG kernels of
// Sec. 3.2 (three dot products in one pass with the SpMV, paired vector updates).
#include "solve.cuh"

namespace cwm {

constexpr int kBlock = 256;

// All T lanes of every tile of the warp call this together (warp-uniform loops), so the
// full-mask shuffles are well defined; inactive tiles contribute zero.
template <class V, int T>
__device__ __forceinline__ V tile_row_dot(const int *__restrict__ rp, const int *__restrict__ ci,
                                          const V *__restrict__ val, const V *__restrict__ x, long long row,
                                          bool active, int lane) {
  V s = V(0);
  if (active && x) {
    const int b = rp[row], e = rp[row + 1];
    for (int k = b + lane; k < e; k += T) s += val[k] * __ldg(x + ci[k]);
  }
#pragma unroll
  for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
  return s;
}

#define CWM_TILE_LOOP(T, n)                                                         \
  const int lane = threadIdx.x & (T - 1);                                           \
  const int sub = (threadIdx.x & 31) / T;                                           \
  constexpr int kRowsPerWarp = 32 / T;                                              \
  const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; \
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;                \
  for (long long base = warp_id * kRowsPerWarp; base < (n); base += nwarps * kRowsPerWarp)

static int rows_grid(long long n, int T) {
  const long long warps = (n * T + 31) / 32;
  return grid_for(warps * 32, kBlock, num_sms() * 8);
}

#define CWM_DISPATCH_T(T, ...)                 \
  switch (T) {                                 \
    case 4: { constexpr int kT = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int kT = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int kT = 16; __VA_ARGS__; } break; \
    default: { constexpr int kT = 32; __VA_ARGS__; } break; \
  }

// ------------------------------------------------------------ block sums ----
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += ws[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// ------------------------------------------------------------ elementwise ----
template <class V>
__global__ void k_scale(int n, const V *__restrict__ dinv, const V *__restrict__ b, V *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = dinv[i] * b[i];
}

template <class V>
amg_status scale(int n, const V *dinv, const V *b, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("scale", 3.0 * sizeof(V) * n, s);
  k_scale<V><<<grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s>>>(n, dinv, b, y);
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
__global__ void k_prolong(int n, const int *__restrict__ agg, const V *__restrict__ p, const V *__restrict__ xc,
                          const V *__restrict__ x, V *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const V base = x ? x[i] : V(0);
    y[i] = base + p[i] * __ldg(xc + agg[i]);
  }
}

template <class V>
amg_status prolong(int n, const int *agg, const V *p, const V *xc, const V *x, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("prolong", (4.0 + (x ? 3.0 : 2.0) * sizeof(V)) * n, s);
  k_prolong<V><<<grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s>>>(n, agg, p, xc, x, y);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ l1-Jacobi ----
template <class V, int T>
__global__ void __launch_bounds__(kBlock) k_jacobi(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const V *__restrict__ val, const V *__restrict__ dinv,
                                                   const V *__restrict__ b, const V *__restrict__ x,
                                                   V *__restrict__ y) {
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const V dot = tile_row_dot<V, T>(rp, ci, val, x, row, active, lane);
    if (active && lane == 0) y[row] = x[row] + dinv[row] * (b[row] - dot);
  }
}

template <class V>
amg_status jacobi(const CsrView<V> &A, const V *dinv, const V *b, const V *x, V *y, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("jacobi", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 4.0 * sizeof(V) * A.n, s);
  CWM_DISPATCH_T(A.tile, (k_jacobi<V, kT><<<rows_grid(A.n, kT), kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, dinv, b, x, y)));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ residual + restriction ----
// One tile per coarse row I; its members' residual rows are formed in turn and
// accumulated in member order (ascending), so the result is deterministic.
template <class V, int T>
__global__ void __launch_bounds__(kBlock)
    k_resid_restrict(int nc, const int *__restrict__ rp, const int *__restrict__ ci, const V *__restrict__ val,
                     const int *__restrict__ mptr, const int *__restrict__ mlist, const V *__restrict__ p,
                     const V *__restrict__ b, const V *__restrict__ x, V *__restrict__ bc) {
  CWM_TILE_LOOP(T, nc) {
    const long long I = base + sub;
    const bool active = I < nc;
    int ms = 0, me = 0;
    if (active) { ms = mptr[I]; me = mptr[I + 1]; }
    // members per tile differ: loop to the warp's maximum so the shuffles stay uniform
    int cnt = me - ms, cmax = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    V acc = V(0);
    for (int t = 0; t < cmax; ++t) {
      const bool has = t < cnt;
      const int m = has ? mlist[ms + t] : 0;
      const V dot = tile_row_dot<V, T>(rp, ci, val, x, m, has, lane);
      if (has) acc += p[m] * (b[m] - dot);
    }
    if (active && lane == 0) bc[I] = acc;
  }
}

template <class V>
amg_status resid_restrict(const CsrView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                          const V *b, const V *x, V *bc, cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  CWM_TRACE("resid_restrict", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + (3.0 * sizeof(V) + 4.0) * A.n +
                                  (4.0 + sizeof(V)) * nc, s);
  CWM_DISPATCH_T(A.tile, (k_resid_restrict<V, kT><<<rows_grid(nc, kT), kBlock, 0, s>>>(nc, A.rp, A.ci, A.val, mptr,
                                                                                      mlist, p, b, x, bc)));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ coarsest solve ----
// One block; x ping-pongs between two shared-memory copies; thread per row.
template <class V>
__global__ void __launch_bounds__(1024) k_coarse_block(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const V *__restrict__ val, const V *__restrict__ dinv,
                                                       const V *__restrict__ b, V *__restrict__ x, int sweeps) {
  extern __shared__ unsigned char smem_raw[];
  V *xa = reinterpret_cast<V *>(smem_raw);
  V *xb = xa + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xa[i] = V(0);
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      V dot = V(0);
      for (int k = rp[i]; k < rp[i + 1]; ++k) dot += val[k] * xa[ci[k]];
      xb[i] = xa[i] + dinv[i] * (b[i] - dot);
    }
    __syncthreads();
    V *t = xa; xa = xb; xb = t;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xa[i];
}

template <class V>
amg_status coarse_solve_block(const CsrView<V> &A, const V *dinv, const V *b, V *x, int sweeps, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  if (A.n > kCoarseBlockMax) {
    set_error("coarse_solve_block: n = %d exceeds %d", A.n, kCoarseBlockMax);
    return AMG_ERR_UNSUPPORTED;
  }
  CWM_TRACE("coarse", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
  const size_t sm = 2 * (size_t)A.n * sizeof(V);
  k_coarse_block<V><<<1, 1024, sm, s>>>(A.n, A.rp, A.ci, A.val, dinv, b, x, sweeps);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ residual ----
template <int T>
__global__ void __launch_bounds__(kBlock) k_residual(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const double *__restrict__ val, const double *__restrict__ b,
                                                     const double *__restrict__ x, double *__restrict__ r) {
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const double dot = tile_row_dot<double, T>(rp, ci, val, x, row, active, lane);
    if (active && lane == 0) r[row] = b[row] - dot;
  }
}

amg_status residual(const CsrView<double> &A, const double *b, const double *x, double *r, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("residual", 4.0 * (A.n + 1) + 12.0 * A.nnz + 24.0 * A.n, s);
  CWM_DISPATCH_T(A.tile, (k_residual<kT><<<rows_grid(A.n, kT), kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, b, x, r)));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ l1 norms ----
template <int T>
__global__ void __launch_bounds__(kBlock) k_l1(int n, const int *__restrict__ rp, const double *__restrict__ val,
                                               double *__restrict__ d) {
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    double a = 0.0;
    if (row < n)
      for (int k = rp[row] + lane; k < rp[row + 1]; k += T) a += fabs(val[k]);
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, T);
    if (row < n && lane == 0) d[row] = a;
  }
}

amg_status l1_norms(const CsrView<double> &A, double *d, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("l1_norms", 4.0 * (A.n + 1) + 8.0 * A.nnz + 8.0 * A.n, s);
  CWM_DISPATCH_T(A.tile, (k_l1<kT><<<rows_grid(A.n, kT), kBlock, 0, s>>>(A.n, A.rp, A.val, d)));
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void k_recip(int n, const double *__restrict__ x, double *__restrict__ y, float *__restrict__ y32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double r = 1.0 / x[i];
    y[i] = r;
    if (y32) y32[i] = (float)r;
  }
}

amg_status reciprocal(int n, const double *x, double *y, float *y32, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  k_recip<<<grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s>>>(n, x, y, y32);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ FCG ----
int fcg_partial_blocks(int n) {
  (void)n;
  return num_sms() * 8;
}

// v = A w fused with the three dot products of Algorithm 3 (w is read once per row).
template <int T>
__global__ void __launch_bounds__(kBlock)
    k_spmv_dots(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ val,
                const double *__restrict__ w, const double *__restrict__ r, const double *__restrict__ q,
                double *__restrict__ v, double *__restrict__ part) {
  double sa = 0.0, sb = 0.0, sg = 0.0;
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const double dot = tile_row_dot<double, T>(rp, ci, val, w, row, active, lane);
    if (active && lane == 0) {
      v[row] = dot;
      const double wi = w[row];
      sa += wi * r[row];
      sb += wi * dot;
      if (q) sg += wi * q[row];
    }
  }
  const double ta = block_sum(sa);
  const double tb = block_sum(sb);
  const double tg = block_sum(sg);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = ta;
    part[3 * blockIdx.x + 1] = tb;
    part[3 * blockIdx.x + 2] = tg;
  }
}

amg_status spmv_dots(const CsrView<double> &A, const double *w, const double *r, const double *q, double *v,
                     double *part, cudaStream_t s) {
  const int g = fcg_partial_blocks(A.n);
  CWM_TRACE("spmv_dots", 4.0 * (A.n + 1) + 12.0 * A.nnz + (q ? 32.0 : 24.0) * A.n, s);
  CWM_DISPATCH_T(A.tile, (k_spmv_dots<kT><<<g, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, w, r, q, v, part)));
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void k_fcg_scalars(int nb, const double *__restrict__ part, double *scal, int first) {
  double a = 0.0, b = 0.0, g = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[3 * i];
    b += part[3 * i + 1];
    g += part[3 * i + 2];
  }
  a = block_sum(a);
  b = block_sum(b);
  g = block_sum(g);
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

amg_status fcg_scalars(int nb, const double *part, double *scal, int first, cudaStream_t s) {
  k_fcg_scalars<<<1, 1024, 0, s>>>(nb, part, scal, first);
  CWM_LAUNCH();
  return AMG_OK;
}

// The two pairs of AXPYs of Algorithm 3, each first result reused from registers:
// d = w - coef d, x += step d;  q = v - coef q, r -= step q;  then partial r.r.
__global__ void __launch_bounds__(kBlock)
    k_fcg_update(int n, const double *__restrict__ w, const double *__restrict__ v, double *__restrict__ d,
                 double *__restrict__ q, double *__restrict__ x, double *__restrict__ r,
                 const double *__restrict__ scal, double *__restrict__ part, int first) {
  if (scal[kFlags] != 0.0) return;  // breakdown: leave x, r, d, q as they were
  const double coef = scal[kCoef], step = scal[kStep];
  double rr = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double di = first ? w[i] : w[i] - coef * d[i];
    const double qi = first ? v[i] : v[i] - coef * q[i];
    d[i] = di;
    q[i] = qi;
    x[i] = x[i] + step * di;
    const double ri = r[i] - step * qi;
    r[i] = ri;
    rr += ri * ri;
  }
  const double t = block_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

amg_status fcg_update(int n, const double *w, const double *v, double *d, double *q, double *x, double *r,
                      const double *scal, double *part, int first, cudaStream_t s) {
  CWM_TRACE("fcg_update", (first ? 64.0 : 80.0) * n, s);
  k_fcg_update<<<fcg_partial_blocks(n), kBlock, 0, s>>>(n, w, v, d, q, x, r, scal, part, first);
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void k_reduce_into(int nb, const double *__restrict__ part, double *scal, int slot) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
  a = block_sum(a);
  if (threadIdx.x == 0) scal[slot] = a;
}

amg_status reduce_into(int nb, const double *part, double *scal, int slot, cudaStream_t s) {
  k_reduce_into<<<1, 1024, 0, s>>>(nb, part, scal, slot);
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void __launch_bounds__(kBlock) k_sqnorm(int n, const double *__restrict__ a, double *__restrict__ part) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i] * a[i];
  const double t = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

amg_status sqnorm_partials(int n, const double *a, double *part, cudaStream_t s) {
  CWM_TRACE("sqnorm", 8.0 * n, s);
  k_sqnorm<<<fcg_partial_blocks(n), kBlock, 0, s>>>(n, a, part);
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void k_to_float(long long n, const double *__restrict__ x, float *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_to_double(long long n, const float *__restrict__ x, double *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
amg_status to_float(long long n, const double *x, float *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  k_to_float<<<grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s>>>(n, x, y);
  CWM_LAUNCH();
  return AMG_OK;
}
amg_status to_double(long long n, const float *x, double *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  k_to_double<<<grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s>>>(n, x, y);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ instantiations ----
#define CWM_INST(V)                                                                                          \
  template amg_status scale<V>(int, const V *, const V *, V *, cudaStream_t);                                \
  template amg_status jacobi<V>(const CsrView<V> &, const V *, const V *, const V *, V *, cudaStream_t);     \
  template amg_status resid_restrict<V>(const CsrView<V> &, int, const int *, const int *, const V *,        \
                                        const V *, const V *, V *, cudaStream_t);                            \
  template amg_status prolong<V>(int, const int *, const V *, const V *, const V *, V *, cudaStream_t);      \
  template amg_status coarse_solve_block<V>(const CsrView<V> &, const V *, const V *, V *, int, cudaStream_t);
CWM_INST(double)
CWM_INST(float)

}  // namespace cwm
