// solve.cu -- solve-phase kernels: CSR row products with a sub-warp ("miniwarp", Sec. 3.1)
// per row, the l1-Jacobi sweep (Sec. 3.2), residual + restriction by the aggregation
// prolongator, prolongation, the one-block coarsest solve, and the fused FCG kernels of
// Sec. 3.2 (three dot products in one pass with the SpMV, paired vector updates).
#include <algorithm>

#include "fcg.cuh"
#include "solve.cuh"

namespace cwm {

constexpr int kBlock = 256;

// All T lanes of every tile of the warp call this together (warp-uniform loops), so the
// full-mask shuffles are well defined; inactive tiles contribute zero.
// NEG: returns init - sum_j a_ij x_j, lane 0 starting from init and every lane subtracting
// its products (no separate FP64 subtraction).
// SCALED: the vector entry is d_j x_j (x = D^{-1} b formed on the fly, d = D^{-1}).
// entries per lane whose loads are in flight together in the tile row walk (8 measured
// slower: elasticity level-2 residual 18.5 -> 20.5 us, lognormal 160^3 41.4 -> 41.9 ms)
#ifndef CWM_TILE_GROUP
#define CWM_TILE_GROUP 4
#endif
#ifndef CWM_TILE_PREFETCH
#define CWM_TILE_PREFETCH 1
#endif
template <class V, int T, bool NEG = false, bool SCALED = false>
__device__ __forceinline__ V tile_row_dot(const int *__restrict__ rp, const int *__restrict__ ci,
                                          const V *__restrict__ val, const V *__restrict__ x, long long row,
                                          bool active, int lane, V init = V(0), const V *__restrict__ d = nullptr) {
  V s = (NEG && lane == 0) ? init : V(0);
  const V sg = NEG ? V(-1) : V(1);
  auto xj = [&](int j) { return SCALED ? __ldg(d + j) * __ldg(x + j) : __ldg(x + j); };
  if (active && x) {
    const int b = rp[row], e = rp[row + 1];
    // four entries per lane in flight, the last group's missing ones predicated off, so that
    // a row of up to 4 T entries costs one round of loads (a long row is a chain of gathers
    // otherwise; a row of 2-3 T entries walked one entry per round trip took three); each
    // lane's products are added in ascending entry order
#if CWM_ROW_PRED
    constexpr int G = CWM_TILE_GROUP;
#if CWM_TILE_PREFETCH
    // the next group's columns one group ahead: a group's value loads and x gathers go out
    // together (elasticity level-2 A P sweep 14.3 -> 13.9 us, lognormal 160^3 41.5 -> 41.1 ms)
    int jn[G];
#pragma unroll
    for (int u = 0; u < G; ++u) jn[u] = b + lane + u * T < e ? ci[b + lane + u * T] : 0;
#endif
    for (int k = b + lane; k < e; k += G * T) {
      int jj[G];
      V aa[G], xx[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const bool ok = k + u * T < e;
#if CWM_TILE_PREFETCH
        jj[u] = jn[u];
#else
        jj[u] = ok ? ci[k + u * T] : 0;
#endif
        aa[u] = ok ? val[k + u * T] : V(0);
      }
#pragma unroll
      for (int u = 0; u < G; ++u) xx[u] = k + u * T < e ? xj(jj[u]) : V(0);
#if CWM_TILE_PREFETCH
#pragma unroll
      for (int u = 0; u < G; ++u) jn[u] = k + (G + u) * T < e ? ci[k + (G + u) * T] : 0;
#endif
#pragma unroll
      for (int u = 0; u < G; ++u)
        if (k + u * T < e) s = fma(sg * aa[u], xx[u], s);
    }
#else
    int k = b + lane;
    for (; k + 3 * T < e; k += 4 * T) {
      const int j0 = ci[k], j1 = ci[k + T], j2 = ci[k + 2 * T], j3 = ci[k + 3 * T];
      const V a0 = val[k], a1 = val[k + T], a2 = val[k + 2 * T], a3 = val[k + 3 * T];
      const V x0 = xj(j0), x1 = xj(j1), x2 = xj(j2), x3 = xj(j3);
      s = fma(sg * a0, x0, s);
      s = fma(sg * a1, x1, s);
      s = fma(sg * a2, x2, s);
      s = fma(sg * a3, x3, s);
    }
    for (; k < e; k += T) s = fma(sg * val[k], xj(ci[k]), s);
#endif
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

// ------------------------------------------------------------ row blocks ----
// A block of kRB threads owns kRB consecutive rows (thread t <-> row r0 + t).  The block's
// entries [rp[r0], rp[r0 + kRB]) are staged in chunks of kRB * kRBE: every thread issues
// kRBE coalesced loads of col and val (streaming cache hint) into shared memory, then each
// thread walks its own row's slice in ascending order, gathering x and accumulating with
// one fused multiply-add per entry.  One FMA per nonzero matters on GB300, whose FP64 pipe
// retires about 500 G instructions/s (a DMUL + DADD pair per nonzero would make the FP64
// SpMV compute-bound).
constexpr int kRB = 256;
static_assert(kRB == kRedBlock, "the row-block kernels reduce with block_sums (fcg.cuh)");
constexpr int kRBE = 8;
constexpr int kRBC = kRB * kRBE;

template <class V>
struct RowBlockSmem {
  V val[kRBC];
  int col[kRBC];
  int rp[kRB + 1];
};

// Stages the row pointers of rows [r0, r0 + nrows] (all threads call it).
__device__ __forceinline__ void rb_stage_rp(const int *__restrict__ rp, int r0, int nrows, int *s_rp) {
  __syncthreads();  // earlier readers of s_rp are done
  for (int i = threadIdx.x; i <= nrows; i += kRB) s_rp[i] = rp[r0 + i];
  __syncthreads();
}

// How the row dot reads its vector: X_PLAIN x_j; X_SCALED d_j x_j (the first l1-Jacobi sweep
// from zero, x = D^{-1} b, formed on the fly); X_PROLONG d_j x_j + p_j xc[agg_j] (that sweep
// plus the coarse correction, formed on the fly).
enum XMode { X_PLAIN = 0, X_SCALED = 1, X_PROLONG = 2 };

template <class V>
struct XSrc {
  const V *x;      // the vector (b for the scaled modes)
  const V *d;      // D^{-1}
  const V *p;      // P values
  const int *agg;  // P columns
  const V *xc;     // coarse correction
};

template <class V, int MODE>
__device__ __forceinline__ V xval(const XSrc<V> &s, int j) {
  if (MODE == X_PLAIN) return __ldg(s.x + j);
  const V xs = __ldg(s.d + j) * __ldg(s.x + j);
  if (MODE == X_SCALED) return xs;
  return fma(__ldg(s.p + j), __ldg(s.xc + __ldg(s.agg + j)), xs);
}

// Row dot of row r0 + threadIdx.x with the vector described by xs (0 for threads beyond
// nrows), same staging as rb_row_dot.
template <class V, int MODE>
__device__ __forceinline__ V rb_row_dot_x(const int *__restrict__ ci, const V *__restrict__ val, const XSrc<V> &xs,
                                          int nrows, RowBlockSmem<V> &sm) {
  const int t = threadIdx.x;
  const int rs = sm.rp[0], re = sm.rp[nrows];
  const int my_s = t < nrows ? sm.rp[t] : 0, my_e = t < nrows ? sm.rp[t + 1] : 0;
  V acc = V(0);
  for (int c0 = rs; c0 < re; c0 += kRBC) {
    const int cend = min(c0 + kRBC, re);
#pragma unroll
    for (int e = 0; e < kRBE; ++e) {
      const int k = c0 + e * kRB + t;
      const bool in = k < cend;
      sm.val[e * kRB + t] = in ? __ldcs(val + k) : V(0);
      sm.col[e * kRB + t] = in ? __ldcs(ci + k) : 0;
    }
    __syncthreads();
    const int lo = max(my_s, c0) - c0, hi = min(my_e, cend) - c0;
    int k = lo;
    for (; k + 4 <= hi; k += 4) {
      const V x0 = xval<V, MODE>(xs, sm.col[k]), x1 = xval<V, MODE>(xs, sm.col[k + 1]);
      const V x2 = xval<V, MODE>(xs, sm.col[k + 2]), x3 = xval<V, MODE>(xs, sm.col[k + 3]);
      acc = fma(sm.val[k], x0, acc);
      acc = fma(sm.val[k + 1], x1, acc);
      acc = fma(sm.val[k + 2], x2, acc);
      acc = fma(sm.val[k + 3], x3, acc);
    }
    for (; k < hi; ++k) acc = fma(sm.val[k], xval<V, MODE>(xs, sm.col[k]), acc);
    __syncthreads();
  }
  return acc;
}

// Row dot of row r0 + threadIdx.x with x (0 for threads beyond nrows); ABS = sum of |a_ij|.
// NEG: init - sum_j a_ij x_j, the products subtracted from init by the FMA chain itself
// (the residual b_i - (A x)_i without a separate FP64 subtraction).
template <class V, bool ABS, bool NEG = false>
__device__ __forceinline__ V rb_row_dot(const int *__restrict__ ci, const V *__restrict__ val,
                                        const V *__restrict__ x, int nrows, RowBlockSmem<V> &sm,
                                        V init = V(0)) {
  const int t = threadIdx.x;
  const int rs = sm.rp[0], re = sm.rp[nrows];
  const int my_s = t < nrows ? sm.rp[t] : 0, my_e = t < nrows ? sm.rp[t + 1] : 0;
  V acc = init;
  for (int c0 = rs; c0 < re; c0 += kRBC) {
    const int cend = min(c0 + kRBC, re);
    int col[kRBE];
    V a[kRBE];
#pragma unroll
    for (int e = 0; e < kRBE; ++e) {
      const int k = c0 + e * kRB + t;
      const bool in = k < cend;
      col[e] = (in && !ABS) ? __ldcs(ci + k) : 0;
      a[e] = in ? __ldcs(val + k) : V(0);
    }
#pragma unroll
    for (int e = 0; e < kRBE; ++e) {
      sm.val[e * kRB + t] = a[e];
      if (!ABS) sm.col[e * kRB + t] = col[e];
    }
    __syncthreads();
    const int lo = max(my_s, c0) - c0, hi = min(my_e, cend) - c0;
    int k = lo;
    if (ABS) {
      for (; k < hi; ++k) acc += fabs(sm.val[k]);
    } else {
      // four independent gathers in flight, then the FMAs in order
      const V sg = NEG ? V(-1) : V(1);
      for (; k + 4 <= hi; k += 4) {
        const V x0 = __ldg(x + sm.col[k]), x1 = __ldg(x + sm.col[k + 1]);
        const V x2 = __ldg(x + sm.col[k + 2]), x3 = __ldg(x + sm.col[k + 3]);
        acc = fma(sg * sm.val[k], x0, acc);
        acc = fma(sg * sm.val[k + 1], x1, acc);
        acc = fma(sg * sm.val[k + 2], x2, acc);
        acc = fma(sg * sm.val[k + 3], x3, acc);
      }
      for (; k < hi; ++k) acc = fma(sg * sm.val[k], __ldg(x + sm.col[k]), acc);
    }
    __syncthreads();
  }
  return acc;
}

static int rb_grid(long long n) { return (int)((n + kRB - 1) / kRB); }

#ifndef CWM_RB_MAX_MEAN
#define CWM_RB_MAX_MEAN 16
#endif
#ifndef CWM_RB_MIN_BLOCKS_PER_SM
#define CWM_RB_MIN_BLOCKS_PER_SM 8
#endif
#ifndef CWM_RB_MAX_ROW
#define CWM_RB_MAX_ROW 64
#endif
#ifndef CWM_TILE64_MEAN_PER_LANE
#define CWM_TILE64_MEAN_PER_LANE 24
#endif
void row_kernel_shape(int n, long long nnz, int max_row, bool fp64, bool *rb, int *tile) {
  const double mean = n > 0 ? (double)nnz / n : 1.0;
  const bool short_rows = mean <= CWM_RB_MAX_MEAN && max_row <= CWM_RB_MAX_ROW;
  if (fp64) {
    *rb = n <= 0 || short_rows;
    int t = 4;
    while (t < 32 && (mean > (double)CWM_TILE64_MEAN_PER_LANE * t || max_row > CWM_TILE_MAX_PER_LANE * t)) t <<= 1;
    *tile = t;
  } else {
    *rb = n <= 0 || short_rows || rb_grid(n) >= (long long)num_sms() * CWM_RB_MIN_BLOCKS_PER_SM;
    *tile = tile_for_rows(mean, max_row);
  }
}

__global__ void k_max_row(int n, const int *__restrict__ rp, int *out) {
  int m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, rp[i + 1] - rp[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

#ifndef CWM_LONG_ROW_MIN
#define CWM_LONG_ROW_MIN 64
#endif
#ifndef CWM_LONG_ROW_FACTOR
#define CWM_LONG_ROW_FACTOR 8
#endif
// A row is long when it is longer than CWM_LONG_ROW_MIN entries and CWM_LONG_ROW_FACTOR
// times the mean: a few hub rows (a lognormal coarse level: mean 5, longest 176) then no
// longer set the tile width and the time of every sweep, while levels whose rows are all
// long (Q1 elasticity: mean 64) keep their shape.  Only levels on sub-warp tiles in some
// precision (rb64 or rb32 false) split.
int long_row_min(int n, long long nnz, int max_row, bool rb64, bool rb32) {
  if (n <= 0 || (rb64 && rb32)) return 0;
  const double mean = (double)nnz / n;
  const double lim = std::max((double)CWM_LONG_ROW_MIN, CWM_LONG_ROW_FACTOR * mean);
  return max_row > lim ? (int)lim : 0;
}

__global__ void k_long_rows(int n, const int *__restrict__ rp, int min_len, int *list, int *count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (rp[i + 1] - rp[i] > min_len) {
      const int q = atomicAdd(count, 1);
      if (list) list[q] = (int)i;
    }
  }
}

amg_status long_row_list(int n, const int *rp, int min_len, int *list, int *d_count, cudaStream_t s) {
  if (n <= 0) return AMG_OK;
  k_long_rows<<<grid_for(n, kBlock, num_sms() * 4), kBlock, 0, s>>>(n, rp, min_len, list, d_count);
  CWM_LAUNCH();
  return AMG_OK;
}

amg_status max_row_length(int n, const int *rp, int *d_out, cudaStream_t s) {
  CWM_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int), s));
  if (n <= 0) return AMG_OK;
  k_max_row<<<grid_for(n, kBlock, num_sms() * 4), kBlock, 0, s>>>(n, rp, d_out);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ elementwise ----
template <class V>
__global__ void k_scale(int n, const V *__restrict__ dinv, const V *__restrict__ b, V *__restrict__ y) {
  pdl_begin();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = dinv[i] * b[i];
}

template <class V>
amg_status scale(int n, const V *dinv, const V *b, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("scale", 3.0 * sizeof(V) * n, s);
  CWM_CUDA(launch_pdl(k_scale<V>, grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s, n, dinv, b, y));
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
__global__ void k_prolong(int n, const int *__restrict__ agg, const V *__restrict__ p, const V *__restrict__ xc,
                          const V *__restrict__ x, V *__restrict__ y) {
  pdl_begin();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const V base = x ? x[i] : V(0);
    y[i] = base + p[i] * __ldg(xc + agg[i]);
  }
}

template <class V>
amg_status prolong(int n, const int *agg, const V *p, const V *xc, const V *x, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("prolong", (4.0 + (x ? 3.0 : 2.0) * sizeof(V)) * n, s);
  CWM_CUDA(launch_pdl(k_prolong<V>, grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s, n, agg, p, xc, x, y));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ l1-Jacobi ----
template <class V, int T>
__global__ void __launch_bounds__(kBlock) k_jacobi(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const V *__restrict__ val, const V *__restrict__ dinv,
                                                   const V *__restrict__ b, const V *__restrict__ x,
                                                   V *__restrict__ y) {
  pdl_begin();
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const V res = tile_row_dot<V, T, true>(rp, ci, val, x, row, active, lane, active && lane == 0 ? b[row] : V(0));
    if (active && lane == 0) y[row] = fma(dinv[row], res, x[row]);
  }
}

// The split sweep: blocks [0, long_blocks) give each listed long row a whole warp; the
// other blocks run the tile loop over all rows and skip the long ones (length > long_min).
template <class V, int T>
__global__ void __launch_bounds__(kBlock)
    k_jacobi_split(int n, const int *__restrict__ rp, const int *__restrict__ ci, const V *__restrict__ val,
                   const V *__restrict__ dinv, const V *__restrict__ b, const V *__restrict__ x, V *__restrict__ y,
                   const int *__restrict__ long_rows, int n_long, int long_min, int long_blocks) {
  pdl_begin();
  if ((int)blockIdx.x < long_blocks) {
    const int lane = threadIdx.x & 31;
    const int nw = long_blocks * (kBlock / 32);
    for (int q = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); q < n_long; q += nw) {
      const int row = long_rows[q];
      const V res = tile_row_dot<V, 32, true>(rp, ci, val, x, row, true, lane, lane == 0 ? b[row] : V(0));
      if (lane == 0) y[row] = fma(dinv[row], res, x[row]);
    }
    return;
  }
  const int lane = threadIdx.x & (T - 1);
  const int sub = (threadIdx.x & 31) / T;
  constexpr int kRowsPerWarp = 32 / T;
  const long long warp_id = ((long long)(blockIdx.x - long_blocks) * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)(gridDim.x - long_blocks) * blockDim.x) >> 5;
  for (long long base = warp_id * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
    const long long row = base + sub;
    const bool active = row < n && rp[row + 1] - rp[row] <= long_min;
    const V res = tile_row_dot<V, T, true>(rp, ci, val, x, row, active, lane, active && lane == 0 ? b[row] : V(0));
    if (active && lane == 0) y[row] = fma(dinv[row], res, x[row]);
  }
}

template <class V>
__global__ void __launch_bounds__(kRB) k_jacobi_rb(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const V *__restrict__ val, const V *__restrict__ dinv,
                                                   const V *__restrict__ b, const V *__restrict__ x,
                                                   V *__restrict__ y) {
  pdl_begin();
  __shared__ RowBlockSmem<V> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  const int r = r0 + threadIdx.x;
  const bool in = threadIdx.x < nrows;
  // the row's own operands are loaded before the row dot, so their latency overlaps it
  const V br = in ? b[r] : V(0), dr = in ? dinv[r] : V(0), xr = in ? x[r] : V(0);
  const V res = rb_row_dot<V, false, true>(ci, val, x, nrows, sm, br);
  if (in) y[r] = fma(dr, res, xr);
}

template <class V>
amg_status jacobi(const CsrView<V> &A, const V *dinv, const V *b, const V *x, V *y, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("jacobi", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 4.0 * sizeof(V) * A.n, s);
  if (A.rb) {
    CWM_CUDA(launch_pdl(k_jacobi_rb<V>, rb_grid(A.n), kRB, 0, s, A.n, A.rp, A.ci, A.val, dinv, b, x, y));
  } else if (A.n_long > 0) {
    const int lb = (int)std::min<long long>((A.n_long + kBlock / 32 - 1) / (kBlock / 32), (long long)num_sms() * 2);
    CWM_DISPATCH_T(A.tile_short, CWM_CUDA(launch_pdl(k_jacobi_split<V, kT>, rows_grid(A.n, kT) + lb, kBlock, 0, s, A.n, A.rp, A.ci,
                                               A.val, dinv, b, x, y, A.long_rows, A.n_long, A.long_min, lb)));
  } else {
    CWM_DISPATCH_T(A.tile, CWM_CUDA(launch_pdl(k_jacobi<V, kT>, rows_grid(A.n, kT), kBlock, 0, s, A.n, A.rp, A.ci, A.val, dinv, b,
                                                                                x, y)));
  }
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ residual + restriction ----
template <class V>
__global__ void k_restrict(int nc, const int *__restrict__ mptr, const int *__restrict__ mlist,
                           const V *__restrict__ p, const V *__restrict__ r, V *__restrict__ bc);

// r = b - A (D^{-1} b): the residual after the first l1-Jacobi sweep from zero, without
// materialising that sweep
template <class V>
__global__ void __launch_bounds__(kRB) k_resid_scaled_rb(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                         const V *__restrict__ val, const V *__restrict__ dinv,
                                                         const V *__restrict__ b, V *__restrict__ r) {
  pdl_begin();
  __shared__ RowBlockSmem<V> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  XSrc<V> xs{b, dinv, nullptr, nullptr, nullptr};
  const V dot = rb_row_dot_x<V, X_SCALED>(ci, val, xs, nrows, sm);
  const int i = r0 + threadIdx.x;
  if (threadIdx.x < nrows) r[i] = b[i] - dot;
}

// x = y + D^{-1} (b - A y) with y = D^{-1} b + P xc formed on the fly: the coarse correction
// of a V-cycle whose pre-smoothing was one sweep from zero, and one post-sweep
template <class V>
__global__ void __launch_bounds__(kRB) k_prolong_jacobi_rb(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ ci, const V *__restrict__ val,
                                                           const V *__restrict__ dinv, const V *__restrict__ b,
                                                           const int *__restrict__ agg, const V *__restrict__ p,
                                                           const V *__restrict__ xc, V *__restrict__ x) {
  pdl_begin();
  __shared__ RowBlockSmem<V> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  XSrc<V> xs{b, dinv, p, agg, xc};
  const V dot = rb_row_dot_x<V, X_PROLONG>(ci, val, xs, nrows, sm);
  const int i = r0 + threadIdx.x;
  if (threadIdx.x < nrows) {
    const V yi = fma(p[i], xc[agg[i]], dinv[i] * b[i]);
    x[i] = yi + dinv[i] * (b[i] - dot);
  }
}

template <class V, int T, bool SCALED = false>
__global__ void __launch_bounds__(kBlock) k_residual(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const V *__restrict__ val, const V *__restrict__ b,
                                                     const V *__restrict__ x, V *__restrict__ r,
                                                     const V *__restrict__ d = nullptr);

template <class V>
amg_status resid_scaled_restrict(const CsrView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                                 const V *dinv, const V *b, V *r_scratch, V *bc, cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  {
    CWM_TRACE("residual", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
    if (A.rb) {
      CWM_CUDA(launch_pdl(k_resid_scaled_rb<V>, rb_grid(A.n), kRB, 0, s, A.n, A.rp, A.ci, A.val, dinv, b, r_scratch));
    } else {
      CWM_DISPATCH_T(A.tile, CWM_CUDA(launch_pdl(k_residual<V, kT, true>, rows_grid(A.n, kT), kBlock, 0, s, A.n,
                                                 A.rp, A.ci, A.val, b, b, r_scratch, dinv)));
    }
    CWM_LAUNCH();
  }
  return restrict_members<V>(A.n, nc, mptr, mlist, p, r_scratch, bc, s);
}

template <class V>
amg_status restrict_members(int n, int nc, const int *mptr, const int *mlist, const V *p, const V *r, V *bc,
                            cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  CWM_TRACE("restrict", (4.0 + 2.0 * sizeof(V)) * n + (4.0 + sizeof(V)) * nc, s);
  CWM_CUDA(launch_pdl(k_restrict<V>, grid_for(nc, kBlock, num_sms() * 8), kBlock, 0, s, nc, mptr, mlist, p, r, bc));
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
amg_status prolong_jacobi(const CsrView<V> &A, const V *dinv, const V *b, const int *agg, const V *p, const V *xc,
                          V *x, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("prolong_jacobi", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + (5.0 * sizeof(V) + 4.0) * A.n, s);
  CWM_CUDA(launch_pdl(k_prolong_jacobi_rb<V>, rb_grid(A.n), kRB, 0, s, A.n, A.rp, A.ci, A.val, dinv, b, agg, p, xc, x));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ A P ----
// Row i of A P: for each aggregate J met among the columns j of row i, (A P)_iJ = the sum
// of a_ij p_j over those j with agg(j) = J, added in the row's stored order.  The distinct J,
// in order of first occurrence, go to ci_pad[rp[i] ..) with their sums in val_pad[rp[i] ..)
// and their number in cnt[i] (at most the row's length, so the padded rows fit A's layout);
// *maxcnt is raised to the longest row of A P.

// Rows of at most MAXL entries, a thread per row: the row's list of aggregates and sums
// stays in registers (fully unrolled, so no local memory).  Longer rows are skipped.
template <int MAXL>
__global__ void __launch_bounds__(kBlock)
    k_ap_short(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ val,
               const int *__restrict__ agg, const double *__restrict__ p, int *__restrict__ ci_pad,
               double *__restrict__ val_pad, int *__restrict__ cnt, int *maxcnt) {
  int dmax = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = rp[i], len = rp[i + 1] - b;
    if (len > MAXL) continue;
    int jl[MAXL];
    double sl[MAXL];
    int d = 0;
#pragma unroll
    for (int e = 0; e < MAXL; ++e) {
      jl[e] = -1;
      sl[e] = 0.0;
      if (e < len) {
        const int j = ci[b + e];
        const int J = agg[j];
        const double t = val[b + e] * p[j];
        bool found = false;
#pragma unroll
        for (int u = 0; u < e; ++u)
          if (u < d && jl[u] == J) { sl[u] += t; found = true; }
#pragma unroll
        for (int u = 0; u <= e; ++u)
          if (!found && u == d) { jl[u] = J; sl[u] = t; }
        d += found ? 0 : 1;
      }
    }
#pragma unroll
    for (int u = 0; u < MAXL; ++u)
      if (u < d) { ci_pad[b + u] = jl[u]; val_pad[b + u] = sl[u]; }
    cnt[i] = d;
    dmax = max(dmax, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0 && dmax > 0) atomicMax(maxcnt, dmax);
}

// Rows longer than min_len, a warp per row: each warp reads the lengths of 32 rows at a time
// and takes their long rows one after the other, in chunks of 32 entries.  Equal J within a
// chunk are grouped by __match_any_sync and summed by the group's first lane, which continues
// the sum of an aggregate already met in an earlier chunk.  The first kApHead list entries
// (aggregate and sum) are kept in shared memory with an open-addressing index (J -> slot) and
// written out when the row is done; later entries live in the padded row and are searched
// there.
constexpr int kApHead = 64;
constexpr int kApHash = 128;  // index size (a power of two, at least twice the head)
constexpr int kApPre = 4;     // chunks whose entries are loaded up front
__device__ __forceinline__ int ap_hash(int J) { return (int)(((unsigned)J * 2654435761u) >> 25); }  // 7 bits

__global__ void __launch_bounds__(kBlock)
    k_ap_long(int n, int min_len, const int *__restrict__ rp, const int *__restrict__ ci,
              const double *__restrict__ val, const int *__restrict__ agg, const double *__restrict__ p,
              int *__restrict__ ci_pad, double *__restrict__ val_pad, int *__restrict__ cnt, int *maxcnt) {
  __shared__ double s_t[kBlock];
  __shared__ int s_key[kBlock / 32][kApHash];
  __shared__ int s_slot[kBlock / 32][kApHash];
  __shared__ int s_hj[kBlock / 32][kApHead];
  __shared__ double s_hv[kBlock / 32][kApHead];
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x & ~31;
  const int w = threadIdx.x >> 5;
  int *key = s_key[w], *slot_of = s_slot[w], *hj = s_hj[w];
  double *hv = s_hv[w];
  const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  int dmax = 0;
  for (long long g = warp_id * 32; g < n; g += nwarps * 32) {
    const long long my = g + lane;
    const int my_b = my < n ? rp[my] : 0;
    const int my_len = my < n ? rp[my + 1] - my_b : 0;
    unsigned todo = __ballot_sync(0xffffffffu, my_len > min_len);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const long long row = g + src;
      const int b = __shfl_sync(0xffffffffu, my_b, src);
      const int len = __shfl_sync(0xffffffffu, my_len, src);
#pragma unroll
      for (int q = 0; q < kApHash / 32; ++q) key[lane + 32 * q] = -1;
      __syncwarp();
      int d = 0;
      // one chunk: entry (J, t) of this lane, has = the lane holds an entry
      auto chunk = [&](int J, double t, bool has) {
        s_t[threadIdx.x] = t;
        const unsigned grp = __match_any_sync(0xffffffffu, J);
        const bool lead = has && (__ffs(grp) - 1) == lane;
        int pos = -1;
        if (lead) {
          // the index holds every head entry, at most kApHead of kApHash places: a probe
          // meets J or an empty place
          for (int it = 0, h = ap_hash(J); it < kApHash; ++it, h = (h + 1) & (kApHash - 1)) {
            const int k = key[h];
            if (k == J) { pos = slot_of[h]; break; }
            if (k < 0) break;
          }
          if (pos < 0)
            for (int u = kApHead; u < d; ++u)
              if (ci_pad[b + u] == J) { pos = u; break; }
        }
        const unsigned fresh = __ballot_sync(0xffffffffu, lead && pos < 0);
        __syncwarp();
        if (lead) {
          const int slot = pos < 0 ? d + __popc(fresh & ((1u << lane) - 1u)) : pos;
          double acc = pos < 0 ? 0.0 : (slot < kApHead ? hv[slot] : val_pad[b + slot]);
          for (unsigned q = grp; q; q &= q - 1) acc += s_t[wbase + __ffs(q) - 1];
          if (slot < kApHead) {
            hj[slot] = J;
            hv[slot] = acc;
            if (pos < 0) {  // index the new head entry (the new J of a chunk are distinct)
              for (int it = 0, h = ap_hash(J); it < kApHash; ++it, h = (h + 1) & (kApHash - 1))
                if (atomicCAS(&key[h], -1, J) == -1) { slot_of[h] = slot; break; }
            }
          } else {
            ci_pad[b + slot] = J;
            val_pad[b + slot] = acc;
          }
        }
        d += __popc(fresh);
        __syncwarp();  // this chunk's entries are visible to the next chunk
      };
      // the entries of the first kApPre chunks are loaded together: one round trip to
      // memory for them instead of one per chunk
      int jp[kApPre];
      double tp[kApPre];
#pragma unroll
      for (int q = 0; q < kApPre; ++q) {
        const int k = 32 * q + lane;
        jp[q] = -1;
        tp[q] = 0.0;
        if (k < len) {
          const int j = ci[b + k];
          jp[q] = agg[j];
          tp[q] = val[b + k] * p[j];
        }
      }
#pragma unroll
      for (int q = 0; q < kApPre; ++q)
        if (32 * q < len) chunk(jp[q], tp[q], 32 * q + lane < len);
      for (int c = 32 * kApPre; c < len; c += 32) {
        const bool has = c + lane < len;
        int J = -1;
        double t = 0.0;
        if (has) {
          const int j = ci[b + c + lane];
          J = agg[j];
          t = val[b + c + lane] * p[j];
        }
        chunk(J, t, has);
      }
      for (int u = lane; u < min(d, kApHead); u += 32) {
        ci_pad[b + u] = hj[u];
        val_pad[b + u] = hv[u];
      }
      __syncwarp();  // the head is read out before the next row resets it
      if (lane == 0) cnt[row] = d;
      dmax = max(dmax, d);
    }
  }
  if (lane == 0 && dmax > 0) atomicMax(maxcnt, dmax);
}

amg_status ap_group(int n, long long nnz, const int *rp, const int *ci, const double *val, const int *agg,
                    const double *p, int max_row, int *ci_pad, double *val_pad, int *cnt, int *maxcnt,
                    cudaStream_t s) {
  if (n == 0) return AMG_OK;
  // A, agg and p read once, the padded rows (at most nnz entries) and the counts written
  CWM_TRACE("ap", 4.0 * (n + 1) + 24.0 * (double)nnz + 16.0 * n, s);
  const int grid = grid_for(n, kBlock, num_sms() * 8);
  const int maxl = max_row <= 8 ? 8 : 16;
  if (maxl == 8)
    k_ap_short<8><<<grid, kBlock, 0, s>>>(n, rp, ci, val, agg, p, ci_pad, val_pad, cnt, maxcnt);
  else
    k_ap_short<16><<<grid, kBlock, 0, s>>>(n, rp, ci, val, agg, p, ci_pad, val_pad, cnt, maxcnt);
  CWM_LAUNCH();
  if (max_row > maxl) {
    k_ap_long<<<grid_for(((long long)n + 31) / 32 * 32, kBlock, num_sms() * 8), kBlock, 0, s>>>(
        n, maxl, rp, ci, val, agg, p, ci_pad, val_pad, cnt, maxcnt);
    CWM_LAUNCH();
  }
  return AMG_OK;
}

// The coarse correction and the first post-sweep through A P:  with y = xs + P xc and
// r = b - A xs (the residual the restriction took), b - A y = r - (A P) xc, so
// x = y + D^{-1} (r - (A P) xc).  xs may be NULL (0); XS_SCALED: xs holds b and the
// pre-sweep result D^{-1} b is formed on the fly (rounded as the scale kernel rounds it).
template <class V, bool XS_SCALED>
__global__ void __launch_bounds__(kRB) k_prolong_jacobi_ap_rb(int n, const int *__restrict__ rp,
                                                              const int *__restrict__ ci, const V *__restrict__ val,
                                                              const V *__restrict__ dinv, const V *__restrict__ r,
                                                              const int *__restrict__ agg, const V *__restrict__ p,
                                                              const V *__restrict__ xc, const V *__restrict__ xs,
                                                              V *__restrict__ x, double *__restrict__ x64) {
  pdl_begin();
  __shared__ RowBlockSmem<V> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  const int i = r0 + threadIdx.x;
  const bool in = threadIdx.x < nrows;
  // the row's own operands are loaded before the row dot, so their latency overlaps it
  V ri = V(0), yi = V(0), di = V(0);
  if (in) {
    ri = r[i];
    di = dinv[i];
    yi = fma(p[i], __ldg(xc + agg[i]), xs ? (XS_SCALED ? di * xs[i] : xs[i]) : V(0));
  }
  const V res = rb_row_dot<V, false, true>(ci, val, xc, nrows, sm, ri);
  if (in) {
    const V xi = fma(di, res, yi);
    x[i] = xi;
    if (x64) x64[i] = (double)xi;
  }
}

template <class V, int T, bool XS_SCALED>
__global__ void __launch_bounds__(kBlock)
    k_prolong_jacobi_ap(int n, const int *__restrict__ rp, const int *__restrict__ ci, const V *__restrict__ val,
                        const V *__restrict__ dinv, const V *__restrict__ r, const int *__restrict__ agg,
                        const V *__restrict__ p, const V *__restrict__ xc, const V *__restrict__ xs,
                        V *__restrict__ x, double *__restrict__ x64) {
  pdl_begin();
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    V ri = V(0), yi = V(0), di = V(0);
    if (active && lane == 0) {
      ri = r[row];
      di = dinv[row];
      yi = fma(p[row], __ldg(xc + agg[row]), xs ? (XS_SCALED ? di * xs[row] : xs[row]) : V(0));
    }
    const V res = tile_row_dot<V, T, true>(rp, ci, val, xc, row, active, lane, ri);
    if (active && lane == 0) {
      const V xi = fma(di, res, yi);
      x[row] = xi;
      if (x64) x64[row] = (double)xi;
    }
  }
}

template <class V, bool XS_SCALED>
static amg_status launch_prolong_jacobi_ap(const CsrView<V> &AP, const V *dinv, const V *r, const int *agg,
                                           const V *p, const V *xc, const V *xs, V *x, double *x64, cudaStream_t s) {
  if (AP.rb) {
    CWM_CUDA(launch_pdl(k_prolong_jacobi_ap_rb<V, XS_SCALED>, rb_grid(AP.n), kRB, 0, s, AP.n, AP.rp, AP.ci, AP.val,
                        dinv, r, agg, p, xc, xs, x, x64));
  } else {
    CWM_DISPATCH_T(AP.tile, CWM_CUDA(launch_pdl(k_prolong_jacobi_ap<V, kT, XS_SCALED>, rows_grid(AP.n, kT), kBlock, 0,
                                                s, AP.n, AP.rp, AP.ci, AP.val, dinv, r, agg, p, xc, xs, x, x64)));
  }
  return AMG_OK;
}

template <class V>
amg_status prolong_jacobi_ap(const CsrView<V> &AP, int nc, const V *dinv, const V *r, const int *agg, const V *p,
                             const V *xc, const V *xs, bool xs_scaled, V *x, cudaStream_t s, double *x64) {
  if (AP.n == 0) return AMG_OK;
  CWM_TRACE("prolong_jacobi_ap", 4.0 * (AP.n + 1) + (4.0 + sizeof(V)) * AP.nnz +
                                     ((xs ? 5.0 : 4.0) * sizeof(V) + 4.0) * AP.n + sizeof(V) * (double)nc +
                                  (x64 ? 8.0 * AP.n : 0.0), s);
  if (xs_scaled) CWM_TRY((launch_prolong_jacobi_ap<V, true>(AP, dinv, r, agg, p, xc, xs, x, x64, s)));
  else CWM_TRY((launch_prolong_jacobi_ap<V, false>(AP, dinv, r, agg, p, xc, xs, x, x64, s)));
  CWM_LAUNCH();
  return AMG_OK;
}

// r = b - A x (x may be NULL: r = b), row blocks
template <class V>
__global__ void __launch_bounds__(kRB) k_resid_rb(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                  const V *__restrict__ val, const V *__restrict__ b,
                                                  const V *__restrict__ x, V *__restrict__ r) {
  pdl_begin();
  __shared__ RowBlockSmem<V> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  const int i = r0 + threadIdx.x;
  const V bi = threadIdx.x < nrows ? b[i] : V(0);
  const V res = x ? rb_row_dot<V, false, true>(ci, val, x, nrows, sm, bi) : bi;
  if (threadIdx.x < nrows) r[i] = res;
}

// r = b - A x (x may be NULL: r = b), a sub-warp tile per row; SCALED: r = b - A (D^{-1} b)
// with x = b and d = D^{-1}
template <class V, int T, bool SCALED>
__global__ void __launch_bounds__(kBlock) k_residual(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const V *__restrict__ val, const V *__restrict__ b,
                                                     const V *__restrict__ x, V *__restrict__ r,
                                                     const V *__restrict__ d) {
  pdl_begin();
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const V res = tile_row_dot<V, T, true, SCALED>(rp, ci, val, x, row, active, lane,
                                                   active && lane == 0 ? b[row] : V(0), d);
    if (active && lane == 0) r[row] = x ? res : b[row];
  }
}

template <class V>
static amg_status launch_residual(const CsrView<V> &A, const V *b, const V *x, V *r, cudaStream_t s) {
  if (A.rb) {
    CWM_CUDA(launch_pdl(k_resid_rb<V>, rb_grid(A.n), kRB, 0, s, A.n, A.rp, A.ci, A.val, b, x, r));
  } else {
    CWM_DISPATCH_T(A.tile, CWM_CUDA(launch_pdl(k_residual<V, kT>, rows_grid(A.n, kT), kBlock, 0, s, A.n, A.rp, A.ci,
                                               A.val, b, x, r, (const V *)nullptr)));
  }
  return AMG_OK;
}

template <class V>
amg_status residual_t(const CsrView<V> &A, const V *b, const V *x, V *r, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("residual", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
  CWM_TRY(launch_residual<V>(A, b, x, r, s));
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
__global__ void k_add_to(int n, const V *__restrict__ x, V *__restrict__ y) {
  pdl_begin();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

template <class V>
amg_status add_to(int n, const V *x, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("add", 3.0 * sizeof(V) * n, s);
  CWM_CUDA(launch_pdl(k_add_to<V>, grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s, n, x, y));
  CWM_LAUNCH();
  return AMG_OK;
}

// bc[I] = sum over the members m of I (ascending) of p_m r_m
template <class V>
__global__ void k_restrict(int nc, const int *__restrict__ mptr, const int *__restrict__ mlist,
                           const V *__restrict__ p, const V *__restrict__ r, V *__restrict__ bc) {
  pdl_begin();
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += (long long)gridDim.x * blockDim.x) {
    const int s = mptr[I], e = mptr[I + 1];
    V acc = V(0);
    for (int k = s; k < e; ++k) {
      const int m = mlist[k];
      acc = fma(p[m], r[m], acc);
    }
    bc[I] = acc;
  }
}

template <class V>
amg_status resid_restrict_rb(const CsrView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                             const V *b, const V *x, V *r_scratch, V *bc, cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  {
    CWM_TRACE("residual", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
    CWM_TRY(launch_residual<V>(A, b, x, r_scratch, s));
    CWM_LAUNCH();
  }
  return restrict_members<V>(A.n, nc, mptr, mlist, p, r_scratch, bc, s);
}


// ------------------------------------------------------------ coarsest solve ----
// One block; x ping-pongs between two shared-memory copies; thread per row.
template <class V>
__global__ void __launch_bounds__(1024) k_coarse_block(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const V *__restrict__ val, const V *__restrict__ dinv,
                                                       const V *__restrict__ b, V *__restrict__ x, int sweeps) {
  pdl_begin();
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

// The whole coarsest system staged in shared memory (matrix, D^{-1}, b, two x copies).
template <class V>
__global__ void __launch_bounds__(1024) k_coarse_smem(int n, int nnz, const int *__restrict__ rp,
                                                      const int *__restrict__ ci, const V *__restrict__ val,
                                                      const V *__restrict__ dinv, const V *__restrict__ b,
                                                      V *__restrict__ x, int sweeps) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *s_val = reinterpret_cast<V *>(smem_raw);
  V *s_dinv = s_val + nnz;
  V *s_b = s_dinv + n;
  V *xa = s_b + n;
  V *xb = xa + n;
  int *s_rp = reinterpret_cast<int *>(xb + n);
  int *s_ci = s_rp + n + 1;
  for (int k = threadIdx.x; k < nnz; k += blockDim.x) {
    s_val[k] = val[k];
    s_ci[k] = ci[k];
  }
  for (int i = threadIdx.x; i <= n; i += blockDim.x) s_rp[i] = rp[i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s_dinv[i] = dinv[i];
    s_b[i] = b[i];
    xa[i] = V(0);
  }
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      V dot = V(0);
      for (int k = s_rp[i]; k < s_rp[i + 1]; ++k) dot += s_val[k] * xa[s_ci[k]];
      xb[i] = xa[i] + s_dinv[i] * (s_b[i] - dot);
    }
    __syncthreads();
    V *t = xa; xa = xb; xb = t;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xa[i];
}

template <class V>
static size_t coarse_smem_bytes(int n, long long nnz) {
  return (size_t)nnz * (sizeof(V) + sizeof(int)) + (size_t)n * 4 * sizeof(V) + ((size_t)n + 1) * sizeof(int);
}
constexpr size_t kCoarseSmemMax = 200 * 1024;

template <class V>
amg_status coarse_solve_block(const CsrView<V> &A, const V *dinv, const V *b, V *x, int sweeps, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  if (A.n > kCoarseBlockMax) {
    set_error("coarse_solve_block: n = %d exceeds %d", A.n, kCoarseBlockMax);
    return AMG_ERR_UNSUPPORTED;
  }
  CWM_TRACE("coarse", 4.0 * (A.n + 1) + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
  const size_t big = coarse_smem_bytes<V>(A.n, A.nnz);
  if (big <= kCoarseSmemMax) {
    static bool attr[64] = {false};
    int dev = 0;
    CWM_CUDA(cudaGetDevice(&dev));
    if (!attr[dev & 63]) {
      CWM_CUDA(cudaFuncSetAttribute(k_coarse_smem<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kCoarseSmemMax));
      attr[dev & 63] = true;
    }
    CWM_CUDA(launch_pdl(k_coarse_smem<V>, 1, 1024, big, s, A.n, (int)A.nnz, A.rp, A.ci, A.val, dinv, b, x, sweeps));
  } else {
    const size_t sm = 2 * (size_t)A.n * sizeof(V);
    CWM_CUDA(launch_pdl(k_coarse_block<V>, 1, 1024, sm, s, A.n, A.rp, A.ci, A.val, dinv, b, x, sweeps));
  }
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ dense coarsest operator ----
// `sweeps` l1-Jacobi sweeps from zero are the fixed linear map
//   x = B b,  B = sum_{k < sweeps} (I - D^{-1} A)^k D^{-1},
// built once at setup by running the sweeps on every unit vector at once (X <- X + D^{-1}(I - A X),
// X_0 = 0, one thread per entry of the row-major X).  Applying it is then one dense
// matrix-vector product spread over many SMs, instead of `sweeps` dependent passes inside one
// block (FP64 throughput per SM is small on GB300).
__global__ void k_dense_sweep(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ val, const double *__restrict__ dinv,
                              const double *__restrict__ X, double *__restrict__ Y, int first) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), c = (int)(idx % n);
  const double e = i == c ? 1.0 : 0.0;
  if (first) {  // X_0 = 0: X_1 = D^{-1}
    Y[idx] = dinv[i] * e;
    return;
  }
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s = fma(val[k], X[(long long)ci[k] * n + c], s);
  Y[idx] = X[idx] + dinv[i] * (e - s);
}

// For symmetric A every X_k is symmetric: (I - D^{-1} A)^j D^{-1} = D^{-1/2} (I - S)^j D^{-1/2}
// with S = D^{-1/2} A D^{-1/2}.  So a sweep computes the upper triangle (c >= i) and writes
// each entry to both (i, c) and (c, i): half the FP64 multiply-adds, and every X_k exactly
// symmetric.  A warp takes row i and 32 kDenseCpt consecutive columns, so each lane keeps
// kDenseCpt independent FMA chains; each entry is still summed in ascending k.  Measured on
// the 832-row coarsest level of Q1 elasticity 64^3 (20 sweeps, on the second stream beside
// the last setup kernels): 1.90 -> 1.62 ms, setup 12.4-12.7 -> 12.0-12.1 ms.
// CWM_DENSE_SYM=0 restores one thread per entry of the full square.
#ifndef CWM_DENSE_SYM
#define CWM_DENSE_SYM 1
#endif
constexpr int kDenseCpt = 2;
__global__ void k_dense_sweep_sym(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                  const double *__restrict__ val, const double *__restrict__ dinv,
                                  const double *__restrict__ X, double *__restrict__ Y) {
  constexpr int W = 32 * kDenseCpt;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nch = (n + W - 1) / W;
  if (warp >= (long long)n * nch) return;
  const int i = (int)(warp / nch), c0 = (int)(warp % nch) * W;
  if (c0 + W <= i) return;  // below the diagonal: written by the mirror stores
  double sum[kDenseCpt];
#pragma unroll
  for (int u = 0; u < kDenseCpt; ++u) sum[u] = 0.0;
  const int b = rp[i], e = rp[i + 1];
#pragma unroll 4
  for (int k = b; k < e; ++k) {
    const double a = val[k];
    const double *xr = X + (long long)ci[k] * n;
#pragma unroll
    for (int u = 0; u < kDenseCpt; ++u) {
      const int c = c0 + lane + 32 * u;
      if (c < n) sum[u] = fma(a, xr[c], sum[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < kDenseCpt; ++u) {
    const int c = c0 + lane + 32 * u;
    if (c >= i && c < n) {
      const long long ic = (long long)i * n + c;
      const double y = X[ic] + dinv[i] * ((i == c ? 1.0 : 0.0) - sum[u]);
      Y[ic] = y;
      if (c != i) Y[(long long)c * n + i] = y;
    }
  }
}

amg_status dense_coarse_build(const CsrView<double> &A, const double *dinv, int sweeps, double *X, double *tmp,
                              cudaStream_t s) {
  const long long nn = (long long)A.n * A.n;
  if (nn == 0) return AMG_OK;
  CWM_TRACE("dense_coarse_build", 8.0 * nn * 2.0 * sweeps, s);
  if (sweeps <= 0) {
    CWM_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * nn, s));
    return AMG_OK;
  }
  // ping-pong so that the last sweep lands in X
  double *bufs[2] = {(sweeps % 2) ? X : tmp, (sweeps % 2) ? tmp : X};
  const int g = grid_for(nn, kBlock, 1 << 30);
  const long long sym_warps = (long long)A.n * ((A.n + 32 * kDenseCpt - 1) / (32 * kDenseCpt));
  const int g_sym = grid_for(sym_warps * 32, kBlock, 1 << 30);
  for (int k = 0; k < sweeps; ++k) {
    const double *src = bufs[(k + 1) & 1];
    double *dst = bufs[k & 1];
    if (CWM_DENSE_SYM && k > 0)
      k_dense_sweep_sym<<<g_sym, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, dinv, src, dst);
    else
      k_dense_sweep<<<g, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, dinv, src, dst, k == 0);
    CWM_LAUNCH();
  }
  return AMG_OK;
}

// y = X b, one warp per row of X (row-major).  Each lane keeps kDenseAcc partial sums over
// the columns lane + 32 (kDenseAcc m + k), so that kDenseAcc loads of the row are in flight
// together (one load per round trip made the 832-row coarsest operator of elasticity take
// 14 us), then adds them in k order and the warp in a fixed shuffle order.
#ifndef CWM_DENSE_ACC
#define CWM_DENSE_ACC 8
#endif
constexpr int kDenseAcc = CWM_DENSE_ACC;
template <class V>
__global__ void k_dense_matvec(int n, const V *__restrict__ X, const V *__restrict__ b, V *__restrict__ y) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < n; i += nw) {
    const V *row = X + i * n;
    V acc[kDenseAcc];
#pragma unroll
    for (int k = 0; k < kDenseAcc; ++k) acc[k] = V(0);
    for (int c0 = 0; c0 < n; c0 += 32 * kDenseAcc) {
      V xv[kDenseAcc], bv[kDenseAcc];
#pragma unroll
      for (int k = 0; k < kDenseAcc; ++k) {
        const int c = c0 + 32 * k + lane;
        xv[k] = c < n ? row[c] : V(0);
        bv[k] = c < n ? b[c] : V(0);
      }
#pragma unroll
      for (int k = 0; k < kDenseAcc; ++k) acc[k] = fma(xv[k], bv[k], acc[k]);
    }
    V a = acc[0];
#pragma unroll
    for (int k = 1; k < kDenseAcc; ++k) a += acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) y[i] = a;
  }
}

template <class V>
amg_status dense_coarse_apply(int n, const V *X, const V *b, V *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("coarse", (double)sizeof(V) * ((double)n * n + 2.0 * n), s);
  CWM_CUDA(launch_pdl(k_dense_matvec<V>, grid_for((long long)n * 32, 128, 1 << 30), 128, 0, s, n, X, b, y));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ residual ----

amg_status residual(const CsrView<double> &A, const double *b, const double *x, double *r, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("residual", 4.0 * (A.n + 1) + 12.0 * A.nnz + 24.0 * A.n, s);
  CWM_TRY(launch_residual<double>(A, b, x, r, s));
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

__global__ void __launch_bounds__(kRB) k_l1_rb(int n, const int *__restrict__ rp, const double *__restrict__ val,
                                               double *__restrict__ d) {
  __shared__ RowBlockSmem<double> sm;
  const int r0 = blockIdx.x * kRB;
  const int nrows = min(kRB, n - r0);
  rb_stage_rp(rp, r0, nrows, sm.rp);
  const double a = rb_row_dot<double, true>(nullptr, val, nullptr, nrows, sm);
  if (threadIdx.x < nrows) d[r0 + threadIdx.x] = a;
}

amg_status l1_norms(const CsrView<double> &A, double *d, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("l1_norms", 4.0 * (A.n + 1) + 8.0 * A.nnz + 8.0 * A.n, s);
  if (A.rb) {
    k_l1_rb<<<rb_grid(A.n), kRB, 0, s>>>(A.n, A.rp, A.val, d);
  } else {
    CWM_DISPATCH_T(A.tile, (k_l1<kT><<<rows_grid(A.n, kT), kBlock, 0, s>>>(A.n, A.rp, A.val, d)));
  }
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
// Blocks of the grid-stride FCG reductions: at most kDotsBlocksPerSm per SM, so that the
// FP64 block reductions are paid once per several row blocks.
#ifndef CWM_DOTS_BLOCKS_PER_SM
#define CWM_DOTS_BLOCKS_PER_SM 12
#endif
constexpr int kDotsBlocksPerSm = CWM_DOTS_BLOCKS_PER_SM;
int fcg_partial_blocks(int n) {
  const int rb = rb_grid(n > 0 ? n : 1);
  const int cap = num_sms() * kDotsBlocksPerSm;
  return rb < cap ? rb : cap;
}
// double2 steps per thread of the FCG update: 2 (756 blocks on elasticity 64^3) gave a
// 45.1 ms solve against 45.6 ms with 4 (378 blocks, two or three per SM); 1 measured as 2
#ifndef CWM_UPD_STEPS
#define CWM_UPD_STEPS 2
#endif
constexpr int kUpdChunk = 2 * CWM_UPD_STEPS * kRB;  // entries per fcg_update block (double2 steps)
int fcg_update_blocks(int n) { return (int)(((n > 0 ? n : 1) + kUpdChunk - 1LL) / kUpdChunk); }

__global__ void __launch_bounds__(kRB)
    k_spmv_dots_rb(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ val,
                   const double *__restrict__ w, const double *__restrict__ r, const double *__restrict__ q,
                   double *__restrict__ v, double *__restrict__ part, double *scal, unsigned *tick, int first) {
  pdl_begin();
  __shared__ RowBlockSmem<double> sm;
  double sa = 0.0, sb = 0.0, sg = 0.0;
  // grid-stride over row blocks: each thread accumulates its rows' contributions, so the
  // block-wide FP64 reduction is paid once per block, not once per 256 rows
  for (int r0 = blockIdx.x * kRB; r0 < n; r0 += gridDim.x * kRB) {
    const int nrows = min(kRB, n - r0);
    const int i = r0 + threadIdx.x;
    const bool in = threadIdx.x < nrows;
    // the row's own w_i, r_i, q_i are loaded before the row dot, so their latency overlaps it
    const double wi = in ? w[i] : 0.0, ri = in ? r[i] : 0.0, qi = (in && q) ? q[i] : 0.0;
    rb_stage_rp(rp, r0, nrows, sm.rp);
    const double dot = rb_row_dot<double, false>(ci, val, w, nrows, sm);
    if (in) {
      v[i] = dot;
      sa = fma(wi, ri, sa);
      sb = fma(wi, dot, sb);
      if (q) sg = fma(wi, qi, sg);
    }
  }
  fcg_dots_finish(sa, sb, sg, part, scal, tick, first);
}

// Same with a sub-warp tile per row (levels on sub-warp tiles, see row_blocks_for).
template <int T>
__global__ void __launch_bounds__(kBlock)
    k_spmv_dots_tile(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ val,
                     const double *__restrict__ w, const double *__restrict__ r, const double *__restrict__ q,
                     double *__restrict__ v, double *__restrict__ part, double *scal, unsigned *tick, int first) {
  pdl_begin();
  double sa = 0.0, sb = 0.0, sg = 0.0;
  CWM_TILE_LOOP(T, n) {
    const long long row = base + sub;
    const bool active = row < n;
    const double dot = tile_row_dot<double, T>(rp, ci, val, w, row, active, lane);
    if (active && lane == 0) {
      v[row] = dot;
      const double wi = w[row];
      sa = fma(wi, r[row], sa);
      sb = fma(wi, dot, sb);
      if (q) sg = fma(wi, q[row], sg);
    }
  }
  fcg_dots_finish(sa, sb, sg, part, scal, tick, first);
}

#ifndef CWM_DOTS_RB_MAX_MEAN
#define CWM_DOTS_RB_MAX_MEAN 1e30
#endif
#ifndef CWM_DOTS_ENTRIES_PER_BLOCK
#define CWM_DOTS_ENTRIES_PER_BLOCK 8192
#endif
// Row-block grid of spmv_dots: kDotsBlocksPerSm per SM, or more when that would give a block
// more than ~8K nonzeros (long rows: a block's row blocks are walked one after the other).
int fcg_dots_blocks(int n, long long nnz) {
  const long long rb = rb_grid(n > 0 ? n : 1);
  long long g = (long long)num_sms() * kDotsBlocksPerSm;
  const long long by_nnz = nnz / CWM_DOTS_ENTRIES_PER_BLOCK;
  if (by_nnz > g) g = by_nnz;
  return (int)(rb < g ? rb : g);
}
int fcg_dots_blocks_max(int n, long long nnz) {
  const int a = fcg_dots_blocks(n, nnz), b = num_sms() * 8;
  return a > b ? a : b;
}

amg_status spmv_dots_scalars(const CsrView<double> &A, const double *w, const double *r, const double *q,
                             double *v, double *part, double *scal, unsigned *tick, int first, cudaStream_t s) {
  CWM_TRACE("spmv_dots", 4.0 * (A.n + 1) + 12.0 * A.nnz + (q ? 32.0 : 24.0) * A.n, s);
  if (A.rb && (A.n == 0 || (double)A.nnz / A.n <= CWM_DOTS_RB_MAX_MEAN)) {
    CWM_CUDA(launch_pdl(k_spmv_dots_rb, fcg_dots_blocks(A.n, A.nnz), kRB, 0, s, A.n, A.rp, A.ci, A.val, w, r, q, v, part, scal, tick,
                                                          first));
  } else {
    // at most num_sms() * 8 blocks (rows_grid), within fcg_dots_blocks_max
    CWM_DISPATCH_T(A.tile, CWM_CUDA(launch_pdl(k_spmv_dots_tile<kT>, wave_cap(k_spmv_dots_tile<kT>, rows_grid(A.n, kT), kBlock),
                                               kBlock, 0, s, A.n, A.rp, A.ci, A.val, w, r,
                                                                                    q, v, part, scal, tick, first)));
  }
  CWM_LAUNCH();
  return AMG_OK;
}

// The two pairs of AXPYs of Algorithm 3, each first result reused from registers:
// d = w - coef d, x += step d;  q = v - coef q, r -= step q;  then partial r.r.
__global__ void __launch_bounds__(kBlock)
    k_fcg_update(int n, const double *__restrict__ w, const double *__restrict__ v, double *__restrict__ d,
                 double *__restrict__ q, double *__restrict__ x, double *__restrict__ r, float *__restrict__ r32,
                 double *__restrict__ scal, double *__restrict__ part, unsigned *tick, int first, int vec) {
  pdl_begin();
  const bool broken = scal[kFlags] != 0.0;  // breakdown: leave x, r, d, q as they were
  const double coef = scal[kCoef], step = scal[kStep];
  double rr = 0.0;
  // the block owns kUpdChunk consecutive entries: CWM_UPD_STEPS coalesced double2 steps per thread
  const long long base = (long long)blockIdx.x * kUpdChunk;
  if (!broken) {
#pragma unroll
    for (int m = 0; m < kUpdChunk / (2 * kRB); ++m) {
      const long long i = base + 2 * (threadIdx.x + (long long)m * kRB);
      if (vec && i + 1 < n) {
        const double2 w2 = *reinterpret_cast<const double2 *>(w + i);
        const double2 v2 = *reinterpret_cast<const double2 *>(v + i);
        const double2 x2 = *reinterpret_cast<const double2 *>(x + i);
        const double2 r2 = *reinterpret_cast<const double2 *>(r + i);
        double2 d2, q2;
        if (first) {
          d2 = w2;
          q2 = v2;
        } else {
          const double2 dd = *reinterpret_cast<const double2 *>(d + i);
          const double2 qq = *reinterpret_cast<const double2 *>(q + i);
          d2 = make_double2(fma(-coef, dd.x, w2.x), fma(-coef, dd.y, w2.y));
          q2 = make_double2(fma(-coef, qq.x, v2.x), fma(-coef, qq.y, v2.y));
        }
        *reinterpret_cast<double2 *>(d + i) = d2;
        *reinterpret_cast<double2 *>(q + i) = q2;
        *reinterpret_cast<double2 *>(x + i) = make_double2(fma(step, d2.x, x2.x), fma(step, d2.y, x2.y));
        const double2 rn = make_double2(fma(-step, q2.x, r2.x), fma(-step, q2.y, r2.y));
        *reinterpret_cast<double2 *>(r + i) = rn;
        if (r32) *reinterpret_cast<float2 *>(r32 + i) = make_float2((float)rn.x, (float)rn.y);
        rr = fma(rn.x, rn.x, rr);
        rr = fma(rn.y, rn.y, rr);
      } else {
        for (long long j = i; j < i + 2 && j < n; ++j) {
          const double dj = first ? w[j] : fma(-coef, d[j], w[j]);
          const double qj = first ? v[j] : fma(-coef, q[j], v[j]);
          d[j] = dj;
          q[j] = qj;
          x[j] = fma(step, dj, x[j]);
          const double rj = fma(-step, qj, r[j]);
          r[j] = rj;
          if (r32) r32[j] = (float)rj;
          rr = fma(rj, rj, rr);
        }
      }
    }
  }
  {
    const double in1[1] = {rr};
    double o1[1];
    block_sums<1>(in1, o1);
    if (threadIdx.x == 0) part[blockIdx.x] = o1[0];
  }
  if (last_block(tick)) {
    const double a = strided_sum<1, 0>((int)gridDim.x, part);
    const double in1[1] = {a};
    double o1[1];
    block_sums<1>(in1, o1);
    if (threadIdx.x == 0) {
      scal[kRR] = o1[0];
      *tick = 0u;
    }
  }
}

amg_status fcg_update(int n, const double *w, const double *v, double *d, double *q, double *x, double *r,
                      float *r32, double *scal, double *part, unsigned *tick, int first, cudaStream_t s) {
  CWM_TRACE("fcg_update", (first ? 64.0 : 80.0) * n + (r32 ? 4.0 * n : 0.0), s);
  auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  const int vec = al(w) && al(v) && al(d) && al(q) && al(x) && al(r) && (((uintptr_t)r32 & 7u) == 0);
  CWM_CUDA(launch_pdl(k_fcg_update, fcg_update_blocks(n), kRB, 0, s, n, w, v, d, q, x, r, r32, scal, part, tick, first,
                      vec));
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
  k_sqnorm<<<fcg_partial_blocks(n), kRB, 0, s>>>(n, a, part);
  CWM_LAUNCH();
  return AMG_OK;
}

__global__ void k_to_float(long long n, const double *__restrict__ x, float *__restrict__ y) {
  pdl_begin();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_to_double(long long n, const float *__restrict__ x, double *__restrict__ y) {
  pdl_begin();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
// y = (float)x for the first *count entries (a count only the device knows yet)
__global__ void k_to_float_count(const int *__restrict__ count, const double *__restrict__ x, float *__restrict__ y) {
  const long long n = *count;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
amg_status to_float_count(const int *count, long long cap, const double *x, float *y, cudaStream_t s) {
  if (cap <= 0) return AMG_OK;
  k_to_float_count<<<grid_for(cap, kBlock, num_sms() * 8), kBlock, 0, s>>>(count, x, y);
  CWM_LAUNCH();
  return AMG_OK;
}
amg_status to_float(long long n, const double *x, float *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_CUDA(launch_pdl(k_to_float, grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s, n, x, y));
  CWM_LAUNCH();
  return AMG_OK;
}
amg_status to_double(long long n, const float *x, double *y, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_CUDA(launch_pdl(k_to_double, grid_for(n, kBlock, num_sms() * 8), kBlock, 0, s, n, x, y));
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ instantiations ----
#define CWM_INST(V)                                                                                          \
  template amg_status scale<V>(int, const V *, const V *, V *, cudaStream_t);                                \
  template amg_status jacobi<V>(const CsrView<V> &, const V *, const V *, const V *, V *, cudaStream_t);     \
  template amg_status prolong<V>(int, const int *, const V *, const V *, const V *, V *, cudaStream_t);      \
  template amg_status resid_restrict_rb<V>(const CsrView<V> &, int, const int *, const int *, const V *,     \
                                           const V *, const V *, V *, V *, cudaStream_t);                    \
  template amg_status coarse_solve_block<V>(const CsrView<V> &, const V *, const V *, V *, int, cudaStream_t); \
  template amg_status dense_coarse_apply<V>(int, const V *, const V *, V *, cudaStream_t);                  \
  template amg_status residual_t<V>(const CsrView<V> &, const V *, const V *, V *, cudaStream_t);          \
  template amg_status resid_scaled_restrict<V>(const CsrView<V> &, int, const int *, const int *, const V *,  \
                                               const V *, const V *, V *, V *, cudaStream_t);               \
  template amg_status prolong_jacobi<V>(const CsrView<V> &, const V *, const V *, const int *, const V *,    \
                                        const V *, V *, cudaStream_t);                                       \
  template amg_status prolong_jacobi_ap<V>(const CsrView<V> &, int, const V *, const V *, const int *, const V *, \
                                           const V *, const V *, bool, V *, cudaStream_t, double *);          \
  template amg_status add_to<V>(int, const V *, V *, cudaStream_t);                                          \
  template amg_status restrict_members<V>(int, int, const int *, const int *, const V *, const V *, V *,      \
                                          cudaStream_t);
CWM_INST(double)
CWM_INST(float)

}  // namespace cwm
