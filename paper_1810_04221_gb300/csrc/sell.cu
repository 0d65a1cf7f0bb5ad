// sell.cu -- a sliced copy of a long-row level operator (or of its product A P) and the
// V-cycle kernels that stream it: the residual after the first l1-Jacobi sweep (Sec. 3.2,
// Algorithm 1) and the coarse correction + post-sweep through A P.
//
// The CSR kernels stage each row block's entries in shared memory, so on rows of 40-100
// entries a chunk holds few rows, few threads work and the rest wait at the barrier (the
// binary32 residual of Q1 elasticity's level 1 ran at 0.38 of the copy bandwidth).  Here K
// lanes own a row (K = 1 .. 32, set by the longest row so that no lane walks more than about
// two dozen entries: a lane's entries are a chain of dependent column -> vector loads, and
// on a small level the longest chain sets the kernel's time), and the entries are laid out
// so that the 32 lanes of a warp read consecutive words at each step (sliced ELL): rows are
// sorted by length, longest first, within windows of kSellWin rows (perm[p] = the row at
// position p); a slice holds R = 32 / K positions; entry e of position p = R s + r sits at
// slot sptr[s] + 32 (e / K) + K r + e % K.  A slice is padded to its first (longest) row;
// a lane stops at its row's length, so padding is never read.  Sorting within windows keeps
// the padding small (a few percent on the elasticity levels, against 15-35% for unsorted
// slices) while the vector entries a window reads and writes stay within a few cache lines.
#include "solve.cuh"

namespace cwm {

constexpr int kSellWin = 256;  // rows sorted together (one block)
// Entries per lane whose loads are in flight together in binary32 (4 in binary64), in
// predicated groups: 8 measured 50.8 / 22.9 us on Q1 elasticity 64^3 levels 0 / 1 (A P),
// 16 gave 53.0 / 27.0 (56 registers); whole groups with a one-at-a-time remainder gave
// 59.0 / 31.0 at 16.  Loading the next group's columns one group ahead (as the tile walk
// does) measured slower here: 52.4 / 23.2 us at 44 registers.
#ifndef CWM_SELL_UNROLL32
#define CWM_SELL_UNROLL32 8
#endif
constexpr int kSellBlock = 128;

// Window w's rows sorted by (length descending, index ascending): perm and len per position.
__global__ void __launch_bounds__(kSellWin) k_sell_sort(int n, const int *__restrict__ rp, int *__restrict__ perm,
                                                        int *__restrict__ len) {
  __shared__ unsigned long long key[kSellWin];
  const int t = threadIdx.x;
  const int r = blockIdx.x * kSellWin + t;
  if (r < n) key[t] = ((unsigned long long)(unsigned)(0x7fffffff - (rp[r + 1] - rp[r])) << 32) | (unsigned)r;
  else key[t] = ~0ull;
  __syncthreads();
  for (int k = 2; k <= kSellWin; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int l = t ^ j;
      if (l > t) {
        const unsigned long long a = key[t], b = key[l];
        if ((a > b) == ((t & k) == 0)) { key[t] = b; key[l] = a; }
      }
      __syncthreads();
    }
  }
  if (r < n) {
    const unsigned long long q = key[t];
    perm[r] = (int)(q & 0xffffffffu);
    len[r] = 0x7fffffff - (int)(q >> 32);
  }
}

// slen[s] = 32 * ceil(length of the first (longest) position of slice s / K), R = 32 / K
__global__ void k_sell_slice_len(int n, int K, const int *__restrict__ len, int *__restrict__ slen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int R = 32 / K;
  const int ns = (n + R - 1) / R;
  if (s < ns) slen[s] = 32 * ((len[R * s] + K - 1) / K);
}

int sell_lanes(int max_row) {
  int K = 1;
  while (K < 32 && max_row > 24 * K) K <<= 1;
  return K;
}

int sell_slices(int n, int K) { return (n + 32 / K - 1) / (32 / K); }

amg_status sell_plan(int n, int K, const int *rp, int *perm, int *len, int *slen, int *sptr, int *scan_scratch,
                     cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("sell_build", 16.0 * n, s);
  k_sell_sort<<<(n + kSellWin - 1) / kSellWin, kSellWin, 0, s>>>(n, rp, perm, len);
  CWM_LAUNCH();
  const int ns = sell_slices(n, K);
  k_sell_slice_len<<<grid_for(ns, 256, 1 << 30), 256, 0, s>>>(n, K, len, slen);
  CWM_LAUNCH();
  return exclusive_scan(slen, sptr, ns, scan_scratch, s);
}

// A thread per position: copies its row's columns and values into its slots.
template <class V>
__global__ void k_sell_fill(int n, int K, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ val, const int *__restrict__ perm,
                            const int *__restrict__ len, const int *__restrict__ sptr, int *__restrict__ col,
                            V *__restrict__ sval) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int R = 32 / K;
  const int row = perm[p], L = len[p];
  const int src = rp[row];
  const long long base = (long long)sptr[p / R] + (long long)K * (p % R);
  for (int e = 0; e < L; ++e) {
    const long long slot = base + 32LL * (e / K) + e % K;
    col[slot] = ci[src + e];
    sval[slot] = (V)val[src + e];
  }
}

template <class V>
amg_status sell_fill(int n, const int *rp, const int *ci, const double *val, const SellView<V> &S, int *col,
                     V *sval, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("sell_build", 4.0 * n + 12.0 * S.nnz + (4.0 + sizeof(V)) * S.nnz, s);
  k_sell_fill<V><<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, S.lanes, rp, ci, val, S.perm, S.len, S.sptr, col,
                                                            sval);
  CWM_LAUNCH();
  return AMG_OK;
}

// The K lanes of one row (all 32 lanes of the warp call this together): lane j sums
// -val x[col] over the row's entries e = j, j + K, ... (U entries' loads in flight:
// CWM_SELL_UNROLL32 in binary32, 4 in binary64), the K partial sums are added
// by shuffles and init joins them; every lane returns the total.
template <class V, int K, bool SCALED>
__device__ __forceinline__ V sell_row(const SellView<V> &A, long long base, int L, int j, const V *__restrict__ x,
                                      const V *__restrict__ d, V init) {
  constexpr int U = sizeof(V) == 4 ? CWM_SELL_UNROLL32 : 4;
  V acc = V(0);
  const int steps = L > j ? (L - j + K - 1) / K : 0;  // this lane's entries
#if CWM_ROW_PRED
  // groups of U entries, the last one's missing entries predicated off: a lane's row costs
  // one round of loads per U entries (its remainder walked one entry per round trip before:
  // 12 dependent gathers for a 44-entry row); products added in ascending entry order
  for (int t = 0; t < steps; t += U) {
    int c[U];
    V a[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = t + u < steps;
      c[u] = ok ? __ldcs(A.col + base + 32LL * (t + u)) : 0;
      a[u] = ok ? __ldcs(A.val + base + 32LL * (t + u)) : V(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      xv[u] = t + u < steps ? (SCALED ? __ldg(d + c[u]) * __ldg(x + c[u]) : __ldg(x + c[u])) : V(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (t + u < steps) acc = fma(-a[u], xv[u], acc);
  }
#else
  int t = 0;
  for (; t + U <= steps; t += U) {
    int c[U];
    V a[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = __ldcs(A.col + base + 32LL * (t + u));
      a[u] = __ldcs(A.val + base + 32LL * (t + u));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = SCALED ? __ldg(d + c[u]) * __ldg(x + c[u]) : __ldg(x + c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc = fma(-a[u], xv[u], acc);
  }
  for (; t < steps; ++t) {
    const int c = __ldcs(A.col + base + 32LL * t);
    const V xv = SCALED ? __ldg(d + c) * __ldg(x + c) : __ldg(x + c);
    acc = fma(-__ldcs(A.val + base + 32LL * t), xv, acc);
  }
#endif
#pragma unroll
  for (int o = K / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, K);
  return init + acc;
}

// Position and entry base of the calling lane: slice = global warp, r = lane / K, j = lane % K.
#define CWM_SELL_LANE(A, K)                                                          \
  const int lane = threadIdx.x & 31, j = lane % (K), R = 32 / (K);                   \
  const long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;      \
  const long long pos = sl * R + lane / (K);                                         \
  const bool in = pos < (A).n;                                                       \
  const int row = in ? (A).perm[pos] : 0;                                            \
  const int L = in ? (A).len[pos] : 0;                                               \
  const long long base = in ? (long long)(A).sptr[sl] + lane : 0;

// r = b - A x, or (SCALED) r = b - A (D^{-1} b)
template <class V, int K, bool SCALED>
__global__ void __launch_bounds__(kSellBlock) k_sell_resid(SellView<V> A, const V *__restrict__ b,
                                                           const V *__restrict__ x, const V *__restrict__ d,
                                                           V *__restrict__ r) {
  pdl_begin();
  CWM_SELL_LANE(A, K)
  const V bi = in && j == 0 ? b[row] : V(0);
  const V res = sell_row<V, K, SCALED>(A, base, L, j, SCALED ? b : x, d, bi);
  if (in && j == 0) r[row] = res;
}

#define CWM_SELL_DISPATCH(K, ...)                              \
  switch (K) {                                                 \
    case 1: { constexpr int kK = 1; __VA_ARGS__; } break;      \
    case 2: { constexpr int kK = 2; __VA_ARGS__; } break;      \
    case 4: { constexpr int kK = 4; __VA_ARGS__; } break;      \
    case 8: { constexpr int kK = 8; __VA_ARGS__; } break;      \
    case 16: { constexpr int kK = 16; __VA_ARGS__; } break;    \
    default: { constexpr int kK = 32; __VA_ARGS__; } break;    \
  }

template <class V>
amg_status sell_residual(const SellView<V> &A, const V *b, const V *x, const V *dinv, V *r, cudaStream_t s) {
  if (A.n == 0) return AMG_OK;
  CWM_TRACE("residual_sl", 16.0 * A.n + (4.0 + sizeof(V)) * A.nnz + 3.0 * sizeof(V) * A.n, s);
  const int grid = grid_for((long long)sell_slices(A.n, A.lanes) * 32, kSellBlock, 1 << 30);
  if (dinv)
    CWM_SELL_DISPATCH(A.lanes, CWM_CUDA(launch_pdl(k_sell_resid<V, kK, true>, grid, kSellBlock, 0, s, A, b,
                                                   (const V *)nullptr, dinv, r)))
  else
    CWM_SELL_DISPATCH(A.lanes, CWM_CUDA(launch_pdl(k_sell_resid<V, kK, false>, grid, kSellBlock, 0, s, A, b, x,
                                                   (const V *)nullptr, r)))
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
amg_status sell_resid_restrict(const SellView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                               const V *b, const V *x, const V *dinv, V *r_scratch, V *bc, cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  CWM_TRY(sell_residual<V>(A, b, x, dinv, r_scratch, s));
  return restrict_members<V>(A.n, nc, mptr, mlist, p, r_scratch, bc, s);
}

// x = y + D^{-1} (r - (A P) xc), y = xs + P xc (XS_SCALED: xs holds b, the pre-sweep result
// is D^{-1} b; xs NULL: 0) -- prolong_jacobi_ap on the sliced A P
template <class V, int K, bool XS_SCALED>
__global__ void __launch_bounds__(kSellBlock)
    k_sell_prolong_jacobi_ap(SellView<V> AP, const V *__restrict__ dinv, const V *__restrict__ r,
                             const int *__restrict__ agg, const V *__restrict__ p, const V *__restrict__ xc,
                             const V *__restrict__ xs, V *__restrict__ x, double *__restrict__ x64) {
  pdl_begin();
  CWM_SELL_LANE(AP, K)
  V ri = V(0), di = V(0), yi = V(0);
  if (in && j == 0) {
    ri = r[row];
    di = dinv[row];
    yi = fma(p[row], __ldg(xc + agg[row]), xs ? (XS_SCALED ? di * xs[row] : xs[row]) : V(0));
  }
  const V res = sell_row<V, K, false>(AP, base, L, j, xc, nullptr, ri);
  if (in && j == 0) {
    const V xi = fma(di, res, yi);
    x[row] = xi;
    if (x64) x64[row] = (double)xi;
  }
}

template <class V>
amg_status sell_prolong_jacobi_ap(const SellView<V> &AP, int nc, const V *dinv, const V *r, const int *agg,
                                  const V *p, const V *xc, const V *xs, bool xs_scaled, V *x, cudaStream_t s,
                                  double *x64) {
  if (AP.n == 0) return AMG_OK;
  CWM_TRACE("prolong_jacobi_sl", 16.0 * AP.n + (4.0 + sizeof(V)) * AP.nnz +
                                     ((xs ? 5.0 : 4.0) * sizeof(V) + 4.0) * AP.n + sizeof(V) * (double)nc +
                                     (x64 ? 8.0 * AP.n : 0.0), s);
  const int grid = grid_for((long long)sell_slices(AP.n, AP.lanes) * 32, kSellBlock, 1 << 30);
  if (xs_scaled)
    CWM_SELL_DISPATCH(AP.lanes, CWM_CUDA(launch_pdl(k_sell_prolong_jacobi_ap<V, kK, true>, grid, kSellBlock, 0, s,
                                                    AP, dinv, r, agg, p, xc, xs, x, x64)))
  else
    CWM_SELL_DISPATCH(AP.lanes, CWM_CUDA(launch_pdl(k_sell_prolong_jacobi_ap<V, kK, false>, grid, kSellBlock, 0, s,
                                                    AP, dinv, r, agg, p, xc, xs, x, x64)))
  CWM_LAUNCH();
  return AMG_OK;
}

#define CWM_SELL_INST(V)                                                                                         \
  template amg_status sell_fill<V>(int, const int *, const int *, const double *, const SellView<V> &, int *, V *,  \
                                   cudaStream_t);                                                                \
  template amg_status sell_residual<V>(const SellView<V> &, const V *, const V *, const V *, V *, cudaStream_t);    \
  template amg_status sell_resid_restrict<V>(const SellView<V> &, int, const int *, const int *, const V *,         \
                                             const V *, const V *, const V *, V *, V *, cudaStream_t);             \
  template amg_status sell_prolong_jacobi_ap<V>(const SellView<V> &, int, const V *, const V *, const int *,       \
                                                const V *, const V *, const V *, bool, V *, cudaStream_t, double *);
CWM_SELL_INST(double)
CWM_SELL_INST(float)

}  // namespace cwm
