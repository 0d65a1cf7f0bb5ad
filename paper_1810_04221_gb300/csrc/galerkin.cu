// galerkin.cu -- Galerkin product A_c = P^T A P (Sec. 2.1; the costliest setup step per
// Sec. 3.1) for the pairwise P of one matching sweep, in one grouping pass: each coarse row
// is written at a padded offset (the sum of its member rows' lengths, an upper bound on its
// length) together with its number of distinct columns; a scan of those counts gives the
// row pointers, and a compaction copies the rows into place.  (A separate counting pass
// repeated the whole grouping -- the sorts of long rows included -- only to size the
// output.)
//
// Coarse row I has members i1 < i2 (or i1 alone).  Rows of at most 32 entries group equal
// J = agg(j) in registers (__match_any_sync); longer ones key their fine entries by
// (J, local slot) and sort them (bitonic: in registers by a warp up to kWarpCap entries,
// in shared memory by a block beyond, up to kBlockCap entries), so equal J are adjacent.
// Each run of equal J holds at most four terms (two members each side); the run's value
// sums t_ij = (p_i p_j) a_ij from +0.0 in ascending (min(i,j), max(i,j), i) order with
// round-to-nearest intrinsics, which makes the result independent of the thread schedule
// and bit-symmetric.  The grouping has a binary32 variant
// (Acc = float): p_i, p_j and a_ij rounded to float, terms and sums in float in the same
// order, each entry stored as the double of its float.
#include <climits>

#include "coarsen.cuh"

namespace cwm {

constexpr int kWarpCap = 256;     // keys per warp (sorted in registers, kept in shared memory)
constexpr int kWarpsPerBlock = 8;
constexpr int kBlockCap = 8192;   // keys per long row (64 KB of dynamic shared memory)
constexpr int kLongThreads = 256;
#ifndef CWM_GALERKIN_KEY32
#define CWM_GALERKIN_KEY32 1
#endif

struct RowSrc {
  int i1, i2;  // members (i2 < 0: singleton)
  int s1, L1;  // first slot and length of row i1
  int s2, L2;  // same for row i2
};

__device__ __forceinline__ RowSrc row_src(int I, const int *__restrict__ m1, const int *__restrict__ m2,
                                          const int *__restrict__ rp) {
  RowSrc r;
  r.i1 = m1[I];
  r.i2 = m2[I];
  r.s1 = rp[r.i1];
  r.L1 = rp[r.i1 + 1] - r.s1;
  if (r.i2 >= 0) {
    r.s2 = rp[r.i2];
    r.L2 = rp[r.i2 + 1] - r.s2;
  } else {
    r.s2 = 0;
    r.L2 = 0;
  }
  return r;
}

__device__ __forceinline__ unsigned long long make_key(const RowSrc &r, int q, const int *__restrict__ ci,
                                                       const int *__restrict__ agg) {
  const int k = q < r.L1 ? r.s1 + q : r.s2 + (q - r.L1);
  const unsigned J = (unsigned)agg[ci[k]];
  return ((unsigned long long)J << 32) | (unsigned)q;
}

// Round-to-nearest arithmetic of the accumulation type (no contraction into FMA).
template <class Acc>
struct Arith;
template <>
struct Arith<double> {
  static __device__ __forceinline__ double in(double x) { return x; }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
};
template <>
struct Arith<float> {
  static __device__ __forceinline__ float in(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};

// Acc(0) + t without an FP operation: t itself, except -0 which becomes +0 (the sum of a
// run starts from +0.0).  FP64 instructions issue at a low rate on GB300.
__device__ __forceinline__ double plus_zero(double t) {
  return (unsigned long long)__double_as_longlong(t) == 0x8000000000000000ull ? 0.0 : t;
}
__device__ __forceinline__ float plus_zero(float t) { return __float_as_uint(t) == 0x80000000u ? 0.0f : t; }

// t_ij = (p_i p_j) a_ij in the accumulation type
template <class Acc>
__device__ __forceinline__ Acc term(double pi, double pj, double a) {
  using M = Arith<Acc>;
  return M::mul(M::mul(M::in(pi), M::in(pj)), M::in(a));
}

// Sum of one run of equal J (length len <= 4) starting at sorted position q.
template <class Acc>
__device__ __forceinline__ double run_value(const RowSrc &r, const unsigned long long *keys, int q, int len,
                                            const int *__restrict__ ci, const double *__restrict__ val,
                                            const double *__restrict__ p) {
  int kmin[4], kmax[4], ii[4];
  Acc t[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e < len) {
      const int local = (int)(keys[q + e] & 0xffffffffu);
      const bool first = local < r.L1;
      const int i = first ? r.i1 : r.i2;
      const int k = first ? r.s1 + local : r.s2 + (local - r.L1);
      const int j = ci[k];
      t[e] = term<Acc>(p[i], p[j], val[k]);
      kmin[e] = i < j ? i : j;
      kmax[e] = i < j ? j : i;
      ii[e] = i;
    } else {
      t[e] = Acc(0);
      kmin[e] = kmax[e] = ii[e] = INT_MAX;
    }
  }
  // insertion sort of <= 4 terms by (kmin, kmax, i)
#pragma unroll
  for (int a = 1; a < 4; ++a) {
#pragma unroll
    for (int b = a; b > 0; --b) {
      const bool swap = kmin[b] < kmin[b - 1] ||
                        (kmin[b] == kmin[b - 1] && (kmax[b] < kmax[b - 1] ||
                                                    (kmax[b] == kmax[b - 1] && ii[b] < ii[b - 1])));
      if (swap) {
        int x;
        Acc y;
        x = kmin[b]; kmin[b] = kmin[b - 1]; kmin[b - 1] = x;
        x = kmax[b]; kmax[b] = kmax[b - 1]; kmax[b - 1] = x;
        x = ii[b]; ii[b] = ii[b - 1]; ii[b - 1] = x;
        y = t[b]; t[b] = t[b - 1]; t[b - 1] = y;
      }
    }
  }
  Acc sum = plus_zero(t[0]);
#pragma unroll
  for (int e = 1; e < 4; ++e)
    if (e < len) sum = Arith<Acc>::add(sum, t[e]);
  return (double)sum;
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ------------------------------------------------------------ register rows ----
// A coarse row with L <= G entries held one per lane by a group of G lanes (G = 16 or 32,
// gmask = the group's lanes).  Lanes with equal J are found with __match_any_sync, so no
// sort is needed: the lowest lane of each equal-J group leads it, counts it, and in the
// fill pass gathers the group's (at most four) terms with shuffles, orders them by
// (min(i,j), max(i,j), i), sums them from +0.0, and writes at its rank among the leaders.
template <class Acc>
__device__ __forceinline__ void galerkin_row_reg(const RowSrc &r, int I, unsigned gmask, int gbase, int glen,
                                                 const int *__restrict__ ci, const double *__restrict__ val,
                                                 const int *__restrict__ agg, const double *__restrict__ p,
                                                 int *__restrict__ cnt, const int *__restrict__ rpc,
                                                 int *__restrict__ cic, double *__restrict__ valc,
                                                 double *__restrict__ diag_c, int *err) {
  const int lane = threadIdx.x & 31;
  const int gl = lane - gbase;
  const int L = r.L1 + r.L2;
  const bool act = gl < L;
  int k = 0, i = 0, j = 0;
  unsigned J = 0x80000000u | (unsigned)lane;  // unique per lane, never a real column
  if (act) {
    const bool first = gl < r.L1;
    i = first ? r.i1 : r.i2;
    k = first ? r.s1 + gl : r.s2 + (gl - r.L1);
    j = ci[k];
    J = (unsigned)agg[j];
  }
  const unsigned mm = __match_any_sync(gmask, J);
  const bool leader = act && lane == __ffs(mm) - 1;
  const unsigned lead = __ballot_sync(gmask, leader) & gmask;
  if (gl == 0 && cnt) cnt[I] = __popc(lead);
  Acc t = Acc(0);
  int kmin = 0, kmax = 0;
  if (act) {
    t = term<Acc>(p[i], p[j], val[k]);
    kmin = min(i, j);
    kmax = max(i, j);
  }
  const int members = __popc(mm);
  int src[4];
  unsigned rest = mm;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    src[m] = rest ? __ffs(rest) - 1 : lane;
    rest &= rest - 1u;
  }
  Acc tm[4];
  int kmn[4], kmx[4], im[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    tm[m] = __shfl_sync(gmask, t, src[m]);
    kmn[m] = __shfl_sync(gmask, kmin, src[m]);
    kmx[m] = __shfl_sync(gmask, kmax, src[m]);
    im[m] = __shfl_sync(gmask, i, src[m]);
  }
  int rank = 0;
  for (int l = gbase; l < gbase + glen; ++l) {
    const unsigned Jl = __shfl_sync(gmask, J, l);
    if (((lead >> l) & 1u) && Jl < J) ++rank;
  }
  if (!leader) return;
  if (members > 4) atomicOr(err, kErrInvalid);
  const int len = members < 4 ? members : 4;
#pragma unroll
  for (int m = 0; m < 4; ++m)
    if (m >= len) { kmn[m] = kmx[m] = im[m] = INT_MAX; tm[m] = Acc(0); }
#pragma unroll
  for (int a = 1; a < 4; ++a) {
#pragma unroll
    for (int b = a; b > 0; --b) {
      const bool swap = kmn[b] < kmn[b - 1] ||
                        (kmn[b] == kmn[b - 1] && (kmx[b] < kmx[b - 1] || (kmx[b] == kmx[b - 1] && im[b] < im[b - 1])));
      if (swap) {
        int x;
        Acc y;
        x = kmn[b]; kmn[b] = kmn[b - 1]; kmn[b - 1] = x;
        x = kmx[b]; kmx[b] = kmx[b - 1]; kmx[b - 1] = x;
        x = im[b]; im[b] = im[b - 1]; im[b - 1] = x;
        y = tm[b]; tm[b] = tm[b - 1]; tm[b - 1] = y;
      }
    }
  }
  Acc acc = plus_zero(tm[0]);
#pragma unroll
  for (int m = 1; m < 4; ++m)
    if (m < len) acc = Arith<Acc>::add(acc, tm[m]);
  const double sum = (double)acc;
  const int out = rpc[I] + rank;
  cic[out] = (int)J;
  valc[out] = sum;
  if ((int)J == I && diag_c) diag_c[I] = sum;
}

// ------------------------------------------------------------ shared-memory rows ----
// Bitonic sort of the warp's 32 * E keys held in registers, key q = lane * E + e: stages
// with j < E compare within a lane, the others exchange with lane ^ (j / E) by shuffles.
// All loops unroll, so the array stays in registers.
template <int E, class K>
__device__ __forceinline__ void warp_bitonic(K (&a)[E], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < E) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int f = e ^ j;
          if (f > e) {
            const bool up = ((lane * E + e) & k) == 0;
            const K x = a[e], y = a[f];
            if ((x > y) == up) { a[e] = y; a[f] = x; }
          }
        }
      } else {
        const int lm = j / E;
        const bool lower = (lane & lm) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const K o = __shfl_xor_sync(0xffffffffu, a[e], lm);
          const bool up = ((lane * E + e) & k) == 0;
          a[e] = (lower == up) ? (a[e] < o ? a[e] : o) : (a[e] < o ? o : a[e]);
        }
      }
    }
  }
}

// Keys (J, slot) of a coarse row with L <= 32 * E entries, sorted into keys[0 .. 32E) as
// (J << 32) | slot.  K32 (every J below 2^24 - 1): the register sort runs on 32-bit keys
// (J << 8) | slot -- slots are below 256 -- half the shuffles and compares of 64-bit keys.
template <int E, bool K32>
__device__ __forceinline__ void sort_row_keys(const RowSrc &r, int L, unsigned long long *keys,
                                              const int *__restrict__ ci, const int *__restrict__ agg, int lane) {
  if (K32) {
    unsigned a[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = lane * E + e;
      const unsigned long long k = q < L ? make_key(r, q, ci, agg) : 0ull;
      a[e] = q < L ? (unsigned)((k >> 32) << 8) | (unsigned)(k & 0xffu) : ~0u;
    }
    warp_bitonic<E>(a, lane);
#pragma unroll
    for (int e = 0; e < E; ++e)
      keys[lane * E + e] = ((unsigned long long)(a[e] >> 8) << 32) | (unsigned long long)(a[e] & 0xffu);
  } else {
    unsigned long long a[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = lane * E + e;
      a[e] = q < L ? make_key(r, q, ci, agg) : ~0ull;
    }
    warp_bitonic<E>(a, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) keys[lane * E + e] = a[e];
  }
  __syncwarp();
}

// A coarse row with 32 < L <= kWarpCap entries: keys (J, slot) sorted by the warp in
// registers (bitonic), then two passes over the sorted positions.  Pass 1, every lane: the
// term t = (p_i p_j) a_ij of each position, its canonical key (min(i,j), max(i,j), i) packed in
// 64 bits (into keys[], whose (J, slot) is no longer needed) and its J (jq[]).  Pass 2, the
// first position of each run of equal J: orders the run's (at most four) terms by their
// canonical keys and sums them.  The FP64 products then run on full warps; only the few
// additions of each run run on its first lane.
template <class Acc, bool K32>
__device__ __forceinline__ void galerkin_row_smem(const RowSrc &r, int I, unsigned long long *keys, double *tq,
                                                  unsigned *jq, const int *__restrict__ ci,
                                                  const double *__restrict__ val, const int *__restrict__ agg,
                                                  const double *__restrict__ p, int *__restrict__ cnt,
                                                  const int *__restrict__ rpc, int *__restrict__ cic,
                                                  double *__restrict__ valc, double *__restrict__ diag_c, int *err) {
  const int lane = threadIdx.x & 31;
  const int L = r.L1 + r.L2;
  if (L <= 64) sort_row_keys<2, K32>(r, L, keys, ci, agg, lane);
  else if (L <= 128) sort_row_keys<4, K32>(r, L, keys, ci, agg, lane);
  else sort_row_keys<8, K32>(r, L, keys, ci, agg, lane);
  for (int q = lane; q < L; q += 32) {
    const unsigned long long key = keys[q];
    const int local = (int)(key & 0xffffffffu);
    const bool first = local < r.L1;
    const int i = first ? r.i1 : r.i2;
    const int k = first ? r.s1 + local : r.s2 + (local - r.L1);
    const int j = ci[k];
    tq[q] = (double)term<Acc>(p[i], p[j], val[k]);
    jq[q] = (unsigned)(key >> 32);
    const unsigned long long lo = (unsigned)min(i, j), hi = (unsigned)max(i, j);
    keys[q] = (lo << 33) | (hi << 1) | (unsigned long long)(i == max(i, j) && i != j);
  }
  __syncwarp();
  int base = 0;
  for (int q0 = 0; q0 < L; q0 += 32) {
    const int q = q0 + lane;
    bool head = false;
    unsigned J = 0;
    if (q < L) {
      J = jq[q];
      head = q == 0 || jq[q - 1] != J;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, head);
    if (head) {
      int len = 1;
      while (len < 5 && q + len < L && jq[q + len] == J) ++len;
      if (len > 4) { atomicOr(err, kErrInvalid); len = 4; }
      unsigned long long ck[4];
      Acc t[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ck[e] = e < len ? keys[q + e] : ~0ull;
        t[e] = e < len ? (Acc)tq[q + e] : Acc(0);
      }
#pragma unroll
      for (int a = 1; a < 4; ++a) {
#pragma unroll
        for (int b = a; b > 0; --b) {
          if (ck[b] < ck[b - 1]) {
            const unsigned long long x = ck[b]; ck[b] = ck[b - 1]; ck[b - 1] = x;
            const Acc y = t[b]; t[b] = t[b - 1]; t[b - 1] = y;
          }
        }
      }
      Acc sum = plus_zero(t[0]);
#pragma unroll
      for (int e = 1; e < 4; ++e)
        if (e < len) sum = Arith<Acc>::add(sum, t[e]);
      const int out = rpc[I] + base + __popc(ball & ((1u << lane) - 1u));
      cic[out] = (int)J;
      valc[out] = (double)sum;
      if ((int)J == I && diag_c) diag_c[I] = (double)sum;
    }
    base += __popc(ball);
  }
  if (cnt && lane == 0) cnt[I] = base;
  __syncwarp();
}

// ------------------------------------------------------------ warp kernel ----
// Each warp takes two consecutive coarse rows.  When both gather <= 16 entries each half
// warp handles one in registers; otherwise the warp handles them in turn (registers up to
// 32 entries, the warp's register sort up to kWarpCap, longer rows queued for the block
// kernel).
// Columns and values of row I at rpc[I] (the padded offsets), and cnt[I] = its number of
// distinct J.
template <class Acc, bool K32>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_galerkin_warp(int nc, const int *__restrict__ rp, const int *__restrict__ ci,
                    const double *__restrict__ val, const int *__restrict__ m1,
                    const int *__restrict__ m2, const int *__restrict__ agg,
                    const double *__restrict__ p, int *__restrict__ cnt,
                    const int *__restrict__ rpc, int *__restrict__ cic, double *__restrict__ valc,
                    double *__restrict__ diag_c, int *__restrict__ long_rows, int *__restrict__ n_long, int *err) {
  __shared__ unsigned long long sbuf[kWarpsPerBlock][kWarpCap];
  __shared__ double stq[kWarpsPerBlock][kWarpCap];
  __shared__ unsigned sjq[kWarpsPerBlock][kWarpCap];
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4;
  unsigned long long *keys = sbuf[threadIdx.x >> 5];
  double *tq = stq[threadIdx.x >> 5];
  unsigned *jq = sjq[threadIdx.x >> 5];
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp0 * 2; base < nc; base += nwarps * 2) {
    const int Ih = (int)(base + half);
    RowSrc rh{};
    int Lh = 0;
    if (Ih < nc) {
      rh = row_src(Ih, m1, m2, rp);
      Lh = rh.L1 + rh.L2;
    }
    const int L0 = __shfl_sync(0xffffffffu, Lh, 0), L1 = __shfl_sync(0xffffffffu, Lh, 16);
    if (L0 <= 16 && L1 <= 16) {
      if (Ih < nc)
        galerkin_row_reg<Acc>(rh, Ih, half ? 0xffff0000u : 0x0000ffffu, half * 16, 16, ci, val, agg, p, cnt, rpc,
                               cic, valc, diag_c, err);
      __syncwarp();
      continue;
    }
    for (int h = 0; h < 2; ++h) {
      const int I = (int)base + h;
      if (I >= nc) break;
      const RowSrc r = row_src(I, m1, m2, rp);
      const int L = r.L1 + r.L2;
      if (L <= 32) {
        galerkin_row_reg<Acc>(r, I, 0xffffffffu, 0, 32, ci, val, agg, p, cnt, rpc, cic, valc, diag_c, err);
      } else if (L <= kWarpCap) {
        galerkin_row_smem<Acc, K32>(r, I, keys, tq, jq, ci, val, agg, p, cnt, rpc, cic, valc, diag_c, err);
      } else if (long_rows && lane == 0) {
        long_rows[atomicAdd(n_long, 1)] = I;
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------ long rows ----
template <class Acc>
__global__ void __launch_bounds__(kLongThreads)
    k_galerkin_block(const int *__restrict__ rp, const int *__restrict__ ci,
                     const double *__restrict__ val, const int *__restrict__ m1,
                     const int *__restrict__ m2, const int *__restrict__ agg,
                     const double *__restrict__ p, int *__restrict__ cnt,
                     const int *__restrict__ rpc, int *__restrict__ cic, double *__restrict__ valc,
                     double *__restrict__ diag_c, double *__restrict__ dl1_c,
                     const int *__restrict__ long_rows, const int *__restrict__ n_long, int *err) {
  extern __shared__ unsigned long long keys[];
  __shared__ int wsum[kLongThreads / 32 + 1];
  __shared__ double wl1[kLongThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kLongThreads / 32;
  const int nrows = *n_long;
  for (int b = blockIdx.x; b < nrows; b += gridDim.x) {
    const int I = long_rows[b];
    const RowSrc r = row_src(I, m1, m2, rp);
    const int L = r.L1 + r.L2;
    if (L > kBlockCap) {
      if (tid == 0) {
        atomicOr(err, kErrUnsupported);
        if (cnt) cnt[I] = 0;
      }
      continue;
    }
    const int P = next_pow2(L < kLongThreads ? kLongThreads : L);
    for (int q = tid; q < P; q += kLongThreads) keys[q] = q < L ? make_key(r, q, ci, agg) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = tid; q < P; q += kLongThreads) {
          const int l = q ^ j;
          if (l > q) {
            const unsigned long long a = keys[q], bb = keys[l];
            if ((a > bb) == ((q & k) == 0)) { keys[q] = bb; keys[l] = a; }
          }
        }
        __syncthreads();
      }
    }
    int base = 0;
    double l1 = 0.0;
    for (int q0 = 0; q0 < L; q0 += kLongThreads) {
      const int q = q0 + tid;
      bool head = false;
      unsigned J = 0;
      if (q < L) {
        J = (unsigned)(keys[q] >> 32);
        head = q == 0 || (unsigned)(keys[q - 1] >> 32) != J;
      }
      const unsigned ball = __ballot_sync(0xffffffffu, head);
      if (lane == 0) wsum[warp] = __popc(ball);
      __syncthreads();
      int before = 0, chunk = 0;
      for (int w = 0; w < nw; ++w) {
        if (w < warp) before += wsum[w];
        chunk += wsum[w];
      }
      if (head) {
        int len = 1;
        while (len < 5 && q + len < L && (unsigned)(keys[q + len] >> 32) == J) ++len;
        if (len > 4) { atomicOr(err, kErrInvalid); len = 4; }
        const double s = run_value<Acc>(r, keys, q, len, ci, val, p);
        const int out = rpc[I] + base + before + __popc(ball & ((1u << lane) - 1u));
        cic[out] = (int)J;
        valc[out] = s;
        if ((int)J == I && diag_c) diag_c[I] = s;
        l1 += fabs(s);
      }
      base += chunk;
      __syncthreads();
    }
    if (cnt && tid == 0) cnt[I] = base;
    if (dl1_c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
      if (lane == 0) wl1[warp] = l1;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += wl1[w];
        dl1_c[I] = t;
      }
    }
    __syncthreads();
  }
}

static amg_status galerkin_attrs() {
  static bool attr_set[64] = {false};
  int dev = 0;
  CWM_CUDA(cudaGetDevice(&dev));
  bool &attr = attr_set[dev & 63];
  if (!attr) {
    CWM_CUDA(cudaFuncSetAttribute(k_galerkin_block<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kBlockCap * 8));
    CWM_CUDA(cudaFuncSetAttribute(k_galerkin_block<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kBlockCap * 8));
    attr = true;
  }
  return AMG_OK;
}

// cnt[I] = L1 + L2: the number of fine entries that coarse row I gathers, an upper bound
// on its length (its padded row length).
__global__ void k_gather_lengths(int nc, const int *__restrict__ rp, const int *__restrict__ m1,
                                 const int *__restrict__ m2, int *__restrict__ cnt, int *__restrict__ n_long) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I == 0) *n_long = 0;  // the long-row queue starts empty
  if (I >= nc) return;
  const int i1 = m1[I], i2 = m2[I];
  cnt[I] = rp[i1 + 1] - rp[i1] + (i2 >= 0 ? rp[i2 + 1] - rp[i2] : 0);
}

// Copies row I from its padded place [rpu[I], rpu[I] + len) to [rpc[I], rpc[I+1]); an
// 8-lane tile per row.
__global__ void k_galerkin_compact(int nc, const int *__restrict__ rpu, const int *__restrict__ rpc,
                                   const int *__restrict__ ci_pad, const double *__restrict__ val_pad,
                                   int *__restrict__ cic, double *__restrict__ valc) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int lane = threadIdx.x & 7;
  const long long nt = ((long long)gridDim.x * blockDim.x) >> 3;
  for (long long I = t; I < nc; I += nt) {
    const int src = rpu[I], dst = rpc[I], len = rpc[I + 1] - dst;
    for (int q = lane; q < len; q += 8) {
      cic[dst + q] = ci_pad[src + q];
      valc[dst + q] = val_pad[src + q];
    }
  }
}

amg_status galerkin_group(const int *rp, const int *ci, const double *val, int nc, const int *m1,
                          const int *m2, const int *agg, const double *p, int *rpc, double *diag_c,
                          double *dl1_c, const GalerkinWork &work, bool fp32, int *d_err, cudaStream_t s) {
  if (nc == 0) {
    CWM_CUDA(cudaMemsetAsync(rpc, 0, sizeof(int), s));
    return AMG_OK;
  }
  CWM_TRY(galerkin_attrs());
  // members and row bounds, ci, agg(ci), val and p of both member rows; the padded rows
  // written (columns and values), the counts and both scans
  CWM_TRACE("galerkin", 16.0 * work.nnz_fine + 16.0 * work.n_fine + 72.0 * nc + 12.0 * work.nnz_fine, s);
  k_gather_lengths<<<grid_for(nc, 256, 1 << 30), 256, 0, s>>>(nc, rp, m1, m2, work.cnt, work.n_long);
  CWM_LAUNCH();
  CWM_TRY(exclusive_scan(work.cnt, work.rpu, nc, work.scan, s));
  const int block = kWarpsPerBlock * 32;
  const int grid = grid_for((long long)nc * 16, block, num_sms() * 8);
  // 32-bit sort keys (J << 8) | slot when every J leaves the all-ones key free for padding and
  // the fine rows are long enough for coarse rows to reach the sort path (2 x mean > 32).
  // Measured (elasticity 64^3, 78 entries per row): level-0 sweeps 2001 -> 1243 and 963 ->
  // 586 us, setup 15.1 -> 13.6 ms; on the 7-entry rows of 3D Poisson 128^3, where the register
  // path does the work, that kernel variant was 4% slower (its registers capped lower).
  const double mean_row = work.n_fine > 0 ? (double)work.nnz_fine / work.n_fine : 0.0;
  const bool k32 = CWM_GALERKIN_KEY32 && nc < (1 << 24) - 1 && mean_row > 16.0;
#define CWM_GAL_LAUNCH(ACC)                                                                                     \
  if (k32)                                                                                                     \
    k_galerkin_warp<ACC, true><<<grid, block, 0, s>>>(nc, rp, ci, val, m1, m2, agg, p, work.cnt, work.rpu,        \
                                                      work.ci_pad, work.val_pad, diag_c, work.long_rows,        \
                                                      work.n_long, d_err);                                      \
  else                                                                                                         \
    k_galerkin_warp<ACC, false><<<grid, block, 0, s>>>(nc, rp, ci, val, m1, m2, agg, p, work.cnt, work.rpu,       \
                                                       work.ci_pad, work.val_pad, diag_c, work.long_rows,       \
                                                       work.n_long, d_err);                                     \
  CWM_LAUNCH();                                                                                                \
  k_galerkin_block<ACC><<<num_sms() * 2, kLongThreads, kBlockCap * 8, s>>>(                                    \
      rp, ci, val, m1, m2, agg, p, work.cnt, work.rpu, work.ci_pad, work.val_pad, diag_c, dl1_c, work.long_rows, \
      work.n_long, d_err);
  if (fp32) {
    CWM_GAL_LAUNCH(float)
  } else {
    CWM_GAL_LAUNCH(double)
  }
#undef CWM_GAL_LAUNCH
  CWM_LAUNCH();
  return exclusive_scan(work.cnt, rpc, nc, work.scan, s);
}

amg_status galerkin_compact(int nc, const int *rpc, int *cic, double *valc, const GalerkinWork &work,
                            cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  k_galerkin_compact<<<grid_for((long long)nc * 8, 256, num_sms() * 8), 256, 0, s>>>(
      nc, work.rpu, rpc, work.ci_pad, work.val_pad, cic, valc);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ members from agg ----
__global__ void k_members_init(int nc, int *m1, int *m2, int *cnt) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < nc) { m1[I] = INT_MAX; m2[I] = -1; cnt[I] = 0; }
}

__global__ void k_members_scatter(int n, int nc, const int *__restrict__ agg, int *m1, int *m2, int *cnt,
                                  int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int I = agg[i];
  if (I < 0 || I >= nc) { atomicOr(err, kErrInvalid); return; }
  atomicMin(m1 + I, i);
  atomicMax(m2 + I, i);
  atomicAdd(cnt + I, 1);
}

__global__ void k_members_final(int nc, int *m1, int *m2, const int *cnt, int *err) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const int c = cnt[I];
  if (c < 1 || c > 2) {
    atomicOr(err, kErrInvalid);
    m1[I] = 0;
    m2[I] = -1;
    return;
  }
  if (c == 1) m2[I] = -1;
}

amg_status members_from_agg(int n, int nc, const int *agg, int *m1, int *m2, int *cnt, int *d_err,
                            cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  k_members_init<<<grid_for(nc, 256, 1 << 30), 256, 0, s>>>(nc, m1, m2, cnt);
  CWM_LAUNCH();
  if (n > 0) {
    k_members_scatter<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, nc, agg, m1, m2, cnt, d_err);
    CWM_LAUNCH();
  }
  k_members_final<<<grid_for(nc, 256, 1 << 30), 256, 0, s>>>(nc, m1, m2, cnt, d_err);
  CWM_LAUNCH();
  return AMG_OK;
}

}  // namespace cwm
