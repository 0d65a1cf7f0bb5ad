// block3.cu -- the input operator of a vector problem with three unknowns per node (3D
// elasticity, dof-interleaved) in 3x3 blocks: a sliced-ELL layout over 32 block rows, and
// the level-0 solve kernels that stream it (the residual of the l1-Jacobi V-cycle, Sec. 3.2
// and Algorithm 1; the SpMV with the fused dot products of the flexible CG, Sec. 3.2 and
// Algorithm 3).
//
// When every block row (rows 3b, 3b+1, 3b+2) stores the same columns in whole aligned
// triples (3c, 3c+1, 3c+2) -- the assembled pattern of a nodal vector discretisation --
// the column indices collapse to one per 3x3 block: 4.44 bytes per entry instead of 8 in
// binary32 and 8.44 instead of 12 in binary64, and every x gather fetches three adjacent
// values.  Layout: block row b belongs to slice b / 32 and lane b % 32; its t-th block sits
// in slot sptr[b / 32] + 32 t + b % 32, so the 32 threads of a warp, one per block row of a
// slice, read consecutive slots.  Block columns go to bci[slot]; the nine values go to nine
// planes val[e * slots + slot], e = 3 * (row in block) + (column in block), so each value
// load of a warp is one contiguous 128- or 256-byte line.  A slice is padded to its longest
// block row; a thread stops at its own row's length (blen), so padding is never read.
//
// A thread owns a block row: three FMA chains, one per row, each in the row's column order
// within a block and block order within the row (the same products as the CSR row, in a
// different summation order than the CSR kernels), one FMA per stored entry.
#include "fcg.cuh"
#include "solve.cuh"

namespace cwm {

constexpr int kS3 = 32;           // block rows per slice (one warp)
constexpr int kS3Block = 128;     // threads per block of the residual kernels
constexpr int kS3DotsBlock = 256; // threads per block of the SpMV + dots kernel (block_sums layout)
// Resident blocks per SM that the SpMV + dots kernel's registers must allow, and blocks per
// step.  Measured on Q1 elasticity 64^3 (average per launch over a solve): 2 blocks and 2 per
// step (116 registers, a fifth of the warp slots, FP64 pipe 75% busy) 145 us; 3 blocks and
// 1 per step (80 registers) 155 us; 4 and 1 (64 registers) 156 us -- the FP64-issue-bound
// chains want independent FMAs more than warps.
#ifndef CWM_B3_DOTS_MIN_BLOCKS
#define CWM_B3_DOTS_MIN_BLOCKS 2
#endif
#ifndef CWM_B3_DOTS_UNROLL
#define CWM_B3_DOTS_UNROLL 2
#endif
// Blocks per step of the binary32 residual (binary64 takes 2): 4 measured 54.5 us against
// 59.6 us with 2 (Q1 elasticity 64^3, level 0).
#ifndef CWM_B3_RESID_UNROLL32
#define CWM_B3_RESID_UNROLL32 4
#endif

// ------------------------------------------------------------ detection ----
// A warp per block row.  flag |= 1 when rows 3b..3b+2 differ in length or columns, or a
// column triple is not (3c, 3c+1, 3c+2); smax[b / 32] = max over the slice of blocks per
// block row.
__global__ void k_block3_detect(int nbr, const int *__restrict__ rp, const int *__restrict__ ci, int *flag,
                                int *smax) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nbr) return;
  const int b = (int)wid;
  const int s0 = rp[3 * b], s1 = rp[3 * b + 1], s2 = rp[3 * b + 2], s3 = rp[3 * b + 3];
  const int L = s1 - s0;
  bool bad = (s2 - s1) != L || (s3 - s2) != L || (L % 3) != 0 || L <= 0;
  if (!bad) {
    for (int k = lane; k < L; k += 32) {
      const int c = ci[s0 + k];
      const int lead = ci[s0 + k - (k % 3)];
      if ((lead % 3) != 0 || c != lead + (k % 3) || ci[s1 + k] != c || ci[s2 + k] != c) bad = true;
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (bad) atomicOr(flag, 1);
    else atomicMax(smax + b / kS3, L / 3);
  }
}

amg_status block3_detect(int n, const int *rp, const int *ci, int *d_flag, int *d_smax, cudaStream_t s) {
  const int nbr = n / 3;
  if (nbr == 0) return AMG_OK;
  CWM_TRACE("block3_detect", 4.0 * (n + 1), s);
  k_block3_detect<<<grid_for((long long)nbr * 32, 256, 1 << 30), 256, 0, s>>>(nbr, rp, ci, d_flag, d_smax);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ fill ----
// A thread per (slice, lane): walks the slice's slots t = 0 .. smax-1 of its block row,
// writing block column and the nine values of each block (padding: column 0, values 0).
// Writes are coalesced across the warp; the row reads are served from cache after the
// first touch of each line.
__global__ void k_block3_fill(int nbr, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ val, const int *__restrict__ sptr, int *__restrict__ blen,
                              int *__restrict__ bci, double *__restrict__ v64, float *__restrict__ v32,
                              long long slots) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long sl = tid >> 5;
  const int lane = threadIdx.x & 31;
  const int nsl = (nbr + kS3 - 1) / kS3;
  if (sl >= nsl) return;
  const int b = (int)(sl * kS3 + lane);
  const bool in = b < nbr;
  const int base = sptr[sl], tmax = (sptr[sl + 1] - base) / kS3;
  int r0 = 0, r1 = 0, r2 = 0, len = 0;
  if (in) {
    r0 = rp[3 * b];
    r1 = rp[3 * b + 1];
    r2 = rp[3 * b + 2];
    len = (r1 - r0) / 3;
    blen[b] = len;
  }
  for (int t = 0; t < tmax; ++t) {
    const long long slot = base + (long long)t * kS3 + lane;
    const bool live = in && t < len;
    bci[slot] = live ? ci[r0 + 3 * t] / 3 : 0;
    const int rows[3] = {r0, r1, r2};
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double a = live ? val[rows[rr] + 3 * t + c] : 0.0;
        v64[(3 * rr + c) * slots + slot] = a;
        if (v32) v32[(3 * rr + c) * slots + slot] = (float)a;
      }
  }
}

amg_status block3_fill(int n, const int *rp, const int *ci, const double *val, const int *sptr, int *blen,
                       int *bci, double *v64, float *v32, long long slots, cudaStream_t s) {
  const int nbr = n / 3;
  if (nbr == 0) return AMG_OK;
  const int nsl = (nbr + kS3 - 1) / kS3;
  CWM_TRACE("block3_fill", 4.0 * n + (152.0 + (v32 ? 36.0 : 0.0)) * slots, s);
  k_block3_fill<<<grid_for((long long)nsl * 32, 256, 1 << 30), 256, 0, s>>>(nbr, rp, ci, val, sptr, blen, bci, v64,
                                                                           v32, slots);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ row products ----
// The three rows of block row b against x: acc[i] = init[i] - sum over the row's blocks of
// a_(3b+i, 3c+j) x_(3c+j) (NEG) or + (otherwise).  SCALED reads x_j = d_j * x_j on the fly
// (the first l1-Jacobi sweep from zero, x = D^{-1} b).  UB blocks per step, their loads
// issued before the FMAs.  With CWM_B3_PREFETCH the block columns of the next step are
// loaded one step ahead, so that a step's value loads and its x gathers go out together
// (one round trip per step instead of two): Q1 elasticity 64^3, SpMV+dots 143.8 -> 137.7 us,
// binary32 residual 54.9 -> 53.2 us (96 registers against 72; 2 or 3 blocks per step there
// measured 55.5 and 57.4 us).
#ifndef CWM_B3_PREFETCH
#define CWM_B3_PREFETCH 1
#endif
template <class V, bool NEG, bool SCALED, int UB>
__device__ __forceinline__ void block3_rows(const Sell3View<V> &A, long long base, int len, int tmax,
                                            const V *__restrict__ x, const V *__restrict__ d, V (&acc)[3]) {
  const long long P = A.slots;
  const V sg = NEG ? V(-1) : V(1);
#if CWM_B3_PREFETCH
  int cn[UB];
#pragma unroll
  for (int u = 0; u < UB; ++u) cn[u] = u < len ? __ldcs(A.bci + base + (long long)u * kS3) : 0;
#endif
  for (int t = 0; t < tmax; t += UB) {
    int c[UB];
    V a[UB][9], xv[UB][3];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const bool live = t + u < len;
      const long long q = base + (long long)(t + u) * kS3;
#if CWM_B3_PREFETCH
      c[u] = cn[u];
#else
      c[u] = live ? __ldcs(A.bci + q) : 0;
#endif
#pragma unroll
      for (int e = 0; e < 9; ++e) a[u][e] = live ? __ldcs(A.val + e * P + q) : V(0);
    }
#if CWM_B3_PREFETCH
#pragma unroll
    for (int u = 0; u < UB; ++u)
      cn[u] = t + UB + u < len ? __ldcs(A.bci + base + (long long)(t + UB + u) * kS3) : 0;
#endif
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const bool live = t + u < len;
#pragma unroll
      for (int jj = 0; jj < 3; ++jj)
        xv[u][jj] = live ? (SCALED ? __ldg(d + 3 * c[u] + jj) * __ldg(x + 3 * c[u] + jj) : __ldg(x + 3 * c[u] + jj))
                         : V(0);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      if (t + u < len) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) acc[i] = fma(sg * a[u][3 * i + jj], xv[u][jj], acc[i]);
      }
    }
  }
}

// r = b - A x (SCALED: x = D^{-1} b formed on the fly, x unused)
template <class V, bool SCALED>
__global__ void __launch_bounds__(kS3Block) k_block3_resid(Sell3View<V> A, const V *__restrict__ b,
                                                           const V *__restrict__ x, const V *__restrict__ d,
                                                           V *__restrict__ r) {
  pdl_begin();
  const long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nsl = (A.nbr + kS3 - 1) / kS3;
  if (sl >= nsl) return;
  const int br = (int)(sl * kS3 + lane);
  const bool in = br < A.nbr;
  const int s0 = A.sptr[sl];
  const int tmax = (A.sptr[sl + 1] - s0) / kS3;
  const int len = in ? A.blen[br] : 0;
  V acc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[i] = in ? b[3 * br + i] : V(0);
  block3_rows<V, true, SCALED, sizeof(V) == 4 ? CWM_B3_RESID_UNROLL32 : 2>(A, s0 + lane, len, tmax, SCALED ? b : x, d,
                                                                            acc);
  if (in) {
#pragma unroll
    for (int i = 0; i < 3; ++i) r[3 * br + i] = acc[i];
  }
}

template <class V>
amg_status block3_residual(const Sell3View<V> &A, const V *b, const V *x, const V *dinv, V *r, cudaStream_t s) {
  if (A.nbr == 0) return AMG_OK;
  // planes, block columns, lengths; b and x (or b and D^{-1}) read once, r written
  CWM_TRACE("residual_b3", (9.0 * sizeof(V) + 4.0) * A.nblocks + 4.0 * A.nbr + 3.0 * sizeof(V) * A.n, s);
  const int nsl = (A.nbr + kS3 - 1) / kS3;
  const int grid = grid_for((long long)nsl * 32, kS3Block, 1 << 30);
  if (dinv) CWM_CUDA(launch_pdl(k_block3_resid<V, true>, grid, kS3Block, 0, s, A, b, (const V *)nullptr, dinv, r));
  else CWM_CUDA(launch_pdl(k_block3_resid<V, false>, grid, kS3Block, 0, s, A, b, x, (const V *)nullptr, r));
  CWM_LAUNCH();
  return AMG_OK;
}

template <class V>
amg_status block3_resid_restrict(const Sell3View<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                                 const V *b, const V *x, const V *dinv, V *r_scratch, V *bc, cudaStream_t s) {
  if (nc == 0) return AMG_OK;
  CWM_TRY(block3_residual<V>(A, b, x, dinv, r_scratch, s));
  return restrict_members<V>(A.n, nc, mptr, mlist, p, r_scratch, bc, s);
}

// ------------------------------------------------------------ FCG SpMV + dots ----
// v = A w with the partial sums of w.r, w.v and w.q (q may be NULL) of Algorithm 3; the
// last block turns every block's partials into the FCG scalars (fcg_scalars_from).  Each
// warp takes a contiguous range of slices (below).
__global__ void __launch_bounds__(kS3DotsBlock, CWM_B3_DOTS_MIN_BLOCKS)
    k_block3_spmv_dots(Sell3View<double> A, const double *__restrict__ w, const double *__restrict__ r,
                       const double *__restrict__ q, double *__restrict__ v, double *__restrict__ part, double *scal,
                       unsigned *tick, int first) {
  pdl_begin();
  const int nsl = (A.nbr + kS3 - 1) / kS3;
  const int lane = threadIdx.x & 31;
  double sa = 0.0, sb = 0.0, sg = 0.0;
  // One resident wave (the grid is capped at the blocks that fit at once); warp g of W
  // takes the contiguous slices [g nsl / W, (g+1) nsl / W), so every SM gets the same
  // number of slices to within one per warp.  A grid of one slice per warp ran 3.3 waves,
  // the last a third full, and left FP64 issue idle on most SMs at the end (145.4 against
  // 142.9 us on Q1 elasticity 64^3).
  const long long W = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long sl_end = (g + 1) * nsl / W;
  for (long long sl = g * nsl / W; sl < sl_end; ++sl) {
    const int br = (int)(sl * kS3 + lane);
    const bool in = br < A.nbr;
    const int s0 = A.sptr[sl];
    const int tmax = (A.sptr[sl + 1] - s0) / kS3;
    const int len = in ? A.blen[br] : 0;
    double wi[3], ri[3], qi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      wi[i] = in ? w[3 * br + i] : 0.0;
      ri[i] = in ? r[3 * br + i] : 0.0;
      qi[i] = (in && q) ? q[3 * br + i] : 0.0;
    }
    double acc[3] = {0.0, 0.0, 0.0};
    block3_rows<double, false, false, CWM_B3_DOTS_UNROLL>(A, s0 + lane, len, tmax, w, nullptr, acc);
    if (in) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        v[3 * br + i] = acc[i];
        sa = fma(wi[i], ri[i], sa);
        sb = fma(wi[i], acc[i], sb);
        if (q) sg = fma(wi[i], qi[i], sg);
      }
    }
  }
  fcg_dots_finish(sa, sb, sg, part, scal, tick, first);
}

int block3_dots_blocks(int n) {
  const int nsl = (n / 3 + kS3 - 1) / kS3;
  return (nsl + kS3DotsBlock / 32 - 1) / (kS3DotsBlock / 32);
}

amg_status block3_spmv_dots(const Sell3View<double> &A, const double *w, const double *r, const double *q, double *v,
                            double *part, int part_blocks, double *scal, unsigned *tick, int first, cudaStream_t s) {
  CWM_TRACE("spmv_dots_b3", 76.0 * A.nblocks + 4.0 * A.nbr + (q ? 32.0 : 24.0) * A.n, s);
  int grid = wave_cap(k_block3_spmv_dots, block3_dots_blocks(A.n), kS3DotsBlock);
  if (grid > part_blocks) grid = part_blocks;
  if (grid < 1) grid = 1;
  CWM_CUDA(launch_pdl(k_block3_spmv_dots, grid, kS3DotsBlock, 0, s, A, w, r, q, v, part, scal, tick, first));
  CWM_LAUNCH();
  return AMG_OK;
}

#define CWM_B3_INST(V)                                                                                           \
  template amg_status block3_residual<V>(const Sell3View<V> &, const V *, const V *, const V *, V *, cudaStream_t); \
  template amg_status block3_resid_restrict<V>(const Sell3View<V> &, int, const int *, const int *, const V *,     \
                                               const V *, const V *, const V *, V *, V *, cudaStream_t);
CWM_B3_INST(double)
CWM_B3_INST(float)

}  // namespace cwm
