// solve.cuh -- host launchers of the solve-phase kernels (solve.cu): CSR SpMV family,
// l1-Jacobi (Sec. 3.2), restriction / prolongation with the aggregation P (Sec. 3.2),
// the one-block coarsest solve, and the flexible-CG vector kernels (Sec. 3.2, Algorithm 3).
#pragma once

#include "common.cuh"

namespace cwm {

// Row walks of the tile and sliced kernels in predicated groups (1) or whole groups followed
// by one entry per round trip (0, the earlier form, kept for measurement).
#ifndef CWM_ROW_PRED
#define CWM_ROW_PRED 1
#endif

template <class V>
struct CsrView {
  int n = 0;
  long long nnz = 0;
  const int *rp = nullptr;
  const int *ci = nullptr;
  const V *val = nullptr;
  int tile = 8;  // sub-warp width chosen from the row lengths (tile_for_rows)
  bool rb = true;  // row-block kernels (else a sub-warp tile per row): row_kernel_shape()
  int max_row = 0;  // longest row (0: unknown)
  // Rows longer than long_min (listed in long_rows[0 .. n_long)) are taken by a whole warp
  // in the l1-Jacobi sweep of a sub-warp-tile level; the tile width then follows the
  // remaining rows.  n_long = 0: no split.
  const int *long_rows = nullptr;
  int n_long = 0;
  int long_min = 0;
  int tile_short = 8;  // tile width of the split sweep's other rows
};

// Shape of a level's solve kernels: row blocks (a thread per row, CSR chunks staged in
// shared memory) or a sub-warp tile of *tile lanes per row.  Row blocks suit short rows.
// With long rows a chunk holds few rows, so few threads (spread over two warps) work while
// the rest wait at the block barrier; in FP64, which GB300 issues per warp instruction at
// a low rate, the half-empty warps double the cost, so FP64 long rows take narrow tiles
// (about a dozen entries per lane, few shuffle steps per row).  FP32 keeps row blocks on
// levels large enough to fill the GPU and takes wide tiles on small ones.  max_row: the
// longest row (0: unknown).
void row_kernel_shape(int n, long long nnz, int max_row, bool fp64, bool *rb, int *tile);
// *d_out = the longest row of the CSR pattern rp (device int; asynchronous)
amg_status max_row_length(int n, const int *rp, int *d_out, cudaStream_t s);
// Length above which a row of a sub-warp-tile level is a "long row" for the split sweep
// (0: the level keeps one tile width for all rows).
int long_row_min(int n, long long nnz, int max_row, bool rb64, bool rb32);
// *d_count = number of rows longer than min_len; with list != NULL they are also written
// to list (in no particular order).  d_count must be zeroed by the caller.
amg_status long_row_list(int n, const int *rp, int min_len, int *list, int *d_count, cudaStream_t s);

// Largest coarsest level solved by the one-block kernel (x kept in shared memory).
constexpr int kCoarseBlockMax = 2048;

// y = dinv .* b
template <class V>
amg_status scale(int n, const V *dinv, const V *b, V *y, cudaStream_t s);
// y = x + dinv .* (b - A x)   (x, y distinct)
template <class V>
amg_status jacobi(const CsrView<V> &A, const V *dinv, const V *b, const V *x, V *y, cudaStream_t s);
// Largest coarsest level whose sweeps are turned into a dense operator at setup.
constexpr int kDenseCoarseMax = 2048;
// X (n*n, row-major) = the linear map of `sweeps` l1-Jacobi sweeps from zero; tmp: n*n
amg_status dense_coarse_build(const CsrView<double> &A, const double *dinv, int sweeps, double *X, double *tmp,
                              cudaStream_t s);
// y = X b
template <class V>
amg_status dense_coarse_apply(int n, const V *X, const V *b, V *y, cudaStream_t s);
// r = b - A x into r_scratch (row blocks), then bc[I] = sum_{m in I} p_m r_m
template <class V>
amg_status resid_restrict_rb(const CsrView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                             const V *b, const V *x, V *r_scratch, V *bc, cudaStream_t s);
// r = b - A (D^{-1} b) into r_scratch, then bc = P^T r (the first sweep from zero fused in;
// row blocks or sub-warp tiles as A's shape says)
template <class V>
amg_status resid_scaled_restrict(const CsrView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                                 const V *dinv, const V *b, V *r_scratch, V *bc, cudaStream_t s);
// x = y + D^{-1}(b - A y) with y = D^{-1} b + P xc formed on the fly
template <class V>
amg_status prolong_jacobi(const CsrView<V> &A, const V *dinv, const V *b, const int *agg, const V *p, const V *xc,
                          V *x, cudaStream_t s);
// Row i of A P (P: one entry p_i in column agg_i per row) into A's padded layout: the
// distinct aggregates J of row i's columns, in order of first occurrence, at ci_pad[rp[i] ..),
// (A P)_iJ = sum of a_ij p_j in the row's order at val_pad[rp[i] ..), their number at cnt[i];
// *maxcnt (zeroed by the caller) is raised to the longest row of A P.  max_row: the
// longest row of A.
amg_status ap_group(int n, long long nnz, const int *rp, const int *ci, const double *val, const int *agg,
                    const double *p, int max_row, int *ci_pad, double *val_pad, int *cnt, int *maxcnt,
                    cudaStream_t s);
// x = y + D^{-1} (r - (A P) xc) with y = xs + P xc and r = b - A xs: the coarse correction
// and one post-sweep (xs may be NULL: 0; xs_scaled: xs holds b and the pre-sweep result is
// D^{-1} b); AP: the stored product A P, nc: columns of P; x64 != NULL: x also written in
// binary64 there
template <class V>
amg_status prolong_jacobi_ap(const CsrView<V> &AP, int nc, const V *dinv, const V *r, const int *agg, const V *p,
                             const V *xc, const V *xs, bool xs_scaled, V *x, cudaStream_t s, double *x64 = nullptr);
// r = b - A x (any value type)
template <class V>
amg_status residual_t(const CsrView<V> &A, const V *b, const V *x, V *r, cudaStream_t s);
// y += x
template <class V>
amg_status add_to(int n, const V *x, V *y, cudaStream_t s);
// y = x + p .* xc[agg]; x may be NULL (0)
template <class V>
amg_status prolong(int n, const int *agg, const V *p, const V *xc, const V *x, V *y, cudaStream_t s);
// x = `sweeps` l1-Jacobi sweeps from zero on a level with n <= kCoarseBlockMax
template <class V>
amg_status coarse_solve_block(const CsrView<V> &A, const V *dinv, const V *b, V *x, int sweeps,
                              cudaStream_t s);
// The coarse end of the V-cycle in one cooperative launch (tail.cu): every level from
// the first with at most kTailMaxRows rows down to the coarsest.
constexpr int kTailMaxRows = 65536;  // default of amg_params.tail_rows
constexpr int kTailMaxLevels = 12;
template <class V>
struct TailLevel {
  int n;
  long long rp_host_nnz;  // nnz, for the tracer's byte count
  const int *rp, *ci;
  const V *val, *dinv;
  const int *agg, *mptr, *mlist;  // transfer to the next level (unused on the coarsest)
  const V *p;
  V *b, *x, *t1, *t2;
  const V *dense;  // coarsest only: the dense operator of the coarse sweeps, or NULL
};
template <class V>
struct TailArgs {
  int nlev;
  int pre, post, coarse_sweeps;
  unsigned spin_cap;  // bound on each grid-barrier wait (polls)
  int grid;           // blocks of the cooperative launch (0: one per SM)
  TailLevel<V> lev[kTailMaxLevels];
};
// x0 = V-cycle of the tail's first level applied to b0; bar: two zeroed unsigned ints (grid
// barrier), err: the device error word
// (a: the host copy, d_a: the same table in device memory)
template <class V>
amg_status vcycle_tail(const TailArgs<V> &a, const TailArgs<V> *d_a, const V *b0, V *x0, unsigned *bar, int *err,
                       cudaStream_t s);
// r = b - A x
amg_status residual(const CsrView<double> &A, const double *b, const double *x, double *r, cudaStream_t s);
// bc[I] = sum over the members m of aggregate I (ascending) of p_m r_m (the restriction P^T r)
template <class V>
amg_status restrict_members(int n, int nc, const int *mptr, const int *mlist, const V *p, const V *r, V *bc,
                            cudaStream_t s);

// ---------------------------------------------------------------- 3x3 blocks ----
// An operator whose block rows (rows 3b, 3b+1, 3b+2) all store the same columns in whole
// aligned triples, held as 3x3 blocks in a sliced-ELL layout over 32 block rows (block3.cu):
// block row b's t-th block at slot sptr[b / 32] + 32 t + b % 32, its block column at
// bci[slot], its values in nine planes val[e * slots + slot] (e = 3 * row + column within
// the block); blen[b] blocks per block row.
template <class V>
struct Sell3View {
  int n = 0;              // scalar rows (3 nbr)
  int nbr = 0;            // block rows
  long long nblocks = 0;  // stored blocks (nnz / 9)
  long long slots = 0;    // plane length (blocks plus slice padding)
  const int *sptr = nullptr;
  const int *blen = nullptr;
  const int *bci = nullptr;
  const V *val = nullptr;
};
// *d_flag |= 1 unless the CSR pattern (n rows) is 3x3-blocked as above; d_smax[s] (zeroed by
// the caller, one per slice of 32 block rows) = the most blocks of a block row of slice s
amg_status block3_detect(int n, const int *rp, const int *ci, int *d_flag, int *d_smax, cudaStream_t s);
// The sliced layout from the CSR arrays: sptr (slice offsets, the scan of 32 d_smax), blen,
// bci, the binary64 planes and (v32 != NULL) their binary32 copy
amg_status block3_fill(int n, const int *rp, const int *ci, const double *val, const int *sptr, int *blen,
                       int *bci, double *v64, float *v32, long long slots, cudaStream_t s);
// r = b - A x, or with dinv != NULL r = b - A (D^{-1} b) (the residual after the first
// l1-Jacobi sweep from zero; x unused)
template <class V>
amg_status block3_residual(const Sell3View<V> &A, const V *b, const V *x, const V *dinv, V *r, cudaStream_t s);
// the residual above into r_scratch, then bc = P^T r
template <class V>
amg_status block3_resid_restrict(const Sell3View<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                                 const V *b, const V *x, const V *dinv, V *r_scratch, V *bc, cudaStream_t s);
// ---------------------------------------------------------------- sliced rows ----
// A long-row operator (or A P) in sliced ELL (sell.cu): rows sorted by length, longest
// first, within windows of 256 rows (perm[p] = the row at position p, len[p] its length);
// `lanes` (K) lanes per row, R = 32 / K positions per slice; entry e of position p = R s + r
// at slot sptr[s] + 32 (e / K) + K r + e % K (col, val).
template <class V>
struct SellView {
  int n = 0;          // rows (0: no sliced copy)
  int lanes = 1;      // K
  long long nnz = 0;  // stored entries
  const int *sptr = nullptr;
  const int *perm = nullptr;
  const int *len = nullptr;
  const int *col = nullptr;
  const V *val = nullptr;
};
// Lanes per row for rows of at most max_row entries (no lane walks more than ~24), and the
// number of slices of n rows
int sell_lanes(int max_row);
int sell_slices(int n, int K);
// perm, len (n ints each), slen (one slice length per slice, scratch) and sptr (their
// exclusive scan, sell_slices(n, K) + 1 ints; sptr[last] = the slots to allocate)
amg_status sell_plan(int n, int K, const int *rp, int *perm, int *len, int *slen, int *sptr, int *scan_scratch,
                     cudaStream_t s);
// col and sval (sptr[last] slots each) from the CSR arrays, values rounded to V
template <class V>
amg_status sell_fill(int n, const int *rp, const int *ci, const double *val, const SellView<V> &S, int *col,
                     V *sval, cudaStream_t s);
// r = b - A x, or with dinv != NULL r = b - A (D^{-1} b) (x unused)
template <class V>
amg_status sell_residual(const SellView<V> &A, const V *b, const V *x, const V *dinv, V *r, cudaStream_t s);
// the residual above into r_scratch, then bc = P^T r
template <class V>
amg_status sell_resid_restrict(const SellView<V> &A, int nc, const int *mptr, const int *mlist, const V *p,
                               const V *b, const V *x, const V *dinv, V *r_scratch, V *bc, cudaStream_t s);
// prolong_jacobi_ap on the sliced A P
template <class V>
amg_status sell_prolong_jacobi_ap(const SellView<V> &AP, int nc, const V *dinv, const V *r, const int *agg,
                                  const V *p, const V *xc, const V *xs, bool xs_scaled, V *x, cudaStream_t s,
                                  double *x64 = nullptr);

// spmv_dots_scalars on the 3x3-block layout (part holds 3 * part_blocks doubles)
amg_status block3_spmv_dots(const Sell3View<double> &A, const double *w, const double *r, const double *q, double *v,
                            double *part, int part_blocks, double *scal, unsigned *tick, int first, cudaStream_t s);

// FCG device scalars (one array of doubles on the device).
enum FcgSlot { kAlpha = 0, kBeta, kGamma, kRho, kRhoPrev, kCoef, kStep, kRR, kBB, kFlags, kFcgSlots };
int fcg_partial_blocks(int n);   // partial sums written by sqnorm_partials
int fcg_dots_blocks(int n, long long nnz);      // row-block grid of spmv_dots
int fcg_dots_blocks_max(int n, long long nnz);  // largest spmv_dots grid of either form (part: 3 per block)
int fcg_update_blocks(int n);    // partial sums written by fcg_update
// v = A w with per-block partial sums of w.r, w.v, w.q (q may be NULL) into part[3 * nb];
// the last block to finish turns them into alpha, beta, gamma, rho, coef = gamma/rho_prev
// and step = alpha/rho in scal (tick: a zeroed counter, left zeroed)
amg_status spmv_dots_scalars(const CsrView<double> &A, const double *w, const double *r, const double *q,
                             double *v, double *part, double *scal, unsigned *tick, int first, cudaStream_t s);
// d = w - coef d; q = v - coef q; x += step d; r -= step q; r.r into scal[kRR] (last block)
// (r32 != NULL: also r32 = the new r rounded to binary32, the next float32 V-cycle's input)
amg_status fcg_update(int n, const double *w, const double *v, double *d, double *q, double *x, double *r,
                      float *r32,
                      double *scal, double *part, unsigned *tick, int first, cudaStream_t s);
// scal[slot] = sum of part[0..nb)
amg_status reduce_into(int nb, const double *part, double *scal, int slot, cudaStream_t s);
// partial sums of a.a into part[nb]
amg_status sqnorm_partials(int n, const double *a, double *part, cudaStream_t s);
// d[i] = sum_j |a_ij| (l1 row norms, Sec. 3.2)
amg_status l1_norms(const CsrView<double> &A, double *d, cudaStream_t s);
// y = 1 / x (and a float copy when y32 is not NULL)
amg_status reciprocal(int n, const double *x, double *y, float *y32, cudaStream_t s);
// float64 <-> float32 copies
amg_status to_float(long long n, const double *x, float *y, cudaStream_t s);
// the same for the first *count (device) of at most cap entries
amg_status to_float_count(const int *count, long long cap, const double *x, float *y, cudaStream_t s);
amg_status to_double(long long n, const float *x, double *y, cudaStream_t s);

}  // namespace cwm
