/*
 * cwm_amg.h -- C ABI of the GB300 (sm_103a) compatible-weighted-matching AMG library.
 *
 * Method: Bernaschi, D'Ambra, Pasquini, "AMG based on compatible weighted matching for
 * GPUs".  The library builds the AMG hierarchy of an s.p.d. sparse matrix A (Sec. 1,
 * system Ax = b) by coarsening based on compatible weighted matching (Sec. 2.2, Sec. 3.1)
 * and applies it as an l1-Jacobi V-cycle (Sec. 2.1 Algorithm 1, Sec. 3.2) inside a
 * flexible CG (Sec. 3.2 Algorithm 3).
 *
 * Conventions for every call:
 *   - Matrices are CSR with int32 row pointers (n+1) and int32 column indices, strictly
 *     ascending within each row, float64 values.  nnz must be < 2^31.
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device; the caller owns
 *     them.  Pointers named h_* or passed as plain structs are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *     work is ordered on it.  A call returns once its work is queued, except where stated
 *     ("synchronises"): then it has waited for `stream`.
 *   - Every call returns an amg_status; none aborts the process.  On error,
 *     amg_last_error() gives a one-line message for the calling thread.
 *   - Numbers and layouts are fixed-width: int32_t indices, int64_t nnz counts, double.
 */
#ifndef CWM_AMG_H
#define CWM_AMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMG_OK = 0,
  AMG_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, malformed or non-symmetric CSR */
  AMG_ERR_NOT_SPD = 2,       /* a diagonal entry is missing or not positive */
  AMG_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  AMG_ERR_OOM = 4,           /* device allocation failed */
  AMG_ERR_TIMEOUT = 5,       /* a bounded device loop hit its iteration cap */
  AMG_ERR_BREAKDOWN = 6,     /* FCG: rho <= 0 or not finite */
  AMG_ERR_NOT_CONVERGED = 7, /* FCG: itmax reached; x and info are still filled */
  AMG_ERR_UNSUPPORTED = 8    /* a size beyond what this build handles (stated per call) */
} amg_status;

/* Parameters of the hierarchy and of the cycle (defaults from Sec. 5 of the paper). */
typedef struct {
  int sweeps_per_level; /* pairwise matching sweeps composed per level: 1, 2, 3 give
                           aggregates of at most 2, 4, 8 (default 2, Sec. 5) */
  int coarse_max;       /* stop coarsening once n <= coarse_max (default 40); -1: the
                           paper's setting floor(40 n^(1/3)) of the input size n (Sec. 5) */
  int max_levels;       /* at most this many levels, finest included (default 40) */
  int pre_sweeps;       /* l1-Jacobi sweeps before the coarse correction (default 1) */
  int post_sweeps;      /* l1-Jacobi sweeps after it (default 1) */
  int coarse_sweeps;    /* l1-Jacobi sweeps from zero on the coarsest level (default 20) */
  int vcycle_fp32;      /* 1: the V-cycle runs on float32 copies of the hierarchy values
                           (FCG recurrences stay float64); 0: all float64 (default 0) */
  int check_input;      /* 1: amg_setup verifies CSR structure and bit symmetry of A on
                           the device before coarsening (default 1).  0: the caller
                           vouches for both; the coarse operators' edge weights and
                           the coarsest level's dense operator (built on its upper
                           triangle) then rely on symmetry (an unchecked non-symmetric
                           input gives an undefined, though terminating, hierarchy) */
  int keep_sweeps;      /* 1: keep every sweep's matching for amg_sweep_mate (default 0) */
  int64_t loop_cap;     /* cap on iterations of any one device retry loop or wait (Suitor
                           proposal chains, grid-barrier polls in the V-cycle); 0 = derived
                           from the sizes (never reached by valid input) */
  int trace;            /* 1: time kernel classes from the start of amg_setup (see
                           amg_trace_*); 0: no tracing (default 0) */
  char trace_filter[32];/* with trace = 1: only classes whose name starts with this
                           NUL-terminated prefix ("" = every class) */
  int tail_rows;        /* levels with at most this many rows (down to the coarsest) run
                           as one cooperative launch per V-cycle; 0 = 65536, -1 = never
                           (default -1: on GB300 the grid barriers cost more than the
                           small launches they replace) */
  double stall_ratio;   /* > 0: stop after a level whose coarsening ratio n_k / n_{k+1}
                           is below this (the paper has no such rule; with strongly
                           heterogeneous coefficients the pairwise matching can grow one
                           aggregate into a hub and coarsen by a few rows per level);
                           0 = off (default) */
  int gamma;            /* coarse cycles per level: 1 = V-cycle (default), 2 = W-cycle
                           (Sec. 5.1; its cost grows as 2^levels) */
  int galerkin_fp32_from; /* k >= 1: the operators of levels k, k+1, ... (and the
                           intermediate operators of their sweeps) come from a binary32
                           Galerkin product: p_i, p_j, a_ij rounded to float, terms and
                           sums in float in the canonical order, stored as doubles (the
                           precision trade-off of Sec. 3.2 carried over to the setup; the
                           finest operator stays the caller's); 0 = off (default) */
  int coupled_post;     /* coarse correction + the post-sweep (post_sweeps = 1) as one pass
                           over the stored product A^k P^k: since b - A(xs + P xc) =
                           (b - A xs) - (A P) xc and the restriction already formed
                           b - A xs, the sweep streams A P (one column per aggregate)
                           instead of A and the separate prolongation pass goes.
                           0 = auto (default: levels with more than 16 entries per row
                           on average that do not take the fused small-level kernels;
                           on short rows building A P costs about what one solve
                           gains); 1 = every level below the coarsest;
                           -1 = off.  Levels with rows longer than 1024 entries never
                           take it. */
  int block3;           /* 0 = auto (default): when every block row of the input operator
                           (rows 3b, 3b+1, 3b+2) stores the same columns in whole aligned
                           triples (3c, 3c+1, 3c+2) -- a nodal 3D vector problem with
                           interleaved unknowns and its assembled pattern -- the finest
                           level's residual in the V-cycle and the FCG's SpMV with its dot
                           products stream a copy of it in 3x3 blocks (one column index
                           per block; the same products summed in block order); -1 = never */
  int sliced;           /* sliced copies (rows sorted by length within windows of 256,
                           one or more lanes per row, the lanes of a warp reading
                           consecutive words) streamed by the V-cycle on the levels that
                           take the coarse correction and post-sweep through A P
                           (coupled_post): 0 = auto (default: A P on such levels with at
                           least 131072 rows and more than 16 entries per row on average,
                           one lane per row), 1 = A and A P on every such level, lanes per
                           row from the longest row, -1 = never */
} amg_params;

/* Statistics filled by amg_pcg_solve and amg_stats. */
typedef struct {
  int iters;             /* FCG iterations (updates of x) */
  double rel_res;        /* recursive ||r||/||b|| at exit */
  double rel_res_true;   /* ||b - A x|| / ||b|| recomputed at exit */
  int nl;                /* number of levels */
  double vcmplx;         /* sum_k nnz(A^k) / nnz(A^1)  (Sec. 5.2) */
  double cratio;         /* (1/nl) sum_{k>=2} n_{k-1}/n_k (Sec. 5.2) */
  double t_setup_ms;     /* wall time of the last amg_setup (synchronised) */
  double t_solve_ms;     /* wall time of the last amg_pcg_solve */
} amg_info;

typedef struct amg_hierarchy *amg_handle; /* opaque; owned by the library */

/* Fills *p with the defaults listed above. */
void amg_default_params(amg_params *p);

/* Builds the hierarchy {A^k, P^k, v^k} of Sec. 2.1 by Sec. 2.2/3.1 coarsening.
 *   n, nnz          size of A (n >= 1, 0 <= nnz < 2^31)
 *   d_row_ptr/col/val  CSR of A.  A must be structurally and numerically
 *                   (bit-for-bit) symmetric with positive diagonal entries.
 *   d_v             smooth vector (n doubles) driving the weights and P.
 *   params          NULL = defaults.
 *   out             receives the handle (NULL on failure).
 * Each of the four input arrays may be device memory or host memory.  Page-locked host
 * memory (cudaHostAlloc, cudaHostRegister, a pinned framework tensor) is read by the
 * library's copy kernel through its device mapping; pageable host memory is copied with
 * cudaMemcpyAsync.  The inputs are copied; the caller may free them on return.  Synchronises.
 * Errors: INVALID_ARG (sizes, NULL, malformed or non-symmetric CSR when check_input),
 * NOT_SPD (diagonal missing or <= 0), OOM, CUDA, TIMEOUT. */
amg_status amg_setup(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                     const double *d_val, const double *d_v, const amg_params *params,
                     void *stream, amg_handle *out);

/* w = B(r): one V-cycle (Algorithm 1) with x^1 = 0.  d_r, d_w: device, n doubles each,
 * must not overlap.  Errors: INVALID_ARG, CUDA. */
amg_status amg_vcycle(amg_handle h, const double *d_r, double *d_w, void *stream);

/* Flexible CG (Algorithm 3) preconditioned by amg_vcycle for A x = b.
 *   d_b     n doubles.   d_x  n doubles: initial guess in, solution out.
 *           Each may be device or host memory (page-locked or pageable, as for
 *           amg_setup); host arrays are solved through device copies that the handle
 *           keeps, and a host x is written back before the call returns (also on
 *           NOT_CONVERGED and BREAKDOWN; on other errors its contents are unspecified).
 *   rtol    stop once ||r||/||b|| <= rtol (recursive residual).   itmax >= 0.
 *   info    may be NULL; else receives iterations, residuals and timings.
 * Synchronises (the host reads ||r|| once per iteration).
 * Errors: INVALID_ARG, BREAKDOWN, NOT_CONVERGED (x and info filled), CUDA. */
amg_status amg_pcg_solve(amg_handle h, const double *d_b, double *d_x, double rtol, int itmax,
                         void *stream, amg_info *info);

/* Releases the hierarchy.  NULL-safe.  Synchronises with the setup stream. */
void amg_free(amg_handle h);

/* Hierarchy statistics (nl, Vcmplx, cratio, t_setup_ms) into *info.  Host only. */
amg_status amg_stats(amg_handle h, amg_info *info);

/* Number of levels (>= 1), or -1 for a NULL handle. */
int amg_num_levels(amg_handle h);

/* Size of level k: n, nnz and the number of sweeps that built level k+1 (0 on the
 * coarsest).  Host only. */
amg_status amg_level_info(amg_handle h, int level, int *n, int64_t *nnz, int *nsweeps);

/* Copies level k out to caller-owned DEVICE buffers (any may be NULL to skip):
 * row_ptr (n+1), col (nnz), val (nnz), v (n), dl1 = l1 row norms (n), and, below the
 * coarsest level, agg (n, the column of P^k in each row) and p (n, its value).
 * Synchronises. */
amg_status amg_level_export(amg_handle h, int level, int32_t *d_row_ptr, int32_t *d_col,
                            double *d_val, double *d_v, double *d_dl1, int32_t *d_agg,
                            double *d_p, void *stream);

/* The matching of sweep s (0-based) of level k, kept when params.keep_sweeps = 1:
 * d_mate receives (*n) int32 partners (-1 = unmatched) and *n the operator size of that
 * sweep.  Pass d_mate = NULL to query *n only.  Synchronises. */
amg_status amg_sweep_mate(amg_handle h, int level, int sweep, int32_t *d_mate, int *n,
                          void *stream);

/* ---- The hot-path steps one at a time (each one sweep of Sec. 2.2 / Sec. 3.1) ---- */

/* Edge weights (Sec. 2.2, C(A, v)): for every stored slot k of row i with column j,
 *   d_w[k] = 1 - 2 a_ab v_a v_b / (a_aa v_a^2 + a_bb v_b^2),  a = min(i,j), b = max(i,j),
 * evaluated without FMA as ((2 a_ab) v_a) v_b over ((a_aa v_a) v_a) + ((a_bb v_b) v_b);
 * 0 on the diagonal, on stored zeros and where the weight is not positive.  A must be
 * symmetric, as for amg_setup (operators of short rows evaluate each edge once and copy
 * it to the mirror slot; long-row operators evaluate every slot from its own value).
 * The quotient is the correctly rounded one, formed on the integer pipes (cwm_div_check).
 * d_w: device, nnz doubles.  Errors: INVALID_ARG, NOT_SPD.  Synchronises. */
amg_status cwm_edge_weights(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                            const double *d_val, const double *d_v, double *d_w, void *stream);

/* Suitor matching (Sec. 3.1) on the graph whose edges are the slots with d_w > 0, under
 * the strict order: heavier first, ties to the larger index (the result is the greedy
 * matching in decreasing (w, max, min) order).  d_w must be symmetric per edge.
 * d_mate: device, n int32 (-1 = unmatched).  Uses 16n bytes of device scratch memory,
 * allocated from the stream-ordered pool.  Errors: INVALID_ARG, TIMEOUT, OOM.
 * Synchronises. */
amg_status cwm_suitor_match(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                            const double *d_w, int32_t *d_mate, void *stream);

/* cwm_suitor_match for callers that cannot allocate device memory -- code running where
 * cudaMalloc is forbidden or would stall (a real-time loop, a host callback, a process
 * whose device memory is owned by another allocator or reserved up front).  The paper has
 * no counterpart: this is an interface variant, not a step of the method.
 * Same arguments, result and errors as cwm_suitor_match, but the 16 bytes of scratch per
 * vertex come from a fixed array inside the library (16 MiB, held by every GPU that loads
 * the library until the process exits), so no call allocates or frees device memory.
 *   - n is limited to 1,048,576 vertices; larger n returns AMG_ERR_UNSUPPORTED.
 *   - Every call looks up the array's address on the current device (no allocation), so
 *     the call stays valid after the host application resets the device.
 *   - Every call uses the same array, so calls whose GPU work overlaps (different streams,
 *     or different threads on one device) race and corrupt each other's result; order
 *     them on one stream.  The scratch contents left by a call are cleared by the next.
 * Synchronises (it reads the device error word back): do not call it while `stream` is
 * being captured into a CUDA graph. */
amg_status cwm_suitor_match_noalloc(int n, int64_t nnz, const int32_t *d_row_ptr,
                                   const int32_t *d_col, const double *d_w, int32_t *d_mate,
                                   void *stream);

/* Pairwise aggregation (Sec. 2.2, Algorithm 2, ids ascending by smallest member) and the
 * prolongator by orthonormal projection of v (Sec. 2.2):
 *   d_agg (n int32): aggregate of each vertex;  d_p (n doubles): the one entry of each
 *   row of P;  d_vc (at least n doubles): v_c = P^T v in its first n_c entries.
 *   h_nc, h_npairs: host ints receiving n_c and the number of pairs.
 * Errors: INVALID_ARG (mate not symmetric is not checked).  Synchronises. */
amg_status cwm_aggregate(int n, const int32_t *d_mate, const double *d_v, int32_t *d_agg,
                         double *d_p, double *d_vc, int *h_nc, int *h_npairs, void *stream);

/* Galerkin product A_c = P^T A P (Sec. 2.1, Sec. 3.1) for a pairwise P (every aggregate
 * has one or two members): entry (I,J) sums (p_i p_j) a_ij from +0.0 in ascending
 * (min(i,j), max(i,j), i) order; every hit (I,J) is stored, columns ascending.
 *   d_rpc (nc+1), d_colc and d_valc (capacity entries each) are device outputs;
 *   capacity >= nnz always suffices.  h_nnzc receives nnz(A_c).
 *   Scratch (stream-ordered pool, freed on return): nnz ints and nnz doubles holding each
 *   coarse row at a padded offset before the compaction into d_colc/d_valc.
 *   fp32 = 1: the binary32 variant (p_i, p_j, a_ij rounded to float, terms and sums in
 *   float in the same order, each entry stored as the double of its float); 0: float64.
 * Errors: INVALID_ARG (an aggregate with more than two members), UNSUPPORTED (a coarse
 * row gathering more than 8192 fine entries), OOM.  Synchronises. */
amg_status cwm_galerkin(int n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                        int nc, const int32_t *d_agg, const double *d_p, int32_t *d_rpc,
                        int32_t *d_colc, double *d_valc, int64_t capacity, int64_t *h_nnzc,
                        int fp32, void *stream);

/* ---- Differentiation of a solve x = A^{-1} b ---- */

/* The sampled outer product on the pattern of A: d_out[k] = alpha * (lambda_i * x_j) for
 * every stored slot k = (i, j).  With lambda = A^{-1} dL/dx (the adjoint solve, A symmetric)
 * and alpha = -1 this is dL/dA_ij of a loss L(x) (Sec. 1: A x = b; the differentiation is an
 * extension of the paper's solver).  d_lambda, d_x: device, n doubles; d_out: device, nnz
 * doubles.  Errors: INVALID_ARG.  Asynchronous on stream. */
amg_status cwm_pattern_outer(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                             const double *d_lambda, const double *d_x, double alpha, double *d_out,
                             void *stream);

/* ---- Tracing: per kernel class, CUDA events recorded on the launching stream ---- */

/* One kernel class ("jacobi@0" = the l1-Jacobi kernel on level 0): launches, summed
 * event-measured milliseconds, and the algorithmic bytes those launches move (each CSR
 * array and vector counted once per launch; gathers counted once). */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
  double bytes;
} amg_trace_entry;

/* Turns tracing on (on = 1) or off for later calls on h.  filter: NULL or "" traces every
 * class; otherwise only classes whose name starts with it.  Host only. */
amg_status amg_trace_enable(amg_handle h, int on, const char *filter);
/* Clears the accumulated entries.  Synchronises. */
amg_status amg_trace_reset(amg_handle h);
/* Number of entries after waiting for every recorded event (-1 for a NULL handle).
 * Synchronises. */
int amg_trace_count(amg_handle h);
/* Entry i (0 <= i < amg_trace_count(h)) into *out.  Host only. */
amg_status amg_trace_get(amg_handle h, int i, amg_trace_entry *out);
/* Kernel launches made by this library in this process so far (all handles, all calls). */
int64_t amg_launch_count(void);

/* Measured FP64 issue rates of the current device (the paper has no counterpart: these are
 * the denominators against which the FP64-bound kernels are reported).  *fma_per_s: fused
 * multiply-adds per second, all SMs, independent chains; *div_per_s: correctly rounded
 * divisions per second, measured the same way.  Host pointers.  Ordered on `stream`; takes
 * a few milliseconds and allocates 8 bytes of device memory.  Errors: INVALID_ARG (NULL
 * output), CUDA.  Synchronises. */
amg_status cwm_fp64_rates(double *fma_per_s, double *div_per_s, void *stream);

/* Copies `bytes` bytes between device memory and device or host memory, the way amg_setup
 * and amg_pcg_solve move host arrays: page-locked host memory by an SM copy kernel through
 * its device mapping (on GB300 the copy engines' host-to-device transfers stalled for tens of
 * milliseconds about every half second; the kernel's did not), pageable host memory by
 * cudaMemcpyAsync (the call then waits for it), device to device by cudaMemcpyAsync.  At
 * least one of dst, src must be device memory (bytes = 0 does nothing and accepts any
 * pointers); the ranges must not overlap.  Ordered on `stream` and asynchronous for
 * page-locked host memory: the caller leaves a host source unchanged, and reads a host
 * destination only, after synchronising with the stream.  Errors: INVALID_ARG (NULL
 * pointer, bytes < 0, no device side), CUDA.  The paper has no counterpart. */
amg_status cwm_copy(void *dst, const void *src, int64_t bytes, void *stream);

/* Self-check of the edge weights' quotient (Sec. 2.2: c = 1 - num / den is evaluated with a
 * correctly rounded division that runs on the integer pipes, not on the FP64 pipe).  For
 * i = 0 .. n-1 the device derives an operand pair (x_i, y_i) from (seed, i) by splitmix64 --
 * raw bit patterns (zeros, subnormals, infinities, NaNs), nearby exponents, quotients next
 * to rounding boundaries (x = RN(y q)), powers of two, equal and extreme significands, and
 * exponents at the edges of the normal range -- and compares the bits of that quotient with
 * the hardware's IEEE division.  *mismatches: pairs whose bits differ (0 expected);
 * *first: the smallest such i, or -1.  Host pointers.  Ordered on `stream`; allocates 16
 * bytes of device memory.  Errors: INVALID_ARG (NULL output, n < 0), CUDA.  Synchronises.
 * The paper has no counterpart. */
amg_status cwm_div_check(long long n, unsigned long long seed, long long *mismatches, long long *first,
                         void *stream);

/* Human-readable name of a status, and the last error message of the calling thread. */
const char *amg_status_string(amg_status s);
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CWM_AMG_H */
