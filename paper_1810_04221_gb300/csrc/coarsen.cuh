// coarsen.cuh -- host launchers of the coarsening kernels (coarsen.cu, galerkin.cu).
#pragma once

#include "common.cuh"

namespace cwm {

constexpr int kMaxSweeps = 8;

// Per-sweep aggregate maps and prolongator values, passed by value to k_compose.
struct SweepMaps {
  const int *agg[kMaxSweeps];
  const double *p[kMaxSweeps];
  int count;
};

amg_status check_input(int n, long long nnz, const int *rp, const int *ci, const double *val,
                       bool check_sym, int *d_err, cudaStream_t s);
amg_status extract_diag(int n, const int *rp, const int *ci, const double *val, double *diag,
                        int *d_err, cudaStream_t s);
// dv_scratch: n doubles (per-vertex (a_ii v_i) v_i)
amg_status edge_weights(int n, long long nnz, const int *rp, const int *ci, const double *val,
                        const double *diag, const double *v, double *w, double *dv_scratch, cudaStream_t s,
                        bool clear = true);
// Suitor matching (Sec. 3.1) into mate[n].  scratch: suitor_scratch_bytes(n) bytes (16 per
// vertex, the packed suitor keys), which suitor_match clears itself before the proposals
// start, so it may hold anything on entry; d_err: the device error word (not cleared here).
size_t suitor_scratch_bytes(int n);
amg_status suitor_match(int n, long long nnz, const int *rp, const int *ci, const double *w,
                        void *scratch, int *mate, long long cap, int *d_err, cudaStream_t s);
// d_counts[0] <- n_c, d_counts[1] <- number of pairs.  id_scratch: n+1 ints.
amg_status aggregate(int n, const int *mate, const double *v, int *agg, double *p, double *vc,
                     int *m1, int *m2, int *id_scratch, int *scan_scratch, int *d_counts,
                     cudaStream_t s);
amg_status compose(int n, const SweepMaps &maps, int *agg_out, double *p_out, cudaStream_t s);
// cnt_scratch: nc+1 ints.
amg_status member_lists(int n, int nc, const int *agg, int *mptr, int *mlist, int *cnt_scratch,
                        int *scan_scratch, cudaStream_t s);

// Galerkin product for a pairwise P (galerkin.cu).
struct GalerkinWork {
  int *cnt = nullptr;         // nc + 1 ints: padded lengths, then distinct-column counts
  int *rpu = nullptr;         // nc + 1 ints: padded row starts
  int *long_rows = nullptr;   // nc ints: coarse rows too long for the warp kernel
  int *n_long = nullptr;      // 1 int
  int *scan = nullptr;        // scan scratch
  int *ci_pad = nullptr;      // nnz_fine ints: padded columns
  double *val_pad = nullptr;  // nnz_fine doubles: padded values
  int n_fine = 0;             // fine size and nnz
  long long nnz_fine = 0;
};
// Groups the entries of every coarse row into the padded arrays and writes the row
// pointers of A_c to rpc (rpc[nc] = nnz(A_c) on the device); diag_c (nc) and dl1_c (nc)
// may be NULL.  fp32: terms and sums in binary32 (values stored as doubles of floats).
amg_status galerkin_group(const int *rp, const int *ci, const double *val, int nc, const int *m1,
                          const int *m2, const int *agg, const double *p, int *rpc, double *diag_c,
                          double *dl1_c, const GalerkinWork &work, bool fp32, int *d_err, cudaStream_t s);
// Copies the padded rows to cic/valc at rpc (capacity rpc[nc]).
amg_status galerkin_compact(int nc, const int *rpc, int *cic, double *valc, const GalerkinWork &work,
                            cudaStream_t s);
// m1/m2 from agg when the caller only has agg (cwm_galerkin): members in ascending order;
// an empty aggregate or one with more than two members raises kErrInvalid.  cnt: nc ints.
amg_status members_from_agg(int n, int nc, const int *agg, int *m1, int *m2, int *cnt, int *d_err,
                            cudaStream_t s);

}  // namespace cwm
