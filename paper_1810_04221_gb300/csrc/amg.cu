// amg.cu -- the hierarchy driver (Sec. 2.1 setup, Sec. 5 parameters), the V-cycle
// (Sec. 2.1, Algorithm 1), the flexible CG (Sec. 3.2, Algorithm 3) and the C ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "coarsen.cuh"
#include "solve.cuh"
#include "trace.cuh"

namespace cwm {
const char *last_error();
}

using namespace cwm;

namespace {

// A sliced copy of a level operator or of its A P (sell.cu), in the V-cycle's precision.
struct SellBuf {
  int n = 0, lanes = 1;
  long long nnz = 0, slots = 0;
  DBuf<int> sptr, perm, len, col;
  DBuf<double> v64;
  DBuf<float> v32;
  template <class V>
  SellView<V> view(const V *values) const {
    SellView<V> a;
    if (!values) return a;
    a.n = n; a.lanes = lanes; a.nnz = nnz; a.sptr = sptr.get(); a.perm = perm.get(); a.len = len.get();
    a.col = col.get();
    a.val = values;
    return a;
  }
};

struct Level {
  int n = 0;
  long long nnz = 0;
  int max_row = 0;  // longest row (selects the solve kernels: row_kernel_shape)
  DBuf<int> rp, ci;
  DBuf<double> val, v, diag, dl1, dinv;
  DBuf<float> val32, dinv32;
  // transfer to level k+1 (empty on the coarsest level)
  DBuf<int> agg, mptr, mlist;
  DBuf<double> p;
  DBuf<float> p32;
  int nsweeps = 0;
  std::vector<int> sweep_n;
  std::vector<DBuf<int>> sweep_mate;
  // V-cycle work vectors
  DBuf<double> b, x, t1, t2;
  DBuf<float> b32, x32, t132, t232;
  // coarsest level only: the dense operator of the coarse sweeps (n <= kDenseCoarseMax)
  DBuf<double> xdense;
  DBuf<float> xdense32;

  // rows longer than long_min, taken by a whole warp in the l1-Jacobi sweep (n_long = 0: none)
  DBuf<int> long_rows;
  int n_long = 0, long_min = 0;
  // A P (n rows, one column per aggregate of the next level; empty: not built), for the
  // coarse correction + post-sweep of cycle_level
  DBuf<int> ap_rp, ap_ci;
  DBuf<double> ap_val;
  DBuf<float> ap_val32;
  long long ap_nnz = 0;
  int ap_max_row = 0;
  // the finest operator in 3x3 blocks (block3.cu), when its pattern is 3x3-blocked
  DBuf<int> b3_sptr, b3_blen, b3_bci;
  DBuf<double> b3_val;
  DBuf<float> b3_val32;
  long long b3_slots = 0;
  // sliced copies of A and of A P (levels with A P and long rows; see build_sell)
  SellBuf sa, sap;

  template <class V>
  void split(CsrView<V> &a, bool fp64) const {
    a.max_row = max_row;
    if (a.rb || n_long <= 0) return;
    bool rb_unused = false;
    a.long_rows = long_rows.get();
    a.n_long = n_long;
    a.long_min = long_min;
    row_kernel_shape(n, nnz, long_min, fp64, &rb_unused, &a.tile_short);
  }
  CsrView<double> view64() const {
    CsrView<double> a;
    a.n = n; a.nnz = nnz; a.rp = rp.get(); a.ci = ci.get(); a.val = val.get();
    row_kernel_shape(n, nnz, max_row, true, &a.rb, &a.tile);
    split(a, true);
    return a;
  }
  CsrView<float> view32() const {
    CsrView<float> a;
    a.n = n; a.nnz = nnz; a.rp = rp.get(); a.ci = ci.get(); a.val = val32.get();
    row_kernel_shape(n, nnz, max_row, false, &a.rb, &a.tile);
    split(a, false);
    return a;
  }
  template <class V>
  Sell3View<V> block3_view(const V *values) const {
    Sell3View<V> a;
    if (!values) return a;  // nbr = 0: no block layout
    a.n = n;
    a.nbr = n / 3;
    a.nblocks = nnz / 9;
    a.slots = b3_slots;
    a.sptr = b3_sptr.get();
    a.blen = b3_blen.get();
    a.bci = b3_bci.get();
    a.val = values;
    return a;
  }
  template <class V>
  CsrView<V> ap_view(const V *values) const {
    CsrView<V> a;
    a.n = n; a.nnz = ap_nnz; a.rp = ap_rp.get(); a.ci = ap_ci.get(); a.val = values;
    a.max_row = ap_max_row;
    row_kernel_shape(n, ap_nnz, ap_max_row, sizeof(V) == 8, &a.rb, &a.tile);
    return a;
  }
};

// One matching sweep's products (owned until moved into a level).
struct SweepOut {
  int n = 0;
  long long nnz = 0;
  int max_row = 0;
  DBuf<int> rp, ci, agg;
  DBuf<double> val, diag, dl1, v, p;
};

// Pinned host mailbox for the few device -> host reads.
struct Mailbox {
  int *ints = nullptr;        // 16
  double *dbls = nullptr;     // 16
  amg_status init() {
    if (!ints) CWM_CUDA(cudaMallocHost((void **)&ints, 16 * sizeof(int)));
    if (!dbls) CWM_CUDA(cudaMallocHost((void **)&dbls, 16 * sizeof(double)));
    return AMG_OK;
  }
  ~Mailbox() {
    if (ints) cudaFreeHost(ints);
    if (dbls) cudaFreeHost(dbls);
  }
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct amg_hierarchy {
  amg_params prm{};
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<Level> lev;
  DBuf<int> err;
  Mailbox box;
  // FCG vectors and reductions
  DBuf<double> r, w, d, vv, q, part, part2, scal;
  DBuf<double> bdev, xdev;  // device copies of a solve's host b and x (amg_pcg_solve)
  DBuf<int> ap_stat;         // per level: nnz(A P) and its longest row, written by build_ap_level
  DBuf<unsigned> tick;  // last-block tickets of the fused reductions (kept at zero between launches)
  double t_setup_ms = 0.0, t_solve_ms = 0.0;
  Tracer trace;
  // the FCG iteration replayed as CUDA graphs on a library-owned stream
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // [0]: iterations >= 1, [1]: the first
  std::vector<Tracer::Pending> gscopes[2];        // tracer scopes recorded inside each graph
  long long gkernels[2] = {0, 0};                 // kernels in each graph (launch accounting)
  double *graph_x = nullptr;                      // the solution pointer the graphs use
  bool graphs_failed = false;
  // the fused coarse end of the V-cycle
  int tail_start = -1;  // first level run by vcycle_tail, -1: none
  TailArgs<double> tail64{};
  TailArgs<float> tail32{};
  DBuf<unsigned> bar;   // grid-barrier state (count, generation)
  DBuf<unsigned char> tail_dev;  // device copies of tail64 and tail32
  // float32 cycle: where the finest level's last kernel also writes its result in binary64
  // (set by apply_vcycle; cycle_level reports in out64_written whether it did)
  double *out64 = nullptr;
  bool out64_written = false;
  void drop_graphs() {
    for (int g = 0; g < 2; ++g) {
      if (gexec[g]) cudaGraphExecDestroy(gexec[g]);
      gexec[g] = nullptr;
      trace.release(gscopes[g]);
    }
    graph_x = nullptr;
  }
  ~amg_hierarchy() {
    drop_graphs();
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (solve_stream) cudaStreamDestroy(solve_stream);
  }
};

namespace {

// Installs h's tracer for the calling thread for the lifetime of the guard.
struct TraceGuard {
  Tracer *prev;
  int prev_level;
  explicit TraceGuard(amg_hierarchy *h) : prev(g_tracer), prev_level(g_trace_level) {
    g_tracer = h->trace.on ? &h->trace : nullptr;
    g_trace_level = -1;
  }
  ~TraceGuard() {
    g_tracer = prev;
    g_trace_level = prev_level;
  }
};

struct LevelTag {
  int prev;
  explicit LevelTag(int k) : prev(g_trace_level) { g_trace_level = k; }
  ~LevelTag() { g_trace_level = prev; }
};

// Tags the setup classes of a level's later matching sweeps (s >= 1) as @k.s, so that the
// @k classes time the first sweep, the one on the level operator itself.
struct SweepTag {
  int prev;
  explicit SweepTag(int s) : prev(g_trace_sweep) { g_trace_sweep = s; }
  ~SweepTag() { g_trace_sweep = prev; }
};

amg_status read_err(amg_hierarchy *h, const char *where) {
  CWM_CUDA(cudaMemcpyAsync(h->box.ints + 8, h->err.get(), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CWM_CUDA(cudaStreamSynchronize(h->stream));
  int bits = h->box.ints[8];
  if (bits) {
    CWM_CUDA(cudaMemsetAsync(h->err.get(), 0, sizeof(int), h->stream));
    return status_from_device_bits(bits, where);
  }
  return AMG_OK;
}

// A device error raised inside the solve (a bounded wait that gave up): report it and reset
// the error word and the grid-barrier state for later calls.
amg_status solve_device_error(amg_hierarchy *h, const char *where) {
  const int bits = h->box.ints[8];
  if (!bits) return AMG_OK;
  cudaMemsetAsync(h->err.get(), 0, sizeof(int), h->stream);
  if (h->bar.get()) cudaMemsetAsync(h->bar.get(), 0, 2 * sizeof(unsigned), h->stream);
  cudaStreamSynchronize(h->stream);
  h->box.ints[8] = 0;
  return status_from_device_bits(bits, where);
}

long long default_cap(const amg_params &prm, long long n, long long nnz) {
  return prm.loop_cap > 0 ? prm.loop_cap : nnz + n + 1024;
}

// Builds level k+1 from level k by up to S sweeps; *made = false when no pair formed.
amg_status coarsen_level(amg_hierarchy *h, bool *made) {
  cudaStream_t s = h->stream;
  Level &F = h->lev.back();
  const int S = h->prm.sweeps_per_level;
  // the level being built is lev.size(); its operators use the binary32 product from
  // level galerkin_fp32_from on
  const bool fp32_galerkin =
      h->prm.galerkin_fp32_from > 0 && (int)h->lev.size() >= h->prm.galerkin_fp32_from;
  *made = false;
  LevelTag tag((int)h->lev.size() - 1);

  // scratch sized for the largest (first) sweep
  const int nf = F.n;
  const long long nnzf = F.nnz;
  DBuf<double> w, dv;
  DBuf<unsigned char> skeys;
  DBuf<int> mate, m1, m2, ids, scan, cnt, longr, misc, cpad;
  CWM_TRY(w.alloc(nnzf, s));
  CWM_TRY(cpad.alloc(nnzf, s));
  CWM_TRY(dv.alloc(nf, s));
  CWM_TRY(skeys.alloc(suitor_scratch_bytes(nf), s));
  CWM_TRY(mate.alloc(nf, s));
  CWM_TRY(m1.alloc(nf, s));
  CWM_TRY(m2.alloc(nf, s));
  CWM_TRY(ids.alloc((size_t)nf + 1, s));
  CWM_TRY(scan.alloc(scan_scratch_ints(nf), s));
  CWM_TRY(cnt.alloc((size_t)nf + 1, s));
  CWM_TRY(longr.alloc(nf, s));
  CWM_TRY(misc.alloc(4, s));

  std::vector<SweepOut> sw;
  sw.reserve(S);
  // the operator matched by the current sweep
  int cn = F.n;
  long long cnnz = F.nnz;
  const int *crp = F.rp.get(), *cci = F.ci.get();
  const double *cval = F.val.get(), *cdiag = F.diag.get(), *cv = F.v.get();
  F.sweep_n.clear();
  F.sweep_mate.clear();

  for (int sweep = 0; sweep < S; ++sweep) {
    SweepTag stag(sweep);
    // every operator after the input is symmetric by construction (P^T A P of a symmetric
    // A), so only the input's weights need the cleared array
    CWM_TRY(edge_weights(cn, cnnz, crp, cci, cval, cdiag, cv, w.get(), dv.get(), s,
                         h->lev.size() == 1 && sweep == 0));
    CWM_TRY(suitor_match(cn, cnnz, crp, cci, w.get(), skeys.get(), mate.get(),
                         default_cap(h->prm, cn, cnnz), h->err.get(), s));
    SweepOut o;
    CWM_TRY(o.agg.alloc(cn, s));
    CWM_TRY(o.p.alloc(cn, s));
    CWM_TRY(o.v.alloc(cn, s));
    CWM_TRY(aggregate(cn, mate.get(), cv, o.agg.get(), o.p.get(), o.v.get(), m1.get(), m2.get(), ids.get(),
                      scan.get(), misc.get(), s));
    CWM_CUDA(cudaMemcpyAsync(h->box.ints, misc.get(), 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CWM_TRY(read_err(h, "amg_setup (matching)"));  // synchronises
    const int nc = h->box.ints[0], npairs = h->box.ints[1];
    if (h->prm.keep_sweeps) {
      DBuf<int> keep;
      CWM_TRY(keep.alloc(cn, s));
      CWM_CUDA(cudaMemcpyAsync(keep.get(), mate.get(), sizeof(int) * (size_t)cn, cudaMemcpyDeviceToDevice, s));
      F.sweep_mate.push_back(std::move(keep));
      F.sweep_n.push_back(cn);
    }
    if (npairs == 0) break;
    // Galerkin product into arrays of capacity cnnz (nnz(A_c) <= nnz(A) always)
    o.n = nc;
    CWM_TRY(o.rp.alloc((size_t)nc + 1, s));
    CWM_TRY(o.ci.alloc(cnnz, s));
    CWM_TRY(o.val.alloc(cnnz, s));
    CWM_TRY(o.diag.alloc(nc, s));
    GalerkinWork gw;
    gw.cnt = cnt.get();
    gw.rpu = ids.get();  // the aggregation's scan output is free again
    gw.long_rows = longr.get();
    gw.n_long = misc.get() + 2;
    gw.scan = scan.get();
    gw.ci_pad = cpad.get();
    gw.val_pad = w.get();  // this sweep's weights are no longer needed
    gw.n_fine = cn;
    gw.nnz_fine = cnnz;
    CWM_TRY(galerkin_group(crp, cci, cval, nc, m1.get(), m2.get(), o.agg.get(), o.p.get(), o.rp.get(),
                           o.diag.get(), nullptr, gw, fp32_galerkin, h->err.get(), s));
    CWM_TRY(galerkin_compact(nc, o.rp.get(), o.ci.get(), o.val.get(), gw, s));
    CWM_TRY(max_row_length(nc, o.rp.get(), misc.get() + 3, s));
    CWM_CUDA(cudaMemcpyAsync(h->box.ints + 4, o.rp.get() + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
    CWM_CUDA(cudaMemcpyAsync(h->box.ints + 5, misc.get() + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CWM_TRY(read_err(h, "amg_setup (Galerkin)"));
    o.nnz = h->box.ints[4];
    o.max_row = h->box.ints[5];
    sw.push_back(std::move(o));
    SweepOut &last = sw.back();
    cn = last.n;
    cnnz = last.nnz;
    crp = last.rp.get();
    cci = last.ci.get();
    cval = last.val.get();
    cdiag = last.diag.get();
    cv = last.v.get();
  }
  F.nsweeps = (int)sw.size();
  if (sw.empty()) return AMG_OK;

  // composed prolongator of level k, and its transpose as member lists
  SweepMaps maps{};
  maps.count = (int)sw.size();
  for (int i = 0; i < maps.count; ++i) {
    maps.agg[i] = sw[i].agg.get();
    maps.p[i] = sw[i].p.get();
  }
  const int nc = sw.back().n;
  CWM_TRY(F.agg.alloc(F.n, s));
  CWM_TRY(F.p.alloc(F.n, s));
  CWM_TRY(compose(F.n, maps, F.agg.get(), F.p.get(), s));
  CWM_TRY(F.mptr.alloc((size_t)nc + 1, s));
  CWM_TRY(F.mlist.alloc(F.n, s));
  CWM_TRY(member_lists(F.n, nc, F.agg.get(), F.mptr.get(), F.mlist.get(), cnt.get(), scan.get(), s));

  // the new level takes the last sweep's operator
  SweepOut &last = sw.back();
  Level C;
  C.n = last.n;
  C.nnz = last.nnz;
  C.max_row = last.max_row;
  C.rp = std::move(last.rp);
  C.ci = std::move(last.ci);
  C.val = std::move(last.val);
  C.v = std::move(last.v);
  C.diag = std::move(last.diag);
  CWM_TRY(C.dl1.alloc(C.n, s));
  CWM_TRY(l1_norms(C.view64(), C.dl1.get(), s));
  h->lev.push_back(std::move(C));
  *made = (int)sw.size() == S;  // a sweep without pairs ends the hierarchy after this level
  return AMG_OK;
}

// Largest level whose cycle uses the fused kernels (see cycle_level), per precision.  The
// fused forms rebuild x_j per nonzero (D^{-1} b, and D^{-1} b + P x_c), two or three FP64
// operations per nonzero instead of one; where GB300's FP64 pipe binds, that costs more
// than the passes saved.  3D Poisson 128^3, FP64 V-cycle: limits of 300000 / 65536 / 0 rows
// gave 11.61 / 11.41 / 11.62 ms per solve (level 1 has 262,144 rows).
#ifndef CWM_FUSE_MAX_ROWS64
#define CWM_FUSE_MAX_ROWS64 65536
#endif
template <class V>
constexpr int fuse_max_rows() { return sizeof(V) == 8 ? CWM_FUSE_MAX_ROWS64 : 300000; }

// Longest row of A for which A P is built (its grouping searches the row's list of
// aggregates once per chunk of 32 entries).
constexpr int kApMaxRow = 1024;

// In auto mode A P is built for levels whose mean row is longer than this.  Measured on
// GB300 (setup + one solve): Q1 elasticity 64^3 (64 entries per row, A P a little over half
// of them) 71.4 -> 68.8 ms; on the 7-entry rows of 3D Poisson 128^3 and the lognormal 160^3
// levels the solve gained what building A P cost (FP64 17.98 -> 18.01 ms, FP32 16.18 ->
// 16.24 ms, lognormal 44.9 -> 45.5 ms), so short-row levels keep the separate passes.
constexpr double kApAutoMinMean = 16.0;

// Whether level L gets A P (built by build_ap_level).
bool wants_ap(const amg_hierarchy *h, const Level &L) {
  const amg_params &P = h->prm;
  if (!L.agg.get() || P.coupled_post < 0 || P.post_sweeps != 1 || L.max_row > kApMaxRow || L.nnz == 0) return false;
  if (P.coupled_post == 1) return true;
  // auto: long-row levels that do not take the fused small-level kernels
  if ((double)L.nnz <= kApAutoMinMean * L.n) return false;
  const bool f32 = P.vcycle_fp32 != 0;
  bool rb = true;
  int t = 0;
  row_kernel_shape(L.n, L.nnz, L.max_row, !f32, &rb, &t);
  const int lim = f32 ? fuse_max_rows<float>() : fuse_max_rows<double>();
  return !(P.pre_sweeps == 1 && rb && L.n <= lim);
}

// Builds A P for the levels that take the coarse correction and their post-sweep through it
// (cycle_level): with y = xs + P xc, b - A y = (b - A xs) - (A P) xc, and the residual
// b - A xs is the one the restriction already formed, so the sweep streams A P (one entry per
// aggregate met in a row) instead of A, and the separate prolongation pass goes.  A level's
// A P is built on the library's second stream as soon as the level's prolongator is known,
// while the setup stream coarsens the next level: its rows are grouped at padded offsets,
// scanned and compacted into arrays allocated at nnz(A) (an upper bound), so no host
// synchronisation is needed; its sizes are read once, after the coarsening (ap_sizes).
amg_status build_ap_level(amg_hierarchy *h, int k, cudaStream_t side) {
  Level &L = h->lev[k];
  LevelTag tag(k);
  DBuf<int> ci_pad, cnt, scan;
  DBuf<double> val_pad;
  int *stat = h->ap_stat.get() + 2 * k;
  CWM_TRY(ci_pad.alloc(L.nnz, side));
  CWM_TRY(val_pad.alloc(L.nnz, side));
  CWM_TRY(cnt.alloc((size_t)L.n + 1, side));
  CWM_TRY(scan.alloc(scan_scratch_ints(L.n), side));
  CWM_TRY(L.ap_rp.alloc((size_t)L.n + 1, side));
  CWM_CUDA(cudaMemsetAsync(stat, 0, 2 * sizeof(int), side));
  CWM_TRY(ap_group(L.n, L.nnz, L.rp.get(), L.ci.get(), L.val.get(), L.agg.get(), L.p.get(), L.max_row, ci_pad.get(),
                   val_pad.get(), cnt.get(), stat + 1, side));
  CWM_TRY(exclusive_scan(cnt.get(), L.ap_rp.get(), L.n, scan.get(), side));
  CWM_CUDA(cudaMemcpyAsync(stat, L.ap_rp.get() + L.n, sizeof(int), cudaMemcpyDeviceToDevice, side));
  // A P has at most as many entries as A: allocated at that bound, no synchronisation
  CWM_TRY(L.ap_ci.alloc(L.nnz, side));
  CWM_TRY(L.ap_val.alloc(L.nnz, side));
  GalerkinWork gw;
  gw.rpu = L.rp.get();
  gw.ci_pad = ci_pad.get();
  gw.val_pad = val_pad.get();
  CWM_TRY(galerkin_compact(L.n, L.ap_rp.get(), L.ap_ci.get(), L.ap_val.get(), gw, side));
  if (h->prm.vcycle_fp32) {
    CWM_TRY(L.ap_val32.alloc(L.nnz, side));
    CWM_TRY(to_float_count(stat, L.nnz, L.ap_val.get(), L.ap_val32.get(), side));
  }
  return AMG_OK;  // the scratch buffers are released in order on `side`
}

// After the side stream has been joined: the sizes of every A P built.
amg_status ap_sizes(amg_hierarchy *h) {
  const int nl = (int)h->lev.size();
  std::vector<int> hs(2 * (size_t)nl);
  CWM_CUDA(cudaMemcpyAsync(hs.data(), h->ap_stat.get(), 2 * sizeof(int) * (size_t)nl, cudaMemcpyDeviceToHost,
                           h->stream));
  CWM_TRY(read_err(h, "amg_setup (A P)"));  // synchronises
  for (int k = 0; k < nl; ++k) {
    Level &L = h->lev[k];
    if (!L.ap_rp.get()) continue;
    L.ap_nnz = hs[2 * k];
    L.ap_max_row = hs[2 * k + 1];
  }
  return AMG_OK;
}

// The finest operator in 3x3 blocks (block3.cu), when its pattern qualifies and block3 >= 0:
// one synchronisation reads the detection flag and the per-slice lengths; the slice offsets
// are scanned on the host.
amg_status build_block3(amg_hierarchy *h) {
  Level &L = h->lev[0];
  if (h->prm.block3 < 0 || L.n < 3 || L.n % 3 != 0 || L.nnz % 9 != 0) return AMG_OK;
  cudaStream_t s = h->stream;
  LevelTag tag(0);
  const int nbr = L.n / 3, nsl = (nbr + 31) / 32;
  DBuf<int> smax;
  CWM_TRY(smax.alloc(nsl, s));
  CWM_CUDA(cudaMemsetAsync(smax.get(), 0, sizeof(int) * (size_t)nsl, s));
  int *flag = h->err.get() + 1;  // scratch word next to the error bits
  CWM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  CWM_TRY(block3_detect(L.n, L.rp.get(), L.ci.get(), flag, smax.get(), s));
  std::vector<int> hs((size_t)nsl + 1, 0);
  CWM_CUDA(cudaMemcpyAsync(h->box.ints + 6, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaMemcpyAsync(hs.data(), smax.get(), sizeof(int) * (size_t)nsl, cudaMemcpyDeviceToHost, s));
  CWM_TRY(read_err(h, "amg_setup (3x3 blocks)"));  // synchronises
  if (h->box.ints[6] != 0) return AMG_OK;          // not 3x3-blocked: the CSR kernels serve
  long long slots = 0;
  for (int q = 0; q < nsl; ++q) {
    const long long len = hs[q];
    hs[q] = (int)slots;
    slots += 32 * len;
    if (slots >= (long long)INT32_MAX) return AMG_OK;  // slot offsets are int32
  }
  hs[nsl] = (int)slots;
  CWM_TRY(L.b3_sptr.alloc((size_t)nsl + 1, s));
  CWM_CUDA(cudaMemcpyAsync(L.b3_sptr.get(), hs.data(), sizeof(int) * ((size_t)nsl + 1), cudaMemcpyHostToDevice, s));
  CWM_TRY(L.b3_blen.alloc(nbr, s));
  CWM_TRY(L.b3_bci.alloc((size_t)slots, s));
  CWM_TRY(L.b3_val.alloc(9 * (size_t)slots, s));
  if (h->prm.vcycle_fp32) CWM_TRY(L.b3_val32.alloc(9 * (size_t)slots, s));
  L.b3_slots = slots;
  CWM_TRY(block3_fill(L.n, L.rp.get(), L.ci.get(), L.val.get(), L.b3_sptr.get(), L.b3_blen.get(), L.b3_bci.get(),
                      L.b3_val.get(), L.b3_val32.get(), slots, s));
  CWM_CUDA(cudaStreamSynchronize(s));  // hs is released on return
  return AMG_OK;
}

// Sliced copies (sell.cu) for the levels that take the coarse correction and post-sweep
// through A P, in the V-cycle's precision.  sliced = 1: A and A P of every such level (A not
// where the finest operator has its 3x3-block layout), lanes per row from the longest row.
// sliced = 0 (auto): A P only, on such levels with at least kSellAutoMinRows rows and a mean
// row longer than kApAutoMinMean, one lane per row.  Measured on Q1 elasticity 64^3
// (binary32): the sliced A P took the coarse correction + post-sweep of level 0 (774K rows)
// from 78.5 to 57 us and of level 1 (194K rows) from 47 to 29 us; the sliced residuals were
// no faster than the CSR row blocks on level 1 (44-45 against 47 us) and slower on the
// smaller levels, where a few long rows per warp leave the kernel latency-bound (level 2:
// 25 against 18 us; levels 3-4: 14-18 against 8-10 us), and several lanes per row cost
// level 0's A P 8 us.  Every matrix is planned first (sorted windows, slice lengths and
// their scan), then one synchronisation reads the slot counts, then the copies are filled.
constexpr int kSellAutoMinRows = 131072;
amg_status build_sell(amg_hierarchy *h) {
  const amg_params &P = h->prm;
  if (P.sliced < 0) return AMG_OK;
  cudaStream_t s = h->stream;
  const bool f32 = P.vcycle_fp32 != 0;
  struct Job {
    int k;
    bool is_ap;
  };
  std::vector<Job> jobs;
  for (int k = 0; k + 1 < (int)h->lev.size(); ++k) {
    Level &L = h->lev[k];
    if (L.ap_nnz <= 0 || !L.ap_val.get()) continue;
    if (P.sliced == 0 && ((double)L.nnz <= kApAutoMinMean * L.n || L.n < kSellAutoMinRows)) continue;
    // slot offsets are int32: skip a matrix whose padded layout could exceed them (at most
    // 32 slots per row and step)
    const long long n32 = ((long long)L.n + 31) / 32 * 32;
    if (P.sliced == 1 && !(k == 0 && L.b3_val.get()) && n32 * (L.max_row + 32) < (long long)INT32_MAX)
      jobs.push_back({k, false});
    if (n32 * (L.ap_max_row + 32) < (long long)INT32_MAX) jobs.push_back({k, true});
  }
  if (jobs.empty()) return AMG_OK;
  int nmax = 0;
  for (const Job &j : jobs) nmax = std::max(nmax, h->lev[j.k].n);
  DBuf<int> slen, scan, totals;
  CWM_TRY(slen.alloc((size_t)nmax + 1, s));
  CWM_TRY(scan.alloc(scan_scratch_ints((long long)nmax + 1), s));
  CWM_TRY(totals.alloc(jobs.size(), s));
  for (size_t q = 0; q < jobs.size(); ++q) {
    Level &L = h->lev[jobs[q].k];
    LevelTag tag(jobs[q].k);
    SellBuf &S = jobs[q].is_ap ? L.sap : L.sa;
    const int *rp = jobs[q].is_ap ? L.ap_rp.get() : L.rp.get();
    S.lanes = P.sliced == 1 ? sell_lanes(jobs[q].is_ap ? L.ap_max_row : L.max_row) : 1;
    const int ns = sell_slices(L.n, S.lanes);
    CWM_TRY(S.perm.alloc(L.n, s));
    CWM_TRY(S.len.alloc(L.n, s));
    CWM_TRY(S.sptr.alloc((size_t)ns + 1, s));
    CWM_TRY(sell_plan(L.n, S.lanes, rp, S.perm.get(), S.len.get(), slen.get(), S.sptr.get(), scan.get(), s));
    CWM_CUDA(cudaMemcpyAsync(totals.get() + q, S.sptr.get() + ns, sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  std::vector<int> tot(jobs.size());
  CWM_CUDA(cudaMemcpyAsync(tot.data(), totals.get(), sizeof(int) * jobs.size(), cudaMemcpyDeviceToHost, s));
  CWM_TRY(read_err(h, "amg_setup (sliced copies)"));  // synchronises
  for (size_t q = 0; q < jobs.size(); ++q) {
    Level &L = h->lev[jobs[q].k];
    LevelTag tag(jobs[q].k);
    SellBuf &S = jobs[q].is_ap ? L.sap : L.sa;
    S.n = L.n;
    S.nnz = jobs[q].is_ap ? L.ap_nnz : L.nnz;
    S.slots = tot[q];
    const int *rp = jobs[q].is_ap ? L.ap_rp.get() : L.rp.get();
    const int *ci = jobs[q].is_ap ? L.ap_ci.get() : L.ci.get();
    const double *val = jobs[q].is_ap ? L.ap_val.get() : L.val.get();
    CWM_TRY(S.col.alloc((size_t)S.slots, s));
    if (f32) {
      CWM_TRY(S.v32.alloc((size_t)S.slots, s));
      CWM_TRY(sell_fill<float>(L.n, rp, ci, val, S.view<float>(S.v32.get()), S.col.get(), S.v32.get(), s));
    } else {
      CWM_TRY(S.v64.alloc((size_t)S.slots, s));
      CWM_TRY(sell_fill<double>(L.n, rp, ci, val, S.view<double>(S.v64.get()), S.col.get(), S.v64.get(), s));
    }
  }
  return AMG_OK;
}

amg_status finish_level(amg_hierarchy *h, Level &L) {
  cudaStream_t s = h->stream;
  {  // the long rows of a sub-warp-tile level (see long_row_min)
    bool rb64 = true, rb32 = true;
    int t = 0;
    row_kernel_shape(L.n, L.nnz, L.max_row, true, &rb64, &t);
    row_kernel_shape(L.n, L.nnz, L.max_row, false, &rb32, &t);
    const int lim = long_row_min(L.n, L.nnz, L.max_row, rb64, rb32);
    if (lim > 0) {
      int *cnt = h->err.get() + 1;  // scratch word next to the error bits
      CWM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
      CWM_TRY(long_row_list(L.n, L.rp.get(), lim, nullptr, cnt, s));
      CWM_CUDA(cudaMemcpyAsync(h->box.ints + 6, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
      CWM_TRY(read_err(h, "amg_setup (long rows)"));
      const int nlong = h->box.ints[6];
      if (nlong > 0) {
        CWM_TRY(L.long_rows.alloc(nlong, s));
        CWM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        CWM_TRY(long_row_list(L.n, L.rp.get(), lim, L.long_rows.get(), cnt, s));
        L.n_long = nlong;
        L.long_min = lim;
      }
    }
  }
  CWM_TRY(L.dinv.alloc(L.n, s));
  const bool f32 = h->prm.vcycle_fp32 != 0;
  if (f32) CWM_TRY(L.dinv32.alloc(L.n, s));
  CWM_TRY(reciprocal(L.n, L.dl1.get(), L.dinv.get(), f32 ? L.dinv32.get() : nullptr, s));
  CWM_TRY(L.b.alloc(L.n, s));
  CWM_TRY(L.x.alloc(L.n, s));
  CWM_TRY(L.t1.alloc(L.n, s));
  CWM_TRY(L.t2.alloc(L.n, s));
  if (f32) {
    CWM_TRY(L.val32.alloc(L.nnz, s));
    CWM_TRY(to_float(L.nnz, L.val.get(), L.val32.get(), s));
    CWM_TRY(L.b32.alloc(L.n, s));
    CWM_TRY(L.x32.alloc(L.n, s));
    CWM_TRY(L.t132.alloc(L.n, s));
    CWM_TRY(L.t232.alloc(L.n, s));
    if (L.p.get()) {
      CWM_TRY(L.p32.alloc(L.n, s));
      CWM_TRY(to_float(L.n, L.p.get(), L.p32.get(), s));
    }
  }
  return AMG_OK;
}

// ------------------------------------------------------------ V-cycle ----
template <class V>
struct LevelVec;
template <class V>
TailArgs<V> &tail_args(amg_hierarchy *h);
template <>
struct LevelVec<double> {
  static CsrView<double> A(const Level &L) { return L.view64(); }
  static const double *dinv(const Level &L) { return L.dinv.get(); }
  static const double *p(const Level &L) { return L.p.get(); }
  static double *b(Level &L) { return L.b.get(); }
  static double *x(Level &L) { return L.x.get(); }
  static double *t1(Level &L) { return L.t1.get(); }
  static double *t2(Level &L) { return L.t2.get(); }
  static const double *dense(const Level &L) { return L.xdense.get(); }
  static bool has_ap(const Level &L) { return L.ap_nnz > 0 && L.ap_val.get(); }
  static CsrView<double> AP(const Level &L) { return L.ap_view<double>(L.ap_val.get()); }
  static Sell3View<double> B3(const Level &L) { return L.block3_view<double>(L.b3_val.get()); }
  static SellView<double> SA(const Level &L) { return L.sa.view<double>(L.sa.v64.get()); }
  static SellView<double> SAP(const Level &L) { return L.sap.view<double>(L.sap.v64.get()); }
};
template <>
struct LevelVec<float> {
  static CsrView<float> A(const Level &L) { return L.view32(); }
  static const float *dinv(const Level &L) { return L.dinv32.get(); }
  static const float *p(const Level &L) { return L.p32.get(); }
  static float *b(Level &L) { return L.b32.get(); }
  static float *x(Level &L) { return L.x32.get(); }
  static float *t1(Level &L) { return L.t132.get(); }
  static float *t2(Level &L) { return L.t232.get(); }
  static const float *dense(const Level &L) { return L.xdense32.get(); }
  static bool has_ap(const Level &L) { return L.ap_nnz > 0 && L.ap_val32.get(); }
  static CsrView<float> AP(const Level &L) { return L.ap_view<float>(L.ap_val32.get()); }
  static Sell3View<float> B3(const Level &L) { return L.block3_view<float>(L.b3_val32.get()); }
  static SellView<float> SA(const Level &L) { return L.sa.view<float>(L.sa.v32.get()); }
  static SellView<float> SAP(const Level &L) { return L.sap.view<float>(L.sap.v32.get()); }
};

template <>
TailArgs<double> &tail_args<double>(amg_hierarchy *h) { return h->tail64; }
template <>
TailArgs<float> &tail_args<float>(amg_hierarchy *h) { return h->tail32; }
template <class V>
const TailArgs<V> *tail_dev_args(amg_hierarchy *h);
template <>
const TailArgs<double> *tail_dev_args<double>(amg_hierarchy *h) {
  return reinterpret_cast<const TailArgs<double> *>(h->tail_dev.get());
}
template <>
const TailArgs<float> *tail_dev_args<float>(amg_hierarchy *h) {
  return reinterpret_cast<const TailArgs<float> *>(h->tail_dev.get() + sizeof(TailArgs<double>));
}

template <class V>
void fill_tail(amg_hierarchy *h, int k0, TailArgs<V> &a) {
  using LV = LevelVec<V>;
  a.nlev = (int)h->lev.size() - k0;
  a.pre = h->prm.pre_sweeps;
  a.post = h->prm.post_sweeps;
  a.coarse_sweeps = h->prm.coarse_sweeps;
  a.spin_cap = h->prm.loop_cap > 0 ? (unsigned)(h->prm.loop_cap < (1ll << 31) ? h->prm.loop_cap : (1ll << 31))
                                   : (1u << 24);
  for (int l = 0; l < a.nlev; ++l) {
    Level &L = h->lev[k0 + l];
    TailLevel<V> &t = a.lev[l];
    const CsrView<V> A = LV::A(L);
    t.n = L.n;
    t.rp_host_nnz = L.nnz;
    t.rp = A.rp;
    t.ci = A.ci;
    t.val = A.val;
    t.dinv = LV::dinv(L);
    t.agg = L.agg.get();
    t.mptr = L.mptr.get();
    t.mlist = L.mlist.get();
    t.p = LV::p(L);
    t.b = LV::b(L);
    t.x = LV::x(L);
    t.t1 = LV::t1(L);
    t.t2 = LV::t2(L);
    t.dense = LV::dense(L);
  }
}

// x^k = V-cycle(k, b^k) from x^k = 0 (Algorithm 1); b and x must not be t1/t2 of level k.
template <class V>
amg_status cycle_level(amg_hierarchy *h, int k, const V *b, V *x, bool zero_init);

// x^k = V-cycle(k, b^k) from x^k = 0 (Algorithm 1); b and x must not be t1/t2 of level k.
template <class V>
amg_status vcycle_level(amg_hierarchy *h, int k, const V *b, V *x) {
  return cycle_level<V>(h, k, b, x, true);
}

// One cycle on level k from the starting guess in x (zero_init: x = 0, not read).  The
// coarse correction runs `gamma` cycles on level k+1 (1: V-cycle; 2: W-cycle, Sec. 5.1), the
// first from zero and the others from the previous result.  A starting guess other than
// zero only occurs on levels k >= 1, where x is the level's own vector.
template <class V>
amg_status cycle_level(amg_hierarchy *h, int k, const V *b, V *x, bool zero_init) {
  using LV = LevelVec<V>;
  cudaStream_t s = h->stream;
  Level &L = h->lev[k];
  LevelTag tag(k);
  const int gamma = h->prm.gamma < 1 ? 1 : h->prm.gamma;
  if (k == h->tail_start && zero_init && gamma == 1)
    return vcycle_tail<V>(tail_args<V>(h), tail_dev_args<V>(h), b, x, h->bar.get(), h->err.get(), s);
  const CsrView<V> A = LV::A(L);
  const V *dinv = LV::dinv(L);
  V *t1 = LV::t1(L), *t2 = LV::t2(L);
  const int nl = (int)h->lev.size();
  if (k == nl - 1) {  // coarsest: l1-Jacobi sweeps from the starting guess
    const int sweeps = h->prm.coarse_sweeps;
    if (!zero_init) {
      if (sweeps <= 0) return AMG_OK;
      if (LV::dense(L)) {  // x += B (b - A x) with B the dense operator of the sweeps
        CWM_TRY(residual_t<V>(A, b, x, t1, s));
        CWM_TRY(dense_coarse_apply<V>(A.n, LV::dense(L), t1, t2, s));
        return add_to<V>(A.n, t2, x, s);
      }
      const V *cur = x;
      for (int i = 0; i < sweeps; ++i) {
        V *dst = cur == t1 ? t2 : t1;
        CWM_TRY(jacobi<V>(A, dinv, b, cur, dst, s));
        cur = dst;
      }
      CWM_CUDA(cudaMemcpyAsync(x, cur, sizeof(V) * (size_t)A.n, cudaMemcpyDeviceToDevice, s));
      return AMG_OK;
    }
    if (LV::dense(L)) return dense_coarse_apply<V>(A.n, LV::dense(L), b, x, s);
    if (A.n <= kCoarseBlockMax) return coarse_solve_block<V>(A, dinv, b, x, sweeps, s);
    if (sweeps <= 0) { CWM_CUDA(cudaMemsetAsync(x, 0, sizeof(V) * (size_t)A.n, s)); return AMG_OK; }
    const V *cur = nullptr;
    for (int i = 0; i < sweeps; ++i) {
      V *dst = i == sweeps - 1 ? x : (cur == t1 ? t2 : t1);
      if (i == 0) CWM_TRY(scale<V>(A.n, dinv, b, dst, s));
      else CWM_TRY(jacobi<V>(A, dinv, b, cur, dst, s));
      cur = dst;
    }
    return AMG_OK;
  }
  Level &C0 = h->lev[k + 1];
  // The default cycle from zero (one pre- and one post-sweep) on a small level: the first
  // sweep x = D^{-1} b is formed on the fly inside the residual and the coarse correction
  // inside the post-sweep, two kernels fewer.  On large levels the extra gathers per
  // nonzero cost more than the passes they save (measured), so they keep separate kernels;
  // so do levels on sub-warp tiles (the fused forms exist as row-block kernels only).  A
  // level with A P (built for the levels that skip the fused kernels, or for every level with
  // coupled_post = 1) takes the coarse correction and the post-sweep through it instead.
  const bool ap = h->prm.post_sweeps == 1 && LV::has_ap(L);
  // the finest operator in 3x3 blocks, or sliced copies of A and A P: the residual and the
  // coarse correction + post-sweep stream those layouts
  const Sell3View<V> B3 = k == 0 ? LV::B3(L) : Sell3View<V>{};
  const SellView<V> SA = LV::SA(L), SAP = LV::SAP(L);
  if (ap && zero_init && h->prm.pre_sweeps == 1 && (B3.nbr > 0 || SA.n > 0 || A.n <= fuse_max_rows<V>())) {
    // the first sweep from zero, xs = D^{-1} b, formed on the fly inside the residual
    // r = b - A xs and inside the coarse correction + post-sweep through A P (no separate
    // scale pass; in FP64 on CSR only up to the fused-kernel size limit, where the extra
    // multiply per nonzero costs less than the pass)
    Level &C = h->lev[k + 1];
    if (B3.nbr > 0)
      CWM_TRY(block3_resid_restrict<V>(B3, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), b, nullptr, dinv, t1,
                                       LV::b(C), s));
    else if (SA.n > 0)
      CWM_TRY(sell_resid_restrict<V>(SA, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), b, nullptr, dinv, t1,
                                     LV::b(C), s));
    else
      CWM_TRY(resid_scaled_restrict<V>(A, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), dinv, b, t1, LV::b(C), s));
    for (int g = 0; g < gamma; ++g) CWM_TRY(cycle_level<V>(h, k + 1, LV::b(C), LV::x(C), g == 0));
    double *x64 = (k == 0 && sizeof(V) == 4) ? h->out64 : nullptr;
    if (x64) h->out64_written = true;
    if (SAP.n > 0)
      return sell_prolong_jacobi_ap<V>(SAP, C.n, dinv, t1, L.agg.get(), LV::p(L), LV::x(C), b, true, x, s, x64);
    return prolong_jacobi_ap<V>(LV::AP(L), C.n, dinv, t1, L.agg.get(), LV::p(L), LV::x(C), b, true, x, s, x64);
  }
  if (!ap && B3.nbr == 0 && zero_init && h->prm.pre_sweeps == 1 && h->prm.post_sweeps == 1 &&
      A.n <= fuse_max_rows<V>() && A.rb) {
    CWM_TRY(resid_scaled_restrict<V>(A, C0.n, L.mptr.get(), L.mlist.get(), LV::p(L), dinv, b, t1, LV::b(C0), s));
    for (int g = 0; g < gamma; ++g) CWM_TRY(cycle_level<V>(h, k + 1, LV::b(C0), LV::x(C0), g == 0));
    return prolong_jacobi<V>(A, dinv, b, L.agg.get(), LV::p(L), LV::x(C0), x, s);
  }
  // pre-smoothing; from zero the first sweep is x = D^{-1} b
  const V *xs = zero_init ? nullptr : x;
  for (int i = 0; i < h->prm.pre_sweeps; ++i) {
    V *dst = (xs == t1) ? t2 : t1;
    if (i == 0 && zero_init) CWM_TRY(scale<V>(A.n, dinv, b, dst, s));
    else CWM_TRY(jacobi<V>(A, dinv, b, xs, dst, s));
    xs = dst;
  }
  Level &C = h->lev[k + 1];
  V *rtmp = (xs == t1) ? t2 : t1;  // free until the prolongation writes it
  if (B3.nbr > 0 && xs)
    CWM_TRY(block3_resid_restrict<V>(B3, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), b, xs, nullptr, rtmp, LV::b(C),
                                     s));
  else if (SA.n > 0 && xs)
    CWM_TRY(sell_resid_restrict<V>(SA, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), b, xs, nullptr, rtmp, LV::b(C),
                                   s));
  else
    CWM_TRY(resid_restrict_rb<V>(A, C.n, L.mptr.get(), L.mlist.get(), LV::p(L), b, xs, rtmp, LV::b(C), s));
  for (int g = 0; g < gamma; ++g) CWM_TRY(cycle_level<V>(h, k + 1, LV::b(C), LV::x(C), g == 0));
  if (ap && SAP.n > 0)  // rtmp still holds b - A xs
    return sell_prolong_jacobi_ap<V>(SAP, C.n, dinv, rtmp, L.agg.get(), LV::p(L), LV::x(C), xs, false, x, s);
  if (ap)
    return prolong_jacobi_ap<V>(LV::AP(L), C.n, dinv, rtmp, L.agg.get(), LV::p(L), LV::x(C), xs, false, x, s);
  V *y = (xs == t1) ? t2 : t1;
  CWM_TRY(prolong<V>(A.n, L.agg.get(), LV::p(L), LV::x(C), xs, y, s));
  const int post = h->prm.post_sweeps;
  if (post <= 0) {
    CWM_CUDA(cudaMemcpyAsync(x, y, sizeof(V) * (size_t)A.n, cudaMemcpyDeviceToDevice, s));
    return AMG_OK;
  }
  const V *cur = y;
  for (int i = 0; i < post; ++i) {
    V *dst = i == post - 1 ? x : (cur == t1 ? t2 : t1);
    CWM_TRY(jacobi<V>(A, dinv, b, cur, dst, s));
    cur = dst;
  }
  return AMG_OK;
}

// w = B(r).  float32 cycle: r32_ready says that the finest level's float input already holds
// r rounded to binary32 (written by the FCG update); the result comes back in binary64
// from the finest level's last kernel where it can write it, else from a conversion pass.
amg_status apply_vcycle(amg_hierarchy *h, const double *r, double *w, bool r32_ready = false) {
  if (!h->prm.vcycle_fp32) return vcycle_level<double>(h, 0, r, w);
  Level &L0 = h->lev[0];
  if (!r32_ready) CWM_TRY(to_float(L0.n, r, L0.b32.get(), h->stream));
  h->out64 = w;
  h->out64_written = false;
  const amg_status st = vcycle_level<float>(h, 0, L0.b32.get(), L0.x32.get());
  h->out64 = nullptr;
  CWM_TRY(st);
  if (h->out64_written) return AMG_OK;
  return to_double(L0.n, L0.x32.get(), w, h->stream);
}

amg_status validate_handle(amg_handle h) {
  if (!h) {
    set_error("NULL handle");
    return AMG_ERR_INVALID_ARG;
  }
  return AMG_OK;
}

}  // namespace

// ============================================================ C ABI ====
extern "C" {

void amg_default_params(amg_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->sweeps_per_level = 2;
  p->coarse_max = 40;
  p->max_levels = 40;
  p->pre_sweeps = 1;
  p->post_sweeps = 1;
  p->coarse_sweeps = 20;
  p->vcycle_fp32 = 0;
  p->check_input = 1;
  p->keep_sweeps = 0;
  p->loop_cap = 0;
  p->trace = 0;
  p->tail_rows = -1;
  p->stall_ratio = 0.0;
  p->gamma = 1;
  p->galerkin_fp32_from = 0;
  p->coupled_post = 0;
  p->block3 = 0;
  p->sliced = 0;
}

const char *amg_status_string(amg_status s) {
  switch (s) {
    case AMG_OK: return "AMG_OK";
    case AMG_ERR_INVALID_ARG: return "AMG_ERR_INVALID_ARG";
    case AMG_ERR_NOT_SPD: return "AMG_ERR_NOT_SPD";
    case AMG_ERR_CUDA: return "AMG_ERR_CUDA";
    case AMG_ERR_OOM: return "AMG_ERR_OOM";
    case AMG_ERR_TIMEOUT: return "AMG_ERR_TIMEOUT";
    case AMG_ERR_BREAKDOWN: return "AMG_ERR_BREAKDOWN";
    case AMG_ERR_NOT_CONVERGED: return "AMG_ERR_NOT_CONVERGED";
    case AMG_ERR_UNSUPPORTED: return "AMG_ERR_UNSUPPORTED";
  }
  return "AMG_ERR_UNKNOWN";
}

const char *amg_last_error(void) { return cwm::last_error(); }

static amg_status setup_impl(int n, int64_t nnz, const int32_t *rp, const int32_t *ci, const double *val,
                             const double *v, const amg_params *params, void *stream, amg_hierarchy *h) {
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  CWM_CUDA(cudaGetDevice(&h->device));
  if (params) h->prm = *params;
  else amg_default_params(&h->prm);
  amg_params &P = h->prm;
  h->trace.on = P.trace != 0;
  P.trace_filter[sizeof(P.trace_filter) - 1] = '\0';
  h->trace.filter = P.trace_filter;
  TraceGuard tg(h);
  if (P.coarse_max == -1) {  // the paper's default (Sec. 5): floor(40 n^(1/3)) = icbrt(64000 n)
    const long long X = 64000LL * (long long)n;
    long long lo = 0, hi = 1LL << 21;
    while (lo < hi) {
      const long long mid = (lo + hi + 1) / 2;
      if (mid * mid * mid <= X) lo = mid;
      else hi = mid - 1;
    }
    P.coarse_max = (int)lo;
  }
  if (P.sweeps_per_level < 1 || P.sweeps_per_level > kMaxSweeps || P.max_levels < 1 || P.pre_sweeps < 0 ||
      P.post_sweeps < 0 || P.coarse_sweeps < 0 || P.coarse_max < 0 || P.galerkin_fp32_from < 0 ||
      P.coupled_post < -1 || P.coupled_post > 1 || P.block3 < -1 || P.block3 > 0 || P.sliced < -1 || P.sliced > 1) {
    set_error("amg_setup: parameter out of range");
    return AMG_ERR_INVALID_ARG;
  }
  retain_pool_memory();
  CWM_TRY(h->box.init());
  CWM_TRY(h->err.alloc(2, s));  // [0] error bits, [1] scratch for one device -> host int
  CWM_CUDA(cudaMemsetAsync(h->err.get(), 0, 2 * sizeof(int), s));

  h->lev.emplace_back();
  Level &L0 = h->lev[0];
  L0.n = n;
  L0.nnz = nnz;
  CWM_TRY(L0.rp.alloc((size_t)n + 1, s));
  CWM_TRY(L0.ci.alloc(nnz, s));
  CWM_TRY(L0.val.alloc(nnz, s));
  CWM_TRY(L0.v.alloc(n, s));
  CWM_TRY(L0.diag.alloc(n, s));
  CWM_TRY(L0.dl1.alloc(n, s));
  // the inputs may be device, page-locked host or pageable host memory (copy_in)
  CWM_TRY(copy_in(L0.rp.get(), rp, sizeof(int) * ((size_t)n + 1), s));
  if (nnz) {
    CWM_TRY(copy_in(L0.ci.get(), ci, sizeof(int) * (size_t)nnz, s));
    CWM_TRY(copy_in(L0.val.get(), val, sizeof(double) * (size_t)nnz, s));
  }
  CWM_TRY(copy_in(L0.v.get(), v, sizeof(double) * (size_t)n, s));
  if (P.check_input) {
    CWM_TRY(check_input(n, nnz, L0.rp.get(), L0.ci.get(), L0.val.get(), true, h->err.get(), s));
    CWM_TRY(read_err(h, "amg_setup (input check)"));
  }
  CWM_TRY(extract_diag(n, L0.rp.get(), L0.ci.get(), L0.val.get(), L0.diag.get(), h->err.get(), s));
  CWM_TRY(max_row_length(n, L0.rp.get(), h->err.get() + 1, s));
  CWM_CUDA(cudaMemcpyAsync(h->box.ints + 5, h->err.get() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CWM_TRY(read_err(h, "amg_setup (diagonal)"));
  L0.max_row = h->box.ints[5];
  CWM_TRY(l1_norms(L0.view64(), L0.dl1.get(), s));

  CWM_CUDA(cudaStreamCreateWithFlags(&h->solve_stream, cudaStreamNonBlocking));
  CWM_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CWM_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  // Work on the library's second stream (the A P of each level while the next level is
  // coarsened, the coarsest level's dense operator while the setup stream builds the 3x3-block
  // and sliced copies): the setup stream waits for it before anything else is released or
  // returned, on every path out of this function (Join runs before the buffers it uses are
  // freed).
  DBuf<double> dense_tmp;
  struct Join {
    cudaStream_t side = nullptr, main = nullptr;
    cudaEvent_t ev = nullptr;
    ~Join() {
      if (!side) return;
      cudaEventRecord(ev, side);
      cudaStreamWaitEvent(main, ev, 0);
    }
  } join;
  cudaStream_t side = h->solve_stream;
  CWM_TRY(h->ap_stat.alloc(2 * (size_t)P.max_levels, s));
  while ((int)h->lev.size() < P.max_levels && h->lev.back().n > P.coarse_max) {
    bool made = false;
    const size_t before = h->lev.size();
    CWM_TRY(coarsen_level(h, &made));
    if (h->lev.size() == before) break;  // no pair at all: the current level is the coarsest
    {  // the level just coarsened has its prolongator: its A P on the second stream
      const int k = (int)h->lev.size() - 2;
      if (wants_ap(h, h->lev[k])) {
        CWM_CUDA(cudaEventRecord(h->ev_in, s));
        CWM_CUDA(cudaStreamWaitEvent(side, h->ev_in, 0));
        join.side = side;
        join.main = s;
        join.ev = h->ev_out;
        CWM_TRY(build_ap_level(h, k, side));
      }
    }
    if (!made) break;
    const Level &Fl = h->lev[h->lev.size() - 2], &Cl = h->lev.back();
    if (P.stall_ratio > 0.0 && (double)Fl.n < P.stall_ratio * (double)Cl.n) break;
  }
  for (Level &L : h->lev) CWM_TRY(finish_level(h, L));
  h->lev.back().nsweeps = 0;
  if (join.side) {  // the A P builds are done before their sizes are read
    CWM_CUDA(cudaEventRecord(h->ev_out, side));
    CWM_CUDA(cudaStreamWaitEvent(s, h->ev_out, 0));
    join.side = nullptr;
    CWM_TRY(ap_sizes(h));
  }
  {
    Level &Lc = h->lev.back();
    LevelTag tag((int)h->lev.size() - 1);
    if (Lc.n <= kDenseCoarseMax) {
      const size_t nn = (size_t)Lc.n * Lc.n;
      CWM_TRY(Lc.xdense.alloc(nn, s));
      CWM_TRY(dense_tmp.alloc(nn, s));
      if (P.vcycle_fp32) CWM_TRY(Lc.xdense32.alloc(nn, s));
      CWM_CUDA(cudaEventRecord(h->ev_in, s));
      CWM_CUDA(cudaStreamWaitEvent(side, h->ev_in, 0));
      join.side = side;
      join.main = s;
      join.ev = h->ev_out;
      CWM_TRY(dense_coarse_build(Lc.view64(), Lc.dinv.get(), P.coarse_sweeps, Lc.xdense.get(), dense_tmp.get(),
                                 side));
      if (P.vcycle_fp32) CWM_TRY(to_float((long long)nn, Lc.xdense.get(), Lc.xdense32.get(), side));
    }
  }
  CWM_TRY(build_block3(h));

  // the fused coarse end of the V-cycle
  {
    const int nl = (int)h->lev.size();
    const int limit = P.tail_rows > 0 ? P.tail_rows : (P.tail_rows == 0 ? kTailMaxRows : -1);
    // measured on GB300 with the default cycle, the cooperative launch and its grid barriers
    // cost more than the small kernels they replace, so the tail is opt-in (tail_rows > 0)
    int k0 = nl;
    while (limit > 0 && k0 > 0 && h->lev[k0 - 1].n <= limit) --k0;
    if (k0 < nl && nl - k0 <= kTailMaxLevels) {
      h->tail_start = k0;
      CWM_TRY(h->bar.alloc(2, s));
      CWM_CUDA(cudaMemsetAsync(h->bar.get(), 0, 2 * sizeof(unsigned), s));
      fill_tail<double>(h, k0, h->tail64);
      if (P.vcycle_fp32) fill_tail<float>(h, k0, h->tail32);
      CWM_TRY(h->tail_dev.alloc(sizeof(TailArgs<double>) + sizeof(TailArgs<float>), s));
      CWM_CUDA(cudaMemcpyAsync(h->tail_dev.get(), &h->tail64, sizeof(TailArgs<double>), cudaMemcpyHostToDevice, s));
      CWM_CUDA(cudaMemcpyAsync(h->tail_dev.get() + sizeof(TailArgs<double>), &h->tail32, sizeof(TailArgs<float>),
                               cudaMemcpyHostToDevice, s));
    }
  }
  CWM_TRY(build_sell(h));
  // FCG work vectors
  CWM_TRY(h->r.alloc(n, s));
  CWM_TRY(h->w.alloc(n, s));
  CWM_TRY(h->d.alloc(n, s));
  CWM_TRY(h->vv.alloc(n, s));
  CWM_TRY(h->q.alloc(n, s));
  const int nb = fcg_partial_blocks(n);
  CWM_TRY(h->part.alloc(3 * (size_t)fcg_dots_blocks_max(n, nnz), s));
  // part2 takes the partial sums of sqnorm_partials and of fcg_update, whose grids differ
  CWM_TRY(h->part2.alloc((size_t)std::max(nb, fcg_update_blocks(n)), s));
  CWM_TRY(h->scal.alloc(kFcgSlots, s));
  CWM_TRY(h->tick.alloc(4, s));
  CWM_CUDA(cudaMemsetAsync(h->tick.get(), 0, 4 * sizeof(unsigned), s));
  if (join.side) {  // join the dense build before the final synchronisation
    CWM_CUDA(cudaEventRecord(h->ev_out, join.side));
    CWM_CUDA(cudaStreamWaitEvent(s, h->ev_out, 0));
    join.side = nullptr;
  }
  CWM_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
}

amg_status amg_setup(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                     const double *d_v, const amg_params *params, void *stream, amg_handle *out) {
  if (!out) {
    set_error("amg_setup: out is NULL");
    return AMG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (n < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX || !d_row_ptr || !d_v || (nnz > 0 && (!d_col || !d_val))) {
    set_error("amg_setup: invalid size or NULL pointer (n=%d, nnz=%lld)", n, (long long)nnz);
    return AMG_ERR_INVALID_ARG;
  }
  const double t0 = now_ms();
  amg_hierarchy *h = new (std::nothrow) amg_hierarchy();
  if (!h) return AMG_ERR_OOM;
  amg_status st = setup_impl(n, nnz, d_row_ptr, d_col, d_val, d_v, params, stream, h);
  if (st != AMG_OK) {
    cudaDeviceSynchronize();
    (void)cudaGetLastError();
    g_sync_free = true;
    delete h;
    g_sync_free = false;
    return st;
  }
  h->t_setup_ms = now_ms() - t0;
  *out = h;
  return AMG_OK;
}

void amg_free(amg_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  g_sync_free = true;
  delete h;
  g_sync_free = false;
  (void)cudaGetLastError();
}

int amg_num_levels(amg_handle h) { return h ? (int)h->lev.size() : -1; }

amg_status amg_level_info(amg_handle h, int level, int *n, int64_t *nnz, int *nsweeps) {
  CWM_TRY(validate_handle(h));
  if (level < 0 || level >= (int)h->lev.size()) {
    set_error("amg_level_info: level %d out of range", level);
    return AMG_ERR_INVALID_ARG;
  }
  const Level &L = h->lev[level];
  if (n) *n = L.n;
  if (nnz) *nnz = L.nnz;
  if (nsweeps) *nsweeps = L.nsweeps;
  return AMG_OK;
}

amg_status amg_stats(amg_handle h, amg_info *info) {
  CWM_TRY(validate_handle(h));
  if (!info) return AMG_ERR_INVALID_ARG;
  const int nl = (int)h->lev.size();
  double z = 0.0, c = 0.0;
  for (int k = 0; k < nl; ++k) z += (double)h->lev[k].nnz;
  for (int k = 1; k < nl; ++k) c += (double)h->lev[k - 1].n / (double)h->lev[k].n;
  info->nl = nl;
  info->vcmplx = h->lev[0].nnz ? z / (double)h->lev[0].nnz : 0.0;
  info->cratio = c / nl;
  info->t_setup_ms = h->t_setup_ms;
  info->t_solve_ms = h->t_solve_ms;
  return AMG_OK;
}

amg_status amg_level_export(amg_handle h, int level, int32_t *d_row_ptr, int32_t *d_col, double *d_val,
                            double *d_v, double *d_dl1, int32_t *d_agg, double *d_p, void *stream) {
  CWM_TRY(validate_handle(h));
  if (level < 0 || level >= (int)h->lev.size()) {
    set_error("amg_level_export: level %d out of range", level);
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CWM_CUDA(cudaStreamSynchronize(h->stream));
  const Level &L = h->lev[level];
  const size_t n = L.n, z = L.nnz;
  auto cp = [&](void *dst, const void *src, size_t bytes) -> amg_status {
    if (dst && src && bytes) CWM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return AMG_OK;
  };
  CWM_TRY(cp(d_row_ptr, L.rp.get(), sizeof(int) * (n + 1)));
  CWM_TRY(cp(d_col, L.ci.get(), sizeof(int) * z));
  CWM_TRY(cp(d_val, L.val.get(), sizeof(double) * z));
  CWM_TRY(cp(d_v, L.v.get(), sizeof(double) * n));
  CWM_TRY(cp(d_dl1, L.dl1.get(), sizeof(double) * n));
  if (level + 1 < (int)h->lev.size()) {
    CWM_TRY(cp(d_agg, L.agg.get(), sizeof(int) * n));
    CWM_TRY(cp(d_p, L.p.get(), sizeof(double) * n));
  }
  CWM_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
}

amg_status amg_sweep_mate(amg_handle h, int level, int sweep, int32_t *d_mate, int *n, void *stream) {
  CWM_TRY(validate_handle(h));
  if (level < 0 || level >= (int)h->lev.size() || sweep < 0 || sweep >= (int)h->lev[level].sweep_mate.size()) {
    set_error("amg_sweep_mate: no kept matching for level %d sweep %d (keep_sweeps=%d)", level, sweep,
              h->prm.keep_sweeps);
    return AMG_ERR_INVALID_ARG;
  }
  const Level &L = h->lev[level];
  const int m = L.sweep_n[sweep];
  if (n) *n = m;
  if (d_mate) {
    CWM_CUDA(cudaStreamSynchronize(h->stream));
    CWM_CUDA(cudaMemcpyAsync(d_mate, L.sweep_mate[sweep].get(), sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    CWM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  }
  return AMG_OK;
}

amg_status amg_vcycle(amg_handle h, const double *d_r, double *d_w, void *stream) {
  CWM_TRY(validate_handle(h));
  if (!d_r || !d_w || d_r == d_w) {
    set_error("amg_vcycle: NULL or aliased vectors");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t prev = h->stream;
  h->stream = (cudaStream_t)stream;
  TraceGuard tg(h);
  amg_status st = apply_vcycle(h, d_r, d_w);
  if (st == AMG_OK && h->tail_start >= 0) {  // the fused tail has a bounded wait: check it
    cudaError_t e = cudaMemcpyAsync(h->box.ints + 8, h->err.get(), sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    st = e == cudaSuccess ? solve_device_error(h, "amg_vcycle") : cuda_fail(e, "amg_vcycle", __FILE__, __LINE__);
  }
  h->stream = prev;
  return st;
}

}  // extern "C"

namespace {

// One FCG iteration (Algorithm 3): w = B(r), v = A w with the three dot products and the
// scalars, the paired updates with ||r||^2, and the copy of the scalars to the host.
amg_status fcg_iteration(amg_hierarchy *h, double *d_x, int first) {
  cudaStream_t s = h->stream;
  const Level &L0 = h->lev[0];
  const CsrView<double> A = L0.view64();
  double *scal = h->scal.get();
  // the float32 cycle's input: r in binary32, written by the previous iteration's update
  const bool f32 = h->prm.vcycle_fp32 != 0;
  CWM_TRY(apply_vcycle(h, h->r.get(), h->w.get(), f32 && !first));
  const Sell3View<double> B3 = LevelVec<double>::B3(L0);
  if (B3.nbr > 0)
    CWM_TRY(block3_spmv_dots(B3, h->w.get(), h->r.get(), first ? nullptr : h->q.get(), h->vv.get(), h->part.get(),
                             fcg_dots_blocks_max(L0.n, L0.nnz), scal, h->tick.get(), first, s));
  else
    CWM_TRY(spmv_dots_scalars(A, h->w.get(), h->r.get(), first ? nullptr : h->q.get(), h->vv.get(), h->part.get(),
                              scal, h->tick.get(), first, s));
  CWM_TRY(fcg_update(L0.n, h->w.get(), h->vv.get(), h->d.get(), h->q.get(), d_x, h->r.get(),
                     f32 ? h->lev[0].b32.get() : nullptr, scal, h->part2.get(),
                     h->tick.get() + 1, first, s));
  CWM_CUDA(cudaMemcpyAsync(h->box.dbls, scal, sizeof(double) * kFcgSlots, cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaMemcpyAsync(h->box.ints + 8, h->err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  return AMG_OK;
}

// Captures the two iteration graphs (first / later iterations) for solution pointer d_x.
// On any capture failure the solver falls back to plain launches for this handle.
void capture_graphs(amg_hierarchy *h, double *d_x) {
  h->drop_graphs();
  if (h->graphs_failed) return;
  for (int g = 0; g < 2; ++g) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      h->graphs_failed = true;
      break;
    }
    h->trace.capturing = true;
    const long long before = launch_count();
    amg_status st = fcg_iteration(h, d_x, g);
    // captured launches are not executed: take them back out and count them per replay
    h->gkernels[g] = launch_count() - before;
    count_launches(-h->gkernels[g]);
    h->trace.capturing = false;
    h->gscopes[g].swap(h->trace.graph_pending);
    h->trace.graph_pending.clear();
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (st != AMG_OK || e != cudaSuccess || !graph ||
        cudaGraphInstantiate(&h->gexec[g], graph, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      h->graphs_failed = true;
      break;
    }
    cudaGraphDestroy(graph);
  }
  if (h->graphs_failed) h->drop_graphs();
  else h->graph_x = d_x;
}

}  // namespace

extern "C" amg_status amg_pcg_solve(amg_handle h, const double *d_b, double *d_x, double rtol, int itmax,
                                    void *stream, amg_info *info) {
  CWM_TRY(validate_handle(h));
  if (!d_b || !d_x || itmax < 0 || !(rtol >= 0.0)) {
    set_error("amg_pcg_solve: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  const double t0 = now_ms();
  cudaStream_t prev = h->stream;
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t s = h->solve_stream;
  struct Restore {
    amg_hierarchy *h;
    cudaStream_t s;
    ~Restore() { h->stream = s; }
  } restore{h, prev};
  h->stream = s;
  TraceGuard tg(h);
  // order after the caller's stream, run on the library's stream
  CWM_CUDA(cudaEventRecord(h->ev_in, user));
  CWM_CUDA(cudaStreamWaitEvent(s, h->ev_in, 0));

  const Level &L0 = h->lev[0];
  const CsrView<double> A = L0.view64();
  const int n = L0.n;
  const int nb = fcg_partial_blocks(n);
  // b and x in host memory are solved through device copies owned by the handle (so the
  // iteration graphs captured for them stay valid from call to call); x is copied back
  // before the call returns
  double *const x_user = d_x;
  const bool x_host = mem_kind(d_x, nullptr) != MemKind::kDevice;
  if (mem_kind(d_b, nullptr) != MemKind::kDevice) {
    if (!h->bdev.get()) CWM_TRY(h->bdev.alloc(n, s));
    CWM_TRY(copy_in(h->bdev.get(), d_b, sizeof(double) * (size_t)n, s));
    d_b = h->bdev.get();
  }
  if (x_host) {
    if (!h->xdev.get()) CWM_TRY(h->xdev.alloc(n, s));
    CWM_TRY(copy_in(h->xdev.get(), x_user, sizeof(double) * (size_t)n, s));
    d_x = h->xdev.get();
  }
  double *scal = h->scal.get();
  CWM_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * kFcgSlots, s));
  CWM_TRY(residual(A, d_b, d_x, h->r.get(), s));
  CWM_TRY(sqnorm_partials(n, d_b, h->part2.get(), s));
  CWM_TRY(reduce_into(nb, h->part2.get(), scal, kBB, s));
  CWM_TRY(sqnorm_partials(n, h->r.get(), h->part2.get(), s));
  CWM_TRY(reduce_into(nb, h->part2.get(), scal, kRR, s));
  CWM_CUDA(cudaMemcpyAsync(h->box.dbls, scal, sizeof(double) * kFcgSlots, cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  const double nb2 = std::sqrt(h->box.dbls[kBB]);
  double nr = std::sqrt(h->box.dbls[kRR]);
  amg_status status = (nb2 == 0.0 || nr <= rtol * nb2) ? AMG_OK : AMG_ERR_NOT_CONVERGED;
  if (status != AMG_OK && itmax > 0 && h->graph_x != d_x) capture_graphs(h, d_x);
  int it = 0;
  while (status != AMG_OK && it < itmax) {
    const int first = it == 0;
    if (h->gexec[first] && h->graph_x == d_x) {
      CWM_CUDA(cudaGraphLaunch(h->gexec[first], s));
      count_launches(h->gkernels[first]);
      CWM_CUDA(cudaStreamSynchronize(s));
      if (h->trace.on) h->trace.collect(h->gscopes[first]);
    } else {
      CWM_TRY(fcg_iteration(h, d_x, first));
      CWM_CUDA(cudaStreamSynchronize(s));
    }
    {
      const amg_status dst = solve_device_error(h, "amg_pcg_solve");
      if (dst != AMG_OK) return dst;
    }
    if (h->box.dbls[kFlags] != 0.0) {
      status = AMG_ERR_BREAKDOWN;
      set_error("amg_pcg_solve: breakdown at iteration %d (rho = %g)", it, h->box.dbls[kRho]);
      break;
    }
    ++it;
    nr = std::sqrt(h->box.dbls[kRR]);
    if (nr <= rtol * nb2) status = AMG_OK;
  }
  if (status == AMG_ERR_NOT_CONVERGED) set_error("amg_pcg_solve: itmax = %d reached", itmax);
  // true residual
  CWM_TRY(residual(A, d_b, d_x, h->vv.get(), s));
  CWM_TRY(sqnorm_partials(n, h->vv.get(), h->part2.get(), s));
  CWM_TRY(reduce_into(nb, h->part2.get(), scal, kBB, s));  // slot reused: true ||r||^2
  CWM_CUDA(cudaMemcpyAsync(h->box.dbls + 12, scal + kBB, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (x_host) CWM_TRY(copy_out(x_user, d_x, sizeof(double) * (size_t)n, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  CWM_CUDA(cudaEventRecord(h->ev_out, s));
  CWM_CUDA(cudaStreamWaitEvent(user, h->ev_out, 0));
  const double nr_true = std::sqrt(h->box.dbls[12]);
  h->t_solve_ms = now_ms() - t0;
  if (info) {
    amg_stats(h, info);
    info->iters = it;
    info->rel_res = nb2 > 0.0 ? nr / nb2 : 0.0;
    info->rel_res_true = nb2 > 0.0 ? nr_true / nb2 : 0.0;
    info->t_solve_ms = h->t_solve_ms;
  }
  return status;
}

extern "C" {

// ------------------------------------------------------------ tracing ----
amg_status amg_trace_enable(amg_handle h, int on, const char *filter) {
  CWM_TRY(validate_handle(h));
  h->trace.on = on != 0;
  h->trace.filter = filter ? filter : "";
  return AMG_OK;
}

amg_status amg_trace_reset(amg_handle h) {
  CWM_TRY(validate_handle(h));
  h->trace.flush();
  h->trace.entries.clear();
  return AMG_OK;
}

int amg_trace_count(amg_handle h) {
  if (!h) return -1;
  h->trace.flush();
  return (int)h->trace.entries.size();
}

amg_status amg_trace_get(amg_handle h, int i, amg_trace_entry *out) {
  CWM_TRY(validate_handle(h));
  if (!out || i < 0 || i >= (int)h->trace.entries.size()) {
    set_error("amg_trace_get: index %d out of range", i);
    return AMG_ERR_INVALID_ARG;
  }
  const TraceEntry &e = h->trace.entries[i];
  std::memset(out, 0, sizeof(*out));
  std::strncpy(out->name, e.name.c_str(), sizeof(out->name) - 1);
  out->launches = e.launches;
  out->total_ms = e.ms;
  out->bytes = e.bytes;
  return AMG_OK;
}

int64_t amg_launch_count(void) { return cwm::launch_count(); }

// ------------------------------------------------------------ step entry points ----
static amg_status read_bits(int *d_err, int *h_slot, cudaStream_t s, const char *where) {
  CWM_CUDA(cudaMemcpyAsync(h_slot, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  return status_from_device_bits(*h_slot, where);
}

amg_status cwm_edge_weights(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                            const double *d_v, double *d_w, void *stream) {
  if (n < 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX || (n > 0 && (!d_row_ptr || !d_v)) ||
      (nnz > 0 && (!d_col || !d_val || !d_w))) {
    set_error("cwm_edge_weights: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  if (n == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<double> diag, dv;
  DBuf<int> err;
  int h_err = 0;
  CWM_TRY(diag.alloc(n, s));
  CWM_TRY(dv.alloc(n, s));
  CWM_TRY(err.alloc(1, s));
  CWM_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  CWM_TRY(extract_diag(n, d_row_ptr, d_col, d_val, diag.get(), err.get(), s));
  CWM_TRY(edge_weights(n, nnz, d_row_ptr, d_col, d_val, diag.get(), d_v, d_w, dv.get(), s));
  return read_bits(err.get(), &h_err, s, "cwm_edge_weights");
}

amg_status cwm_suitor_match(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_w,
                            int32_t *d_mate, void *stream) {
  if (n < 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX || (n > 0 && (!d_row_ptr || !d_mate)) ||
      (nnz > 0 && (!d_col || !d_w))) {
    set_error("cwm_suitor_match: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  if (n == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<unsigned char> keys;
  DBuf<int> err;
  int h_err = 0;
  CWM_TRY(keys.alloc(suitor_scratch_bytes(n), s));
  CWM_TRY(err.alloc(1, s));
  CWM_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  CWM_TRY(suitor_match(n, nnz, d_row_ptr, d_col, d_w, keys.get(), d_mate, nnz + n + 1024, err.get(), s));
  return read_bits(err.get(), &h_err, s, "cwm_suitor_match");
}

amg_status cwm_aggregate(int n, const int32_t *d_mate, const double *d_v, int32_t *d_agg, double *d_p, double *d_vc,
                         int *h_nc, int *h_npairs, void *stream) {
  if (n < 0 || (n > 0 && (!d_mate || !d_v || !d_agg || !d_p || !d_vc))) {
    set_error("cwm_aggregate: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<int> ids, scan, counts;
  CWM_TRY(ids.alloc((size_t)n + 1, s));
  CWM_TRY(scan.alloc(scan_scratch_ints(n), s));
  CWM_TRY(counts.alloc(2, s));
  CWM_TRY(aggregate(n, d_mate, d_v, d_agg, d_p, d_vc, nullptr, nullptr, ids.get(), scan.get(), counts.get(), s));
  int hc[2] = {0, 0};
  CWM_CUDA(cudaMemcpyAsync(hc, counts.get(), sizeof(hc), cudaMemcpyDeviceToHost, s));
  CWM_CUDA(cudaStreamSynchronize(s));
  if (h_nc) *h_nc = hc[0];
  if (h_npairs) *h_npairs = hc[1];
  return AMG_OK;
}

amg_status cwm_galerkin(int n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val, int nc,
                        const int32_t *d_agg, const double *d_p, int32_t *d_rpc, int32_t *d_colc, double *d_valc,
                        int64_t capacity, int64_t *h_nnzc, int fp32, void *stream) {
  if (n < 0 || nc < 0 || nc > n || (n > 0 && (!d_row_ptr || !d_agg || !d_p)) || !d_rpc || capacity < 0) {
    set_error("cwm_galerkin: invalid argument");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<int> m1, m2, cnt, longr, misc, scan, err;
  CWM_TRY(m1.alloc(nc, s));
  CWM_TRY(m2.alloc(nc, s));
  CWM_TRY(cnt.alloc((size_t)nc + 1, s));
  CWM_TRY(longr.alloc(nc, s));
  CWM_TRY(misc.alloc(1, s));
  CWM_TRY(scan.alloc(scan_scratch_ints(nc), s));
  CWM_TRY(err.alloc(1, s));
  CWM_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  CWM_TRY(members_from_agg(n, nc, d_agg, m1.get(), m2.get(), cnt.get(), err.get(), s));
  int nnz_in = 0;  // nnz of the fine operator: the padded rows' capacity
  if (n > 0) CWM_CUDA(cudaMemcpyAsync(&nnz_in, d_row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  int h_err = 0;
  CWM_TRY(read_bits(err.get(), &h_err, s, "cwm_galerkin (aggregates)"));  // synchronises
  if (nnz_in < 0) {
    set_error("cwm_galerkin: row_ptr[n] = %d is negative", nnz_in);
    return AMG_ERR_INVALID_ARG;
  }
  DBuf<int> rpu, cpad;
  DBuf<double> vpad;
  CWM_TRY(rpu.alloc((size_t)nc + 1, s));
  CWM_TRY(cpad.alloc(nnz_in, s));
  CWM_TRY(vpad.alloc(nnz_in, s));
  GalerkinWork gw;
  gw.cnt = cnt.get();
  gw.rpu = rpu.get();
  gw.long_rows = longr.get();
  gw.n_long = misc.get();
  gw.scan = scan.get();
  gw.ci_pad = cpad.get();
  gw.val_pad = vpad.get();
  gw.n_fine = n;
  gw.nnz_fine = nnz_in;
  CWM_TRY(galerkin_group(d_row_ptr, d_col, d_val, nc, m1.get(), m2.get(), d_agg, d_p, d_rpc, nullptr, nullptr, gw,
                         fp32 != 0, err.get(), s));
  int nnzc = 0;
  CWM_CUDA(cudaMemcpyAsync(&nnzc, d_rpc + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
  CWM_TRY(read_bits(err.get(), &h_err, s, "cwm_galerkin (grouping)"));
  if (h_nnzc) *h_nnzc = nnzc;
  if (nnzc > capacity) {
    set_error("cwm_galerkin: nnz(A_c) = %d exceeds capacity %lld", nnzc, (long long)capacity);
    return AMG_ERR_INVALID_ARG;
  }
  if (nnzc > 0 && (!d_colc || !d_valc)) {
    set_error("cwm_galerkin: NULL output arrays");
    return AMG_ERR_INVALID_ARG;
  }
  CWM_TRY(galerkin_compact(nc, d_rpc, d_colc, d_valc, gw, s));
  return read_bits(err.get(), &h_err, s, "cwm_galerkin (compaction)");
}

}  // extern "C"
