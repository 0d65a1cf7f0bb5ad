// coarsen.cu -- one pairwise coarsening sweep: input checks, diagonal, edge weights
// (Sec. 2.2), Suitor matching (Sec. 3.1), aggregation (Sec. 2.2, Algorithm 2), the
// orthonormal prolongator (Sec. 2.2), and the composition of sweeps (Sec. 5).
#include "coarsen.cuh"
#include "divint.cuh"

namespace cwm {

// ------------------------------------------------------------ input checks ----
// One thread per row: ascending in-range columns, positive stored diagonal, and (when
// check_sym) a bit-equal mirror entry for every stored (i, j).
__global__ void k_check_csr(int n, long long nnz, const int *__restrict__ rp,
                            const int *__restrict__ ci, const double *__restrict__ val,
                            int check_sym, int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = rp[i], e = rp[i + 1];
  if (s < 0 || e < s || e > nnz || (i == 0 && s != 0) || (i == n - 1 && e != nnz)) {
    atomicOr(err, kErrInvalid);
    return;
  }
  bool has_diag = false;
  for (int k = s; k < e; ++k) {
    int j = ci[k];
    if (j < 0 || j >= n || (k > s && j <= ci[k - 1])) { atomicOr(err, kErrInvalid); return; }
    if (j == i) {
      has_diag = true;
      if (!(val[k] > 0.0)) atomicOr(err, kErrNotSpd);
    }
    if (check_sym && j != i) {
      const int rs = rp[j], re = rp[j + 1];
      if (rs < 0 || re < rs || re > nnz) { atomicOr(err, kErrInvalid); return; }  // row j malformed
      int lo = rs, hi = re - 1, pos = -1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == i) { pos = mid; break; }
        if (c < i) lo = mid + 1; else hi = mid - 1;
      }
      if (pos < 0 || __double_as_longlong(val[pos]) != __double_as_longlong(val[k]))
        atomicOr(err, kErrInvalid);
    }
  }
  if (!has_diag) atomicOr(err, kErrNotSpd);
}

amg_status check_input(int n, long long nnz, const int *rp, const int *ci, const double *val,
                       bool check_sym, int *d_err, cudaStream_t s) {
  CWM_TRACE("check_input", 4.0 * (n + 1) + 12.0 * nnz, s);
  k_check_csr<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, nnz, rp, ci, val, check_sym ? 1 : 0, d_err);
  CWM_LAUNCH();
  return AMG_OK;
}

// Diagonal by binary search in each (sorted) row; a missing or non-positive diagonal
// raises kErrNotSpd.
__global__ void k_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                       const double *__restrict__ val, double *__restrict__ diag, int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = rp[i], hi = rp[i + 1] - 1;
  double d = 0.0;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int c = ci[mid];
    if (c == i) { d = val[mid]; break; }
    if (c < i) lo = mid + 1; else hi = mid - 1;
  }
  if (!(d > 0.0)) atomicOr(err, kErrNotSpd);
  diag[i] = d;
}

amg_status extract_diag(int n, const int *rp, const int *ci, const double *val, double *diag,
                        int *d_err, cudaStream_t s) {
  CWM_TRACE("diag", 4.0 * (n + 1) + 20.0 * n, s);
  k_diag<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, rp, ci, val, diag, d_err);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ edge weights ----
// Sec. 2.2, C(A, v).  No FMA: every product and sum is an explicit round-to-nearest
// intrinsic in the order ((2 a) v_a) v_b over ((a_aa v_a) v_a) + ((a_bb v_b) v_b),
// a = min(i,j).  The quotient is the correctly rounded one, formed on the integer pipes
// (div_rn_int), and 2 a is an exponent increment, which leaves four binary64 operations per
// evaluation on the scarce FP64 pipe.

// 2 a, exactly: the exponent field incremented when a is normal and 2 a finite (no FP64
// instruction), else the multiply.
__device__ __forceinline__ double twice_f64(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const unsigned e = (unsigned)((b >> 52) & 0x7ff);
  return e - 1u < 2045u ? __longlong_as_double((long long)(b + (1ull << 52))) : __dmul_rn(2.0, a);
}
// Operators whose rows average more than this many stored slots take k_edge_weights_all
// (every slot from its own row: twice the FP64 work, no mirror searches), the others
// k_edge_weights_rb.  Measured on GB300: elasticity levels (78 to a few hundred slots per
// row) 2.69 -> 2.35 ms of weights per setup; Poisson and lognormal (7 to 27 per row) lost
// 25% and 16% with every slot evaluated.
constexpr double kWeightsAllMean = 32.0;

// Row blocks, evaluating each edge once.  A block of kWB
// threads owns kWB consecutive rows.  Each row's thread finds where its upper part
// (columns > i) starts, writes 0 into its diagonal slot, and the block packs the upper
// slots of all its rows into one dense list (an exclusive scan of the per-row counts);
// threads then take that list in chunks of kWC, so the FP64 work -- a pipe that retires
// whole-warp instructions at a low rate on GB300 -- runs on full warps.  The thread that
// evaluates slot (i, j) also stores the weight into the mirror slot (j, i), found by a
// binary search in row j.
constexpr int kWB = 256;
constexpr int kWE = 8;
constexpr int kWC = kWB * kWE;

__global__ void __launch_bounds__(kWB) k_edge_weights_rb(int n, const int *__restrict__ rp,
                                                         const int *__restrict__ ci,
                                                         const double *__restrict__ val,
                                                         const double *__restrict__ dv,
                                                         const double *__restrict__ v,
                                                         double *__restrict__ w) {
  __shared__ double s_v[kWB], s_d[kWB];
  __shared__ int s_ustart[kWB], s_uoff[kWB + 1];
  __shared__ int s_slot[kWC];
  __shared__ unsigned char s_row[kWC];
  __shared__ int s_wsum[kWB / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int r0 = blockIdx.x * kWB;
  const int nrows = min(kWB, n - r0);
  int ucnt = 0, ustart = 0;
  if (t < nrows) {
    const int i = r0 + t;
    const int s = rp[i], e = rp[i + 1];
    s_v[t] = v[i];
    s_d[t] = dv[i];
    int lo = s, hi = e;  // first slot with column >= i
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ci[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    int k = lo;
    if (k < e && ci[k] == i) {
      w[k] = 0.0;  // the diagonal carries no edge
      ++k;
    }
    ustart = k;
    ucnt = e - k;
  }
  // block exclusive scan of the upper counts
  int incl = ucnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  int wbase = 0;
  for (int q = 0; q < warp; ++q) wbase += s_wsum[q];
  s_ustart[t] = ustart;
  s_uoff[t] = wbase + incl - ucnt;
  if (t == kWB - 1) s_uoff[kWB] = wbase + incl;
  __syncthreads();
  const int U = s_uoff[kWB];
  const int my_s = s_uoff[t], my_e = my_s + ucnt;
  for (int c0 = 0; c0 < U; c0 += kWC) {
    const int cend = min(c0 + kWC, U);
    for (int q = max(my_s, c0); q < min(my_e, cend); ++q) {
      s_slot[q - c0] = ustart + (q - my_s);
      s_row[q - c0] = (unsigned char)t;
    }
    __syncthreads();
    int slot[kWE], col[kWE];
    double a[kWE];
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      const int q = c0 + e * kWB + t;
      slot[e] = q < cend ? s_slot[q - c0] : -1;
      col[e] = slot[e] >= 0 ? __ldg(ci + slot[e]) : 0;
      a[e] = slot[e] >= 0 ? __ldg(val + slot[e]) : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      if (slot[e] < 0) continue;
      const int il = s_row[c0 + e * kWB + t - c0];
      const int i = r0 + il, j = col[e];  // i < j: row i is the smaller index
      double c = 0.0;
      if (nonzero_f64(a[e])) {
        const double va = s_v[il], vb = __ldg(v + j);
        const double num = __dmul_rn(__dmul_rn(twice_f64(a[e]), va), vb);
        const double den = __dadd_rn(s_d[il], __ldg(dv + j));
        if (nonzero_f64(den)) {
          const double cc = __dsub_rn(1.0, div_rn_int(num, den));
          if (pos_f64(cc)) c = cc;
        }
      }
      __stcs(w + slot[e], c);
      int lo = __ldg(rp + j), hi = __ldg(rp + j + 1) - 1;  // mirror slot (j, i)
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = __ldg(ci + mid);
        if (cm == i) {
          __stcs(w + mid, c);
          break;
        }
        if (cm < i) lo = mid + 1;
        else hi = mid - 1;
      }
    }
    __syncthreads();
  }
}

// Every stored slot evaluated from its own row's value: no mirror-slot search, every slot
// written (the diagonal and ineligible slots with 0), and the weights are those of the
// definition slot by slot even where the values are not symmetric.  A block owns kWB
// consecutive rows, whose slots are contiguous; each chunk of kWC of them is spread over the
// block's threads (kWE per thread, full warps) with the slot's row taken from a shared map.
__global__ void __launch_bounds__(kWB) k_edge_weights_all(int n, const int *__restrict__ rp,
                                                          const int *__restrict__ ci,
                                                          const double *__restrict__ val,
                                                          const double *__restrict__ dv,
                                                          const double *__restrict__ v,
                                                          double *__restrict__ w) {
  __shared__ double s_v[kWB], s_d[kWB];
  __shared__ int s_rs[kWB + 1];
  __shared__ unsigned char s_row[kWC];
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * kWB;
  const int nrows = min(kWB, n - r0);
  const int base = rp[r0];
  if (t < nrows) {
    s_v[t] = v[r0 + t];
    s_d[t] = dv[r0 + t];
    s_rs[t] = rp[r0 + t] - base;
  }
  if (t == 0) s_rs[nrows] = rp[r0 + nrows] - base;
  __syncthreads();
  const int U = s_rs[nrows];
  const int my_s = t < nrows ? s_rs[t] : 0, my_e = t < nrows ? s_rs[t + 1] : 0;
  for (int c0 = 0; c0 < U; c0 += kWC) {
    const int cend = min(c0 + kWC, U);
    for (int q = max(my_s, c0); q < min(my_e, cend); ++q) s_row[q - c0] = (unsigned char)t;
    __syncthreads();
    int col[kWE];
    double a[kWE];
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      const int q = c0 + e * kWB + t;
      col[e] = q < cend ? __ldg(ci + base + q) : 0;
      a[e] = q < cend ? __ldg(val + base + q) : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      const int q = c0 + e * kWB + t;
      if (q >= cend) continue;
      const int il = s_row[q - c0];
      const int i = r0 + il, j = col[e];
      double c = 0.0;
      if (j != i && nonzero_f64(a[e])) {
        const double vi = s_v[il], vj = __ldg(v + j), di = s_d[il], dj = __ldg(dv + j);
        const bool lo = i < j;  // the smaller index's values come first
        const double num = __dmul_rn(__dmul_rn(twice_f64(a[e]), lo ? vi : vj), lo ? vj : vi);
        const double den = __dadd_rn(lo ? di : dj, lo ? dj : di);
        if (nonzero_f64(den)) {
          const double cc = __dsub_rn(1.0, div_rn_int(num, den));
          if (pos_f64(cc)) c = cc;
        }
      }
      __stcs(w + base + q, c);
    }
    __syncthreads();
  }
}

// dv[i] = (a_ii v_i) v_i: the per-vertex half of the denominator, rounded exactly as in
// the per-slot expression, so that den = dv[a] + dv[b] is bit-identical.
__global__ void k_vertex_dv(int n, const double *__restrict__ diag, const double *__restrict__ v,
                            double *__restrict__ dv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dv[i] = __dmul_rn(__dmul_rn(diag[i], v[i]), v[i]);
}

amg_status edge_weights(int n, long long nnz, const int *rp, const int *ci, const double *val,
                        const double *diag, const double *v, double *w, double *dv_scratch, cudaStream_t s,
                        bool clear) {
  if (n == 0) return AMG_OK;
  // rp, ci, val, w written; v and diag of each row (gathers of neighbours counted once)
  CWM_TRACE("weights", 4.0 * (n + 1) + 20.0 * nnz + 32.0 * n, s);
  k_vertex_dv<<<grid_for(n, 256, num_sms() * 8), 256, 0, s>>>(n, diag, v, dv_scratch);
  CWM_LAUNCH();
  // upper-triangle kernel: lower slots without an upper partner (a pattern that is not
  // symmetric) stay 0; a structurally symmetric pattern has every slot written, so the
  // caller may skip the clear.  The every-slot kernel writes every slot.
  if ((double)nnz > kWeightsAllMean * n) {
    k_edge_weights_all<<<(n + kWB - 1) / kWB, kWB, 0, s>>>(n, rp, ci, val, dv_scratch, v, w);
  } else {
    if (clear) CWM_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * (size_t)nnz, s));
    k_edge_weights_rb<<<(n + kWB - 1) / kWB, kWB, 0, s>>>(n, rp, ci, val, dv_scratch, v, w);
  }
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ Suitor ----
#ifndef CWM_SUITOR_ENTRIES_PER_LANE
#define CWM_SUITOR_ENTRIES_PER_LANE 1
#endif
// Proposal tiles and their order.  One T-lane tile per vertex, blocks of kSuitorBlock
// threads, vertices taken in descending order as the hardware dispatches blocks.  The
// earlier design -- a resident grid whose tiles walked strided lists of ~50 vertices --
// let displacement chains queue behind one tile's list (one tile ran 2,400 proposal steps
// on 3D Poisson 128^3 where a lockstep model of the same proposals needs ~345) and took
// 1.3-4.0 ms for that level's first sweep, varying from run to run.  One vertex per tile
// in ascending order took 1.15-1.3 ms; descending 1.0-1.13 ms (lognormal 160^3: 2.5 ->
// 1.0 ms; Q1 elasticity 64^3: 4.3 -> 0.8 ms).  Small blocks release their slot as soon as
// their few tiles finish (64 vs 256 threads measured equal or slightly better).
constexpr int kSuitorBlock = 64;
// Sec. 3.1.  S[x] = (weight bits, suitor + 1) packed in 16 bytes; weights are positive
// doubles, whose bit patterns order like their values, so the 128-bit pair compares
// lexicographically as (weight, suitor index).  A proposer u beats the current suitor s
// of x iff (w_ux, u) > (w_sx, s); u prefers the neighbour maximising (w_ux, x).
struct __align__(16) SKey {
  unsigned long long lo;  // suitor index + 1 (0: none)
  unsigned long long hi;  // weight bits
};

__device__ __forceinline__ SKey load_key(const SKey *p) {
  SKey k;
  asm volatile(
      "{\n\t.reg .b128 t;\n\t"
      "ld.relaxed.gpu.global.b128 t, [%2];\n\t"
      "mov.b128 {%0, %1}, t;\n\t}"
      : "=l"(k.lo), "=l"(k.hi)
      : "l"(p)
      : "memory");
  return k;
}

__device__ __forceinline__ bool gt(unsigned long long h1, unsigned long long l1,
                                   unsigned long long h2, unsigned long long l2) {
  return h1 > h2 || (h1 == h2 && l1 > l2);
}

__global__ void k_clear_keys(long long n, SKey *S) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { S[i].lo = 0ull; S[i].hi = 0ull; }
}

// One T-lane tile per vertex u.  The tile finds the best neighbour that would accept the
// current proposer; the lane that found it installs the proposal with a 128-bit CAS,
// taking the key it has just read as the expected value (one dependent memory round trip
// less per proposal), and a displaced suitor becomes the next proposer (the chain is
// followed by the same tile).  Each lane takes up to two entries per round trip, issuing
// the column, weight and key loads of both before comparing, so that a step costs four
// dependent round trips (row pointers, row entries, keys, CAS) whatever the row length up
// to 2T.  Every loop is capped; hitting a cap raises kErrTimeout and ends the tile.
template <int T>
__global__ void __launch_bounds__(kSuitorBlock, 2048 / kSuitorBlock) k_suitor(int n, const int *__restrict__ rp,
                                                                            const int *__restrict__ ci,
                                                                            const double *__restrict__ w, SKey *S,
                                                                            long long cap, int *err) {
  auto tile = cg::tiled_partition<T>(cg::this_thread_block());
  const int lane = tile.thread_rank();
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / T;
  if (t >= n) return;
  int current = (int)(n - 1 - t);
  long long steps = 0;
  for (;;) {
    if (++steps > cap) {
      if (lane == 0) atomicOr(err, kErrTimeout);
      break;
    }
    const unsigned long long me = (unsigned long long)current + 1ull;
    unsigned long long mc = 0ull;  // this lane's best candidate and the key it read there
    int mx = -1;
    SKey mk;
    mk.lo = mk.hi = 0ull;
    const int s = rp[current], e = rp[current + 1];
    for (int k0 = s + lane; k0 < e; k0 += 2 * T) {
      const int k1 = k0 + T;
      const bool has1 = k1 < e;
      const double c0 = w[k0];
      const int x0 = ci[k0];
      const double c1 = has1 ? w[k1] : 0.0;
      const int x1 = has1 ? ci[k1] : 0;
      const bool ok0 = pos_f64(c0), ok1 = pos_f64(c1);
      SKey key0, key1;
      key0.lo = key0.hi = key1.lo = key1.hi = 0ull;
      if (ok0) key0 = load_key(S + x0);
      if (ok1) key1 = load_key(S + x1);
      const unsigned long long cb0 = (unsigned long long)__double_as_longlong(c0);
      const unsigned long long cb1 = (unsigned long long)__double_as_longlong(c1);
      if (ok0 && (cb0 > mc || (cb0 == mc && x0 > mx)) && gt(cb0, me, key0.hi, key0.lo)) {
        mc = cb0; mx = x0; mk = key0;
      }
      if (ok1 && (cb1 > mc || (cb1 == mc && x1 > mx)) && gt(cb1, me, key1.hi, key1.lo)) {
        mc = cb1; mx = x1; mk = key1;
      }
    }
    unsigned long long bc = mc;
    int bx = mx;
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
      const unsigned long long oc = tile.shfl_xor(bc, o);
      const int ox = tile.shfl_xor(bx, o);
      if (oc > bc || (oc == bc && ox > bx)) { bc = oc; bx = ox; }
    }
    if (bx < 0) break;  // nobody would accept `current`: it stays unmatched
    const int src = __ffs(tile.ballot(mx == bx)) - 1;  // the lane holding bx (>= 1 lane)
    int next = -2;      // -2: beaten while proposing, rescan
    if (lane == src) {
      SKey mine;
      mine.lo = me;
      mine.hi = bc;
      SKey expect = mk;
      for (int q = 0; q < (1 << 22); ++q) {
        if (!gt(bc, me, expect.hi, expect.lo)) break;
        const SKey old = atomicCAS(S + bx, expect, mine);
        if (old.lo == expect.lo && old.hi == expect.hi) {
          next = (int)old.lo - 1;  // -1: x had no suitor
          break;
        }
        expect = old;
      }
    }
    next = tile.shfl(next, src);
    if (next == -2) continue;
    if (next < 0) break;
    current = next;
  }
}

__global__ void k_suitor_mate(int n, const SKey *__restrict__ S, int *__restrict__ mate) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = (int)S[i].lo - 1;
  mate[i] = (s >= 0 && (int)S[s].lo - 1 == i) ? s : -1;
}

size_t suitor_scratch_bytes(int n) { return (size_t)n * sizeof(SKey); }

amg_status suitor_match(int n, long long nnz, const int *rp, const int *ci, const double *w,
                        void *scratch, int *mate, long long cap, int *d_err, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  // one proposal pass: rp, ci, w; S cleared, read once per vertex, read for the mates; mate
  CWM_TRACE("suitor", 4.0 * (n + 1) + 12.0 * nnz + 52.0 * n, s);
  SKey *S = reinterpret_cast<SKey *>(scratch);
  k_clear_keys<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, S);
  CWM_LAUNCH();
  if (cap <= 0) cap = nnz + (long long)n + 1024;
  const double mean = n ? (double)nnz / n : 1.0;
  // Proposals are latency-bound: a tile of half the row length (two entries per lane)
  // keeps twice as many proposal chains in flight.
  const int T = tile_for_mean(mean / CWM_SUITOR_ENTRIES_PER_LANE);
  const int block = kSuitorBlock;
  const unsigned grid = (unsigned)(((long long)n * T + block - 1) / block);
  switch (T) {
    case 4: k_suitor<4><<<grid, block, 0, s>>>(n, rp, ci, w, S, cap, d_err); break;
    case 8: k_suitor<8><<<grid, block, 0, s>>>(n, rp, ci, w, S, cap, d_err); break;
    case 16: k_suitor<16><<<grid, block, 0, s>>>(n, rp, ci, w, S, cap, d_err); break;
    default: k_suitor<32><<<grid, block, 0, s>>>(n, rp, ci, w, S, cap, d_err); break;
  }
  CWM_LAUNCH();
  k_suitor_mate<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, S, mate);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ aggregation ----
// Sec. 2.2, Algorithm 2 with U scanned in ascending order: vertex i starts an aggregate
// iff it is unmatched or the smaller end of its pair, and the aggregate id is the number
// of such leaders before i (an exclusive scan).  The leader writes both members' agg
// and p, v_c, and the member list.
// Leader flags, and the pairs counted with one atomic per block.
__global__ void k_leader_flags(int n, const int *__restrict__ mate, int *__restrict__ flag, int *npairs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = i < n ? mate[i] : -1;
  if (i < n) flag[i] = (m < 0 || i < m) ? 1 : 0;
  const int c = __syncthreads_count(i < n && m > i);
  if (threadIdx.x == 0 && c) atomicAdd(npairs, c);
}

__global__ void k_aggregate_fill(int n, const int *__restrict__ mate, const int *__restrict__ id,
                                 const double *__restrict__ v, int *__restrict__ agg,
                                 double *__restrict__ p, double *__restrict__ vc,
                                 int *__restrict__ m1, int *__restrict__ m2, int *__restrict__ nc_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *nc_out = id[n];  // the number of aggregates (the scan's total)
  if (i >= n) return;
  const int j = mate[i];
  if (j >= 0 && j < i) return;  // the follower is written by its leader
  const int I = id[i];
  const double vi = v[i];
  agg[i] = I;
  if (m1) m1[I] = i;
  if (j > i) {
    const double vj = v[j];
    const double s = __dsqrt_rn(__dadd_rn(__dmul_rn(vi, vi), __dmul_rn(vj, vj)));
    p[i] = __ddiv_rn(vi, s);
    p[j] = __ddiv_rn(vj, s);
    agg[j] = I;
    vc[I] = s;
    if (m2) m2[I] = j;
  } else {
    const double a = fabs(vi);
    p[i] = a > 0.0 ? __ddiv_rn(vi, a) : 1.0;
    vc[I] = a;
    if (m2) m2[I] = -1;
  }
}

amg_status aggregate(int n, const int *mate, const double *v, int *agg, double *p, double *vc,
                     int *m1, int *m2, int *id_scratch, int *scan_scratch, int *d_counts,
                     cudaStream_t s) {
  // d_counts[0] = n_c, d_counts[1] = n_pairs
  CWM_CUDA(cudaMemsetAsync(d_counts, 0, 2 * sizeof(int), s));
  if (n == 0) return AMG_OK;
  CWM_TRACE("aggregate", 52.0 * n, s);
  const int g = grid_for(n, 256, 1 << 30);
  k_leader_flags<<<g, 256, 0, s>>>(n, mate, id_scratch, d_counts + 1);
  CWM_LAUNCH();
  CWM_TRY(exclusive_scan(id_scratch, id_scratch, n, scan_scratch, s));
  k_aggregate_fill<<<g, 256, 0, s>>>(n, mate, id_scratch, v, agg, p, vc, m1, m2, d_counts);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ composition ----
// Row i of P_1 ... P_S has column agg_S[...agg_1[i]] and value
// ((p_1[i] * p_2[agg_1[i]]) * p_3[agg_2[agg_1[i]]]) ..., multiplied left to right.
__global__ void k_compose(int n, SweepMaps maps, int *__restrict__ agg_out, double *__restrict__ p_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = maps.agg[0][i];
  double pp = maps.p[0][i];
  for (int s = 1; s < maps.count; ++s) {
    pp = __dmul_rn(pp, maps.p[s][a]);
    a = maps.agg[s][a];
  }
  agg_out[i] = a;
  p_out[i] = pp;
}

amg_status compose(int n, const SweepMaps &maps, int *agg_out, double *p_out, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  CWM_TRACE("compose", 24.0 * n, s);
  k_compose<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, maps, agg_out, p_out);
  CWM_LAUNCH();
  return AMG_OK;
}

// ------------------------------------------------------------ member lists ----
// The transpose of the composed P as lists: members of aggregate I in ascending order
// (count, scan, scatter, then a tiny insertion sort per list, so the order does not
// depend on the scatter's atomics).
__global__ void k_count_members(int n, const int *__restrict__ agg, int *__restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + agg[i], 1);
}

__global__ void k_scatter_members(int n, const int *__restrict__ agg, const int *__restrict__ mptr,
                                  int *__restrict__ cursor, int *__restrict__ mlist) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int I = agg[i];
  const int pos = atomicAdd(cursor + I, 1);
  mlist[mptr[I] + pos] = i;
}

__global__ void k_sort_members(int nc, const int *__restrict__ mptr, int *__restrict__ mlist) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const int s = mptr[I], e = mptr[I + 1];
  for (int a = s + 1; a < e; ++a) {
    const int x = mlist[a];
    int b = a - 1;
    while (b >= s && mlist[b] > x) { mlist[b + 1] = mlist[b]; --b; }
    mlist[b + 1] = x;
  }
}

amg_status member_lists(int n, int nc, const int *agg, int *mptr, int *mlist, int *cnt_scratch,
                        int *scan_scratch, cudaStream_t s) {
  CWM_TRACE("members", 16.0 * n + 16.0 * nc, s);
  CWM_CUDA(cudaMemsetAsync(cnt_scratch, 0, sizeof(int) * ((size_t)nc + 1), s));
  const int g = grid_for(n, 256, 1 << 30);
  k_count_members<<<g, 256, 0, s>>>(n, agg, cnt_scratch);
  CWM_LAUNCH();
  CWM_TRY(exclusive_scan(cnt_scratch, mptr, nc, scan_scratch, s));
  CWM_CUDA(cudaMemsetAsync(cnt_scratch, 0, sizeof(int) * ((size_t)nc + 1), s));
  k_scatter_members<<<g, 256, 0, s>>>(n, agg, mptr, cnt_scratch, mlist);
  CWM_LAUNCH();
  k_sort_members<<<grid_for(nc, 256, 1 << 30), 256, 0, s>>>(nc, mptr, mlist);
  CWM_LAUNCH();
  return AMG_OK;
}

}  // namespace cwm
