/*
 * cwm_oracle.c -- plain, sequential FP64 CPU oracle for AMG coarsening based on
 * compatible weighted matching (Bernaschi, D'Ambra, Pasquini, "AMG based on
 * compatible weighted matching for GPUs"), together with the l1-Jacobi V-cycle
 * and the flexible CG that validate the hierarchy it builds.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Build:  gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared  (no FMA contraction:
 * every a*b+c below is two IEEE roundings, evaluated in the order written).
 *
 * Readings of the paper taken here (the paper leaves them open):
 *   - Edge set (Sec. 2.2): off-diagonal stored entries with a_ij != 0.
 *   - Edge weight (Sec. 2.2 names C(A,w) but does not print it):
 *       c_ab = 1 - (2 a_ab v_a v_b) / (a_aa v_a^2 + a_bb v_b^2),  a = min(i,j), b = max(i,j),
 *     evaluated as num = ((2*a_ab)*v_a)*v_b, den = ((a_aa*v_a)*v_a) + ((a_bb*v_b)*v_b),
 *     c = 1 - num/den.  Ordering the factors by vertex index makes c_ij == c_ji bit for
 *     bit whenever a_ij == a_ji.  den == 0 or c <= 0 (or NaN) makes the edge ineligible;
 *     an ineligible slot carries weight 0.
 *   - Matching (Sec. 3.1, Suitor): the Suitor result under the strict total order
 *     key(e) = (c_e, b, a) on edges e = {a < b}.  That is the greedy matching in
 *     decreasing key order.  For edges sharing a vertex the order reduces to
 *     "heavier first, then the larger other endpoint".
 *   - Aggregation (Sec. 2.2, Algorithm 2): "pick i in U" picks the smallest index left,
 *     so aggregate ids follow the smallest member.
 *   - Prolongator (Sec. 2.2): orthonormal projection of v on each aggregate:
 *     pair {i<j}: s = sqrt(v_i*v_i + v_j*v_j), p_i = v_i/s, p_j = v_j/s, v_c = s;
 *     singleton:  p_i = v_i/|v_i|, v_c = |v_i| (p_i = 1, v_c = 0 when v_i = 0).
 *   - Galerkin product A_c = P^T A P (Sec. 2.1): entry (I,J) sums the terms
 *     t_ij = (p_i*p_j)*a_ij over stored (i,j) with agg(i)=I, agg(j)=J, starting from +0.0
 *     and adding left to right in ascending order of (min(i,j), max(i,j), i).  The order
 *     depends only on the unordered pair, so A_c is bit-symmetric when A is.  Every hit
 *     (I,J) is stored, structural zeros included; columns ascend.
 *   - Single-precision Galerkin variant (the precision trade-off of Sec. 3.2 carried over
 *     to the setup): for the levels chosen, p_i, p_j and a_ij are rounded to binary32, the
 *     term is (p_i*p_j)*a_ij in binary32, and each entry sums its terms in binary32 from
 *     +0.0 in the same order; the entry is then stored as the double of that float.
 *   - Several sweeps per level (Sec. 2.2, Sec. 5): sweep s matches the operator made by
 *     sweep s-1; the level prolongator is the composition of the sweeps' prolongators.
 *   - l1-Jacobi (Sec. 3.2): D_ii = sum_j |a_ij|; one sweep x <- x + (b - A x)/D.
 *   - V-cycle (Sec. 2.1, Algorithm 1) with the coarsest solve done by l1-Jacobi sweeps
 *     from zero (Sec. 5).
 *   - Flexible CG (Sec. 3.2, Algorithm 3) with the residual update r <- r - (alpha/rho) q
 *     and the recurrence coefficient gamma_i / rho_{i-1}; stop on ||r||/||b|| <= rtol.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_SPD 2
#define OR_ERR_OOM 4
#define OR_ERR_BREAKDOWN 6
#define OR_ERR_NOT_CONVERGED 7

#define OR_MAX_LEVELS 64
#define OR_MAX_SWEEPS 8

/* ------------------------------------------------------------------------- */
/* Small helpers                                                              */
/* ------------------------------------------------------------------------- */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* a_ii by a linear scan of row i; returns 0 when the diagonal is not stored. */
static double diag_entry(const int *rp, const int *ci, const double *val, int i) {
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    if (ci[k] == i) return val[k];
  return 0.0;
}

/* ------------------------------------------------------------------------- */
/* Input checks                                                               */
/* ------------------------------------------------------------------------- */

/* 0 when rows have strictly ascending in-range columns; OR_ERR_ARG otherwise. */
int or_check_csr(int n, const int *rp, const int *ci) {
  if (n < 0 || rp[0] != 0) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return OR_ERR_ARG;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n) return OR_ERR_ARG;
      if (k > rp[i] && ci[k] <= ci[k - 1]) return OR_ERR_ARG;
    }
  }
  return OR_OK;
}

/* 0 when A is bit-symmetric (pattern and values); OR_ERR_ARG otherwise. */
int or_check_symmetric(int n, const int *rp, const int *ci, const double *val) {
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      int j = ci[k], found = 0;
      for (int q = rp[j]; q < rp[j + 1]; ++q)
        if (ci[q] == i) {
          found = 1;
          if (memcmp(&val[q], &val[k], sizeof(double)) != 0) return OR_ERR_ARG;
        }
      if (!found) return OR_ERR_ARG;
    }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.2: edge weights C(A, v)                                             */
/* ------------------------------------------------------------------------- */

/* w[k] for every stored slot k: c_ij for an eligible off-diagonal entry, 0 otherwise.
 * Returns OR_ERR_NOT_SPD when a diagonal entry is missing or not positive. */
int or_edge_weights(int n, const int *rp, const int *ci, const double *val,
                    const double *v, double *w) {
  double *d = (double *)xcalloc((size_t)n, sizeof(double));
  if (!d) return OR_ERR_OOM;
  for (int i = 0; i < n; ++i) {
    d[i] = diag_entry(rp, ci, val, i);
    if (!(d[i] > 0.0)) { free(d); return OR_ERR_NOT_SPD; }
  }
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      int j = ci[k];
      w[k] = 0.0;
      if (j == i || val[k] == 0.0) continue;
      int a = i < j ? i : j, b = i < j ? j : i;
      double num = ((2.0 * val[k]) * v[a]) * v[b];
      double den = ((d[a] * v[a]) * v[a]) + ((d[b] * v[b]) * v[b]);
      if (den == 0.0) continue;
      double c = 1.0 - num / den;
      if (c > 0.0) w[k] = c;  /* NaN and c <= 0 stay ineligible */
    }
  free(d);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: matching.  Greedy in decreasing key order = the Suitor result.   */
/* ------------------------------------------------------------------------- */

typedef struct { double c; int a, b; } or_edge;

/* Descending by (c, b, a). */
static int edge_cmp_desc(const void *x, const void *y) {
  const or_edge *e = (const or_edge *)x, *f = (const or_edge *)y;
  if (e->c != f->c) return e->c > f->c ? -1 : 1;
  if (e->b != f->b) return e->b > f->b ? -1 : 1;
  if (e->a != f->a) return e->a > f->a ? -1 : 1;
  return 0;
}

/* mate[i] = partner or -1.  Edges are the upper-triangle slots with w > 0. */
int or_greedy_match(int n, const int *rp, const int *ci, const double *w, int *mate) {
  long m = 0;
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] > i && w[k] > 0.0) ++m;
  or_edge *E = (or_edge *)xcalloc((size_t)m, sizeof(or_edge));
  if (!E) return OR_ERR_OOM;
  m = 0;
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] > i && w[k] > 0.0) { E[m].c = w[k]; E[m].a = i; E[m].b = ci[k]; ++m; }
  qsort(E, (size_t)m, sizeof(or_edge), edge_cmp_desc);
  for (int i = 0; i < n; ++i) mate[i] = -1;
  for (long e = 0; e < m; ++e)
    if (mate[E[e].a] < 0 && mate[E[e].b] < 0) { mate[E[e].a] = E[e].b; mate[E[e].b] = E[e].a; }
  free(E);
  return OR_OK;
}

/* (c1, i1) > (c2, i2) lexicographically. */
static int key_gt(double c1, int i1, double c2, int i2) {
  return c1 > c2 || (c1 == c2 && i1 > i2);
}

/* The sequential Suitor algorithm (Manne and Halappanavar): every vertex proposes to
 * its best neighbour that would accept it, displacing that neighbour's weaker suitor,
 * which then proposes again.  A second, independent route to the same matching. */
int or_suitor_match(int n, const int *rp, const int *ci, const double *w, int *mate) {
  int *suitor = (int *)xcalloc((size_t)n, sizeof(int));
  double *ws = (double *)xcalloc((size_t)n, sizeof(double));
  if (!suitor || !ws) { free(suitor); free(ws); return OR_ERR_OOM; }
  for (int i = 0; i < n; ++i) { suitor[i] = -1; ws[i] = 0.0; }
  for (int u = 0; u < n; ++u) {
    int current = u;
    for (;;) {
      int partner = -1;
      double best = 0.0;
      for (int k = rp[current]; k < rp[current + 1]; ++k) {
        int x = ci[k];
        double c = w[k];
        if (x == current || !(c > 0.0)) continue;
        /* x accepts current only over a weaker suitor; current prefers (c, x) max. */
        if (key_gt(c, current, ws[x], suitor[x]) && (partner < 0 || key_gt(c, x, best, partner))) {
          partner = x;
          best = c;
        }
      }
      if (partner < 0) break;
      int displaced = suitor[partner];
      suitor[partner] = current;
      ws[partner] = best;
      if (displaced < 0) break;
      current = displaced;
    }
  }
  for (int i = 0; i < n; ++i) {
    int s = suitor[i];
    mate[i] = (s >= 0 && suitor[s] == i) ? s : -1;
  }
  free(suitor);
  free(ws);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.2, Algorithm 2: pairwise aggregation                                */
/* ------------------------------------------------------------------------- */

/* agg[i] = aggregate id; returns n_c, and n_p / n_s through the pointers. */
int or_aggregate(int n, const int *mate, int *agg, int *n_pairs, int *n_single) {
  int nc = 0, np = 0, ns = 0;
  for (int i = 0; i < n; ++i) agg[i] = -1;
  for (int i = 0; i < n; ++i) {  /* U scanned in ascending order */
    if (agg[i] >= 0) continue;
    int j = mate[i];
    if (j >= 0 && agg[j] < 0 && j != i) {
      agg[i] = agg[j] = nc;
      ++np;
    } else {
      agg[i] = nc;
      ++ns;
    }
    ++nc;
  }
  if (n_pairs) *n_pairs = np;
  if (n_single) *n_single = ns;
  return nc;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.2: piecewise-constant prolongator by orthonormal projection of v     */
/* ------------------------------------------------------------------------- */

/* p[i] = the single nonzero of row i of P (column agg[i]); vc = P^T v. */
int or_prolongator(int n, int nc, const int *agg, const double *v, double *p, double *vc) {
  int *first = (int *)xcalloc((size_t)nc, sizeof(int));
  int *second = (int *)xcalloc((size_t)nc, sizeof(int));
  if (!first || !second) { free(first); free(second); return OR_ERR_OOM; }
  for (int I = 0; I < nc; ++I) first[I] = second[I] = -1;
  for (int i = 0; i < n; ++i) {
    int I = agg[i];
    if (first[I] < 0) first[I] = i;
    else second[I] = i;
  }
  for (int I = 0; I < nc; ++I) {
    int i = first[I], j = second[I];
    if (j >= 0) {
      double s = sqrt(v[i] * v[i] + v[j] * v[j]);
      p[i] = v[i] / s;
      p[j] = v[j] / s;
      vc[I] = s;
    } else {
      double a = fabs(v[i]);
      p[i] = a > 0.0 ? v[i] / a : 1.0;
      vc[I] = a;
    }
  }
  free(first);
  free(second);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.1 / Sec. 3.1: Galerkin product A_c = P^T A P                         */
/* ------------------------------------------------------------------------- */

typedef struct { int I, J, kmin, kmax, i; double t; float tf; } or_term;

static int term_cmp(const void *x, const void *y) {
  const or_term *a = (const or_term *)x, *b = (const or_term *)y;
  if (a->I != b->I) return a->I < b->I ? -1 : 1;
  if (a->J != b->J) return a->J < b->J ? -1 : 1;
  if (a->kmin != b->kmin) return a->kmin < b->kmin ? -1 : 1;
  if (a->kmax != b->kmax) return a->kmax < b->kmax ? -1 : 1;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  return 0;
}

typedef struct { int n; long nnz; int *rp; int *ci; double *val; } or_csr;

static void csr_free(or_csr *A) {
  free(A->rp); free(A->ci); free(A->val);
  A->rp = NULL; A->ci = NULL; A->val = NULL;
}

/* Builds Ac (allocated here) from A, agg and p; f32 != 0 forms and sums the terms in
 * binary32.  Returns OR_OK or OR_ERR_OOM. */
static int galerkin(const or_csr *A, int nc, const int *agg, const double *p, int f32, or_csr *Ac) {
  long m = A->nnz;
  or_term *T = (or_term *)xcalloc((size_t)m, sizeof(or_term));
  if (!T) return OR_ERR_OOM;
  long q = 0;
  for (int i = 0; i < A->n; ++i)
    for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
      int j = A->ci[k];
      T[q].I = agg[i];
      T[q].J = agg[j];
      T[q].kmin = i < j ? i : j;
      T[q].kmax = i < j ? j : i;
      T[q].i = i;
      T[q].t = (p[i] * p[j]) * A->val[k];
      {
        const float pi = (float)p[i], pj = (float)p[j], a = (float)A->val[k];
        const float pp = pi * pj;
        T[q].tf = pp * a;
      }
      ++q;
    }
  qsort(T, (size_t)m, sizeof(or_term), term_cmp);
  long nnzc = 0;
  for (long e = 0; e < m; ++e)
    if (e == 0 || T[e].I != T[e - 1].I || T[e].J != T[e - 1].J) ++nnzc;
  Ac->n = nc;
  Ac->nnz = nnzc;
  Ac->rp = (int *)xcalloc((size_t)nc + 1, sizeof(int));
  Ac->ci = (int *)xcalloc((size_t)nnzc, sizeof(int));
  Ac->val = (double *)xcalloc((size_t)nnzc, sizeof(double));
  if (!Ac->rp || !Ac->ci || !Ac->val) { csr_free(Ac); free(T); return OR_ERR_OOM; }
  long out = -1;
  float accf = 0.0f;
  for (long e = 0; e < m; ++e) {
    if (e == 0 || T[e].I != T[e - 1].I || T[e].J != T[e - 1].J) {
      ++out;
      Ac->ci[out] = T[e].J;
      Ac->val[out] = 0.0;
      accf = 0.0f;
      Ac->rp[T[e].I + 1]++;
    }
    if (f32) {
      accf = accf + T[e].tf;
      Ac->val[out] = (double)accf;
    } else {
      Ac->val[out] = Ac->val[out] + T[e].t;
    }
  }
  for (int I = 0; I < nc; ++I) Ac->rp[I + 1] += Ac->rp[I];
  free(T);
  return OR_OK;
}

/* C entry: count of A_c nonzeros, then fill (caller allocates). */
long or_galerkin_nnz(int n, const int *rp, const int *ci, const double *val, int nc,
                     const int *agg, const double *p) {
  or_csr A = {n, rp[n], (int *)rp, (int *)ci, (double *)val}, Ac = {0};
  if (galerkin(&A, nc, agg, p, 0, &Ac) != OR_OK) return -1;
  long z = Ac.nnz;
  csr_free(&Ac);
  return z;
}

int or_galerkin(int n, const int *rp, const int *ci, const double *val, int nc,
                const int *agg, const double *p, int f32, int *rpc, int *cic, double *valc) {
  or_csr A = {n, rp[n], (int *)rp, (int *)ci, (double *)val}, Ac = {0};
  int st = galerkin(&A, nc, agg, p, f32, &Ac);
  if (st != OR_OK) return st;
  memcpy(rpc, Ac.rp, sizeof(int) * ((size_t)nc + 1));
  memcpy(cic, Ac.ci, sizeof(int) * (size_t)Ac.nnz);
  memcpy(valc, Ac.val, sizeof(double) * (size_t)Ac.nnz);
  csr_free(&Ac);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* The hierarchy (Sec. 2.1 setup phase, Sec. 5 parameters)                    */
/* ------------------------------------------------------------------------- */

typedef struct {
  or_csr A;          /* A^k */
  double *v;         /* smooth vector restricted to this level */
  double *dl1;       /* l1 row norms */
  int *agg;          /* composed aggregate map to level k+1 (NULL on the coarsest) */
  double *p;         /* composed prolongator values (NULL on the coarsest) */
  int nsweeps;       /* sweeps done to build level k+1 */
  int sweep_n[OR_MAX_SWEEPS];       /* operator size each sweep matched on */
  int sweep_pairs[OR_MAX_SWEEPS];
  int *sweep_mate[OR_MAX_SWEEPS];   /* matching of each sweep */
} or_level;

typedef struct {
  int nl;
  or_level lev[OR_MAX_LEVELS];
  int pre, post, coarse;  /* l1-Jacobi sweeps */
  int gamma;              /* recursive calls per level: 1 = V-cycle, 2 = W-cycle */
} or_hier;

static double *l1_norms(const or_csr *A) {
  double *d = (double *)xcalloc((size_t)A->n, sizeof(double));
  if (!d) return NULL;
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) s = s + fabs(A->val[k]);
    d[i] = s;
  }
  return d;
}

void or_free(or_hier *h) {
  if (!h) return;
  for (int k = 0; k < h->nl; ++k) {
    or_level *L = &h->lev[k];
    csr_free(&L->A);
    free(L->v); free(L->dl1); free(L->agg); free(L->p);
    for (int s = 0; s < OR_MAX_SWEEPS; ++s) free(L->sweep_mate[s]);
  }
  free(h);
}

/* The paper's default coarse size (Sec. 5, solver settings): floor(40 n^(1/3)), taken as
 * the largest m with m^3 <= 64000 n (40^3 = 64000), by bisection on integers so that no
 * rounding of a floating cube root enters. */
int or_paper_coarse_max(int n) {
  const long long X = 64000LL * (long long)n;
  long long lo = 0, hi = 1LL << 21;  /* hi^3 > 64000 * 2^31 */
  while (lo < hi) {
    const long long mid = (lo + hi + 1) / 2;
    if (mid * mid * mid <= X) lo = mid;
    else hi = mid - 1;
  }
  return (int)lo;
}

/* Build the hierarchy: levels while n_k > coarse_max and nl < max_levels; each level
 * does `sweeps` pairwise matching sweeps; stops early when a sweep forms no pair, and,
 * when stall_ratio > 0, after a level whose coarsening ratio n_k / n_{k+1} is below it.
 * galerkin_fp32_from = k >= 1 forms the operators of levels k, k+1, ... (and the
 * intermediate operators of their sweeps) with the binary32 Galerkin product; 0: none. */
or_hier *or_setup(int n, const int *rp, const int *ci, const double *val, const double *v,
                  int sweeps, int coarse_max, int max_levels, double stall_ratio,
                  int galerkin_fp32_from, int *status) {
  *status = OR_OK;
  if (coarse_max == -1 && n > 0) coarse_max = or_paper_coarse_max(n);  /* -1: the paper's default */
  if (n <= 0 || sweeps < 1 || sweeps > OR_MAX_SWEEPS || max_levels < 1 || coarse_max < 0 ||
      max_levels > OR_MAX_LEVELS || or_check_csr(n, rp, ci) != OR_OK) {
    *status = OR_ERR_ARG;
    return NULL;
  }
  or_hier *h = (or_hier *)xcalloc(1, sizeof(or_hier));
  if (!h) { *status = OR_ERR_OOM; return NULL; }
  h->pre = 1; h->post = 1; h->coarse = 20; h->gamma = 1;
  long nnz = rp[n];
  or_level *L0 = &h->lev[0];
  L0->A.n = n;
  L0->A.nnz = nnz;
  L0->A.rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
  L0->A.ci = (int *)xcalloc((size_t)nnz, sizeof(int));
  L0->A.val = (double *)xcalloc((size_t)nnz, sizeof(double));
  L0->v = (double *)xcalloc((size_t)n, sizeof(double));
  memcpy(L0->A.rp, rp, sizeof(int) * ((size_t)n + 1));
  memcpy(L0->A.ci, ci, sizeof(int) * (size_t)nnz);
  memcpy(L0->A.val, val, sizeof(double) * (size_t)nnz);
  memcpy(L0->v, v, sizeof(double) * (size_t)n);
  L0->dl1 = l1_norms(&L0->A);
  h->nl = 1;

  while (h->nl < max_levels && h->lev[h->nl - 1].A.n > coarse_max) {
    or_level *F = &h->lev[h->nl - 1];
    int nf = F->A.n;
    /* composed prolongator, starts as the identity */
    int *agg_tot = (int *)xcalloc((size_t)nf, sizeof(int));
    double *p_tot = (double *)xcalloc((size_t)nf, sizeof(double));
    for (int i = 0; i < nf; ++i) { agg_tot[i] = i; p_tot[i] = 1.0; }
    or_csr cur = F->A;  /* borrowed for sweep 1 */
    int own_cur = 0;
    double *vcur = F->v;
    int own_v = 0;
    int done_sweeps = 0;
    for (int s = 0; s < sweeps; ++s) {
      int ns = cur.n;
      double *w = (double *)xcalloc((size_t)cur.nnz, sizeof(double));
      int *mate = (int *)xcalloc((size_t)ns, sizeof(int));
      int st = or_edge_weights(ns, cur.rp, cur.ci, cur.val, vcur, w);
      if (st == OR_OK) st = or_greedy_match(ns, cur.rp, cur.ci, w, mate);
      free(w);
      if (st != OR_OK) { *status = st; free(mate); break; }
      int *agg = (int *)xcalloc((size_t)ns, sizeof(int));
      int np = 0, nsg = 0;
      int nc = or_aggregate(ns, mate, agg, &np, &nsg);
      F->sweep_n[s] = ns;
      F->sweep_pairs[s] = np;
      F->sweep_mate[s] = mate;
      if (np == 0) { free(agg); break; }
      double *p = (double *)xcalloc((size_t)ns, sizeof(double));
      double *vc = (double *)xcalloc((size_t)nc, sizeof(double));
      or_prolongator(ns, nc, agg, vcur, p, vc);
      or_csr next = {0};
      st = galerkin(&cur, nc, agg, p, galerkin_fp32_from > 0 && h->nl >= galerkin_fp32_from, &next);
      if (st != OR_OK) { *status = st; free(agg); free(p); free(vc); break; }
      /* compose: row i of P_1...P_s has column agg_s[agg_tot[i]] and value
       * p_tot[i] * p_s[agg_tot[i]] */
      for (int i = 0; i < nf; ++i) {
        int a = agg_tot[i];
        p_tot[i] = p_tot[i] * p[a];
        agg_tot[i] = agg[a];
      }
      if (own_cur) csr_free(&cur);
      if (own_v) free(vcur);
      cur = next;
      own_cur = 1;
      vcur = vc;
      own_v = 1;
      free(agg);
      free(p);
      ++done_sweeps;
    }
    F->nsweeps = done_sweeps;
    if (*status != OR_OK || done_sweeps == 0) {
      if (own_cur) csr_free(&cur);
      if (own_v) free(vcur);
      free(agg_tot);
      free(p_tot);
      break;
    }
    F->agg = agg_tot;
    F->p = p_tot;
    or_level *C = &h->lev[h->nl];
    C->A = cur;
    C->v = vcur;
    C->dl1 = l1_norms(&C->A);
    h->nl++;
    if (F->sweep_pairs[done_sweeps - 1] == 0 || done_sweeps < sweeps) break;
    if (stall_ratio > 0.0 && (double)F->A.n < stall_ratio * (double)C->A.n) break;
  }
  if (*status != OR_OK) { or_free(h); return NULL; }
  return h;
}

void or_set_cycle(or_hier *h, int pre, int post, int coarse) {
  h->pre = pre; h->post = post; h->coarse = coarse;
}

void or_set_gamma(or_hier *h, int gamma) { h->gamma = gamma; }
int or_num_levels(const or_hier *h) { return h->nl; }
int or_level_n(const or_hier *h, int k) { return h->lev[k].A.n; }
long or_level_nnz(const or_hier *h, int k) { return h->lev[k].A.nnz; }
int or_level_sweeps(const or_hier *h, int k) { return h->lev[k].nsweeps; }
int or_sweep_n(const or_hier *h, int k, int s) { return h->lev[k].sweep_n[s]; }

/* Copies level k out; agg and p only when k < nl-1 (pass NULL otherwise). */
void or_level_export(const or_hier *h, int k, int *rp, int *ci, double *val, double *v,
                     double *dl1, int *agg, double *p) {
  const or_level *L = &h->lev[k];
  int n = L->A.n;
  if (rp) memcpy(rp, L->A.rp, sizeof(int) * ((size_t)n + 1));
  if (ci) memcpy(ci, L->A.ci, sizeof(int) * (size_t)L->A.nnz);
  if (val) memcpy(val, L->A.val, sizeof(double) * (size_t)L->A.nnz);
  if (v) memcpy(v, L->v, sizeof(double) * (size_t)n);
  if (dl1) memcpy(dl1, L->dl1, sizeof(double) * (size_t)n);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int) * (size_t)n);
  if (p && L->p) memcpy(p, L->p, sizeof(double) * (size_t)n);
}

void or_sweep_mate(const or_hier *h, int k, int s, int *mate) {
  memcpy(mate, h->lev[k].sweep_mate[s], sizeof(int) * (size_t)h->lev[k].sweep_n[s]);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2: l1-Jacobi;  Sec. 2.1, Algorithm 1: V-cycle                        */
/* ------------------------------------------------------------------------- */

static void spmv(const or_csr *A, const double *x, double *y) {
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) s = s + A->val[k] * x[A->ci[k]];
    y[i] = s;
  }
}

/* x <- x + D^{-1}(b - A x), all rows from the old x; tmp has n entries. */
static void l1_jacobi_sweep(const or_csr *A, const double *d, const double *b, double *x,
                            double *tmp) {
  spmv(A, x, tmp);
  for (int i = 0; i < A->n; ++i) tmp[i] = x[i] + (b[i] - tmp[i]) / d[i];
  memcpy(x, tmp, sizeof(double) * (size_t)A->n);
}

void or_l1_jacobi(const or_hier *h, int k, const double *b, double *x, int sweeps) {
  const or_level *L = &h->lev[k];
  double *tmp = (double *)xcalloc((size_t)L->A.n, sizeof(double));
  for (int s = 0; s < sweeps; ++s) l1_jacobi_sweep(&L->A, L->dl1, b, x, tmp);
  free(tmp);
}

/* One multigrid cycle on level k (Algorithm 1) from the starting guess in x: pre-smoothing,
 * the coarse correction x += P x^{k+1} where x^{k+1} comes from gamma cycles on level k+1
 * started from zero (gamma = 1: V-cycle; 2: W-cycle, the second cycle starting from the
 * first one's result), and post-smoothing.  The coarsest level does `coarse` l1-Jacobi
 * sweeps from the starting guess. */
static void cycle(const or_hier *h, int k, const double *b, double *x) {
  const or_level *L = &h->lev[k];
  int n = L->A.n;
  double *tmp = (double *)xcalloc((size_t)n, sizeof(double));
  if (k == h->nl - 1) {
    for (int s = 0; s < h->coarse; ++s) l1_jacobi_sweep(&L->A, L->dl1, b, x, tmp);
    free(tmp);
    return;
  }
  for (int s = 0; s < h->pre; ++s) l1_jacobi_sweep(&L->A, L->dl1, b, x, tmp);
  /* b^{k+1} = P^T (b - A x) */
  int nc = h->lev[k + 1].A.n;
  double *bc = (double *)xcalloc((size_t)nc, sizeof(double));
  double *xc = (double *)xcalloc((size_t)nc, sizeof(double));
  spmv(&L->A, x, tmp);
  for (int i = 0; i < n; ++i) bc[L->agg[i]] = bc[L->agg[i]] + L->p[i] * (b[i] - tmp[i]);
  for (int g = 0; g < h->gamma; ++g) cycle(h, k + 1, bc, xc);
  for (int i = 0; i < n; ++i) x[i] = x[i] + L->p[i] * xc[L->agg[i]];
  for (int s = 0; s < h->post; ++s) l1_jacobi_sweep(&L->A, L->dl1, b, x, tmp);
  free(bc);
  free(xc);
  free(tmp);
}

/* x^k = cycle(k, b^k) with x^k starting from zero. */
static void vcycle(const or_hier *h, int k, const double *b, double *x) {
  memset(x, 0, sizeof(double) * (size_t)h->lev[k].A.n);
  cycle(h, k, b, x);
}

void or_vcycle(const or_hier *h, const double *r, double *w) { vcycle(h, 0, r, w); }

/* ------------------------------------------------------------------------- */
/* Sec. 3.2, Algorithm 3: flexible (preconditioned) CG                        */
/* ------------------------------------------------------------------------- */

static double dot(int n, const double *x, const double *y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = s + x[i] * y[i];
  return s;
}

/* prec: 0 = AMG V-cycle, 1 = identity, 2 = one l1-Jacobi application D^{-1}.
 * x holds u_0 on entry and the solution on exit.  iters = number of updates of u. */
int or_pcg(const or_hier *h, const double *b, double *x, double rtol, int itmax, int prec,
           int *iters, double *relres_rec, double *relres_true) {
  const or_level *L = &h->lev[0];
  const or_csr *A = &L->A;
  int n = A->n;
  double *r = (double *)xcalloc((size_t)n, sizeof(double));
  double *w = (double *)xcalloc((size_t)n, sizeof(double));
  double *d = (double *)xcalloc((size_t)n, sizeof(double));
  double *v = (double *)xcalloc((size_t)n, sizeof(double));
  double *q = (double *)xcalloc((size_t)n, sizeof(double));
  int status = OR_ERR_NOT_CONVERGED, it = 0;
  double nb = sqrt(dot(n, b, b));
  spmv(A, x, r);
  for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
  double nr = sqrt(dot(n, r, r));
  double rho_prev = 0.0;
  if (nb == 0.0 || nr <= rtol * nb) status = OR_OK;
  while (status != OR_OK && it < itmax) {
    /* w_i = B(r_i), v_i = A w_i */
    if (prec == 0) vcycle(h, 0, r, w);
    else if (prec == 1) memcpy(w, r, sizeof(double) * (size_t)n);
    else for (int i = 0; i < n; ++i) w[i] = r[i] / L->dl1[i];
    spmv(A, w, v);
    double alpha = dot(n, w, r), beta = dot(n, w, v);
    double rho, coef;
    if (it == 0) {
      rho = beta;
      coef = 0.0;
      memcpy(d, w, sizeof(double) * (size_t)n);
      memcpy(q, v, sizeof(double) * (size_t)n);
    } else {
      double gamma = dot(n, w, q);
      rho = beta - gamma * gamma / rho_prev;
      coef = gamma / rho_prev;
      for (int i = 0; i < n; ++i) d[i] = w[i] - coef * d[i];
      for (int i = 0; i < n; ++i) q[i] = v[i] - coef * q[i];
    }
    if (!(rho > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    double step = alpha / rho;
    for (int i = 0; i < n; ++i) x[i] = x[i] + step * d[i];
    for (int i = 0; i < n; ++i) r[i] = r[i] - step * q[i];
    rho_prev = rho;
    ++it;
    nr = sqrt(dot(n, r, r));
    if (nr <= rtol * nb) status = OR_OK;
  }
  *iters = it;
  *relres_rec = nb > 0.0 ? nr / nb : 0.0;
  spmv(A, x, v);
  for (int i = 0; i < n; ++i) v[i] = b[i] - v[i];
  *relres_true = nb > 0.0 ? sqrt(dot(n, v, v)) / nb : 0.0;
  free(r); free(w); free(d); free(v); free(q);
  return status;
}

/* Vcmplx = sum_k nnz(A^k) / nnz(A^1);  cratio = (1/nl) sum_{k>=2} n_{k-1}/n_k (Sec. 5.2). */
void or_stats(const or_hier *h, double *vcmplx, double *cratio) {
  double z = 0.0, c = 0.0;
  for (int k = 0; k < h->nl; ++k) z += (double)h->lev[k].A.nnz;
  for (int k = 1; k < h->nl; ++k) c += (double)h->lev[k - 1].A.n / (double)h->lev[k].A.n;
  *vcmplx = z / (double)h->lev[0].A.nnz;
  *cratio = c / (double)h->nl;
}
