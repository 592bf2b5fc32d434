/*
 * CPU oracle for the AMG-preconditioned flexible CG of arXiv:2303.02352.
 * TEST INFRASTRUCTURE ONLY (see orc.h): plain serial FP64 C, natural index
 * order, no blocking or fusion.  Compile with -ffp-contract=off so that no
 * multiply-add is fused: the matching weights must be reproducible bit for bit.
 *
 * Readings of the paper that this file implements (each is also listed in the
 * design notes of the repository):
 *  - matching weight (Sec. 3.1 says only "a suitable function of a smooth
 *    vector w and of the matrix entries"): the compatible weighted-matching
 *    weight w_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2) with w = 1 on
 *    every level; edges with weight <= 0 are never matched;
 *  - strict total order on edges: larger weight first, ties by the smaller
 *    (min endpoint, max endpoint) pair; the half-approximate matching is then
 *    the greedy matching in that order (the suitor algorithm the paper uses
 *    reaches exactly this matching under a strict order);
 *  - pairwise prolongator with unit entries (P 1 = 1), aggregate ids in order of
 *    their smallest member;
 *  - Galerkin sums in canonical order (fine rows ascending, then CSR positions
 *    ascending), upper triangle computed and mirrored to the lower one;
 *  - l1-Jacobi diagonal M_ii = sum_j |a_ij| (Sec. 3.1 prints the sum without the
 *    absolute value, which vanishes on interior Poisson rows);
 *  - V-cycle from the operator B^k of Sec. 3.1: nu pre-sweeps of M^{-1} from
 *    zero, restriction of the residual, recursion, prolongation, nu post-sweeps;
 *    the coarsest level applies a fixed number of l1-Jacobi sweeps (Sec. 3.1,
 *    Sec. 5);
 *  - Alg. 1 with the stop test |r|_2/|b|_2 < tol after each update; the
 *    iteration count is the number of updates of u.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 64
#define ORC_MAXPAIR 256

typedef struct {
  int n;
  int64_t nnz;
  int32_t* rp;
  int32_t* ci;
  double* v;
} ocsr;

struct orc_hier {
  orc_params p;
  int nl;
  ocsr A[ORC_MAXL];
  int32_t* agg[ORC_MAXL];  /* level k row -> level k+1 row (composed pairwise maps) */
  double* l1[ORC_MAXL];    /* l1 row norms */
  double* omega[ORC_MAXL]; /* per-row damping, 1 by default */
  double* dinv[ORC_MAXL];  /* omega / l1 */
  double* wsv[ORC_MAXL];   /* smooth vector w^k of the w-normalised prolongators (NULL for unit P) */
  float* fval[ORC_MAXL];   /* mixed precision: rounded level values */
  float* fdinv[ORC_MAXL];
  double* chol;            /* dense Cholesky factor of the coarsest matrix (pins only) */
  int npair;
  int pair_n[ORC_MAXPAIR];
};

void orc_params_default(orc_params* p) {
  p->aggr_steps = 3;     /* Listing 1: aggrsweeps = 2 (pairs of pairs of pairs), Sec. 5: size <= 8 */
  p->max_levels = 39;    /* Listing 1 */
  p->coarse_size = 0;    /* Sec. 5: 40 * nd */
  p->pre_sweeps = 4;     /* Sec. 5 */
  p->post_sweeps = 4;
  p->coarse_sweeps = 20; /* Sec. 5 */
  p->coarse_solver = ORC_COARSE_L1JACOBI;
  p->precision = ORC_FP64;
  p->true_res_every = 50;
  p->num_parts = 1;
  p->cycle = 0;
  p->relax_type = 4;     /* Listing 1: relax_type 4 (l1-Jacobi) */
  p->prolong_scale = ORC_PROLONG_UNIT;
}

static void* xcalloc(size_t n, size_t s) {
  void* q = calloc(n ? n : 1, s);
  if (!q) abort();
  return q;
}

/* ------------------------------------------------------------------ */
/* matching weights (Alg. 3 "apply MWM(A^k, w^k)"; weight formula is a reading) */

static int find_diag(const int32_t* rp, const int32_t* ci, int i) {
  for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) return p;
  return -1;
}

int orc_weights(int n, const int32_t* rp, const int32_t* ci, const double* v, double* wgt) {
  double* diag = (double*)xcalloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) {
    int p = find_diag(rp, ci, i);
    if (p < 0) {
      free(diag);
      return ORC_ERR_ARG;
    }
    diag[i] = v[p];
  }
  const double wi = 1.0, wj = 1.0; /* unit smooth vector on every level */
  for (int i = 0; i < n; ++i) {
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      if (j == i || v[p] == 0.0) {
        wgt[p] = 0.0; /* not an edge */
        continue;
      }
      double t = 2.0 * v[p];
      t = t * wi;
      t = t * wj;
      double den = diag[i] * wi * wi + diag[j] * wj * wj;
      wgt[p] = 1.0 - t / den;
    }
  }
  free(diag);
  return ORC_OK;
}

/* decoupled aggregation (Sec. 4.1): every task matches only its own rows, so
 * an edge whose ends lie in different row blocks is not an edge */
static int part_of(int i, int np, const int32_t* bnd) {
  int p = 0;
  while (p + 1 < np && i >= bnd[p + 1]) ++p;
  return p;
}

int orc_weights_parts(int n, const int32_t* rp, const int32_t* ci, const double* v, int np, const int32_t* bnd,
                      double* wgt) {
  int st = orc_weights(n, rp, ci, v, wgt);
  if (st != ORC_OK || np <= 1) return st;
  for (int i = 0; i < n; ++i) {
    int pi = part_of(i, np, bnd);
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (part_of(ci[p], np, bnd) != pi) wgt[p] = 0.0;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* greedy matching under the strict order (weight desc, (u,v) lexicographic asc) */

typedef struct {
  double w;
  int32_t u, v;
} oedge;

static int edge_cmp(const void* a, const void* b) {
  const oedge* x = (const oedge*)a;
  const oedge* y = (const oedge*)b;
  if (x->w > y->w) return -1;
  if (x->w < y->w) return 1;
  if (x->u != y->u) return x->u < y->u ? -1 : 1;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  return 0;
}

int orc_match_greedy(int n, const int32_t* rp, const int32_t* ci, const double* wgt, int32_t* mate) {
  int64_t ne = 0;
  for (int i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] > i && wgt[p] > 0.0) ++ne;
  oedge* e = (oedge*)xcalloc((size_t)ne, sizeof(oedge));
  int64_t k = 0;
  for (int i = 0; i < n; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] > i && wgt[p] > 0.0) {
        e[k].w = wgt[p];
        e[k].u = i;
        e[k].v = ci[p];
        ++k;
      }
  qsort(e, (size_t)ne, sizeof(oedge), edge_cmp);
  for (int i = 0; i < n; ++i) mate[i] = -1;
  int pairs = 0;
  for (int64_t q = 0; q < ne; ++q) {
    if (mate[e[q].u] < 0 && mate[e[q].v] < 0) {
      mate[e[q].u] = e[q].v;
      mate[e[q].v] = e[q].u;
      ++pairs;
    }
  }
  free(e);
  return pairs;
}

/* ------------------------------------------------------------------ */
/* pairwise aggregation: vertex i opens an aggregate iff it is unmatched or the
 * smaller end of its pair; ids follow increasing i */

int orc_aggregate(int n, const int32_t* mate, int32_t* agg) {
  int nc = 0;
  for (int i = 0; i < n; ++i) {
    if (mate[i] < 0 || i < mate[i]) {
      agg[i] = nc;
      if (mate[i] >= 0) agg[mate[i]] = nc;
      ++nc;
    }
  }
  return nc;
}

/* ------------------------------------------------------------------ */
/* Galerkin product A_c = P^T A P with unit piecewise-constant P (Alg. 3) */

static int int_cmp(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

int64_t orc_galerkin(int n, const int32_t* rp, const int32_t* ci, const double* v,
                     const int32_t* agg, int nc, int32_t* rp_c, int32_t* ci_c, double* v_c) {
  /* members of each aggregate, ascending */
  int32_t* mptr = (int32_t*)xcalloc((size_t)nc + 1, sizeof(int32_t));
  int32_t* mem = (int32_t*)xcalloc((size_t)n, sizeof(int32_t));
  for (int i = 0; i < n; ++i) mptr[agg[i] + 1]++;
  for (int I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
  int32_t* fill = (int32_t*)xcalloc((size_t)nc, sizeof(int32_t));
  for (int i = 0; i < n; ++i) mem[mptr[agg[i]] + fill[agg[i]]++] = i;

  int32_t* mark = (int32_t*)xcalloc((size_t)nc, sizeof(int32_t));
  for (int I = 0; I < nc; ++I) mark[I] = -1;
  double* acc = (double*)xcalloc((size_t)nc, sizeof(double));
  int32_t* list = (int32_t*)xcalloc((size_t)nc, sizeof(int32_t));

  int64_t nnz_c = 0;
  for (int I = 0; I < nc; ++I) {
    int cnt = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) {
      int i = mem[m];
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int J = agg[ci[p]];
        if (mark[J] != I) {
          mark[J] = I;
          acc[J] = v[p]; /* the sum starts from its first term */
          list[cnt++] = J;
        } else {
          acc[J] = acc[J] + v[p];
        }
      }
    }
    qsort(list, (size_t)cnt, sizeof(int32_t), int_cmp);
    if (rp_c) {
      rp_c[I] = (int32_t)nnz_c;
      for (int q = 0; q < cnt; ++q) {
        ci_c[nnz_c + q] = list[q];
        v_c[nnz_c + q] = acc[list[q]];
      }
    }
    nnz_c += cnt;
  }
  if (rp_c) {
    rp_c[nc] = (int32_t)nnz_c;
    /* mirror: A_c(I,J) := A_c(J,I) for J < I, so that A_c is bitwise symmetric */
    for (int I = 0; I < nc; ++I) {
      for (int32_t p = rp_c[I]; p < rp_c[I + 1]; ++p) {
        int J = ci_c[p];
        if (J >= I) continue;
        int32_t lo = rp_c[J], hi = rp_c[J + 1] - 1, found = -1;
        while (lo <= hi) {
          int32_t mid = lo + (hi - lo) / 2;
          if (ci_c[mid] == I) {
            found = mid;
            break;
          }
          if (ci_c[mid] < I) lo = mid + 1;
          else hi = mid - 1;
        }
        if (found >= 0) v_c[p] = v_c[found];
      }
    }
  }
  free(mptr);
  free(mem);
  free(fill);
  free(mark);
  free(acc);
  free(list);
  return nnz_c;
}

/* ------------------------------------------------------------------ */
/* bf16 round-to-nearest-even of a float (bias-and-truncate method) */

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

float orc_round_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan: truncate, keep nan quiet */
    if (u & 0x007fffffu) u |= 0x00400000u;
    u &= 0xffff0000u;
  } else {
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
  }
  float y;
  memcpy(&y, &u, 4);
  return y;
}

/* ------------------------------------------------------------------ */
/* hierarchy construction: Alg. 3 with s-fold composition of pairwise steps */

static void csr_copy(ocsr* dst, int n, const int32_t* rp, const int32_t* ci, const double* v) {
  dst->n = n;
  dst->nnz = rp[n];
  dst->rp = (int32_t*)xcalloc((size_t)n + 1, sizeof(int32_t));
  dst->ci = (int32_t*)xcalloc((size_t)dst->nnz, sizeof(int32_t));
  dst->v = (double*)xcalloc((size_t)dst->nnz, sizeof(double));
  memcpy(dst->rp, rp, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(dst->ci, ci, sizeof(int32_t) * (size_t)dst->nnz);
  memcpy(dst->v, v, sizeof(double) * (size_t)dst->nnz);
}

static void csr_free(ocsr* a) {
  free(a->rp);
  free(a->ci);
  free(a->v);
  memset(a, 0, sizeof(*a));
}

/* l1 row norms and D = omega / M with M_ii = sum_j |a_ij| (l1-Jacobi) or
 * M_ii = a_ii (Jacobi, Listing 1 relax_type 0).
 *
 * w-normalised prolongators (Sec. 3.1: P's entries come from the smooth vector,
 * w^{k+1} = R w^k): P^k_{i,I} = w^k_i / |w^k restricted to I|, so
 * w^{k+1}_I = |w^k on I|_2 and, by induction from w^0 = 1, the normalised
 * level matrix is W_k^{-1} A^k W_k^{-1} (W_k = diag(w^k)) with A^k the
 * unit-prolongator matrix kept here.  Residuals, corrections and the error
 * propagation map into the unit coordinates through the same W_k, and there
 * the only change is the smoother diagonal: l1-Jacobi on the normalised
 * matrix becomes M_I = sum_J |a_IJ| w_I / w_J, while Jacobi (a_II) and the
 * matching weights (invariant under the scaling) are unchanged. */
static void level_diag(orc_hier* h, int k) {
  ocsr* A = &h->A[k];
  const double* w = h->wsv[k];
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0, d = 0.0, m = 0.0;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      s += fabs(A->v[p]);
      if (w) m += fabs(A->v[p]) * (w[i] / w[A->ci[p]]);
      if (A->ci[p] == i) d = A->v[p];
    }
    h->l1[k][i] = s;
    h->dinv[k][i] = h->omega[k][i] / (h->p.relax_type == 0 ? d : (w ? m : s));
  }
}

static void level_lowprec(orc_hier* h, int k) {
  ocsr* A = &h->A[k];
  free(h->fval[k]);
  free(h->fdinv[k]);
  h->fval[k] = NULL;
  h->fdinv[k] = NULL;
  if (h->p.precision == ORC_FP64 || k == h->nl - 1) return; /* coarsest stays FP64 */
  h->fval[k] = (float*)xcalloc((size_t)A->nnz, sizeof(float));
  h->fdinv[k] = (float*)xcalloc((size_t)A->n, sizeof(float));
  int bf = (h->p.precision == ORC_FP32_BF16FINE && k == 0);
  for (int64_t p = 0; p < A->nnz; ++p) {
    float f = (float)A->v[p];
    h->fval[k][p] = bf ? orc_round_bf16(f) : f;
  }
  for (int i = 0; i < A->n; ++i) h->fdinv[k][i] = (float)h->dinv[k][i];
}

static void build_chol(orc_hier* h) {
  ocsr* A = &h->A[h->nl - 1];
  int n = A->n;
  double* L = (double*)xcalloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i)
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) L[(size_t)i * n + A->ci[p]] = A->v[p];
  for (int j = 0; j < n; ++j) {
    double d = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    d = sqrt(d);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = L[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = s / d;
    }
  }
  h->chol = L;
}

orc_hier* orc_setup(int n, const int32_t* rp, const int32_t* ci, const double* v, const orc_params* p) {
  if (n <= 0 || !rp || !ci || !v || !p) return NULL;
  if (p->relax_type != 0 && p->relax_type != 4) return NULL;
  if (p->prolong_scale != ORC_PROLONG_UNIT && p->prolong_scale != ORC_PROLONG_W_NORMALIZED) return NULL;
  for (int i = 0; i < n; ++i)
    if (find_diag(rp, ci, i) < 0) return NULL;
  orc_hier* h = (orc_hier*)xcalloc(1, sizeof(orc_hier));
  h->p = *p;
  int cs = p->coarse_size > 0 ? p->coarse_size : 40 * (int)lround(cbrt((double)n));
  int s = p->aggr_steps > 0 ? p->aggr_steps : 1;

  csr_copy(&h->A[0], n, rp, ci, v);
  h->nl = 1;
  h->npair = 0;
  ocsr cur;
  csr_copy(&cur, n, rp, ci, v);
  int32_t* comp = (int32_t*)xcalloc((size_t)n, sizeof(int32_t)); /* level rows -> current rows */
  for (int i = 0; i < n; ++i) comp[i] = i;
  int comp_n = n;
  int group = 0;
  /* row blocks of the decoupled aggregation; block boundaries move to the
   * aggregate ids of the blocks' first rows after every pairwise step */
  int np = p->num_parts > 1 ? p->num_parts : 1;
  if (np > n) np = n;
  int32_t* bnd = (int32_t*)xcalloc((size_t)np + 1, sizeof(int32_t));
  for (int q = 0; q <= np; ++q) bnd[q] = (int32_t)(((int64_t)q * n) / np);

  while (cur.n > cs && h->nl < p->max_levels && h->nl < ORC_MAXL - 1 && h->npair < ORC_MAXPAIR) {
    double* wgt = (double*)xcalloc((size_t)cur.nnz, sizeof(double));
    int32_t* mate = (int32_t*)xcalloc((size_t)cur.n, sizeof(int32_t));
    int32_t* agg = (int32_t*)xcalloc((size_t)cur.n, sizeof(int32_t));
    orc_weights_parts(cur.n, cur.rp, cur.ci, cur.v, np, bnd, wgt);
    orc_match_greedy(cur.n, cur.rp, cur.ci, wgt, mate);
    int nc = orc_aggregate(cur.n, mate, agg);
    free(wgt);
    free(mate);
    if (nc == cur.n) { /* no edge matched: no progress */
      free(agg);
      break;
    }
    int64_t nnz_c = orc_galerkin(cur.n, cur.rp, cur.ci, cur.v, agg, nc, NULL, NULL, NULL);
    ocsr nxt;
    nxt.n = nc;
    nxt.nnz = nnz_c;
    nxt.rp = (int32_t*)xcalloc((size_t)nc + 1, sizeof(int32_t));
    nxt.ci = (int32_t*)xcalloc((size_t)nnz_c, sizeof(int32_t));
    nxt.v = (double*)xcalloc((size_t)nnz_c, sizeof(double));
    orc_galerkin(cur.n, cur.rp, cur.ci, cur.v, agg, nc, nxt.rp, nxt.ci, nxt.v);
    for (int i = 0; i < comp_n; ++i) comp[i] = agg[comp[i]];
    for (int q = 0; q < np; ++q) bnd[q] = bnd[q] < cur.n ? agg[bnd[q]] : nc;
    bnd[np] = nc;
    free(agg);
    csr_free(&cur);
    cur = nxt;
    h->pair_n[h->npair++] = cur.n;
    ++group;
    if (group == s || cur.n <= cs) {
      int k = h->nl;
      h->agg[k - 1] = comp;
      csr_copy(&h->A[k], cur.n, cur.rp, cur.ci, cur.v);
      h->nl++;
      comp = (int32_t*)xcalloc((size_t)cur.n, sizeof(int32_t));
      for (int i = 0; i < cur.n; ++i) comp[i] = i;
      comp_n = cur.n;
      group = 0;
    }
  }
  if (group > 0) {
    int k = h->nl;
    h->agg[k - 1] = comp;
    csr_copy(&h->A[k], cur.n, cur.rp, cur.ci, cur.v);
    h->nl++;
  } else {
    free(comp);
  }
  csr_free(&cur);
  free(bnd);

  if (p->prolong_scale == ORC_PROLONG_W_NORMALIZED) {
    /* w^0 = 1; w^{k+1}_I = sqrt(sum over i in I of (w^k_i)^2) */
    h->wsv[0] = (double*)xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) h->wsv[0][i] = 1.0;
    for (int k = 0; k + 1 < h->nl; ++k) {
      double* wc = (double*)xcalloc((size_t)h->A[k + 1].n, sizeof(double));
      for (int i = 0; i < h->A[k].n; ++i) wc[h->agg[k][i]] += h->wsv[k][i] * h->wsv[k][i];
      for (int c = 0; c < h->A[k + 1].n; ++c) wc[c] = sqrt(wc[c]);
      h->wsv[k + 1] = wc;
    }
  }
  for (int k = 0; k < h->nl; ++k) {
    int nk = h->A[k].n;
    h->l1[k] = (double*)xcalloc((size_t)nk, sizeof(double));
    h->dinv[k] = (double*)xcalloc((size_t)nk, sizeof(double));
    h->omega[k] = (double*)xcalloc((size_t)nk, sizeof(double));
    for (int i = 0; i < nk; ++i) h->omega[k][i] = 1.0;
    level_diag(h, k);
    level_lowprec(h, k);
  }
  if (p->coarse_solver == ORC_COARSE_DENSE_CHOL) build_chol(h);
  return h;
}

void orc_free(orc_hier* h) {
  if (!h) return;
  for (int k = 0; k < h->nl; ++k) {
    csr_free(&h->A[k]);
    free(h->agg[k]);
    free(h->l1[k]);
    free(h->wsv[k]);
    free(h->omega[k]);
    free(h->dinv[k]);
    free(h->fval[k]);
    free(h->fdinv[k]);
  }
  free(h->chol);
  free(h);
}

int orc_num_levels(const orc_hier* h) { return h->nl; }
int orc_level_n(const orc_hier* h, int k) { return h->A[k].n; }
int64_t orc_level_nnz(const orc_hier* h, int k) { return h->A[k].nnz; }
void orc_level_csr(const orc_hier* h, int k, int32_t* rp, int32_t* ci, double* v) {
  const ocsr* A = &h->A[k];
  memcpy(rp, A->rp, sizeof(int32_t) * ((size_t)A->n + 1));
  memcpy(ci, A->ci, sizeof(int32_t) * (size_t)A->nnz);
  memcpy(v, A->v, sizeof(double) * (size_t)A->nnz);
}
void orc_level_agg(const orc_hier* h, int k, int32_t* agg) {
  if (k < h->nl - 1) memcpy(agg, h->agg[k], sizeof(int32_t) * (size_t)h->A[k].n);
}
void orc_level_l1(const orc_hier* h, int k, double* l1) {
  memcpy(l1, h->l1[k], sizeof(double) * (size_t)h->A[k].n);
}
int orc_num_pairwise(const orc_hier* h) { return h->npair; }
int orc_pairwise_n(const orc_hier* h, int t) { return h->pair_n[t]; }

int orc_set_omega(orc_hier* h, int k, const double* omega) {
  if (k < 0 || k >= h->nl) return ORC_ERR_ARG;
  for (int i = 0; i < h->A[k].n; ++i) h->omega[k][i] = omega ? omega[i] : 1.0;
  level_diag(h, k);
  level_lowprec(h, k);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* FP64 V-cycle (Alg. 2 read through the operator B^k of Sec. 3.1) */

void orc_spmv(const orc_hier* h, int k, const double* x, double* y) {
  const ocsr* A = &h->A[k];
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
    y[i] = s;
  }
}

/* one l1-Jacobi sweep z <- z + D (r - A z), Jacobi (all rows from the old z) */
static void sweep_d(const ocsr* A, const double* D, const double* r, double* z, double* tmp) {
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * z[A->ci[p]];
    tmp[i] = z[i] + D[i] * (r[i] - s);
  }
  memcpy(z, tmp, sizeof(double) * (size_t)A->n);
}

static void chol_solve(const orc_hier* h, const double* r, double* z) {
  int n = h->A[h->nl - 1].n;
  const double* L = h->chol;
  for (int i = 0; i < n; ++i) {
    double s = r[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * z[k];
    z[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * z[k];
    z[i] = s / L[(size_t)i * n + i];
  }
}

static void smooth_from_zero_d(const ocsr* A, const double* D, const double* r, double* z, int sweeps, double* tmp) {
  if (sweeps <= 0) {
    memset(z, 0, sizeof(double) * (size_t)A->n);
    return;
  }
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n; ++i) z[i] = D[i] * r[i]; /* first sweep from z = 0 */
  for (int s = 1; s < sweeps; ++s) sweep_d(A, D, r, z, tmp);
}

static void vcycle_d(orc_hier* h, int k, const double* r, double* z) {
  const ocsr* A = &h->A[k];
  int n = A->n;
  double* tmp = (double*)xcalloc((size_t)n, sizeof(double));
  if (k == h->nl - 1) {
    if (h->p.coarse_solver == ORC_COARSE_DENSE_CHOL) chol_solve(h, r, z);
    else smooth_from_zero_d(A, h->dinv[k], r, z, h->p.coarse_sweeps, tmp);
    free(tmp);
    return;
  }
  int nc = h->A[k + 1].n;
  const int32_t* agg = h->agg[k];
  smooth_from_zero_d(A, h->dinv[k], r, z, h->p.pre_sweeps, tmp);
  /* residual, then restriction r_c = P^T (r - A z), members in ascending order */
  double* rc = (double*)xcalloc((size_t)nc, sizeof(double));
  double* zc = (double*)xcalloc((size_t)nc, sizeof(double));
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * z[A->ci[p]];
    tmp[i] = r[i] - s;
  }
  for (int i = 0; i < n; ++i) rc[agg[i]] += tmp[i];
  vcycle_d(h, k + 1, rc, zc);
  if (h->p.cycle == 2) {
    /* W-cycle: a second coarse correction on the updated coarse residual */
    double* rc2 = (double*)xcalloc((size_t)nc, sizeof(double));
    double* ec2 = (double*)xcalloc((size_t)nc, sizeof(double));
    orc_spmv(h, k + 1, zc, rc2);
    for (int J = 0; J < nc; ++J) rc2[J] = rc[J] - rc2[J];
    vcycle_d(h, k + 1, rc2, ec2);
    for (int J = 0; J < nc; ++J) zc[J] += ec2[J];
    free(rc2);
    free(ec2);
  }
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) z[i] += zc[agg[i]]; /* prolongation, unit P */
  for (int s = 0; s < h->p.post_sweeps; ++s) sweep_d(A, h->dinv[k], r, z, tmp);
  free(rc);
  free(zc);
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* mixed-precision V-cycle: level values and l1 diagonal in float (bf16 values
 * on level 0 if asked), float arithmetic; the coarsest level stays FP64 and
 * takes a float-rounded input */

static void sweep_f(const ocsr* A, const float* val, const float* D, const float* r, float* z, float* tmp) {
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n; ++i) {
    float s = 0.0f;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += val[p] * z[A->ci[p]];
    tmp[i] = z[i] + D[i] * (r[i] - s);
  }
  memcpy(z, tmp, sizeof(float) * (size_t)A->n);
}

static void vcycle_f(orc_hier* h, int k, const float* r, float* z) {
  const ocsr* A = &h->A[k];
  int n = A->n;
  if (k == h->nl - 1) {
    double* rd = (double*)xcalloc((size_t)n, sizeof(double));
    double* zd = (double*)xcalloc((size_t)n, sizeof(double));
    double* tmp = (double*)xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) rd[i] = (double)r[i];
    if (h->p.coarse_solver == ORC_COARSE_DENSE_CHOL) chol_solve(h, rd, zd);
    else smooth_from_zero_d(A, h->dinv[k], rd, zd, h->p.coarse_sweeps, tmp);
    for (int i = 0; i < n; ++i) z[i] = (float)zd[i];
    free(rd);
    free(zd);
    free(tmp);
    return;
  }
  const float* val = h->fval[k];
  const float* D = h->fdinv[k];
  int nc = h->A[k + 1].n;
  const int32_t* agg = h->agg[k];
  float* tmp = (float*)xcalloc((size_t)n, sizeof(float));
  if (h->p.pre_sweeps <= 0) {
    memset(z, 0, sizeof(float) * (size_t)n);
  } else {
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) z[i] = D[i] * r[i];
    for (int s = 1; s < h->p.pre_sweeps; ++s) sweep_f(A, val, D, r, z, tmp);
  }
  float* rc = (float*)xcalloc((size_t)nc, sizeof(float));
  float* zc = (float*)xcalloc((size_t)nc, sizeof(float));
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += val[p] * z[A->ci[p]];
    tmp[i] = r[i] - s;
  }
  for (int i = 0; i < n; ++i) rc[agg[i]] += tmp[i];
  vcycle_f(h, k + 1, rc, zc);
  if (h->p.cycle == 2) {
    float* rc2 = (float*)xcalloc((size_t)nc, sizeof(float));
    float* ec2 = (float*)xcalloc((size_t)nc, sizeof(float));
    const ocsr* C = &h->A[k + 1];
    if (k + 1 == h->nl - 1) { /* the coarsest level: FP64 values, float vectors */
      for (int J = 0; J < nc; ++J) {
        double s = 0.0;
        for (int32_t q = C->rp[J]; q < C->rp[J + 1]; ++q) s += C->v[q] * (double)zc[C->ci[q]];
        rc2[J] = (float)((double)rc[J] - s);
      }
    } else {
      for (int J = 0; J < nc; ++J) {
        float s = 0.0f;
        for (int32_t q = C->rp[J]; q < C->rp[J + 1]; ++q) s += h->fval[k + 1][q] * zc[C->ci[q]];
        rc2[J] = rc[J] - s;
      }
    }
    vcycle_f(h, k + 1, rc2, ec2);
    for (int J = 0; J < nc; ++J) zc[J] += ec2[J];
    free(rc2);
    free(ec2);
  }
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) z[i] += zc[agg[i]];
  for (int s = 0; s < h->p.post_sweeps; ++s) sweep_f(A, val, D, r, z, tmp);
  free(rc);
  free(zc);
  free(tmp);
}

void orc_vcycle(orc_hier* h, const double* r, double* z) {
  int n = h->A[0].n;
  if (h->p.precision == ORC_FP64 || h->nl == 1) {
    vcycle_d(h, 0, r, z);
    return;
  }
  float* rf = (float*)xcalloc((size_t)n, sizeof(float));
  float* zf = (float*)xcalloc((size_t)n, sizeof(float));
  for (int i = 0; i < n; ++i) rf[i] = (float)r[i];
  vcycle_f(h, 0, rf, zf);
  for (int i = 0; i < n; ++i) z[i] = (double)zf[i];
  free(rf);
  free(zf);
}

/* ------------------------------------------------------------------ */
/* Alg. 1: flexible (Notay) preconditioned CG */

static double dot(int n, const double* x, const double* y) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

static void residual(const orc_hier* h, const double* b, const double* u, double* r) {
  orc_spmv(h, 0, u, r);
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < h->A[0].n; ++i) r[i] = b[i] - r[i];
}

static void apply_B(orc_hier* h, int precflag, const double* r, double* w) {
  if (precflag) orc_vcycle(h, r, w);
  else memcpy(w, r, sizeof(double) * (size_t)h->A[0].n); /* B = I: plain CG */
}

int orc_fcg(orc_hier* h, const double* b, double* u, double tol, int maxit, int precflag,
            int* iters, double* hist, double* true_rel) {
  int n = h->A[0].n;
  double *r = xcalloc((size_t)n, 8), *w = xcalloc((size_t)n, 8), *d = xcalloc((size_t)n, 8);
  double *v = xcalloc((size_t)n, 8), *q = xcalloc((size_t)n, 8);
  int status = ORC_OK, it = 0;
  double nb = sqrt(dot(n, b, b));
  if (nb == 0.0) {
    memset(u, 0, sizeof(double) * (size_t)n);
    if (hist) hist[0] = 0.0;
    *iters = 0;
    *true_rel = 0.0;
    goto done;
  }
  residual(h, b, u, r);
  double res = sqrt(dot(n, r, r)) / nb;
  if (hist) hist[0] = res;
  double rho = 0.0;
  int mixed = h->p.precision != ORC_FP64 && precflag;
  for (;;) {
    if (res < tol) {
      /* recursive residual below tol: confirm with the true residual, and if it
       * is not below tol yet, continue from r = b - A u */
      double* t = w;
      residual(h, b, u, t);
      double tr = sqrt(dot(n, t, t)) / nb;
      if (tr < tol) break;
      memcpy(r, t, sizeof(double) * (size_t)n);
      res = tr;
      if (hist) hist[it] = tr;
    }
    if (it >= maxit) {
      status = ORC_NOT_CONVERGED;
      break;
    }
    apply_B(h, precflag, r, w);
    orc_spmv(h, 0, w, v);
    double alpha = dot(n, w, r);
    if (it == 0) {
      double beta = dot(n, w, v);
      rho = beta;
      if (!(rho > 0.0) || !isfinite(rho)) {
        status = ORC_ERR_BREAKDOWN;
        break;
      }
      memcpy(d, w, sizeof(double) * (size_t)n);
      memcpy(q, v, sizeof(double) * (size_t)n);
      double a = alpha / rho;
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) u[i] += a * d[i];
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] -= a * q[i];
    } else {
      double beta = dot(n, w, v);
      double gamma = dot(n, w, q);
      double rho_new = beta - gamma * gamma / rho;
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        status = ORC_ERR_BREAKDOWN;
        break;
      }
      double g = gamma / rho;
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) d[i] = w[i] - g * d[i];
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) q[i] = v[i] - g * q[i];
      double a = alpha / rho_new;
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) u[i] += a * d[i];
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] -= a * q[i];
      rho = rho_new;
    }
    ++it;
    if (mixed && h->p.true_res_every > 0 && it % h->p.true_res_every == 0) residual(h, b, u, r);
    res = sqrt(dot(n, r, r)) / nb;
    if (hist) hist[it] = res;
  }
  *iters = it;
  {
    residual(h, b, u, w);
    *true_rel = sqrt(dot(n, w, w)) / nb;
  }
done:
  free(r);
  free(w);
  free(d);
  free(v);
  free(q);
  return status;
}

/* ------------------------------------------------------------------ */
/* learned smoother: loss of m stationary V-cycle steps and its adjoint.
 * D_i = omega_i / l1_i on every level, so dD_i/domega_i = 1 / l1_i. */

/* adjoint of s sweeps started from zero: forward iterates recomputed here.
 * lam: in dL/dz_final, out dL/dz_start (unused when started from zero);
 * lr accumulates dL/dr; dom accumulates dL/domega */
static void sweeps_adj(const ocsr* A, const double* D, const double* l1, const double* r,
                       const double* zstart, int sweeps, double* lam, double* lr, double* dom) {
  int n = A->n;
  if (sweeps <= 0) return;
  /* iterates z_0 .. z_{sweeps-1} (the inputs of each sweep) */
  double** zs = (double**)xcalloc((size_t)sweeps, sizeof(double*));
  double* tmp = (double*)xcalloc((size_t)n, sizeof(double));
  for (int s = 0; s < sweeps; ++s) zs[s] = (double*)xcalloc((size_t)n, sizeof(double));
  if (zstart) memcpy(zs[0], zstart, sizeof(double) * (size_t)n);
  for (int s = 1; s < sweeps; ++s) {
    memcpy(zs[s], zs[s - 1], sizeof(double) * (size_t)n);
    sweep_d(A, D, r, zs[s], tmp);
  }
  double* t = (double*)xcalloc((size_t)n, sizeof(double));
  double* dl = (double*)xcalloc((size_t)n, sizeof(double));
  for (int s = sweeps - 1; s >= 0; --s) {
    /* z_{s+1} = z_s + D (r - A z_s) */
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) acc += A->v[p] * zs[s][A->ci[p]];
      t[i] = r[i] - acc;
    }
    for (int i = 0; i < n; ++i) {
      dom[i] += lam[i] * t[i] / l1[i];
      dl[i] = D[i] * lam[i];
      lr[i] += dl[i];
    }
    /* lam <- lam - A^T (D lam); A is symmetric, A^T is applied through the transpose loop */
    for (int i = 0; i < n; ++i)
      for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) lam[A->ci[p]] -= A->v[p] * dl[i];
  }
  for (int s = 0; s < sweeps; ++s) free(zs[s]);
  free(zs);
  free(tmp);
  free(t);
  free(dl);
}

/* returns dL/dr for the V-cycle at level k given dL/dz (lam, overwritten) */
static void vcycle_adj(orc_hier* h, int k, const double* r, double* lam, double* lr, double* const* dom) {
  const ocsr* A = &h->A[k];
  int n = A->n;
  memset(lr, 0, sizeof(double) * (size_t)n);
  if (k == h->nl - 1) {
    sweeps_adj(A, h->dinv[k], h->l1[k], r, NULL, h->p.coarse_sweeps, lam, lr, dom[k]);
    return;
  }
  int nc = h->A[k + 1].n;
  const int32_t* agg = h->agg[k];
  double* tmp = (double*)xcalloc((size_t)n, sizeof(double));
  double* z = (double*)xcalloc((size_t)n, sizeof(double));
  double* rc = (double*)xcalloc((size_t)nc, sizeof(double));
  double* zc = (double*)xcalloc((size_t)nc, sizeof(double));
  /* forward recompute */
  smooth_from_zero_d(A, h->dinv[k], r, z, h->p.pre_sweeps, tmp);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * z[A->ci[p]];
    tmp[i] = r[i] - s;
  }
  for (int i = 0; i < n; ++i) rc[agg[i]] += tmp[i];
  vcycle_d(h, k + 1, rc, zc);
  double* y0 = (double*)xcalloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) y0[i] = z[i] + zc[agg[i]];
  /* backward: post-sweeps */
  sweeps_adj(A, h->dinv[k], h->l1[k], r, y0, h->p.post_sweeps, lam, lr, dom[k]);
  /* prolongation y0 = z + P zc */
  double* lzc = (double*)xcalloc((size_t)nc, sizeof(double));
  for (int i = 0; i < n; ++i) lzc[agg[i]] += lam[i];
  double* lrc = (double*)xcalloc((size_t)nc, sizeof(double));
  vcycle_adj(h, k + 1, rc, lzc, lrc, dom);
  /* restriction rc = P^T (r - A z) */
  double* lres = tmp;
  for (int i = 0; i < n; ++i) lres[i] = lrc[agg[i]];
  for (int i = 0; i < n; ++i) lr[i] += lres[i];
  for (int i = 0; i < n; ++i)
    for (int32_t p = A->rp[i]; p < A->rp[i + 1]; ++p) lam[A->ci[p]] -= A->v[p] * lres[i];
  /* pre-sweeps from zero */
  sweeps_adj(A, h->dinv[k], h->l1[k], r, NULL, h->p.pre_sweeps, lam, lr, dom[k]);
  free(tmp);
  free(z);
  free(rc);
  free(zc);
  free(y0);
  free(lzc);
  free(lrc);
}

static double nrm2(int n, const double* x) { return sqrt(dot(n, x, x)); }

double orc_vcycle_loss(orc_hier* h, const double* r0, int m) {
  int n = h->A[0].n;
  double* r = (double*)xcalloc((size_t)n, sizeof(double));
  double* z = (double*)xcalloc((size_t)n, sizeof(double));
  double* az = (double*)xcalloc((size_t)n, sizeof(double));
  memcpy(r, r0, sizeof(double) * (size_t)n);
  for (int t = 0; t < m; ++t) {
    vcycle_d(h, 0, r, z);
    orc_spmv(h, 0, z, az);
    for (int i = 0; i < n; ++i) r[i] -= az[i];
  }
  double L = (log(nrm2(n, r)) - log(nrm2(n, r0))) / m;
  free(r);
  free(z);
  free(az);
  return L;
}

double orc_vcycle_loss_grad(orc_hier* h, const double* r0, int m, double* const* domega) {
  if (h->p.relax_type != 4 || h->p.cycle != 0 || h->wsv[0]) return NAN; /* dD/domega = 1 / l1 below */
  int n = h->A[0].n;
  double** rs = (double**)xcalloc((size_t)m + 1, sizeof(double*));
  double* z = (double*)xcalloc((size_t)n, sizeof(double));
  double* az = (double*)xcalloc((size_t)n, sizeof(double));
  for (int t = 0; t <= m; ++t) rs[t] = (double*)xcalloc((size_t)n, sizeof(double));
  memcpy(rs[0], r0, sizeof(double) * (size_t)n);
  for (int t = 0; t < m; ++t) {
    vcycle_d(h, 0, rs[t], z);
    orc_spmv(h, 0, z, az);
    for (int i = 0; i < n; ++i) rs[t + 1][i] = rs[t][i] - az[i];
  }
  double nm = nrm2(n, rs[m]);
  double L = (log(nm) - log(nrm2(n, r0))) / m;
  for (int k = 0; k < h->nl; ++k) memset(domega[k], 0, sizeof(double) * (size_t)h->A[k].n);
  double* lam_r = (double*)xcalloc((size_t)n, sizeof(double));
  double* lam_z = (double*)xcalloc((size_t)n, sizeof(double));
  double* lr = (double*)xcalloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) lam_r[i] = rs[m][i] / ((double)m * nm * nm);
  for (int t = m - 1; t >= 0; --t) {
    /* r_{t+1} = r_t - A z_t: dL/dz_t = -A^T lam_r */
    orc_spmv(h, 0, lam_r, lam_z);
    for (int i = 0; i < n; ++i) lam_z[i] = -lam_z[i];
    vcycle_adj(h, 0, rs[t], lam_z, lr, domega);
    for (int i = 0; i < n; ++i) lam_r[i] += lr[i];
  }
  for (int t = 0; t <= m; ++t) free(rs[t]);
  free(rs);
  free(z);
  free(az);
  free(lam_r);
  free(lam_z);
  free(lr);
  return L;
}
