/*
 * FP64 CPU oracle, part 2: smoothed-aggregation algebraic multigrid with a
 * relaxation smoother, the setting in which the paper also runs GS2 -- as
 * the smoother of an AMG V-cycle (the Nalu-Wind experiments of Sec. 11,
 * hypre and Trilinos subsections).  TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Readings (the paper names the AMG flavours it used but not their steps):
 *  - strength of connection: the classical threshold the paper's C-AMG runs
 *    use, theta = 0.25: j != i is strong for i if |a_ij| >= theta max_{k != i}
 *    |a_ik|; the aggregation graph joins i and j if either is strong for the
 *    other;
 *  - aggregation: the three greedy phases of smoothed aggregation, rows in
 *    natural order;
 *  - tentative prolongator: the constant vector on each aggregate, each
 *    column scaled to unit 2-norm;
 *  - smoothed prolongator P = (I - w D^{-1} A) P0 with w = 4 / (3 rho), rho
 *    the Gershgorin bound max_i sum_j |a_ij| / |a_ii| of rho(D^{-1} A);
 *  - Galerkin coarse operator A_c = P^T A P, restriction P^T;
 *  - coarsening stops at max_levels, when a level has at most coarse_size
 *    rows, or when it would not shrink; the coarsest level is solved
 *    exactly (dense LU with partial pivoting);
 *  - V-cycle from a zero start: pre-smoothing from zero, residual,
 *    restriction, coarse correction, prolongation, post-smoothing.  A
 *    symmetric smoother is split as forward pre- and backward
 *    post-smoothing (the combination the Trilinos continuity runs found
 *    best), which keeps the cycle symmetric for SPD A.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t n, m;  /* rows, columns */
  int64_t* rp;
  int32_t* ci;
  double* va;
} csr;

struct ora_amg {
  int nlev;
  csr A[ORA_AMG_MAX_LEVELS];  /* A[0] is a copy of the input */
  csr P[ORA_AMG_MAX_LEVELS];  /* P[l]: n_l x n_{l+1} */
  csr R[ORA_AMG_MAX_LEVELS];  /* R[l] = P[l]^T */
  int32_t* agg[ORA_AMG_MAX_LEVELS];
  double* lu;                 /* coarsest matrix, LU factors in place */
  int64_t* piv;
};

static void csr_free(csr* a) {
  free(a->rp);
  free(a->ci);
  free(a->va);
  memset(a, 0, sizeof(*a));
}

static csr csr_alloc(int64_t n, int64_t m, int64_t nnz) {
  csr a;
  a.n = n;
  a.m = m;
  a.rp = calloc((size_t)n + 1, sizeof(int64_t));
  a.ci = malloc(((size_t)nnz + 1) * sizeof(int32_t));
  a.va = malloc(((size_t)nnz + 1) * sizeof(double));
  return a;
}

/* B = A^T, columns of every row ascending */
static csr csr_transpose(const csr* a) {
  const int64_t nnz = a->rp[a->n];
  csr t = csr_alloc(a->m, a->n, nnz);
  for (int64_t k = 0; k < nnz; ++k) t.rp[a->ci[k] + 1]++;
  for (int64_t j = 0; j < a->m; ++j) t.rp[j + 1] += t.rp[j];
  int64_t* fill = malloc(((size_t)a->m + 1) * sizeof(int64_t));
  memcpy(fill, t.rp, ((size_t)a->m + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < a->n; ++i)
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      const int64_t q = fill[a->ci[k]]++;
      t.ci[q] = (int32_t)i;
      t.va[q] = a->va[k];
    }
  free(fill);
  return t;
}

static int cmp_i32(const void* x, const void* y) {
  const int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* C = A B, row by row with a dense accumulator; every product a_ik b_kj
 * that exists structurally gives an entry (no dropping), columns ascending */
static csr csr_matmul(const csr* a, const csr* b) {
  double* acc = calloc((size_t)b->m + 1, sizeof(double));
  int64_t* mark = malloc(((size_t)b->m + 1) * sizeof(int64_t));
  for (int64_t j = 0; j < b->m; ++j) mark[j] = -1;
  int32_t* cols = malloc(((size_t)b->m + 1) * sizeof(int32_t));
  /* first pass: row lengths */
  int64_t* len = calloc((size_t)a->n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < a->n; ++i) {
    int64_t cnt = 0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      const int64_t r = a->ci[k];
      for (int64_t q = b->rp[r]; q < b->rp[r + 1]; ++q)
        if (mark[b->ci[q]] != i) {
          mark[b->ci[q]] = i;
          cnt++;
        }
    }
    len[i] = cnt;
  }
  int64_t nnz = 0;
  for (int64_t i = 0; i < a->n; ++i) nnz += len[i];
  csr c = csr_alloc(a->n, b->m, nnz);
  for (int64_t i = 0; i < a->n; ++i) c.rp[i + 1] = c.rp[i] + len[i];
  for (int64_t j = 0; j < b->m; ++j) mark[j] = -1;
  for (int64_t i = 0; i < a->n; ++i) {
    int64_t cnt = 0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      const int64_t r = a->ci[k];
      for (int64_t q = b->rp[r]; q < b->rp[r + 1]; ++q) {
        const int32_t j = b->ci[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols[cnt++] = j;
        }
        acc[j] += a->va[k] * b->va[q];
      }
    }
    qsort(cols, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int64_t q = 0; q < cnt; ++q) {
      c.ci[c.rp[i] + q] = cols[q];
      c.va[c.rp[i] + q] = acc[cols[q]];
    }
  }
  free(acc);
  free(mark);
  free(cols);
  free(len);
  return c;
}

/* ------------------------------------------------------------------ */
/* Aggregation                                                          */
/* ------------------------------------------------------------------ */

/* Symmetrised strength graph: adjacency lists (ascending) of the rows j
 * that are strong for i or for which i is strong. */
static void strength_graph(const csr* a, double theta, int64_t** gp_out,
                           int32_t** gi_out) {
  const int64_t n = a->n;
  /* directed strong entries */
  csr s = csr_alloc(n, n, a->rp[n]);
  int64_t q = 0;
  for (int64_t i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k)
      if (a->ci[k] != i && fabs(a->va[k]) > mx) mx = fabs(a->va[k]);
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k)
      if (a->ci[k] != i && mx > 0.0 && fabs(a->va[k]) >= theta * mx) {
        s.ci[q] = a->ci[k];
        s.va[q] = 1.0;
        q++;
      }
    s.rp[i + 1] = q;
  }
  csr st = csr_transpose(&s);
  /* union of the two patterns, per row, ascending without duplicates */
  int64_t* gp = calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* gi = malloc(((size_t)2 * q + 1) * sizeof(int32_t));
  int32_t* buf = malloc(((size_t)n + 1) * sizeof(int32_t));
  int64_t tot = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cnt = 0;
    for (int64_t k = s.rp[i]; k < s.rp[i + 1]; ++k) buf[cnt++] = s.ci[k];
    for (int64_t k = st.rp[i]; k < st.rp[i + 1]; ++k) buf[cnt++] = st.ci[k];
    qsort(buf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int64_t k = 0; k < cnt; ++k)
      if (k == 0 || buf[k] != buf[k - 1]) gi[tot++] = buf[k];
    gp[i + 1] = tot;
  }
  free(buf);
  csr_free(&s);
  csr_free(&st);
  *gp_out = gp;
  *gi_out = gi;
}

/* The three greedy phases in natural order; returns the aggregate count. */
static int64_t aggregate(int64_t n, const int64_t* gp, const int32_t* gi, int32_t* agg) {
  for (int64_t i = 0; i < n; ++i) agg[i] = -1;
  int64_t na = 0;
  /* phase 1: a row whose whole neighbourhood is free seeds an aggregate of
   * itself and its neighbours */
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int free_all = 1;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k)
      if (agg[gi[k]] >= 0) free_all = 0;
    if (!free_all) continue;
    agg[i] = (int32_t)na;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k) agg[gi[k]] = (int32_t)na;
    na++;
  }
  /* phase 2: a free row joins the phase-1 aggregate of its first neighbour
   * (ascending) that has one */
  int32_t* phase1 = malloc(((size_t)n + 1) * sizeof(int32_t));
  memcpy(phase1, agg, (size_t)n * sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) {
    if (phase1[i] >= 0) continue;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k)
      if (phase1[gi[k]] >= 0) {
        agg[i] = phase1[gi[k]];
        break;
      }
  }
  free(phase1);
  /* phase 3: every row still free seeds an aggregate with its free
   * neighbours */
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = (int32_t)na;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k)
      if (agg[gi[k]] < 0) agg[gi[k]] = (int32_t)na;
    na++;
  }
  return na;
}

/* ------------------------------------------------------------------ */
/* Hierarchy                                                            */
/* ------------------------------------------------------------------ */

static csr csr_copy(int64_t n, const int64_t* rp, const int32_t* ci, const double* va) {
  csr a = csr_alloc(n, n, rp[n]);
  memcpy(a.rp, rp, ((size_t)n + 1) * sizeof(int64_t));
  memcpy(a.ci, ci, (size_t)rp[n] * sizeof(int32_t));
  memcpy(a.va, va, (size_t)rp[n] * sizeof(double));
  return a;
}

/* P = (I - w D^{-1} A) P0 for one level; fills agg and returns P */
static csr smoothed_prolongator(const csr* a, double theta, int32_t* agg, int64_t* nagg) {
  const int64_t n = a->n;
  int64_t* gp;
  int32_t* gi;
  strength_graph(a, theta, &gp, &gi);
  const int64_t na = aggregate(n, gp, gi, agg);
  free(gp);
  free(gi);
  *nagg = na;
  /* tentative prolongator: one entry per row, 1/sqrt(|aggregate|) */
  int64_t* size = calloc((size_t)na + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) size[agg[i]]++;
  csr p0 = csr_alloc(n, na, n);
  for (int64_t i = 0; i < n; ++i) {
    p0.rp[i + 1] = i + 1;
    p0.ci[i] = agg[i];
    p0.va[i] = 1.0 / sqrt((double)size[agg[i]]);
  }
  free(size);
  /* diagonal and the Gershgorin bound of rho(D^{-1} A) */
  double* d = malloc(((size_t)n + 1) * sizeof(double));
  double rho = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double di = 0.0, row = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      if (a->ci[k] == i) di = a->va[k];
      row += fabs(a->va[k]);
    }
    d[i] = di;
    if (row / fabs(di) > rho) rho = row / fabs(di);
  }
  const double w = 4.0 / (3.0 * rho);
  csr ap0 = csr_matmul(a, &p0);
  /* P = P0 - (w / a_ii) (A P0): the pattern of A P0 contains that of P0 */
  csr p = csr_alloc(n, na, ap0.rp[n]);
  memcpy(p.rp, ap0.rp, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ap0.rp[i]; k < ap0.rp[i + 1]; ++k) {
      const int32_t c = ap0.ci[k];
      const double p0v = (c == agg[i]) ? p0.va[i] : 0.0;
      p.ci[k] = c;
      p.va[k] = p0v - (w / d[i]) * ap0.va[k];
    }
  free(d);
  csr_free(&p0);
  csr_free(&ap0);
  return p;
}

/* dense LU with partial pivoting, in place, row-major; 0 or 2 (singular) */
static int dense_lu(int64_t n, double* a, int64_t* piv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t pr = k;
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > fabs(a[pr * n + k])) pr = i;
    piv[k] = pr;
    if (a[pr * n + k] == 0.0) return 2;
    if (pr != k)
      for (int64_t j = 0; j < n; ++j) {
        const double t = a[k * n + j];
        a[k * n + j] = a[pr * n + j];
        a[pr * n + j] = t;
      }
    for (int64_t i = k + 1; i < n; ++i) {
      const double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 0;
}

static void dense_lu_solve(int64_t n, const double* lu, const int64_t* piv, const double* b,
                           double* x) {
  memcpy(x, b, (size_t)n * sizeof(double));
  for (int64_t k = 0; k < n; ++k) {
    const double t = x[k];
    x[k] = x[piv[k]];
    x[piv[k]] = t;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < i; ++j) x[i] -= lu[i * n + j] * x[j];
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int64_t j = i + 1; j < n; ++j) x[i] -= lu[i * n + j] * x[j];
    x[i] /= lu[i * n + i];
  }
}

ora_amg* ora_amg_build(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                       double theta, int max_levels, int64_t coarse_size) {
  if (n <= 0 || max_levels < 1 || max_levels > ORA_AMG_MAX_LEVELS || coarse_size < 1)
    return NULL;
  double* d = malloc((size_t)n * sizeof(double));
  const int st = ora_diag(n, rp, ci, va, d);
  free(d);
  if (st) return NULL;
  ora_amg* M = calloc(1, sizeof(ora_amg));
  M->A[0] = csr_copy(n, rp, ci, va);
  M->nlev = 1;
  while (M->nlev < max_levels && M->A[M->nlev - 1].n > coarse_size) {
    const int l = M->nlev - 1;
    const csr* a = &M->A[l];
    int32_t* agg = malloc(((size_t)a->n + 1) * sizeof(int32_t));
    int64_t na = 0;
    csr p = smoothed_prolongator(a, theta, agg, &na);
    if (na >= a->n || na == 0) {
      csr_free(&p);
      free(agg);
      break;
    }
    csr r = csr_transpose(&p);
    csr ap = csr_matmul(a, &p);
    M->A[l + 1] = csr_matmul(&r, &ap);
    csr_free(&ap);
    M->P[l] = p;
    M->R[l] = r;
    M->agg[l] = agg;
    M->nlev++;
  }
  /* coarsest level: dense LU */
  const csr* c = &M->A[M->nlev - 1];
  M->lu = calloc((size_t)(c->n * c->n) + 1, sizeof(double));
  M->piv = malloc(((size_t)c->n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < c->n; ++i)
    for (int64_t k = c->rp[i]; k < c->rp[i + 1]; ++k) M->lu[i * c->n + c->ci[k]] += c->va[k];
  if (dense_lu(c->n, M->lu, M->piv)) {
    ora_amg_free(M);
    return NULL;
  }
  return M;
}

void ora_amg_free(ora_amg* M) {
  if (!M) return;
  for (int l = 0; l < ORA_AMG_MAX_LEVELS; ++l) {
    csr_free(&M->A[l]);
    csr_free(&M->P[l]);
    csr_free(&M->R[l]);
    free(M->agg[l]);
  }
  free(M->lu);
  free(M->piv);
  free(M);
}

int ora_amg_levels(const ora_amg* M) { return M ? M->nlev : 0; }

int ora_amg_level(const ora_amg* M, int l, int64_t* n, int64_t* nnz, int64_t* pnnz) {
  if (!M || l < 0 || l >= M->nlev) return 1;
  if (n) *n = M->A[l].n;
  if (nnz) *nnz = M->A[l].rp[M->A[l].n];
  if (pnnz) *pnnz = (l + 1 < M->nlev) ? M->P[l].rp[M->P[l].n] : 0;
  return 0;
}

static int copy_out(const csr* a, int64_t* rp, int32_t* ci, double* va) {
  if (!a->rp) return 1;
  if (rp) memcpy(rp, a->rp, ((size_t)a->n + 1) * sizeof(int64_t));
  if (ci) memcpy(ci, a->ci, (size_t)a->rp[a->n] * sizeof(int32_t));
  if (va) memcpy(va, a->va, (size_t)a->rp[a->n] * sizeof(double));
  return 0;
}

int ora_amg_get_matrix(const ora_amg* M, int l, int64_t* rp, int32_t* ci, double* va) {
  if (!M || l < 0 || l >= M->nlev) return 1;
  return copy_out(&M->A[l], rp, ci, va);
}

int ora_amg_get_prolongator(const ora_amg* M, int l, int64_t* rp, int32_t* ci, double* va) {
  if (!M || l < 0 || l + 1 >= M->nlev) return 1;
  return copy_out(&M->P[l], rp, ci, va);
}

int ora_amg_get_aggregates(const ora_amg* M, int l, int32_t* agg) {
  if (!M || l < 0 || l + 1 >= M->nlev) return 1;
  memcpy(agg, M->agg[l], (size_t)M->A[l].n * sizeof(int32_t));
  return 0;
}

/* ------------------------------------------------------------------ */
/* V-cycle                                                              */
/* ------------------------------------------------------------------ */

/* `sweeps` relaxation sweeps of the smoother on A x = b from the given x */
static int smooth(const csr* a, const double* b, double* x, int kind, int outer, int inner,
                  double omega, double gamma, int dir) {
  switch (kind) {
    case ORA_PC_GS2:
      return ora_gs2(a->n, a->rp, a->ci, a->va, b, x, outer, inner, omega, gamma, dir);
    case ORA_PC_JR:
      return ora_jr(a->n, a->rp, a->ci, a->va, b, x, outer, omega);
    default:
      return 1;
  }
}

static int vcycle(const ora_amg* M, int l, const double* b, double* x, int kind, int outer,
                  int inner, double omega, double gamma, int dir) {
  const csr* a = &M->A[l];
  const int64_t n = a->n;
  if (l == M->nlev - 1) {
    dense_lu_solve(n, M->lu, M->piv, b, x);
    return 0;
  }
  const int pre = (dir == ORA_SYMMETRIC) ? ORA_FORWARD : dir;
  const int post = (dir == ORA_SYMMETRIC) ? ORA_BACKWARD : dir;
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  int st = smooth(a, b, x, kind, outer, inner, omega, gamma, pre);
  if (st) return st;
  double* r = malloc((size_t)n * sizeof(double));
  ora_spmv(n, a->rp, a->ci, a->va, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  const int64_t nc = M->A[l + 1].n;
  double* bc = malloc((size_t)nc * sizeof(double));
  double* xc = malloc((size_t)nc * sizeof(double));
  ora_spmv(nc, M->R[l].rp, M->R[l].ci, M->R[l].va, r, bc);
  st = vcycle(M, l + 1, bc, xc, kind, outer, inner, omega, gamma, dir);
  if (!st) {
    ora_spmv(n, M->P[l].rp, M->P[l].ci, M->P[l].va, xc, r);
    for (int64_t i = 0; i < n; ++i) x[i] += r[i];
    st = smooth(a, b, x, kind, outer, inner, omega, gamma, post);
  }
  free(r);
  free(bc);
  free(xc);
  return st;
}

int ora_amg_vcycle(const ora_amg* M, const double* b, double* x, int kind, int outer,
                   int inner, double omega, double gamma, int dir) {
  if (!M || (kind != ORA_PC_GS2 && kind != ORA_PC_JR) || outer < 0 || inner < 0)
    return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC) return 1;
  return vcycle(M, 0, b, x, kind, outer, inner, omega, gamma, dir);
}

/* GMRES with one V-cycle as the right preconditioner: ora_gmres with the
 * preconditioner kind ORA_PC_AMG (GS2 smoother) or ORA_PC_AMG_JR (JR
 * smoother), which applies the hierarchy set here. */
_Thread_local const ora_amg* ora_amg_current = NULL;

int ora_gmres_amg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                  const double* b, double* x, int restart, double tol, int max_iters,
                  const ora_amg* M, int kind, int outer, int inner, double omega,
                  double gamma, int dir, ora_info* info) {
  if (!M || M->A[0].n != n || (kind != ORA_PC_GS2 && kind != ORA_PC_JR)) return 1;
  ora_amg_current = M;
  const int pc = (kind == ORA_PC_JR) ? ORA_PC_AMG_JR : ORA_PC_AMG;
  const int st = ora_gmres(n, rp, ci, va, b, x, restart, tol, max_iters, pc, outer, inner,
                           omega, gamma, dir, info, NULL);
  ora_amg_current = NULL;
  return st;
}

/* CG with one symmetric V-cycle as the preconditioner: ora_cg with the AMG
 * preconditioner kind on the hierarchy set here. */
int ora_cg_amg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, double tol, int max_iters, const ora_amg* M,
               int kind, int outer, int inner, double omega, double gamma, int dir,
               ora_info* info) {
  if (!M || M->A[0].n != n || (kind != ORA_PC_GS2 && kind != ORA_PC_JR)) return 1;
  ora_amg_current = M;
  const int pc = (kind == ORA_PC_JR) ? ORA_PC_AMG_JR : ORA_PC_AMG;
  const int st = ora_cg(n, rp, ci, va, b, x, tol, max_iters, pc, outer, inner, omega, gamma,
                        dir, info);
  ora_amg_current = NULL;
  return st;
}
