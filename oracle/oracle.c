/*
 * FP64 CPU oracle: two-stage Gauss-Seidel and the Krylov solvers it
 * preconditions.  TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: one loop per formula, no blocking, no fusion, no reordering beyond
 * what the formula states.  Where the paper is ambiguous the reading taken is
 * stated at the function.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops over rows (or vector entries) in which every iteration writes only
 * its own entry, from the same code in the same order, carry an OpenMP
 * parallel-for: a build with -fopenmp spreads them over the host cores (the
 * multi-core CPU timing), a build without it ignores the pragma, and both
 * give bitwise the same results.  Reductions (inner products, norms) and the
 * recurrences of exact GS stay sequential in every build. */
#ifdef _OPENMP
#include <omp.h>
#define ORA_ROWS_PARALLEL _Pragma("omp parallel for schedule(static)")
#else
#define ORA_ROWS_PARALLEL
#endif

int ora_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Basic pieces                                                         */
/* ------------------------------------------------------------------ */

void ora_spmv(int64_t n, const int64_t* rp, const int32_t* ci,
              const double* va, const double* x, double* y) {
  ORA_ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
    y[i] = s;
  }
}

int ora_diag(int64_t n, const int64_t* rp, const int32_t* ci,
             const double* va, double* d) {
  for (int64_t i = 0; i < n; ++i) {
    double di = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) di += va[k];
    if (di == 0.0) return 2;
    d[i] = di;
  }
  return 0;
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

/* r = b - A x  (the residual of Eq. (1) and Eq. (2)) */
static void residual(int64_t n, const int64_t* rp, const int32_t* ci,
                     const double* va, const double* b, const double* x,
                     double* r) {
  ORA_ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
    r[i] = b[i] - s;
  }
}

/* t = T g with T the strict lower (lower=1) or strict upper (lower=0)
 * triangle of A, selected entry by entry by comparing column and row. */
static void tri_mult(int64_t n, const int64_t* rp, const int32_t* ci,
                     const double* va, int lower, const double* g,
                     double* t) {
  ORA_ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int64_t j = ci[k];
      if ((lower && j < i) || (!lower && j > i)) s += va[k] * g[j];
    }
    t[i] = s;
  }
}

/* ------------------------------------------------------------------ */
/* GS2: Eq. (2) with inner JR sweeps Eq. (3)-(5) and the damping        */
/* factors omega (outer) and gamma (inner) of Sec. 4.                   */
/* ------------------------------------------------------------------ */

/* One non-compact GS2 sweep with triangle T (lower or upper):
 *   r = b - A x
 *   g^(0) = D^{-1} r                                   Eq. (3)
 *   g^(j+1) = (1-gamma) g^(j) + gamma D^{-1}(r - omega T g^(j))
 *                                     (damped form of Eq. (4)-(5))
 *   x = x + omega g^(inner)
 * Reading: the outer damping multiplies the correction, so the inner
 * iteration solves (D + omega T) g = r and omega = 1 gives Eq. (2) exactly.
 * Each inner sweep uses only the previous iterate (Jacobi, not in place). */
static void gs2_sweep(int64_t n, const int64_t* rp, const int32_t* ci,
                      const double* va, const double* d, const double* b,
                      double* x, int inner, double omega, double gamma,
                      int lower, double* r, double* g, double* gn,
                      double* t) {
  residual(n, rp, ci, va, b, x, r);
  ORA_ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) g[i] = r[i] / d[i];
  for (int j = 0; j < inner; ++j) {
    tri_mult(n, rp, ci, va, lower, g, t);
    ORA_ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i)
      gn[i] = (1.0 - gamma) * g[i] + gamma * (r[i] - omega * t[i]) / d[i];
    memcpy(g, gn, (size_t)n * sizeof(double));
  }
  ORA_ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * g[i];
}

int ora_gs2(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
            const double* b, double* x, int outer, int inner, double omega,
            double gamma, int dir) {
  if (n < 0 || outer < 0 || inner < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC)
    return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  double* r = malloc((size_t)n * sizeof(double));
  double* g = malloc((size_t)n * sizeof(double));
  double* gn = malloc((size_t)n * sizeof(double));
  double* t = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  for (int s = 0; st == 0 && s < outer; ++s) {
    if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC)
      gs2_sweep(n, rp, ci, va, d, b, x, inner, omega, gamma, 1, r, g, gn, t);
    if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC)
      gs2_sweep(n, rp, ci, va, d, b, x, inner, omega, gamma, 0, r, g, gn, t);
  }
  free(d); free(r); free(g); free(gn); free(t);
  return st;
}

/* ------------------------------------------------------------------ */
/* Exact GS / SOR: compact row recurrence of the sequential GS listing  */
/* (Sec. 6.1.1); for omega != 1 the SOR form x + omega (D+omega L)^{-1} */
/* (b - A x) of the "Damping factor" paragraph, written row by row.     */
/* ------------------------------------------------------------------ */

static void gs_row(int64_t i, const int64_t* rp, const int32_t* ci,
                   const double* va, const double* b, double* x,
                   double omega) {
  double sum = 0.0, aii = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    if (ci[k] == i) aii += va[k];
    else sum += va[k] * x[ci[k]];
  }
  x[i] = (1.0 - omega) * x[i] + omega * (b[i] - sum) / aii;
}

int ora_gs(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, int sweeps, double omega, int dir) {
  if (n < 0 || sweeps < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC)
    return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  free(d);
  if (st) return st;
  for (int s = 0; s < sweeps; ++s) {
    if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC)
      for (int64_t i = 0; i < n; ++i) gs_row(i, rp, ci, va, b, x, omega);
    if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC)
      for (int64_t i = n - 1; i >= 0; --i) gs_row(i, rp, ci, va, b, x, omega);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Multicolour GS (Sec. 6.1.2): greedy colouring, then the sequential   */
/* row update visiting the rows colour by colour.                       */
/* ------------------------------------------------------------------ */

int ora_coloring(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* color) {
  /* transpose pattern: for every row j, the rows i with a_ij != 0 */
  int64_t* tp = calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) tp[ci[k] + 1]++;
  for (int64_t j = 0; j < n; ++j) tp[j + 1] += tp[j];
  int64_t* fill = malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(fill, tp, ((size_t)n + 1) * sizeof(int64_t));
  int64_t* ti = malloc(((size_t)rp[n] + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) ti[fill[ci[k]]++] = i;
  /* first fit: forbidden[c] == i marks colour c as used by a neighbour of i */
  int64_t* forbidden = malloc(((size_t)n + 1) * sizeof(int64_t));
  for (int64_t c = 0; c <= n; ++c) forbidden[c] = -1;
  int32_t ncolors = 0;
  for (int64_t i = 0; i < n; ++i) color[i] = -1;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i && color[ci[k]] >= 0) forbidden[color[ci[k]]] = i;
    for (int64_t k = tp[i]; k < tp[i + 1]; ++k)
      if (ti[k] != i && color[ti[k]] >= 0) forbidden[color[ti[k]]] = i;
    int32_t c = 0;
    while (forbidden[c] == i) ++c;
    color[i] = c;
    if (c + 1 > ncolors) ncolors = c + 1;
  }
  free(tp); free(fill); free(ti); free(forbidden);
  return ncolors;
}

int ora_mtgs(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
             const double* b, double* x, int sweeps, double omega, int dir) {
  if (n < 0 || sweeps < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC)
    return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  free(d);
  if (st) return st;
  int32_t* color = malloc((size_t)n * sizeof(int32_t));
  const int32_t nc = ora_coloring(n, rp, ci, color);
  for (int s = 0; s < sweeps; ++s) {
    if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC)
      for (int32_t c = 0; c < nc; ++c)
        for (int64_t i = 0; i < n; ++i)
          if (color[i] == c) gs_row(i, rp, ci, va, b, x, omega);
    if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC)
      for (int32_t c = nc - 1; c >= 0; --c)
        for (int64_t i = 0; i < n; ++i)
          if (color[i] == c) gs_row(i, rp, ci, va, b, x, omega);
  }
  free(color);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Jacobi-Richardson: GS2 with zero inner sweeps (Sec. 4), damped.      */
/* ------------------------------------------------------------------ */

int ora_jr(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, int sweeps, double omega) {
  if (n < 0 || sweeps < 0) return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  double* r = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  for (int s = 0; st == 0 && s < sweeps; ++s) {
    residual(n, rp, ci, va, b, x, r);
    ORA_ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * r[i] / d[i];
  }
  free(d); free(r);
  return st;
}

/* ------------------------------------------------------------------ */
/* Level sets of a triangle (level-set scheduling, Sec. 3).             */
/* ------------------------------------------------------------------ */

int ora_levels(int64_t n, const int64_t* rp, const int32_t* ci, int lower,
               int32_t* level) {
  int32_t nlev = 0;
  for (int64_t s = 0; s < n; ++s) {
    int64_t i = lower ? s : n - 1 - s;
    int32_t lv = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int64_t j = ci[k];
      if ((lower && j < i) || (!lower && j > i))
        if (level[j] + 1 > lv) lv = level[j] + 1;
    }
    level[i] = lv;
    if (lv + 1 > nlev) nlev = lv + 1;
  }
  return nlev;
}

/* ------------------------------------------------------------------ */
/* Preconditioner application from a zero start.                        */
/* Reading: the paper does not state the preconditioner's initial      */
/* guess; a zero start makes M^{-1} a fixed linear operator, and makes  */
/* one JR sweep equal omega D^{-1}, which is why the JR(1) row of the   */
/* elasticity omega table (Sec. 8) does not depend on omega.            */
/* ------------------------------------------------------------------ */

int ora_precond(int64_t n, const int64_t* rp, const int32_t* ci,
                const double* va, const double* v, double* z, int kind,
                int outer, int inner, double omega, double gamma, int dir) {
  for (int64_t i = 0; i < n; ++i) z[i] = 0.0;
  switch (kind) {
    case ORA_PC_NONE:
      memcpy(z, v, (size_t)n * sizeof(double));
      return 0;
    case ORA_PC_GS2:
      if (ora_precision != ORA_PREC_FP64)
        return ora_gs2_lp(n, rp, ci, va, v, z, outer, inner, omega, gamma, dir,
                          ora_precision);
      return ora_gs2(n, rp, ci, va, v, z, outer, inner, omega, gamma, dir);
    case ORA_PC_JR:
      return ora_jr(n, rp, ci, va, v, z, outer, omega);
    case ORA_PC_GS:
      return ora_gs(n, rp, ci, va, v, z, outer, omega, dir);
    case ORA_PC_MTGS:
      return ora_mtgs(n, rp, ci, va, v, z, outer, omega, dir);
    case ORA_PC_HYBRID_GS2:
    case ORA_PC_HYBRID_JR:
    case ORA_PC_HYBRID_GS:
      return ora_hybrid(n, rp, ci, va, v, z,
                        kind == ORA_PC_HYBRID_GS2 ? ORA_PC_GS2
                                                  : (kind == ORA_PC_HYBRID_JR ? ORA_PC_JR
                                                                              : ORA_PC_GS),
                        ora_hybrid_parts, outer, ora_hybrid_local, inner, omega, gamma, dir);
    case ORA_PC_GS2_COMPACT:
      return ora_gs2_compact(n, rp, ci, va, v, z, outer, inner, dir);
    case ORA_PC_AMG:
    case ORA_PC_AMG_JR:
      if (!ora_amg_current) return 1;
      return ora_amg_vcycle(ora_amg_current, v, z, kind == ORA_PC_AMG ? ORA_PC_GS2 : ORA_PC_JR,
                            outer, inner, omega, gamma, dir);
    default:
      return 1;
  }
}

/* ------------------------------------------------------------------ */
/* GMRES(m): right preconditioning, classical Gram-Schmidt applied      */
/* twice (CGS2), Givens rotations with the sign convention              */
/*   d = sqrt(f^2 + g^2), c = |f|/d, r = sign(f) d, s = g/r             */
/*   (f = 0: c = 0, s = sign(g), r = |g|; g = 0: c = 1, s = 0, r = f).   */
/* ------------------------------------------------------------------ */

static void givens(double f, double g, double* c, double* s, double* r) {
  if (g == 0.0) {
    *c = 1.0; *s = 0.0; *r = f;
  } else if (f == 0.0) {
    *c = 0.0; *s = (g > 0.0) ? 1.0 : -1.0; *r = fabs(g);
  } else {
    double d = sqrt(f * f + g * g);
    *c = fabs(f) / d;
    *r = (f > 0.0) ? d : -d;
    *s = g / *r;
  }
}

int ora_gmres(int64_t n, const int64_t* rp, const int32_t* ci,
              const double* va, const double* b, double* x, int restart,
              double tol, int max_iters, int pc_kind, int pc_outer,
              int pc_inner, double pc_omega, double pc_gamma, int pc_dir,
              ora_info* info, double* resid_hist) {
  if (n < 0 || restart < 1 || max_iters < 0 || !(tol >= 0.0)) return 1;
  ora_info loc = {0, 0, 0, 0.0};
  const int m = restart;
  double bnorm = nrm2(n, b);
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    if (info) *info = loc;
    return 0;
  }
  double* V = malloc((size_t)(m + 1) * (size_t)n * sizeof(double));
  double* H = calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
  double* cs = malloc((size_t)m * sizeof(double));
  double* sn = malloc((size_t)m * sizeof(double));
  double* gv = malloc((size_t)(m + 1) * sizeof(double));
  double* h1 = malloc((size_t)(m + 1) * sizeof(double));
  double* h2 = malloc((size_t)(m + 1) * sizeof(double));
  double* y = malloc((size_t)m * sizeof(double));
  double* r = malloc((size_t)n * sizeof(double));
  double* z = malloc((size_t)n * sizeof(double));
  double* w = malloc((size_t)n * sizeof(double));
#define HH(i, j) H[(size_t)(i) * (size_t)m + (size_t)(j)]
#define VV(k) (V + (size_t)(k) * (size_t)n)
  int st = 0;
  int breakdown = 0;
  for (;;) {
    residual(n, rp, ci, va, b, x, r);
    double beta = nrm2(n, r);
    loc.true_relres = beta / bnorm;
    if (isnan(beta) || isinf(beta)) { st = 7; break; }
    if (loc.true_relres <= tol) { st = 0; break; }
    if (breakdown) { st = 6; break; }
    if (loc.iters >= max_iters) { st = 5; break; }
    loc.cycles++;
    for (int64_t i = 0; i < n; ++i) VV(0)[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) gv[i] = 0.0;
    gv[0] = beta;
    int k = 0;
    int nan_seen = 0;
    for (int j = 0; j < m; ++j) {
      st = ora_precond(n, rp, ci, va, VV(j), z, pc_kind, pc_outer, pc_inner,
                       pc_omega, pc_gamma, pc_dir);
      if (st) goto done;
      ora_spmv(n, rp, ci, va, z, w);
      /* first classical Gram-Schmidt pass */
      for (int i = 0; i <= j; ++i) h1[i] = dot(n, VV(i), w);
      for (int64_t q = 0; q < n; ++q) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += VV(i)[q] * h1[i];
        w[q] -= s;
      }
      /* second pass (re-orthogonalisation) */
      for (int i = 0; i <= j; ++i) h2[i] = dot(n, VV(i), w);
      for (int64_t q = 0; q < n; ++q) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += VV(i)[q] * h2[i];
        w[q] -= s;
      }
      for (int i = 0; i <= j; ++i) HH(i, j) = h1[i] + h2[i];
      double hn = nrm2(n, w);
      HH(j + 1, j) = hn;
      /* previous rotations, then the new one */
      for (int i = 0; i < j; ++i) {
        double a = HH(i, j), c = HH(i + 1, j);
        HH(i, j) = cs[i] * a + sn[i] * c;
        HH(i + 1, j) = -sn[i] * a + cs[i] * c;
      }
      double rr;
      givens(HH(j, j), HH(j + 1, j), &cs[j], &sn[j], &rr);
      HH(j, j) = rr;
      HH(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      loc.iters++;
      k = j + 1;
      if (resid_hist) resid_hist[loc.iters - 1] = fabs(gv[j + 1]) / bnorm;
      if (isnan(gv[j + 1]) || isnan(hn) || isinf(hn)) { nan_seen = 1; break; }
      if (hn == 0.0) { breakdown = 1; break; }
      for (int64_t q = 0; q < n; ++q) VV(j + 1)[q] = w[q] / hn;
      if (fabs(gv[j + 1]) <= tol * bnorm || loc.iters >= max_iters) break;
    }
    if (nan_seen) { st = 7; break; }
    /* y = R^{-1} g by back substitution, u = V y, x += M^{-1} u */
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int l = i + 1; l < k; ++l) s -= HH(i, l) * y[l];
      y[i] = s / HH(i, i);
    }
    for (int64_t q = 0; q < n; ++q) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += VV(i)[q] * y[i];
      w[q] = s;
    }
    st = ora_precond(n, rp, ci, va, w, z, pc_kind, pc_outer, pc_inner,
                     pc_omega, pc_gamma, pc_dir);
    if (st) break;
    for (int64_t q = 0; q < n; ++q) x[q] += z[q];
  }
done:
#undef HH
#undef VV
  free(V); free(H); free(cs); free(sn); free(gv); free(h1); free(h2);
  free(y); free(r); free(z); free(w);
  if (info) { loc.status = st; *info = loc; }
  return st;
}

/* ------------------------------------------------------------------ */
/* Preconditioned CG (Sec. 9 and 10 run CG with SGS2 on SPD            */
/* matrices; SGS2 from a zero start is a symmetric operator when A is). */
/* ------------------------------------------------------------------ */

int ora_cg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, double tol, int max_iters, int pc_kind,
           int pc_outer, int pc_inner, double pc_omega, double pc_gamma,
           int pc_dir, ora_info* info) {
  if (n < 0 || max_iters < 0 || !(tol >= 0.0)) return 1;
  ora_info loc = {0, 0, 0, 0.0};
  double bnorm = nrm2(n, b);
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    if (info) *info = loc;
    return 0;
  }
  double* r = malloc((size_t)n * sizeof(double));
  double* z = malloc((size_t)n * sizeof(double));
  double* p = malloc((size_t)n * sizeof(double));
  double* q = malloc((size_t)n * sizeof(double));
  int st = 0;
  int fresh = 1; /* start (or restart) the search direction from r */
  double rz = 0.0;
  residual(n, rp, ci, va, b, x, r);
  for (;;) {
    double rn = nrm2(n, r);
    if (isnan(rn) || isinf(rn)) { st = 7; break; }
    if (rn <= tol * bnorm) {
      /* the recursively updated residual says converged: confirm it */
      residual(n, rp, ci, va, b, x, q);
      double tn = nrm2(n, q);
      if (tn <= tol * bnorm) break;
      memcpy(r, q, (size_t)n * sizeof(double));
      fresh = 1;
    }
    if (loc.iters >= max_iters) { st = 5; break; }
    if (fresh) {
      st = ora_precond(n, rp, ci, va, r, z, pc_kind, pc_outer, pc_inner,
                       pc_omega, pc_gamma, pc_dir);
      if (st) break;
      memcpy(p, z, (size_t)n * sizeof(double));
      rz = dot(n, r, z);
      loc.cycles++;
      fresh = 0;
    }
    ora_spmv(n, rp, ci, va, p, q);
    double pq = dot(n, p, q);
    if (pq == 0.0) { st = 6; break; }
    double alpha = rz / pq;
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    loc.iters++;
    if (nrm2(n, r) <= tol * bnorm) continue;
    st = ora_precond(n, rp, ci, va, r, z, pc_kind, pc_outer, pc_inner,
                     pc_omega, pc_gamma, pc_dir);
    if (st) break;
    double rz_new = dot(n, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  residual(n, rp, ci, va, b, x, q);
  loc.true_relres = nrm2(n, q) / bnorm;
  free(r); free(z); free(p); free(q);
  if (info) { loc.status = st; *info = loc; }
  return st;
}

/* ------------------------------------------------------------------ */
/* Compact GS2, Eq. (9): x <- Mhat^{-1}(b + N x).                       */
/* Forward: M = D + L, N = -U; backward: M = D + U, N = -L.             */
/* ------------------------------------------------------------------ */

static void gs2c_sweep(int64_t n, const int64_t* rp, const int32_t* ci,
                       const double* va, const double* d, const double* b,
                       double* x, int inner, int lower, double* c, double* g,
                       double* gn, double* t) {
  /* c = b + N x = b - (other triangle) x */
  tri_mult(n, rp, ci, va, !lower, x, t);
  for (int64_t i = 0; i < n; ++i) c[i] = b[i] - t[i];
  for (int64_t i = 0; i < n; ++i) g[i] = c[i] / d[i];
  for (int j = 0; j < inner; ++j) {
    tri_mult(n, rp, ci, va, lower, g, t);
    for (int64_t i = 0; i < n; ++i) gn[i] = (c[i] - t[i]) / d[i];
    memcpy(g, gn, (size_t)n * sizeof(double));
  }
  memcpy(x, g, (size_t)n * sizeof(double));
}

int ora_gs2_compact(int64_t n, const int64_t* rp, const int32_t* ci,
                    const double* va, const double* b, double* x, int outer,
                    int inner, int dir) {
  if (n < 0 || outer < 0 || inner < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC)
    return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  double* c = malloc((size_t)n * sizeof(double));
  double* g = malloc((size_t)n * sizeof(double));
  double* gn = malloc((size_t)n * sizeof(double));
  double* t = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  for (int s = 0; st == 0 && s < outer; ++s) {
    if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC)
      gs2c_sweep(n, rp, ci, va, d, b, x, inner, 1, c, g, gn, t);
    if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC)
      gs2c_sweep(n, rp, ci, va, d, b, x, inner, 0, c, g, gn, t);
  }
  free(d); free(c); free(g); free(gn); free(t);
  return st;
}
