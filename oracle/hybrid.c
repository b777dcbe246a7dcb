/*
 * Hybrid (block-Jacobi) relaxations of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sec. 3 describes the hybrid Gauss-Seidel of distributed solvers: the rows
 * are split into 1-D blocks (one per process); the processes exchange the
 * solution values on their boundaries and then relax their own rows
 * independently, several local sweeps per exchange, with the values of the
 * other blocks held at what was exchanged.  Block p solves
 *   A^(p) x^(p) = b^(p) - E^(p) y^(p),
 * A^(p) the diagonal block, E^(p) the couplings to the other blocks and y the
 * exchanged values.  The two-stage listing of Sec. 4 runs n_t exchanges, n_k
 * local outer sweeps per exchange and n_j local inner JR sweeps; the
 * symmetric sweep takes its forward and backward halves after one exchange.
 *
 * Readings taken here:
 *  - the blocks are contiguous: block p holds rows [floor(p n / P),
 *    floor((p+1) n / P)), P = parts;
 *  - per exchange t: c = b - E x (E: entries whose column lies outside the
 *    row's block; x as it stands when the exchange happens); then n_k
 *    local sweeps, each a half sweep (or two, symmetric) on A_loc x = c with
 *    A_loc = A - E, exactly as the global sweeps of oracle.c but with L and
 *    U replaced by their local parts;
 *  - P = 1 is the global method with n_t * n_k sweeps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* block index of every row */
static void block_of_rows(int64_t n, int parts, int32_t* blk) {
  for (int p = 0; p < parts; ++p) {
    const int64_t lo = (int64_t)p * n / parts, hi = (int64_t)(p + 1) * n / parts;
    for (int64_t i = lo; i < hi; ++i) blk[i] = p;
  }
}

/* c = b - E x: the couplings to other blocks with the exchanged x */
static void exchange_rhs(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                         const int32_t* blk, const double* b, const double* x, double* c) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (blk[ci[k]] != blk[i]) s += va[k] * x[ci[k]];
    c[i] = b[i] - s;
  }
}

/* r = c - A_loc x */
static void local_residual(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                           const int32_t* blk, const double* c, const double* x, double* r) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (blk[ci[k]] == blk[i]) s += va[k] * x[ci[k]];
    r[i] = c[i] - s;
  }
}

/* t = T_loc g: strict lower (lower = 1) or upper local triangle */
static void local_tri_mult(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                           const int32_t* blk, int lower, const double* g, double* t) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = ci[k];
      if (blk[j] != blk[i]) continue;
      if ((lower && j < i) || (!lower && j > i)) s += va[k] * g[j];
    }
    t[i] = s;
  }
}

/* one local GS2 half sweep: r = c - A_loc x, g0 = D^{-1} r, inner damped JR
 * sweeps with the local triangle, x += omega g */
static void local_gs2_half(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                           const int32_t* blk, const double* d, const double* c, double* x,
                           int inner, double omega, double gamma, int lower, double* r,
                           double* g, double* gn, double* t) {
  local_residual(n, rp, ci, va, blk, c, x, r);
  for (int64_t i = 0; i < n; ++i) g[i] = r[i] / d[i];
  for (int j = 0; j < inner; ++j) {
    local_tri_mult(n, rp, ci, va, blk, lower, g, t);
    for (int64_t i = 0; i < n; ++i)
      gn[i] = (1.0 - gamma) * g[i] + gamma * (r[i] - omega * t[i]) / d[i];
    memcpy(g, gn, (size_t)n * sizeof(double));
  }
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * g[i];
}

/* one local exact GS / SOR row update on A_loc x = c */
static void local_gs_row(int64_t i, const int64_t* rp, const int32_t* ci, const double* va,
                         const int32_t* blk, const double* c, double* x, double omega) {
  double sum = 0.0, aii = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    if (blk[ci[k]] != blk[i]) continue;
    if (ci[k] == i) aii += va[k];
    else sum += va[k] * x[ci[k]];
  }
  x[i] = (1.0 - omega) * x[i] + omega * (c[i] - sum) / aii;
}

int ora_hybrid(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, int kind, int parts, int outer, int local, int inner,
               double omega, double gamma, int dir) {
  if (n < 0 || parts < 1 || outer < 0 || local < 1 || inner < 0) return 1;
  if (kind != ORA_PC_GS2 && kind != ORA_PC_JR && kind != ORA_PC_GS) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC) return 1;
  if (n == 0) return 0;
  if (parts > n) parts = (int)n;
  double* d = malloc((size_t)n * sizeof(double));
  int st = ora_diag(n, rp, ci, va, d);
  if (st) {
    free(d);
    return st;
  }
  int32_t* blk = malloc((size_t)n * sizeof(int32_t));
  double* c = malloc((size_t)n * sizeof(double));
  double* r = malloc((size_t)n * sizeof(double));
  double* g = malloc((size_t)n * sizeof(double));
  double* gn = malloc((size_t)n * sizeof(double));
  double* t = malloc((size_t)n * sizeof(double));
  block_of_rows(n, parts, blk);
  for (int s = 0; s < outer; ++s) {
    exchange_rhs(n, rp, ci, va, blk, b, x, c);
    for (int k = 0; k < local; ++k) {
      if (kind == ORA_PC_JR) {
        /* x += omega D^{-1} (c - A_loc x) */
        local_residual(n, rp, ci, va, blk, c, x, r);
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * (r[i] / d[i]);
        continue;
      }
      if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC) {
        if (kind == ORA_PC_GS2)
          local_gs2_half(n, rp, ci, va, blk, d, c, x, inner, omega, gamma, 1, r, g, gn, t);
        else
          for (int64_t i = 0; i < n; ++i) local_gs_row(i, rp, ci, va, blk, c, x, omega);
      }
      if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC) {
        if (kind == ORA_PC_GS2)
          local_gs2_half(n, rp, ci, va, blk, d, c, x, inner, omega, gamma, 0, r, g, gn, t);
        else
          for (int64_t i = n - 1; i >= 0; --i) local_gs_row(i, rp, ci, va, blk, c, x, omega);
      }
    }
  }
  free(d); free(blk); free(c); free(r); free(g); free(gn); free(t);
  return 0;
}

/* the partition the hybrid preconditioner kinds use inside GMRES / CG */
_Thread_local int ora_hybrid_parts = 1;
_Thread_local int ora_hybrid_local = 1;

void ora_set_hybrid(int parts, int local) {
  ora_hybrid_parts = parts < 1 ? 1 : parts;
  ora_hybrid_local = local < 1 ? 1 : local;
}
