/*
 * GS2 with its inner sweeps in a lower precision than the outer iteration.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Sec. 10 of the paper runs the preconditioner in single precision inside a
 * double-precision Krylov solver and reports that the iteration count is
 * kept.  The library offers that form and one more, FP16 values with a
 * per-row scale; this file states both as definitions, one loop per formula:
 *
 *   r     = b - A x                                  FP64 (the outer residual)
 *   rhat  = fl32(D^{-1} r)                           rounded once, at the boundary
 *   FP32:  t_ij = fl32((D^{-1} T)_ij)
 *   FP16:  m_i = max_j |(D^{-1} T)_ij|,  sigma_i = fl32(m_i),
 *          q_ij = fl16((D^{-1} T)_ij / m_i)  (0 when m_i = 0: a row whose
 *          stored triangle entries are all zero),  t_ij = sigma_i q_ij
 *   g^(0) = rhat
 *   s_i   = sum_j t_ij g_j          FP32 operations, the row's stored order
 *           (FP16: sigma_i (sum_j q_ij g_j), the scale applied once per row)
 *   g^(j+1)_i = (1-gamma') g_i + gamma' (rhat_i - omega' s_i)   FP32,
 *           omega' = fl32(omega), gamma' = fl32(gamma)
 *   x     = x + omega g^(inner)                      FP64
 *
 * T = L (forward half) or U (backward half); symmetric = forward then
 * backward, the residual recomputed in FP64 in between.  Every float
 * operation is one IEEE binary32 operation rounded to nearest (the file is
 * compiled without contraction, so a*b+c is two roundings); fl16 is IEEE
 * binary16 round-to-nearest-even, written out below from its definition.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

_Thread_local int ora_precision = ORA_PREC_FP64;

void ora_set_precision(int prec) { ora_precision = prec; }

/* IEEE 754 binary16 rounding of a real value, round to nearest, ties to
 * even: 11 significant bits for normal numbers (|v| >= 2^-14), a fixed
 * quantum of 2^-24 below that (subnormals), and infinity from the halfway
 * point 65520 = (2 - 2^-11) 2^15 upwards.  Returned as a double (every
 * binary16 value is exact in double). */
double ora_round_half(double v) {
  if (isnan(v)) return v;
  const double a = fabs(v);
  if (a >= 65520.0) return v > 0 ? INFINITY : -INFINITY;
  int e;
  frexp(a, &e);                       /* a = f 2^e, f in [0.5, 1) */
  int qexp = e - 11;                  /* 11 significant bits: quantum 2^(e-11) */
  if (qexp < -24) qexp = -24;         /* subnormal range: quantum 2^-24 */
  const double q = ldexp(1.0, qexp);
  double k = a / q;                   /* exact: scaling by a power of two */
  double fl = floor(k);
  double rem = k - fl;
  if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0)) fl += 1.0;
  const double out = fl * q;
  return v < 0 ? -out : out;
}

/* One half sweep with triangle T (lower = 1: L, lower = 0: U). */
static void lp_half(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                    const double* d, const double* b, double* x, int inner, double omega,
                    double gamma, int lower, int prec, double* r, float* rhat, float* g,
                    float* gn) {
  /* r = b - A x in FP64 */
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
    r[i] = b[i] - s;
  }
  /* rhat = fl32(D^{-1} r); g^(0) = rhat */
  for (int64_t i = 0; i < n; ++i) {
    rhat[i] = (float)(r[i] / d[i]);
    g[i] = rhat[i];
  }
  const float om = (float)omega, ga = (float)gamma;
  const float one_minus_ga = 1.0f - ga;
  for (int j = 0; j < inner; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      /* the row's triangle entries, prescaled by D^{-1} (FP64), then
       * stored in the sweep precision */
      double m = 0.0;
      if (prec == ORA_PREC_FP16_ROWSCALED)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
          const int64_t c = ci[k];
          if ((lower && c < i) || (!lower && c > i)) m = fmax(m, fabs(va[k] / d[i]));
        }
      float s = 0.0f;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int64_t c = ci[k];
        if (!((lower && c < i) || (!lower && c > i))) continue;
        const double t64 = va[k] / d[i];
        float t;
        if (prec == ORA_PREC_FP32) t = (float)t64;
        else t = m > 0.0 ? (float)ora_round_half(t64 / m) : 0.0f;  /* q_ij */
        const float p = t * g[c];
        s = s + p;
      }
      if (prec == ORA_PREC_FP16_ROWSCALED) s = s * (float)m;
      const float upd = rhat[i] - om * s;
      gn[i] = one_minus_ga * g[i] + ga * upd;
    }
    memcpy(g, gn, (size_t)n * sizeof(float));
  }
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * (double)g[i];
}

int ora_gs2_lp(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, int outer, int inner, double omega,
               double gamma, int dir, int prec) {
  if (n < 0 || outer < 0 || inner < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC) return 1;
  if (prec == ORA_PREC_FP64)
    return ora_gs2(n, rp, ci, va, b, x, outer, inner, omega, gamma, dir);
  if (prec != ORA_PREC_FP32 && prec != ORA_PREC_FP16_ROWSCALED) return 1;
  if (n == 0) return 0;
  double* d = malloc((size_t)n * sizeof(double));
  double* r = malloc((size_t)n * sizeof(double));
  float* rhat = malloc((size_t)n * sizeof(float));
  float* g = malloc((size_t)n * sizeof(float));
  float* gn = malloc((size_t)n * sizeof(float));
  int st = ora_diag(n, rp, ci, va, d);
  for (int s = 0; st == 0 && s < outer; ++s) {
    if (dir == ORA_FORWARD || dir == ORA_SYMMETRIC)
      lp_half(n, rp, ci, va, d, b, x, inner, omega, gamma, 1, prec, r, rhat, g, gn);
    if (dir == ORA_BACKWARD || dir == ORA_SYMMETRIC)
      lp_half(n, rp, ci, va, d, b, x, inner, omega, gamma, 0, prec, r, rhat, g, gn);
  }
  free(d); free(r); free(rhat); free(g); free(gn);
  return st;
}
