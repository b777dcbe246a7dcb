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
 *   FP16:  m_i = max_j |(D^{-1} T)_ij| = f 2^e_i with f in [1/2, 1) (e_i = 0
 *          when m_i = 0; e_i clamped to [-126, 127]), sigma_i = 2^e_i,
 *          q_ij = fl16((D^{-1} T)_ij / sigma_i),  t_ij = sigma_i q_ij
 *          (a power-of-two scale: the division and the multiplication by
 *          sigma_i are exact, fl16 is the only rounding)
 *   g^(0) = rhat
 *   s_i   = sum_j t_ij g_j          FP32 operations, the row's stored order
 *           (FP16: sigma_i (sum_j q_ij g_j), the scale applied once per row,
 *           exactly)
 *   g^(j+1)_i = (1-gamma') g_i + gamma' (rhat_i - omega' s_i)   FP32,
 *           omega' = fl32(omega), gamma' = fl32(gamma)
 *   x     = x + omega g^(inner)                      FP64
 *
 * T = L (forward half) or U (backward half); symmetric = forward then
 * backward, the residual recomputed in FP64 in between.
 *
 * Whole-sweep precisions (Sec. 10 runs the outer GS iteration in single
 * precision too): the iterate and the residual are FP32 as well,
 *   x32   = fl32(x),  bhat_i = fl32(b_i / a_ii)
 *   rhat_i = (bhat_i - x32_i) - s_i,  s_i = sum_{j != i} o_ij x32_j     FP32
 *           (o = D^{-1}(L + U): the row's lower entries, then its upper ones,
 *           each in stored order; values fl32(a_ij / a_ii), or row-scaled
 *           FP16 with the row's own power-of-two scale over all its
 *           off-diagonal entries, applied to the sum)
 *   g^(0) = rhat, the inner sweeps as above,  x32 = x32 + fl32(omega) g
 *   x = (double) x32 once the sweeps are done.  Every float
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

/* value of an entry t64 of a prescaled matrix in precision prec (FP32 or
 * FP16 with the row's scale exponent e) */
static float lp_value(double t64, int prec, int e) {
  if (prec == ORA_PREC_FP32) return (float)t64;
  return (float)ora_round_half(ldexp(t64, -e));
}

/* the power-of-two scale exponent of the entries of row i selected by
 * sel (1: j < i, 2: j > i, 3: both) */
static int row_exponent(const int64_t* rp, const int32_t* ci, const double* va,
                        const double* d, int64_t i, int sel) {
  double m = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    const int64_t c = ci[k];
    if (((sel & 1) && c < i) || ((sel & 2) && c > i)) m = fmax(m, fabs(va[k] / d[i]));
  }
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  if (e < -126) e = -126;
  if (e > 127) e = 127;
  return e;
}

/* one inner JR sweep in FP32 on triangle T of the values precision vp:
 * gn = (1-gamma') g + gamma' (rhat - omega' s) */
static void lp_inner(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                     const double* d, int lower, int vp, float om, float ga, const float* rhat,
                     const float* g, float* gn) {
  const float one_minus_ga = 1.0f - ga;
  for (int64_t i = 0; i < n; ++i) {
    const int e = vp == ORA_PREC_FP16_ROWSCALED ? row_exponent(rp, ci, va, d, i, lower ? 1 : 2)
                                                : 0;
    float s = 0.0f;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t c = ci[k];
      if (!((lower && c < i) || (!lower && c > i))) continue;
      const float p = lp_value(va[k] / d[i], vp, e) * g[c];
      s = s + p;
    }
    if (vp == ORA_PREC_FP16_ROWSCALED) s = ldexpf(s, e);
    const float upd = rhat[i] - om * s;
    gn[i] = one_minus_ga * g[i] + ga * upd;
  }
}

/* One half sweep with triangle T (lower = 1: L, lower = 0: U): FP64
 * residual, inner sweeps in the value precision prec. */
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
  for (int j = 0; j < inner; ++j) {
    lp_inner(n, rp, ci, va, d, lower, prec, (float)omega, (float)gamma, rhat, g, gn);
    memcpy(g, gn, (size_t)n * sizeof(float));
  }
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + omega * (double)g[i];
}

/* the whole-sweep precisions (see the header comment) */
static int gs2_sweep_lp(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                        const double* b, double* x, int outer, int inner, double omega,
                        double gamma, int dir, int vp) {
  double* d = malloc((size_t)n * sizeof(double));
  float* x32 = malloc((size_t)n * sizeof(float));
  float* bh = malloc((size_t)n * sizeof(float));
  float* rhat = malloc((size_t)n * sizeof(float));
  float* g = malloc((size_t)n * sizeof(float));
  float* gn = malloc((size_t)n * sizeof(float));
  int st = ora_diag(n, rp, ci, va, d);
  const float om = (float)omega, ga = (float)gamma;
  if (st == 0) {
    for (int64_t i = 0; i < n; ++i) {
      x32[i] = (float)x[i];
      bh[i] = (float)(b[i] / d[i]);
    }
    for (int sw = 0; sw < outer; ++sw) {
      for (int half = 0; half < 2; ++half) {
        const int lower = half == 0;
        if (lower && dir == ORA_BACKWARD) continue;
        if (!lower && dir == ORA_FORWARD) continue;
        /* rhat = (bhat - x32) - O x32, lower entries of the row first */
        for (int64_t i = 0; i < n; ++i) {
          const int e = vp == ORA_PREC_FP16_ROWSCALED ? row_exponent(rp, ci, va, d, i, 3) : 0;
          float s = 0.0f;
          for (int pass = 0; pass < 2; ++pass)
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
              const int64_t c = ci[k];
              if (!((pass == 0 && c < i) || (pass == 1 && c > i))) continue;
              const float p = lp_value(va[k] / d[i], vp, e) * x32[c];
              s = s + p;
            }
          if (vp == ORA_PREC_FP16_ROWSCALED) s = ldexpf(s, e);
          rhat[i] = (bh[i] - x32[i]) - s;
          g[i] = rhat[i];
        }
        for (int j = 0; j < inner; ++j) {
          lp_inner(n, rp, ci, va, d, lower, vp, om, ga, rhat, g, gn);
          memcpy(g, gn, (size_t)n * sizeof(float));
        }
        for (int64_t i = 0; i < n; ++i) x32[i] = x32[i] + om * g[i];
      }
    }
    for (int64_t i = 0; i < n; ++i) x[i] = (double)x32[i];
  }
  free(d); free(x32); free(bh); free(rhat); free(g); free(gn);
  return st;
}

int ora_gs2_lp(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, int outer, int inner, double omega,
               double gamma, int dir, int prec) {
  if (n < 0 || outer < 0 || inner < 0) return 1;
  if (dir != ORA_FORWARD && dir != ORA_BACKWARD && dir != ORA_SYMMETRIC) return 1;
  if (prec == ORA_PREC_FP64)
    return ora_gs2(n, rp, ci, va, b, x, outer, inner, omega, gamma, dir);
  if (prec == ORA_PREC_FP32_SWEEP || prec == ORA_PREC_FP16_SWEEP)
    return n == 0 ? 0
                  : gs2_sweep_lp(n, rp, ci, va, b, x, outer, inner, omega, gamma, dir,
                                 prec == ORA_PREC_FP32_SWEEP ? ORA_PREC_FP32
                                                             : ORA_PREC_FP16_ROWSCALED);
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
