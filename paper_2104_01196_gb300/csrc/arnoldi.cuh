// Device bodies of the Arnoldi step of GMRES with CGS2 (classical
// Gram-Schmidt applied twice) and of the Givens update of the Hessenberg
// least-squares problem.  The single-system kernels (krylov.cu) run them over
// the whole vector with one grid-stride loop; the packed kernels (pack.cu)
// run them over one system's rows of a block-diagonal pack.  V is stored by
// vector: entry i of basis vector k at V[k * ld + i].
#pragma once

#include "internal.cuh"
#include "reduce.cuh"

namespace gs2 {

// acc[k] += sum over this thread's rows i of V_k[i] w[i], k < JC
template <int JC>
__device__ __forceinline__ void dots_rows(int i, int end, int step, int ld,
                                          const double* __restrict__ V,
                                          const double* __restrict__ w, double (&acc)[JC]) {
  for (; i < end; i += step) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < JC; ++k) acc[k] = fma(__ldg(V + (size_t)k * ld + i), wi, acc[k]);
  }
}

// w_i -= sum_k V_k[i] h_k over this thread's rows, then (NORM) acc[0] +=
// w_i^2 or (!NORM) acc[k] += V_k[i] w_i.  hneg holds -h.  The update is one
// FMA chain started at w_i with the negated coefficients, so it issues no
// FP64 instruction beyond its products; at the FP64 issue interval (one warp
// instruction per 64 cycles per scheduler) a dependent chain does not stall.
template <int JC, bool NORM>
__device__ __forceinline__ void update_rows(int i, int end, int step, int ld,
                                            const double* __restrict__ V,
                                            const double* hneg, double* __restrict__ w,
                                            double (&acc)[NORM ? 1 : JC]) {
  for (; i < end; i += step) {
    double wn = w[i];
#pragma unroll
    for (int k = 0; k < JC; ++k) wn = fma(__ldg(V + (size_t)k * ld + i), hneg[k], wn);
    w[i] = wn;
    if (NORM) {
      acc[0] = fma(wn, wn, acc[0]);
    } else {
#pragma unroll
      for (int k = 0; k < JC; ++k) acc[k] = fma(__ldg(V + (size_t)k * ld + i), wn, acc[k]);
    }
  }
}

// Givens step j on one thread's own copies (the solvers whose every block
// or CTA holds the Krylov scalars): col = column j of H with H(j+1, j)
// already in col[j + 1]; the earlier rotations cs/sn[0 .. j) are applied to
// it, the new rotation is formed by the rules of givens_block below and
// applied to col and to g.  Returns the residual estimate |g_{j+1}|.
__device__ __forceinline__ double givens_column(double* col, double* cs, double* sn, double* g,
                                                int j) {
  for (int q = 0; q < j; ++q) {
    const double u = col[q], v = col[q + 1];
    col[q] = cs[q] * u + sn[q] * v;
    col[q + 1] = -sn[q] * u + cs[q] * v;
  }
  const double f = col[j], gg = col[j + 1];
  double c, sg, rr;
  if (gg == 0.0) {
    c = 1.0; sg = 0.0; rr = f;
  } else if (f == 0.0) {
    c = 0.0; sg = gg > 0.0 ? 1.0 : -1.0; rr = fabs(gg);
  } else {
    const double d = sqrt(f * f + gg * gg);
    c = fabs(f) / d;
    rr = f > 0.0 ? d : -d;
    sg = gg / rr;
  }
  cs[j] = c;
  sn[j] = sg;
  col[j] = rr;
  col[j + 1] = 0.0;
  const double gj = g[j];
  g[j + 1] = -sg * gj;
  g[j] = c * gj;
  return fabs(-sg * gj);
}

// Givens step j of one system, run by a whole block: H(j+1, j) = ||w|| from
// the partial sums part[p0 .. p1), the earlier rotations applied to column
// j, the new rotation from (H(j,j), H(j+1,j)) with
//   d = sqrt(f^2 + g^2), c = |f|/d, r = sign(f) d, s = g/r
// (f = 0: c = 0, s = sign(g), r = |g|; g = 0: c = 1, s = 0, r = f), the
// residual estimate |g_{j+1}| and the stop decision of the cycle.  The
// column and the earlier rotations are staged in shared memory by all
// threads; the sequential rotation chain runs on thread 0.  Returns (to
// every thread) whether this step ended the system's cycle.
// Every global value the step needs (the column, the rotations, the norm
// partials, g_j and the state fields) is loaded before the first use of any
// of them, so the loads share one round trip instead of following the
// rotation chain one after another.  With skip_if non-null the block returns
// false without side effects when *skip_if is set (read with the others).
__device__ __forceinline__ bool givens_block(const double* __restrict__ part, int p0, int p1,
                                             double* col, double* cs, double* sn, double* gv,
                                             int j, KrylovState* st,
                                             const int* skip_if = nullptr) {
  __shared__ double red[32];
  __shared__ double col_s[kMaxRestart + 2], cs_s[kMaxRestart + 1], sn_s[kMaxRestart + 1];
  __shared__ int stopped;
  const int skip = skip_if ? *skip_if : 0;
  double gj = 0.0, tol_abs = 0.0;
  int iters = 0, max_iters = 0;
  if (threadIdx.x == 0) {
    gj = gv[j];
    iters = st->iters;
    max_iters = st->max_iters;
    tol_abs = st->tol_abs;
  }
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col_s[i] = col[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs_s[i] = cs[i];
    sn_s[i] = sn[i];
  }
  double s = 0.0;
  for (int b = p0 + threadIdx.x; b < p1; b += blockDim.x) s += part[b];
  if (skip) return false;  // the same value in every thread: a uniform exit
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nrm2 += red[w];
    const double hn = sqrt(nrm2);
    col_s[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = col_s[i], c = col_s[i + 1];
      col_s[i] = cs_s[i] * a + sn_s[i] * c;
      col_s[i + 1] = -sn_s[i] * a + cs_s[i] * c;
    }
    const double f = col_s[j], g = col_s[j + 1];
    double c, sgv, r;
    if (g == 0.0) {
      c = 1.0; sgv = 0.0; r = f;
    } else if (f == 0.0) {
      c = 0.0; sgv = g > 0.0 ? 1.0 : -1.0; r = fabs(g);
    } else {
      const double d = sqrt(f * f + g * g);
      c = fabs(f) / d;
      r = f > 0.0 ? d : -d;
      sgv = g / r;
    }
    cs[j] = c;
    sn[j] = sgv;
    col_s[j] = r;
    col_s[j + 1] = 0.0;
    gv[j + 1] = -sgv * gj;
    gv[j] = c * gj;
    st->iters = iters + 1;
    st->k = j + 1;
    st->hn = hn;
    st->inv_hn = 1.0 / hn;
    const double est = fabs(-sgv * gj);
    int stop = 0;
    if (isnan(est) || isnan(hn) || isinf(hn)) {
      st->status = GS2_ERR_NAN;
      stop = 1;
    } else if (hn == 0.0) {
      st->status = GS2_ERR_BREAKDOWN;
      stop = 1;
    } else if (est <= tol_abs || iters + 1 >= max_iters) {
      stop = 1;
    }
    if (stop) st->stop = 1;
    stopped = stop;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = col_s[i];
  return stopped != 0;
}

// y = R^{-1} g over the k steps of a cycle, run by a whole block:
// column-oriented back substitution, y_i = g_i / R_ii, then every g_l
// (l < i) -= R_li y_i in parallel; g lives in shared memory.
__device__ __forceinline__ void backsolve_block(const double* __restrict__ H, int ldh,
                                                const double* gv, double* y, int k) {
  __shared__ double g_s[kMaxRestart + 1];
  __shared__ double yi_s;
  for (int i = threadIdx.x; i < k; i += blockDim.x) g_s[i] = gv[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double* ci = H + (size_t)i * ldh;
    if (threadIdx.x == 0) {
      yi_s = g_s[i] / ci[i];
      y[i] = yi_s;
    }
    __syncthreads();
    const double yi = yi_s;
    for (int l = threadIdx.x; l < i; l += blockDim.x) g_s[l] -= ci[l] * yi;
    __syncthreads();
  }
}

// u_i = sum_{l < k} V_l[i] ys[l] over this thread's rows, and the
// preconditioner's D^{-1} u in the sweep precision (whichever of rhat64,
// rhat32 is non-null)
template <int MAXK>
__device__ __forceinline__ void combine_rows(int i, int end, int step, size_t ld,
                                             const double* __restrict__ V, const double* ys,
                                             int k, double* u, const double* __restrict__ dinv,
                                             double* rhat64, float* rhat32) {
  for (; i < end; i += step) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < MAXK; ++l)
      if (l < k) s = fma(__ldg(V + (size_t)l * ld + i), ys[l], s);
    u[i] = s;
    if (rhat64) rhat64[i] = dinv[i] * s;
    if (rhat32) rhat32[i] = (float)(dinv[i] * s);
  }
}

// v = w * a and the preconditioner's D^{-1} v over this thread's rows
__device__ __forceinline__ void scale_rows(int i, int end, int step, double a,
                                           const double* __restrict__ w, double* v,
                                           const double* __restrict__ dinv, double* rhat64,
                                           float* rhat32) {
  for (; i < end; i += step) {
    const double x = w[i] * a;
    v[i] = x;
    if (rhat64) rhat64[i] = dinv[i] * x;
    if (rhat32) rhat32[i] = (float)(dinv[i] * x);
  }
}

}  // namespace gs2
