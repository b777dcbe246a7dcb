// Relaxation drivers: GS2 (non-compact Eq. 2 and compact Eq. 9), exact
// GS/SOR by level-scheduled triangular solves, damped JR, and the
// zero-start preconditioner application used by the Krylov solvers.
#include <algorithm>

#include "internal.cuh"

namespace gs2 {

__global__ void k_fill(int n, double* y, double v, const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = v;
}

__global__ void k_copy(int n, double* y, const double* __restrict__ x, const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = x[i];
}

static void launch_fill(gs2_handle* h, double* y, double v, const int* skip) {
  k_fill<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>((int)h->n, y, v, skip);
  GS2_LAUNCH_CHECK();
}

void launch_fill_value(gs2_handle* h, double* y, double v) { launch_fill(h, y, v, nullptr); }

static void launch_copy_skip(gs2_handle* h, double* y, const double* x, const int* skip) {
  KernelTimer tm(h, "copy", 16.0 * h->n);
  k_copy<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>((int)h->n, y, x, skip);
  GS2_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// GS2 pieces
// ---------------------------------------------------------------------------

static void* rhat_buf(gs2_handle* h, int prec) {
  return prec == GS2_FP64 ? (void*)h->rhat : (void*)h->rhat32;
}

// n_j inner JR sweeps (Eq. 4-5, damped), the last one fused with the update
// of x in `last_mode` (x += omega g or x = omega g).
static void inner_sweeps(gs2_handle* h, const DevCsr& T, int prec, const void* rhat,
                         double* x, double omega, double gamma, int inner, int last_mode,
                         const int* skip) {
  void* bufA = prec == GS2_FP64 ? (void*)h->g0 : (void*)h->g32a;
  void* bufB = prec == GS2_FP64 ? (void*)h->g1 : (void*)h->g32b;
  const void* gin = rhat;  // g_0 = D^{-1} r  (Eq. 3)
  for (int j = 0; j < inner; ++j) {
    const bool last = j == inner - 1;
    void* gout = last ? nullptr : (j % 2 == 0 ? bufA : bufB);
    launch_inner(h, T, prec, rhat, gin, gout, x, omega, gamma, last ? last_mode : INNER_MID,
                 skip);
    gin = gout;
  }
}

static void resid_into(gs2_handle* h, const DevCsr& R, int prec, const double* b,
                       const double* x, const int* skip) {
  if (prec == GS2_FP64)
    launch_resid_matrix(h, R, b, x, nullptr, h->rhat, nullptr, skip);
  else
    launch_resid_matrix(h, R, b, x, nullptr, nullptr, h->rhat32, skip);
}

static void compact_rhs_into(gs2_handle* h, int prec, const DevCsr& Tother, const double* b,
                             const double* x, const int* skip) {
  if (prec == GS2_FP64)
    launch_compact_rhs(h, Tother, b, x, h->rhat, nullptr, skip);
  else
    launch_compact_rhs(h, Tother, b, x, nullptr, h->rhat32, skip);
}

// One half sweep of GS2 on triangle T.  x_zero: x is known to be 0 and the
// sweep-precision D^{-1} b is already in the rhat buffer.  R: the matrix of
// the residual (A; the local block in the hybrid form).
static void gs2_half(gs2_handle* h, const gs2_params* p, const DevCsr& T, const DevCsr& Tother,
                     const double* b, double* x, bool x_zero, const int* skip,
                     const DevCsr* R = nullptr) {
  const int prec = p->precision;
  void* rh = rhat_buf(h, prec);
  if (p->form == GS2_COMPACT) {
    // x <- Mhat^{-1} (b + N x): every half sweep overwrites x
    if (!x_zero) compact_rhs_into(h, prec, Tother, b, x, skip);
    if (p->inner == 0)
      launch_rhat_update(h, prec, rh, x, 1.0, false, skip);
    else
      inner_sweeps(h, T, prec, rh, x, 1.0, 1.0, p->inner, INNER_LAST_SET, skip);
    return;
  }
  // non-compact: x += omega Mhat^{-1} (b - A x)
  if (!x_zero) resid_into(h, R ? *R : h->A, prec, b, x, skip);
  const int mode = x_zero ? INNER_LAST_SET : INNER_LAST_ADD;
  if (p->inner == 0)
    launch_rhat_update(h, prec, rh, x, p->omega, !x_zero, skip);
  else
    inner_sweeps(h, T, prec, rh, x, p->omega, p->gamma, p->inner, mode, skip);
}

// One half sweep of a whole-sweep precision (GS2_FP32_SWEEP,
// GS2_FP16_SWEEP) on triangle T, all in FP32 arithmetic on the iterate x32:
//   rhat = fl32(D^{-1} b) - x32 - O x32   (O = D^{-1}(L + U); skipped from
//                                          x32 = 0, where rhat = bhat32)
//   n_j inner sweeps on T from g_0 = rhat, x32 (+)= omega g
// bhat32 = fl32(D^{-1} b) must be prepared.  last: the final half sweep of
// the call, which writes the FP64 x = (double) x32 instead of x32.
static void gs2_half_sweep32(gs2_handle* h, const gs2_params* p, const DevCsr& T, double* x,
                             bool x_zero, bool last, const int* skip) {
  const int vprec = value_precision(p->precision);
  if (!x_zero) launch_resid_sweep(h, vprec, skip);
  const float* rh = x_zero ? h->bhat32 : h->rhat32;
  const int mode = last ? (x_zero ? INNER_LAST_SET32_OUT : INNER_LAST_ADD32_OUT)
                        : (x_zero ? INNER_LAST_SET32 : INNER_LAST_ADD32);
  if (p->inner == 0)
    launch_rhat_update32(h, rh, x, p->omega, mode, skip);
  else
    inner_sweeps(h, T, vprec, rh, x, p->omega, p->gamma, p->inner, mode, skip);
}

// The half sweeps of a whole-sweep-precision application in order; x_zero:
// x = 0 and bhat32 is prepared (the preconditioner), else x32 = fl32(x) and
// bhat32 = fl32(D^{-1} b) are formed first.
static void sweep32_relax(gs2_handle* h, const gs2_params* p, const double* b, double* x,
                          bool x_zero, int sweeps, const int* skip) {
  if (!x_zero) {
    launch_to32(h, x, h->x32, skip);
    launch_prep_rhat(h, b, nullptr, h->bhat32, skip);
  }
  const bool fwd = p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC;
  const bool bwd = p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC;
  bool zero = x_zero;
  for (int s = 0; s < sweeps; ++s) {
    if (fwd) {
      gs2_half_sweep32(h, p, h->L, x, zero, s == sweeps - 1 && !bwd, skip);
      zero = false;
    }
    if (bwd) {
      gs2_half_sweep32(h, p, h->U, x, zero, s == sweeps - 1, skip);
      zero = false;
    }
  }
}

// Sweeps of a GS2 / JR parameter set: n_t = outer exchanges of n_k local
// sweeps each (one block: n_t n_k global sweeps)
static int global_sweeps(const gs2_params* p) {
  return p->outer * std::max(1, p->local_sweeps);
}

// ---------------------------------------------------------------------------
// hybrid (block-Jacobi) form, Sec. 3: per exchange c = b - E x with the other
// blocks' values frozen, then n_k local sweeps on A_loc x = c (GS2 half
// sweeps with the local triangles, or JR).  x_zero: x = 0 and D^{-1} b is in
// the rhat buffer of the sweep precision.
// ---------------------------------------------------------------------------

static void gs_half_levels(gs2_handle* h, const DevCsr& T, const std::vector<int>& ptr,
                           const int* rows, const DevCsr& R, const double* b, double* x,
                           double omega, bool x_zero, const int* skip);

static void hybrid_apply(gs2_handle* h, const gs2_params* p, const Hybrid& Y, const double* b,
                         double* x, bool x_zero, const int* skip) {
  const int nk = std::max(1, p->local_sweeps);
  bool zero = x_zero;
  for (int t = 0; t < p->outer; ++t) {
    const double* c = b;  // E x = 0 while x = 0
    if (!zero) {
      launch_resid_matrix(h, Y.E, b, x, Y.c, nullptr, nullptr, skip);
      c = Y.c;
    }
    for (int k = 0; k < nk; ++k) {
      if (p->kind == GS2_PC_JR) {
        if (zero) {
          launch_rhat_update(h, GS2_FP64, h->rhat, x, p->omega, false, skip);
        } else {
          launch_jr_matrix(h, Y.Aloc, c, x, h->t, p->omega, skip);
          launch_copy_skip(h, x, h->t, skip);
        }
        zero = false;
        continue;
      }
      if (p->kind == GS2_PC_GS) {
        // local exact GS / SOR: the local triangular solves by level sets
        if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC) {
          gs_half_levels(h, Y.Lloc, Y.lev_ptr_L, Y.lev_rows_L, Y.Aloc, c, x, p->omega, zero,
                         skip);
          zero = false;
        }
        if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC) {
          gs_half_levels(h, Y.Uloc, Y.lev_ptr_U, Y.lev_rows_U, Y.Aloc, c, x, p->omega, zero,
                         skip);
          zero = false;
        }
        continue;
      }
      if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC) {
        gs2_half(h, p, Y.Lloc, Y.Uloc, c, x, zero, skip, &Y.Aloc);
        zero = false;
      }
      if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC) {
        gs2_half(h, p, Y.Uloc, Y.Lloc, c, x, zero, skip, &Y.Aloc);
        zero = false;
      }
    }
  }
}

void gs2_relax(gs2_handle* h, const double* b, double* x, const gs2_params* p) {
  if (Hybrid* Y = p->parts > 1 ? ensure_hybrid(h, p) : nullptr) {
    hybrid_apply(h, p, *Y, b, x, false, nullptr);
    return;
  }
  if (p->kind == GS2_PC_JR) {
    jr_relax(h, b, x, global_sweeps(p), p->omega);
    return;
  }
  if (p->kind == GS2_PC_GS) {
    ensure_levels(h);
    gs_relax(h, b, x, global_sweeps(p), p->omega, p->direction);
    return;
  }
  if (p->kind == GS2_PC_MTGS) {
    ensure_colors(h);
    mtgs_relax(h, b, x, p->outer, p->omega, p->direction);
    return;
  }
  if (is_sweep_precision(p->precision)) {
    sweep32_relax(h, p, b, x, false, global_sweeps(p), nullptr);
    return;
  }
  for (int s = 0; s < global_sweeps(p); ++s) {
    if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC)
      gs2_half(h, p, h->L, h->U, b, x, false, nullptr);
    if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC)
      gs2_half(h, p, h->U, h->L, b, x, false, nullptr);
  }
}

// ---------------------------------------------------------------------------
// exact GS / SOR baseline: x += omega (D + omega T)^{-1} (b - A x), the
// triangular solve by level sets (one launch per level)
// ---------------------------------------------------------------------------

// One exact half sweep by level sets of T: r-hat = D^{-1} (b - R x) (R = A;
// the local block in the hybrid form), then the triangular solve level by
// level with the x update.  x_zero: x = 0 and D^{-1} b is in h->rhat.
static void gs_half_levels(gs2_handle* h, const DevCsr& T, const std::vector<int>& ptr,
                           const int* rows, const DevCsr& R, const double* b, double* x,
                           double omega, bool x_zero, const int* skip) {
  if (x_zero) {
    launch_fill(h, x, 0.0, skip);
  } else {
    launch_resid_matrix(h, R, b, x, nullptr, h->rhat, nullptr, skip);
  }
  KernelTimer tm(h, "levels", T.nnz * 12.0 + 4.0 * (h->n + 1) + 32.0 * h->n);
  for (size_t l = 0; l + 1 < ptr.size(); ++l)
    launch_level(h, T, rows, ptr[l], ptr[l + 1], h->rhat, h->g0, x, omega, skip);
}

static void gs_half(gs2_handle* h, bool lower, const double* b, double* x, double omega,
                    bool x_zero, const int* skip) {
  gs_half_levels(h, lower ? h->L : h->U, lower ? h->lev_ptr_L : h->lev_ptr_U,
                 lower ? h->lev_rows_L : h->lev_rows_U, h->A, b, x, omega, x_zero, skip);
}

void gs_relax(gs2_handle* h, const double* b, double* x, int sweeps, double omega,
              int direction) {
  for (int s = 0; s < sweeps; ++s) {
    if (direction == GS2_FORWARD || direction == GS2_SYMMETRIC)
      gs_half(h, true, b, x, omega, false, nullptr);
    if (direction == GS2_BACKWARD || direction == GS2_SYMMETRIC)
      gs_half(h, false, b, x, omega, false, nullptr);
  }
}

// ---------------------------------------------------------------------------
// multicolour GS / SOR baseline (Sec. 6.1.2): the compact row update of
// exact GS, colour by colour (ascending forward, descending backward); rows
// of one colour are independent, so each colour is one parallel launch.
// bhat = D^{-1} b must be in h->rhat.
// ---------------------------------------------------------------------------

static void mtgs_half(gs2_handle* h, bool forward, double* x, double omega,
                      const int* skip) {
  const int nc = (int)h->colors.size();
  for (int s = 0; s < nc; ++s) {
    const int c = forward ? s : nc - 1 - s;
    launch_color(h, h->colors[c], h->color_rows[c], h->rhat, x, omega, skip);
  }
}

void mtgs_relax(gs2_handle* h, const double* b, double* x, int sweeps, double omega,
                int direction) {
  launch_prep_rhat(h, b, h->rhat, nullptr, nullptr);
  for (int s = 0; s < sweeps; ++s) {
    if (direction == GS2_FORWARD || direction == GS2_SYMMETRIC)
      mtgs_half(h, true, x, omega, nullptr);
    if (direction == GS2_BACKWARD || direction == GS2_SYMMETRIC)
      mtgs_half(h, false, x, omega, nullptr);
  }
}

// ---------------------------------------------------------------------------
// damped JR baseline, ping-pong between x and a resident temporary
// ---------------------------------------------------------------------------

void jr_relax(gs2_handle* h, const double* b, double* x, int sweeps, double omega) {
  const double* xin = x;
  double* xout = h->t;
  for (int s = 0; s < sweeps; ++s) {
    launch_jr(h, b, xin, xout, omega, nullptr);
    xin = xout;
    xout = (xout == h->t) ? x : h->t;
  }
  if (xin != x) launch_copy(h, x, xin);
}

// ---------------------------------------------------------------------------
// preconditioner from a zero start: z = M^{-1} v
// ---------------------------------------------------------------------------

bool precond_wants_rhat(const gs2_params* p) {
  return p && (p->kind == GS2_PC_GS2 || p->kind == GS2_PC_JR || p->kind == GS2_PC_GS ||
               p->kind == GS2_PC_MTGS || p->kind == GS2_PC_AMG || p->kind == GS2_PC_AMG_JR);
}

// (the AMG kinds start with the fine-level smoother from zero, which reads
// D^{-1} v like the stand-alone smoother does)
void* precond_rhat_buffer(gs2_handle* h, const gs2_params* p) {
  if (!precond_wants_rhat(p)) return nullptr;
  if (p->kind == GS2_PC_GS2 && is_sweep_precision(p->precision)) return h->bhat32;
  if (p->kind == GS2_PC_GS2 || p->kind == GS2_PC_AMG) return rhat_buf(h, p->precision);
  return h->rhat;
}

void smooth_sweeps(gs2_handle* h, const gs2_params* p, const double* b, double* x,
                   const int* skip) {
  if (p->kind == GS2_PC_JR) {
    const double* xin = x;
    double* xout = h->t;
    for (int s = 0; s < p->outer; ++s) {
      launch_jr(h, b, xin, xout, p->omega, skip);
      xin = xout;
      xout = (xout == h->t) ? x : h->t;
    }
    if (xin != x) launch_copy_skip(h, x, xin, skip);
    return;
  }
  for (int s = 0; s < p->outer; ++s) {
    if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC)
      gs2_half(h, p, h->L, h->U, b, x, false, skip);
    if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC)
      gs2_half(h, p, h->U, h->L, b, x, false, skip);
  }
}

void precond_apply(gs2_handle* h, const gs2_params* p, const double* v, double* z,
                   bool rhat_ready, const int* skip) {
  if (!p || p->kind == GS2_PC_NONE) {
    launch_copy_skip(h, z, v, skip);
    return;
  }
  if ((p->kind == GS2_PC_GS2 || p->kind == GS2_PC_JR || p->kind == GS2_PC_GS) && p->parts > 1) {
    const Hybrid* Y = find_hybrid(h, (int)std::min<int64_t>(p->parts, h->n));
    if (!Y) GS2_THROW(GS2_ERR_INVALID_ARG, "hybrid form not prepared (ensure_precond)");
    if (!rhat_ready) {
      if (p->kind == GS2_PC_GS2 && p->precision != GS2_FP64)
        launch_prep_rhat(h, v, nullptr, h->rhat32, skip);
      else
        launch_prep_rhat(h, v, h->rhat, nullptr, skip);
    }
    hybrid_apply(h, p, *Y, v, z, true, skip);
    return;
  }
  if (p->kind == GS2_PC_GS2 && is_sweep_precision(p->precision)) {
    if (!rhat_ready) launch_prep_rhat(h, v, nullptr, h->bhat32, skip);
    sweep32_relax(h, p, v, z, true, global_sweeps(p), skip);
    return;
  }
  if (p->kind == GS2_PC_GS2) {
    const int prec = p->precision;
    if (!rhat_ready) {
      if (prec == GS2_FP64)
        launch_prep_rhat(h, v, h->rhat, nullptr, skip);
      else
        launch_prep_rhat(h, v, nullptr, h->rhat32, skip);
    }
    bool zero = true;
    for (int s = 0; s < global_sweeps(p); ++s) {
      if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC) {
        gs2_half(h, p, h->L, h->U, v, z, zero, skip);
        zero = false;
      }
      if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC) {
        gs2_half(h, p, h->U, h->L, v, z, zero, skip);
        zero = false;
      }
    }
    return;
  }
  if (p->kind == GS2_PC_JR) {
    if (!rhat_ready) launch_prep_rhat(h, v, h->rhat, nullptr, skip);
    launch_rhat_update(h, GS2_FP64, h->rhat, z, p->omega, false, skip);
    const double* xin = z;
    double* xout = h->t;
    for (int s = 1; s < global_sweeps(p); ++s) {
      launch_jr(h, v, xin, xout, p->omega, skip);
      xin = xout;
      xout = (xout == h->t) ? z : h->t;
    }
    if (xin != z) launch_copy_skip(h, z, xin, skip);
    return;
  }
  if (p->kind == GS2_PC_AMG || p->kind == GS2_PC_AMG_JR) {
    amg_vcycle(h, p, v, z, rhat_ready, skip);
    return;
  }
  if (p->kind == GS2_PC_MTGS) {
    if (!rhat_ready) launch_prep_rhat(h, v, h->rhat, nullptr, skip);
    launch_fill(h, z, 0.0, skip);
    for (int s = 0; s < p->outer; ++s) {
      if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC)
        mtgs_half(h, true, z, p->omega, skip);
      if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC)
        mtgs_half(h, false, z, p->omega, skip);
    }
    return;
  }
  // exact GS: the first half sweep from z = 0 solves with r = v
  if (!rhat_ready) launch_prep_rhat(h, v, h->rhat, nullptr, skip);
  bool zero = true;
  for (int s = 0; s < global_sweeps(p); ++s) {
    if (p->direction == GS2_FORWARD || p->direction == GS2_SYMMETRIC) {
      gs_half(h, true, v, z, p->omega, zero, skip);
      zero = false;
    }
    if (p->direction == GS2_BACKWARD || p->direction == GS2_SYMMETRIC) {
      gs_half(h, false, v, z, p->omega, zero, skip);
      zero = false;
    }
  }
}

}  // namespace gs2
