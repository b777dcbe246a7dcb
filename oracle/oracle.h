/*
 * Plain, slow, single-threaded FP64 CPU oracle for two-stage Gauss-Seidel
 * (GS2), exact Gauss-Seidel (GS/SOR), Jacobi-Richardson (JR) and restarted
 * right-preconditioned GMRES with CGS2 orthogonalisation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU library
 * shares no code with it and never calls it.
 *
 * Matrices are CSR: rowptr[n+1] (int64), col[nnz] (int32), val[nnz] (f64).
 * Column order inside a row is arbitrary; the split A = L + D + U is taken by
 * comparing the column index with the row index (Sec. 3, splitting before
 * Eq. (1)).
 *
 * Return codes follow the library's status enumeration: 0 = OK,
 * 1 = invalid argument, 2 = zero/missing diagonal, 5 = not converged,
 * 6 = breakdown, 7 = NaN/Inf detected.
 */
#ifndef GS2_ORACLE_H
#define GS2_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_FORWARD = 0, ORA_BACKWARD = 1, ORA_SYMMETRIC = 2 };
enum { ORA_PC_NONE = 0, ORA_PC_GS2 = 1, ORA_PC_JR = 2, ORA_PC_GS = 3,
       ORA_PC_MTGS = 4, ORA_PC_AMG = 5, ORA_PC_AMG_JR = 6, ORA_PC_HYBRID_GS2 = 7,
       ORA_PC_HYBRID_JR = 8, ORA_PC_HYBRID_GS = 9, ORA_PC_GS2_COMPACT = 10 };

typedef struct {
  int iters;          /* total Arnoldi steps over all cycles */
  int cycles;         /* restart cycles started */
  int status;         /* 0 converged, 5 not converged, 6 breakdown, 7 NaN */
  double true_relres; /* ||b - A x|| / ||b|| at exit */
} ora_info;

/* y = A x */
void ora_spmv(int64_t n, const int64_t* rp, const int32_t* ci,
              const double* va, const double* x, double* y);

/* Diagonal a_ii of every row; returns 2 if some a_ii is zero or absent. */
int ora_diag(int64_t n, const int64_t* rp, const int32_t* ci,
             const double* va, double* d);

/* Non-compact two-stage GS, Eq. (2)-(5) with the damping factors of the
 * "Damping factor" paragraph of Sec. 4: per outer sweep
 *   r = b - A x;  g0 = D^{-1} r;
 *   g_{j+1} = (1-gamma) g_j + gamma D^{-1} (r - omega T g_j),  j < inner;
 *   x += omega g_inner,
 * with T = L (forward) or U (backward); symmetric = forward then backward.
 * x is updated in place. */
int ora_gs2(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
            const double* b, double* x, int outer, int inner, double omega,
            double gamma, int dir);

/* Exact GS / SOR by the compact row recurrence (Sec. 6.1.1, sequential GS):
 * x_i <- (1-omega) x_i + omega (b_i - sum_{j != i} a_ij x_j) / a_ii in
 * ascending (forward) or descending (backward) row order; symmetric =
 * forward then backward.  x in place. */
int ora_gs(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, int sweeps, double omega, int dir);

/* Damped Jacobi-Richardson: x += omega D^{-1} (b - A x), `sweeps` times
 * (Sec. 4, zero-inner-sweep special case). */
int ora_jr(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, int sweeps, double omega);

/* Level sets of the strict lower (lower=1) or strict upper (lower=0)
 * triangle: level(i) = 1 + max level(j) over dependencies j, level 0 for
 * rows with none.  Returns the number of levels. */
int ora_levels(int64_t n, const int64_t* rp, const int32_t* ci, int lower,
               int32_t* level);

/* First-fit colouring of the symmetrised pattern of A in natural row order:
 * rows i and j with a_ij != 0 or a_ji != 0 (i != j) get different colours.
 * Returns the number of colours. */
int ora_coloring(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* color);

/* Multicolour GS / SOR (Sec. 6.1.2, multi-threaded GS): the compact row
 * update of ora_gs applied colour by colour, colours ascending (forward) or
 * descending (backward), rows of one colour in natural order; symmetric =
 * forward then backward.  x in place. */
int ora_mtgs(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
             const double* b, double* x, int sweeps, double omega, int dir);

/* Apply a preconditioner from a zero start: z = M^{-1} v.
 * kind: ORA_PC_NONE (z = v), ORA_PC_GS2, ORA_PC_JR (outer = sweeps),
 * ORA_PC_GS (exact GS, outer = sweeps), ORA_PC_MTGS (multicolour GS,
 * outer = sweeps), ORA_PC_AMG / ORA_PC_AMG_JR (one V-cycle of the hierarchy
 * ora_gmres_amg installs, GS2 / JR smoother with these parameters),
 * ORA_PC_HYBRID_GS2 / ORA_PC_HYBRID_JR / ORA_PC_HYBRID_GS (ora_hybrid with
 * the partition and local sweeps set by ora_set_hybrid; outer = n_t),
 * ORA_PC_GS2_COMPACT (compact GS2 of Eq. (9), undamped). */
int ora_precond(int64_t n, const int64_t* rp, const int32_t* ci,
                const double* va, const double* v, double* z, int kind,
                int outer, int inner, double omega, double gamma, int dir);

/* Restarted GMRES(m), right preconditioned, CGS2 Arnoldi, Givens rotations.
 * x holds x0 on entry and the solution on exit.  Stops when the implicit
 * residual |g_{j+1}| <= tol ||b|| inside a cycle and the recomputed true
 * residual confirms it, or when max_iters Arnoldi steps have run.
 * resid_hist (may be NULL) receives |g_{j+1}|/||b|| after every step, so it
 * needs max_iters entries. */
int ora_gmres(int64_t n, const int64_t* rp, const int32_t* ci,
              const double* va, const double* b, double* x, int restart,
              double tol, int max_iters, int pc_kind, int pc_outer,
              int pc_inner, double pc_omega, double pc_gamma, int pc_dir,
              ora_info* info, double* resid_hist);

/* Preconditioned conjugate gradients for SPD A (Sec. 9 uses CG with an
 * SGS2 preconditioner).  Same stopping rule on the recursively updated
 * residual, confirmed by the true residual. */
int ora_cg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
           const double* b, double* x, double tol, int max_iters, int pc_kind,
           int pc_outer, int pc_inner, double pc_omega, double pc_gamma,
           int pc_dir, ora_info* info);

/* Compact two-stage GS, Eq. (9): x <- Mhat^{-1} (b + N x) where
 * N = -U (forward) or -L (backward) and Mhat^{-1} is `inner` JR sweeps on
 * (D + T) from g0 = D^{-1}(b + N x).  Undamped (omega = gamma = 1). */
int ora_gs2_compact(int64_t n, const int64_t* rp, const int32_t* ci,
                    const double* va, const double* b, double* x, int outer,
                    int inner, int dir);

/* ------------------------------------------------------------------ */
/* Hybrid (block-Jacobi) relaxation of Sec. 3 with the local sweeps of  */
/* the two-stage listing (hybrid.c; the readings are stated there).     */
/* ------------------------------------------------------------------ */

/* Rows in `parts` contiguous blocks; per exchange (outer = n_t times)
 * c = b - E x with E the couplings between blocks, then `local` = n_k local
 * sweeps on A_loc x = c: kind ORA_PC_GS2 (half sweeps as ora_gs2 with the
 * local triangles, `inner` = n_j, dir), ORA_PC_JR (x += omega D^{-1}
 * (c - A_loc x)) or ORA_PC_GS (exact local SOR, dir).  x in place. */
int ora_hybrid(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, int kind, int parts, int outer, int local, int inner,
               double omega, double gamma, int dir);
/* partition and local sweeps of the hybrid preconditioner kinds */
void ora_set_hybrid(int parts, int local);

/* ------------------------------------------------------------------ */
/* GS2 with lower-precision inner sweeps (lowprec.c; the definitions    */
/* are stated there): FP32 values and vectors, or FP16 values with a    */
/* per-row power-of-two scale, FP32 accumulation; residual and update   */
/* in FP64 -- or, in the whole-sweep precisions, in FP32 as well.       */
/* ------------------------------------------------------------------ */

enum { ORA_PREC_FP64 = 0, ORA_PREC_FP32 = 1, ORA_PREC_FP16_ROWSCALED = 2,
       ORA_PREC_FP32_SWEEP = 3, ORA_PREC_FP16_SWEEP = 4 };

/* GS2 sweeps as ora_gs2 with the inner sweeps in precision `prec`
 * (ORA_PREC_FP64 is ora_gs2 itself).  x in place. */
int ora_gs2_lp(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, int outer, int inner, double omega,
               double gamma, int dir, int prec);
/* IEEE binary16 round-to-nearest-even of v (returned exactly as a double) */
double ora_round_half(double v);
/* inner-sweep precision of the ORA_PC_GS2 preconditioner kind */
void ora_set_precision(int prec);
extern _Thread_local int ora_precision;

/* Threads the row loops run on: the OpenMP thread count in a build with
 * -fopenmp, else 1. */
int ora_threads(void);
extern _Thread_local int ora_hybrid_parts;
extern _Thread_local int ora_hybrid_local;

/* ------------------------------------------------------------------ */
/* Smoothed-aggregation AMG with GS2 (or JR) as the smoother of a       */
/* V-cycle (amg.c; the readings are stated there).                      */
/* ------------------------------------------------------------------ */

#define ORA_AMG_MAX_LEVELS 16
typedef struct ora_amg ora_amg;

/* Build the hierarchy of A: strength threshold theta, at most max_levels
 * levels, stop coarsening at <= coarse_size rows.  NULL on invalid input,
 * a zero diagonal or a singular coarsest matrix. */
ora_amg* ora_amg_build(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                       double theta, int max_levels, int64_t coarse_size);
void ora_amg_free(ora_amg* M);
int ora_amg_levels(const ora_amg* M);
/* sizes of level l: rows, entries of A_l, entries of P_l (0 on the coarsest) */
int ora_amg_level(const ora_amg* M, int l, int64_t* n, int64_t* nnz, int64_t* pnnz);
/* copies of A_l, P_l (rows of level l, columns of level l+1) and the
 * aggregate of every row of level l; arrays sized by ora_amg_level */
int ora_amg_get_matrix(const ora_amg* M, int l, int64_t* rp, int32_t* ci, double* va);
int ora_amg_get_prolongator(const ora_amg* M, int l, int64_t* rp, int32_t* ci, double* va);
int ora_amg_get_aggregates(const ora_amg* M, int l, int32_t* agg);
/* x = M^{-1} b: one V-cycle from a zero start, smoother kind ORA_PC_GS2
 * (outer, inner, omega, gamma) or ORA_PC_JR (outer sweeps, omega) applied
 * before and after the coarse correction; direction SYMMETRIC smooths
 * forward before and backward after. */
int ora_amg_vcycle(const ora_amg* M, const double* b, double* x, int kind, int outer,
                   int inner, double omega, double gamma, int dir);
/* GMRES(restart) right-preconditioned by one V-cycle per application */
int ora_gmres_amg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                  const double* b, double* x, int restart, double tol, int max_iters,
                  const ora_amg* M, int kind, int outer, int inner, double omega,
                  double gamma, int dir, ora_info* info);
/* CG preconditioned by one V-cycle per application (symmetric smoothing) */
int ora_cg_amg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
               const double* b, double* x, double tol, int max_iters, const ora_amg* M,
               int kind, int outer, int inner, double omega, double gamma, int dir,
               ora_info* info);
/* the hierarchy the AMG preconditioner kinds apply (set by ora_gmres_amg and
 * ora_cg_amg) */
extern _Thread_local const ora_amg* ora_amg_current;

#ifdef __cplusplus
}
#endif
#endif
