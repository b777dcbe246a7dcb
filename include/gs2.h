/*
 * gs2.h -- C ABI of the GB300 two-stage Gauss-Seidel library.
 *
 * Two-stage Gauss-Seidel (GS2) replaces the sparse triangular solve of a
 * Gauss-Seidel sweep by a fixed number of inner Jacobi-Richardson (JR)
 * sweeps (Sec. 4, Eq. (2)-(5)); it is used here as a relaxation and as the
 * preconditioner of restarted GMRES.  Exact GS through a level-scheduled
 * triangular solve and damped JR are provided beside it as baselines.
 *
 * Conventions shared by every call:
 *  - Status: every call returns a gs2_status and never throws across the
 *    ABI.  On failure gs2_last_error() returns a message for the calling
 *    thread.
 *  - Matrix: CSR with rowptr int64[n+1], col int32[nnz], val double[nnz].
 *    Columns may appear in any order inside a row; duplicates are rejected.
 *    A = L + D + U is split by comparing column and row index (Sec. 3,
 *    splitting before Eq. (1)).  Every row needs a nonzero diagonal entry.
 *  - Vectors b and x: double[n].  They may be device pointers (of the
 *    handle's device) or host pointers (pageable or pinned); host vectors
 *    are staged through device buffers by the call, which then synchronises
 *    the stream before returning.  With device vectors a call only enqueues
 *    work on the handle's stream, except gmres_solve/cg_solve, which read
 *    back a small status word once per restart cycle.
 *  - Ownership: gs2_setup copies the matrix; no call keeps a pointer to the
 *    caller's vectors after it returns.
 *  - Threads: a handle belongs to one stream and is not thread-safe.
 *    A server (gs2_server_*) is thread-safe.
 *  - Results of one handle are bitwise reproducible run to run on the same
 *    GPU: no floating-point atomics are used.
 */
#ifndef GS2_H
#define GS2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS2_OK = 0,
  GS2_ERR_INVALID_ARG = 1,
  GS2_ERR_ZERO_DIAGONAL = 2,
  GS2_ERR_OOM = 3,
  GS2_ERR_CUDA = 4,
  GS2_ERR_NOT_CONVERGED = 5,
  GS2_ERR_BREAKDOWN = 6,
  GS2_ERR_NAN = 7,
  GS2_ERR_TIMEOUT = 8,
  GS2_ERR_BUSY = 9,
  GS2_ERR_NOT_FOUND = 10
} gs2_status;

typedef enum { GS2_FORWARD = 0, GS2_BACKWARD = 1, GS2_SYMMETRIC = 2 } gs2_direction;

/* Storage and arithmetic of a GS2 sweep.  Sec. 10 runs the preconditioner
 * in single precision (its outer GS and inner JR iterations); FP16 values
 * with a per-row power-of-two scale are an extension of that.
 *   GS2_FP32, GS2_FP16_ROWSCALED: the inner sweeps only (the triangles
 *     D^{-1}L, D^{-1}U and the inner iterate g); the residual r = b - A x
 *     and the iterate x stay FP64.
 *   GS2_FP32_SWEEP, GS2_FP16_SWEEP: the whole sweep: the iterate x32 =
 *     fl32(x), the residual rhat = fl32(D^{-1}b) - x32 - (D^{-1}(L+U)) x32
 *     from FP32 (or row-scaled FP16) values of the prescaled off-diagonal
 *     entries in FP32 arithmetic, the inner sweeps as above, x32 += omega g
 *     in FP32; x = (double) x32 at the end of the call.  GS2 preconditioner
 *     (GMRES, CG, batch, packs, server) and gs2_apply_ex; not with the AMG,
 *     hybrid or compact forms. */
typedef enum {
  GS2_FP64 = 0,
  GS2_FP32 = 1,
  GS2_FP16_ROWSCALED = 2,
  GS2_FP32_SWEEP = 3,
  GS2_FP16_SWEEP = 4
} gs2_precision;

/* Non-compact form Eq. (2) is the paper's default (Sec. 7 setup); the
 * compact form Eq. (9) is x <- Mhat^{-1}(b + N x) (undamped). */
typedef enum { GS2_NONCOMPACT = 0, GS2_COMPACT = 1 } gs2_form;

typedef enum {
  GS2_PC_NONE = 0, /* identity */
  GS2_PC_GS2 = 1,  /* two-stage GS, Eq. (2)-(5) with damping */
  GS2_PC_JR = 2,   /* damped Jacobi-Richardson, `outer` sweeps */
  GS2_PC_GS = 3,   /* exact GS/SOR, level-scheduled, `outer` sweeps */
  GS2_PC_MTGS = 4, /* multicolour GS/SOR, `outer` sweeps (Sec. 6.1.2) */
  GS2_PC_AMG = 5,  /* one AMG V-cycle, GS2 smoother (outer, inner, omega,
                      gamma, precision) on every level */
  GS2_PC_AMG_JR = 6 /* one AMG V-cycle, JR smoother (outer sweeps, omega) */
} gs2_pc_kind;

/* Relaxation / preconditioner parameters in the paper's notation:
 * GS2(n_t, n_j) = `outer` global sweeps with `inner` JR sweeps each (Sec. 7
 * setup; the local sweep count n_k is 1 on one GPU).  omega is the outer
 * (SOR-like) damping factor and gamma the inner one (Sec. 4, "Damping
 * factor"): an outer sweep computes r = b - A x, g_0 = D^{-1} r,
 *   g_{j+1} = (1 - gamma) g_j + gamma D^{-1} (r - omega T g_j),
 * and x += omega g_{inner}, with T = L (forward) or U (backward).
 * As a preconditioner the sweeps start from x = 0. */
typedef struct {
  int kind;      /* gs2_pc_kind */
  int outer;     /* n_t >= 1 (sweeps for JR / GS) */
  int inner;     /* n_j >= 0 */
  double omega;  /* outer damping, > 0 */
  double gamma;  /* inner damping, > 0; 1 = undamped */
  int direction; /* gs2_direction */
  int precision; /* gs2_precision */
  int form;      /* gs2_form */
  int parts;     /* hybrid (block-Jacobi) form of Sec. 3 for kinds GS2 and
                    JR: the rows in `parts` contiguous blocks (block p holds
                    rows [p n / P, (p+1) n / P), more blocks than rows count
                    as n); each of the `outer` sweeps (n_t) freezes the other
                    blocks' values, c = b - E x with E the couplings between
                    blocks, then runs `local_sweeps` (n_k) local sweeps on
                    A_loc x = c, GS2 with the local triangles (n_j = inner)
                    or JR.  It is the preconditioner a 1-D row-block
                    distribution over `parts` processes applies, run here on
                    one GPU.  0 or 1 = the global method. Non-compact only. */
  int local_sweeps; /* n_k >= 1 (0 = 1) */
} gs2_params;

typedef struct {
  int iters;          /* total Krylov iterations (Arnoldi steps for GMRES) */
  int cycles;         /* restart cycles (GMRES) / direction restarts (CG) */
  int status;         /* gs2_status of the solve */
  double true_relres; /* ||b - A x|| / ||b|| recomputed at exit */
} gs2_solve_info;

typedef struct {
  int64_t n, nnz, nnz_lower, nnz_upper;
  int levels_lower, levels_upper; /* 0 until a level-scheduled call */
  int64_t device_bytes;           /* device memory held by the handle */
  int tpr_a, tpr_tri;             /* lanes per row of the tile kernels (A, D^-1 L) */
  int rpt_a, rpt_tri;             /* rows per lane group of the tile kernels */
  int colors;                     /* 0 until a multicolour call */
  int sell_a, sell_tri;           /* 1: A / the triangles run on the sliced-ELL layout */
  double offset_frac_a;           /* share of A's sliced-ELL chunks that store column */
  double offset_frac_tri;         /* offsets instead of columns (stencil rows); D^{-1}L */
  int solve_mode;                 /* gs2_autotune_gmres's choice (1, 2, 3, 4); 0 = not tuned */
  int solve_modes_timed;          /* candidates it timed */
} gs2_handle_stats;

typedef struct gs2_handle gs2_handle;

/* Create a handle for A (Sec. 3 splitting; Sec. 6.1.3 keeps D^{-1}L and
 * D^{-1}U prescaled and explicit; Sec. 6.2 keeps the temporaries resident
 * with A).  Copies A to the current CUDA device, checks it (rowptr
 * monotone with rowptr[0] = 0 and rowptr[n] = nnz, 0 <= col < n, no
 * duplicate (i, j), nonzero a_ii in every row) and prepares the inner-sweep
 * storage for every precision bit set in `precisions` (bit p for
 * gs2_precision p; FP64 is always prepared, other precisions are also
 * prepared on first use).
 *   on_device: 1 if rowptr/col/val are device pointers, 0 if host.
 *   stream: cudaStream_t the handle enqueues on (NULL = legacy default).
 * Errors: INVALID_ARG (bad sizes or structure, n or nnz above 2^31 - 1),
 * ZERO_DIAGONAL, OOM, CUDA. */
gs2_status gs2_setup(int64_t n, int64_t nnz, const int64_t* rowptr,
                     const int32_t* col, const double* val, int on_device,
                     unsigned precisions, void* stream, gs2_handle** out);

/* Release every device and host resource of the handle (NULL is a no-op). */
void gs2_destroy(gs2_handle* h);

/* Change the stream later calls enqueue on. */
gs2_status gs2_set_stream(gs2_handle* h, void* stream);

gs2_status gs2_get_stats(const gs2_handle* h, gs2_handle_stats* out);

/* Autotune the row kernels of A, D^{-1}L and D^{-1}U: for each matrix, time
 * its most frequent kernel (the residual for A, the inner sweep with the x
 * update for a triangle) for every candidate row-tile shape (lanes per row
 * K around the row-length heuristic, rows per lane group 1 or 2), keeping
 * the heuristic shape unless another is at least 2% faster, and, for a
 * matrix with a sliced-ELL copy, keep that layout unless the best tile
 * shape beats it by 2%.  Results are
 * cached by matrix class (size to a factor sqrt(2), mean row length), so
 * matrices of a class already measured are re-tiled without timing.  The
 * numerical results do not change (rows are reduced in the same order for
 * K = 1 and in a different segment split otherwise, within rounding). */
gs2_status gs2_autotune(gs2_handle* h);

/* How gmres_solve issues the Arnoldi steps of a restart cycle:
 * 0 (default): for a small system (restart <= 32, no preconditioner, JR or
 * FP64 non-compact GS2, per-kernel profiling off) the whole solve in one
 * kernel -- inside one thread-block cluster as in mode 4 when the system's
 * rows fit its shared memory, else as one cooperative launch whose blocks
 * meet at bounded grid barriers (n <= 16,384) -- every restart cycle,
 * preconditioner application and Givens step included; otherwise as in
 * mode 1; 1 = each restart cycle's steps
 * as one replayed CUDA graph; 2 = as separate launches; 3 = the one-launch
 * solver, up to n = 65,536 (INVALID_ARG when the solve does not qualify);
 * 4 = the one-cluster solver: the whole GMRES solve inside one cluster of
 * at most 16 CTAs, every row's vectors, Krylov basis entries and matrix
 * entries in the shared memory of the CTA that owns it, other rows' entries
 * read through distributed shared memory, the CTAs meeting at bounded
 * cluster barriers (restart <= 32, no, JR or FP64 non-compact GS2
 * preconditioning, and a system whose rows fit: about 8,000 rows of a
 * 5-point stencil at restart 30; INVALID_ARG otherwise); cg_solve runs the
 * same way in modes 3 and 4; a pack (gs2_pack_gmres) in mode 4 gives every
 * system a cluster of its own, of one shape chosen for the pack (the most
 * systems resident at once against the rows each CTA holds).
 * A graph is captured once per cycle shape (restart, preconditioner,
 * profiling settings) on a private stream joined to the handle's stream;
 * steps after the device has ended the cycle run as no-ops.  Results are
 * the same either way, bit for bit.  With per-kernel profiling enabled the
 * graph carries event nodes around the profiled kernels, and only the steps
 * a cycle ran are counted. */
gs2_status gs2_set_graph_mode(gs2_handle* h, int mode);

/* Autotune how much of a GMRES(restart) solve with this preconditioner is
 * fused into one launch -- the fusion depth: every kernel of an Arnoldi
 * step launched on its own (mode 2), a restart cycle's steps replayed as
 * one CUDA graph (mode 1), the whole solve as one cooperative launch
 * (mode 3) or inside one thread-block cluster (mode 4), where the solve
 * qualifies -- by timing one restart cycle of each
 * candidate on this matrix (the right-hand side is the handle's scratch, the
 * caller's vectors are not touched).  The fastest becomes the handle's
 * automatic choice (graph mode 0), cached by matrix class (size to a factor
 * sqrt(2), mean row length) and preconditioner; *mode_out (may be NULL)
 * receives it.  Results do not change with the choice beyond rounding (the
 * one-launch and one-cluster solvers reduce in another order). */
gs2_status gs2_autotune_gmres(gs2_handle* h, int restart, const gs2_params* precond,
                              int* mode_out);

/* Test hook for the bounded waits of the one-launch and one-cluster
 * solvers: the next such solve on this handle starts with a grid barrier
 * that can never open (one launch) or with one CTA that never arrives at the
 * cluster barriers (one cluster), so every block gives up after its wait
 * limit (about two seconds), the kernel returns, and the solve reports
 * GS2_ERR_TIMEOUT; the handle stays usable. */
gs2_status gs2_test_stall_barrier(gs2_handle* h);

/* Non-compact GS2 relaxation, Eq. (2) with inner JR sweeps Eq. (3)-(5):
 * x is read and overwritten (in/out), b is read.  outer_sweeps = n_t >= 0,
 * inner_sweeps = n_j >= 0 (0 gives JR), damping = omega > 0, direction as
 * gs2_direction (symmetric = forward then backward, Sec. 3).  FP64,
 * gamma = 1. */
gs2_status gs2_apply(gs2_handle* h, const double* b, double* x,
                     int outer_sweeps, int inner_sweeps, double damping,
                     int direction);

/* GS2 with every parameter: gamma, precision and compact form.
 * p->kind is ignored (taken as GS2_PC_GS2). */
gs2_status gs2_apply_ex(gs2_handle* h, const double* b, double* x,
                        const gs2_params* p);

/* The gs2_apply relaxation for callers that cannot allocate device memory
 * (an application that owns all GPU memory through its own allocator, code
 * that must not allocate after start-up).  The paper has no counterpart:
 * this is a library convenience.  No handle is needed and the call
 * allocates nothing: its working memory (D^{-1}, r-hat and two inner
 * iterates) is a fixed 8 MiB array inside the library's device image, held
 * by every GPU that loads the library until the process exits.
 *   n <= 262,144 rows, else GS2_ERR_INVALID_ARG; rowptr int64[n+1],
 *   col int32[nnz], val, b (read) and x (read and overwritten) are device
 *   pointers of the current device; stream as in gs2_setup.  Sweep counts
 *   and damping are bounded as in gs2_apply (outer 0..1000, inner
 *   0..100000, damping finite and > 0), else GS2_ERR_INVALID_ARG.  The
 *   matrix is not validated: a zero or missing diagonal gives inf/NaN in x;
 *   duplicate entries are not detected, and duplicated diagonal entries are
 *   summed (as an SpMV would use them).
 * Every call uses the same array, so calls that overlap on the GPU race:
 * serialise them.  Each call outside stream capture looks the array's
 * device address up on the current device and remembers it; a call on a
 * capturing stream uses the remembered address, so make one uncaptured call
 * on the device before capturing (else GS2_ERR_INVALID_ARG).  Results match
 * gs2_apply to rounding (FP64, gamma = 1). */
gs2_status gs2_apply_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                             const double* val, const double* b, double* x,
                             int outer_sweeps, int inner_sweeps, double damping,
                             int direction, void* stream);

/* Exact GS / SOR baseline: x + omega (D + omega T)^{-1} (b - A x) per half
 * sweep (Sec. 4, "Damping factor"), the triangular solve scheduled by
 * level sets of T (Sec. 3, level-set scheduling).  Levels are computed on
 * the first call. x in/out. */
gs2_status gs_apply(gs2_handle* h, const double* b, double* x, int sweeps,
                    double omega, int direction);

/* Multicolour GS / SOR baseline (Sec. 6.1.2, multi-threaded GS): rows are
 * coloured on the host on the first call, first fit in natural row order
 * on the symmetrised pattern (rows i and j differ in colour whenever a_ij
 * or a_ji is stored, i != j); the paper's greedy colouring is parallel and
 * leaves the order open, this one is deterministic.  A forward sweep
 * relaxes the colours in ascending order, each colour in one parallel
 * launch with
 *   x_i <- (1 - omega) x_i + omega (b_i - sum_{j != i} a_ij x_j) / a_ii,
 * a backward sweep takes the colours in descending order, and symmetric is
 * forward then backward.  Equal to SOR on A with its rows and columns
 * permuted by colour.  x in/out.  Errors: INVALID_ARG (sweeps < 0,
 * omega <= 0, bad direction), OOM and CUDA on the first call. */
gs2_status mtgs_apply(gs2_handle* h, const double* b, double* x, int sweeps,
                      double omega, int direction);

/* ------------------------------------------------------------------------
 * GS2 as a multigrid smoother.  The paper also applies the two-stage
 * iteration as the smoother of an AMG V-cycle (its Nalu-Wind runs, Sec. 11.2:
 * one GS2 sweep per level of hypre's C-AMG).  This library builds a
 * smoothed-aggregation hierarchy: classical strength of connection
 * |a_ij| >= theta max_{k != i} |a_ik| (symmetrised), greedy aggregation in
 * natural row order, unit-norm constant tentative prolongator P0, smoothed
 * prolongator P = (I - w D^{-1} A) P0 with w = 4 / (3 rho) and rho the
 * Gershgorin bound of rho(D^{-1} A), Galerkin coarse operators P^T A P, and
 * an exact solve on the coarsest level.  The hierarchy is set up on the host
 * (once per matrix) and applied on the device.
 * ---------------------------------------------------------------------- */

#define GS2_AMG_MAX_LEVELS 16

typedef struct {
  double theta;        /* strength threshold, 0.25 (the paper's C-AMG value) */
  int max_levels;      /* 1 .. GS2_AMG_MAX_LEVELS, default 10 */
  int64_t coarse_size; /* stop coarsening at this many rows or fewer (64);
                          the coarsest level must have at most 2048 rows */
} gs2_amg_cfg;

/* Build (or rebuild) the handle's hierarchy; cfg NULL = defaults.  A GMRES,
 * CG or batch solve with an AMG preconditioner kind builds the default
 * hierarchy itself when the handle has none.  Errors: INVALID_ARG (bad
 * settings, a coarsest level above 2048 rows, a singular coarsest matrix),
 * OOM, CUDA. */
gs2_status gs2_amg_setup(gs2_handle* h, const gs2_amg_cfg* cfg);

/* Levels of the hierarchy (0 if none) and, per level l < levels, its rows,
 * matrix entries and prolongator entries (0 on the coarsest); each array
 * (may be NULL) holds GS2_AMG_MAX_LEVELS entries. */
gs2_status gs2_amg_info(const gs2_handle* h, int* levels, int64_t* rows, int64_t* nnz,
                        int64_t* pnnz);

/* x = M^{-1} b: one V-cycle from a zero start with the smoother of `p`
 * (kind GS2_PC_AMG or GS2_PC_AMG_JR).  On each level but the coarsest: x =
 * `outer` smoother sweeps from zero on b, r = b - A x, coarse right-hand
 * side P^T r, coarse correction, x += P x_c, `outer` sweeps from x.
 * Direction SYMMETRIC smooths forward before and backward after the coarse
 * correction (a symmetric cycle for SPD A); FORWARD / BACKWARD smooth in
 * that direction both times.  The hierarchy is built with defaults if the
 * handle has none. */
gs2_status gs2_amg_vcycle(gs2_handle* h, const double* b, double* x, const gs2_params* p);

/* The relaxation of p's kind from x (in/out): GS2 (as gs2_apply_ex), JR,
 * exact GS by level sets or multicolour GS, with `outer` sweeps; for GS2, JR
 * and GS the hybrid (block-Jacobi) form when p->parts > 1, local exact GS
 * solving each block's triangle by its own level sets.  Errors: INVALID_ARG
 * for the other kinds and bad parameters, OOM, CUDA. */
gs2_status relax_apply(gs2_handle* h, const double* b, double* x, const gs2_params* p);

/* Damped JR baseline: x += omega D^{-1} (b - A x), `sweeps` times (Sec. 4,
 * zero-inner-sweep case). x in/out. */
gs2_status jr_apply(gs2_handle* h, const double* b, double* x, int sweeps,
                    double omega);

/* y = A x (FP64). */
gs2_status gs2_spmv(gs2_handle* h, const double* x, double* y);

/* Restarted GMRES(restart), right preconditioned by `precond` (NULL = no
 * preconditioner) applied from a zero start, Arnoldi by classical
 * Gram-Schmidt applied twice (CGS2) in FP64, Givens rotations in FP64 on
 * the device (Sec. 7 uses GMRES with GS2; the paper's stopping rule is a
 * relative residual reduction).  x holds x0 on entry and the solution on
 * exit.  Stops when the implicit residual |g_{j+1}| <= tol ||b|| and the
 * recomputed true residual confirms it, or after max_iters Arnoldi steps.
 * Returns OK, NOT_CONVERGED, BREAKDOWN or NAN (also stored in info->status);
 * info may be NULL.  1 <= restart <= 64. */
gs2_status gmres_solve(gs2_handle* h, const double* b, double* x, int restart,
                       double tol, int max_iters, const gs2_params* precond,
                       gs2_solve_info* info);

/* Preconditioned CG for SPD A (Sec. 9 runs CG with SGS2), same
 * conventions as gmres_solve; the preconditioner must be symmetric
 * (GS2/GS/MTGS with direction SYMMETRIC, JR, or none). */
gs2_status cg_solve(gs2_handle* h, const double* b, double* x, double tol,
                    int max_iters, const gs2_params* precond,
                    gs2_solve_info* info);

/* Many independent systems in one call: system i is solved on hs[i] with
 * bs[i], xs[i] (device pointers), all with the same restart, tol,
 * max_iters and preconditioner.  The systems' kernels are interleaved on
 * the first handle's stream so that small systems share the GPU.
 * infos[count] receives each system's result; the return value is OK if
 * every system converged, else the first failing status.  Each system runs
 * the restart-cycle graphs of gmres_solve's graph mode 1. */
gs2_status gs2_batch_solve(gs2_handle* const* hs, const double* const* bs,
                           double* const* xs, int count, int restart,
                           double tol, int max_iters, const gs2_params* precond,
                           gs2_solve_info* infos);

/* ---- packs: many independent systems in one set of launches ------------
 *
 * A pack holds `count` independent systems A_s x_s = b_s as one handle
 * whose matrix is their block-diagonal concatenation diag(A_0, ..., A_{S-1})
 * (system s owns rows offsets[s] .. offsets[s+1]-1).  Every row kernel of a
 * sweep (residual, inner JR sweeps, SpMV, level-scheduled and multicolour
 * GS, JR) covers all systems in one launch: a row reads only its own
 * system's columns, so each system is relaxed exactly as it would be alone
 * (gs2_apply and the other relaxations work on a pack unchanged, vectors
 * concatenated).  gs2_pack_gmres runs restarted GMRES for all systems at
 * once with per-system inner products, Hessenberg matrices, Givens
 * rotations, stopping tests and iteration counts; each restart cycle is one
 * replay of the captured Arnoldi steps for every system still running.
 * Small systems, which alone leave the GPU idle between launches, share the
 * launches of a pack.  A pack small enough to give every row a thread of
 * the co-resident blocks runs in one launch instead: one thread-block
 * cluster per system where every system fits a cluster's shared memory,
 * else every system on its own blocks of one cooperative launch (graph
 * modes 4 and 3 ask for these).  The paper solves one system at a time; packs are a
 * library extension. */

/* Create a pack from host CSR arrays: n[s] rows, rowptr[s] (int64, n[s]+1,
 * rowptr[s][0] = 0), col[s] (int32, columns of system s: 0 .. n[s]-1) and
 * val[s] (double) per system, with the conventions of gs2_setup (diagonal,
 * duplicates; precisions and stream as there).  Errors name the system and
 * its row.  The total rows and entries must stay below 2^31. */
gs2_status gs2_pack_setup(int count, const int64_t* n, const int64_t* const* rowptr,
                          const int32_t* const* col, const double* const* val,
                          unsigned precisions, void* stream, gs2_handle** out);

/* Systems of a pack (0 for a handle made by gs2_setup) and, if offsets is
 * not NULL, their first rows: offsets[count + 1], offsets[count] = n. */
gs2_status gs2_pack_info(const gs2_handle* h, int* count, int64_t* offsets);

/* Restarted GMRES(restart) on every system of a pack, each with the
 * semantics of gmres_solve (right preconditioning by `precond` from a zero
 * start, CGS2, Givens, tol relative to ||b_s||, at most max_iters Arnoldi
 * steps per system).  b and x are the concatenated vectors (double[n],
 * device or host as in gmres_solve; x holds every x_s0 on entry).
 * infos[count] (may be NULL) receives each system's result.  The AMG
 * preconditioner kinds are refused (a hierarchy of the pack would coarsen
 * all systems together).  Returns OK if every system converged, else the
 * first failing system's status.  Per-system results equal gmres_solve's on
 * the system alone up to the rounding of the inner products (the block
 * partition of a reduction differs). */
gs2_status gs2_pack_gmres(gs2_handle* h, const double* b, double* x, int restart, double tol,
                          int max_iters, const gs2_params* precond, gs2_solve_info* infos);

/* Synchronise the handle's stream and report a sticky device-side error:
 * TIMEOUT if a kernel's bounded wait on its own shared-memory copies gave
 * up (the kernel then returned without touching its outputs further).  The
 * word is cleared by this call.  gmres_solve and cg_solve check it once per
 * restart cycle and return the status themselves. */
gs2_status gs2_check(gs2_handle* h);

/* ---- solve server: continuous batching of independent systems ---------- */

/* A server owns one GPU (the device current at creation) and solves
 * submitted systems A x = b with restarted GMRES and the configured
 * preconditioner.  Requests are admitted in arrival order as soon as a slot
 * is free and their estimated device footprint fits both the server's
 * budget and the device's free memory; each admitted request gets its own
 * stream, handle and resident Krylov state, so the work of requests that
 * arrive while others are running overlaps on the GPU.  A result is the
 * same, bit for bit, as the same solve run alone through gmres_solve with
 * graph mode 1 (the one-launch solver gmres_solve picks by default for a
 * small system sums its inner products in another order); with
 * pack_rows set, a packed request's result is the same, bit for bit, as that
 * request solved alone as a pack of one (a pack partitions each system by
 * its own size), and equal to gmres_solve's up to the rounding of the inner
 * products. */
typedef struct gs2_server gs2_server;

typedef struct {
  int64_t hbm_budget_bytes; /* device bytes the server may reserve for admitted
                               requests; 0 = 90% of the free memory at creation */
  int max_slots;            /* requests on the GPU at once, >= 1 */
  int prep_threads;         /* host threads preparing admitted requests, >= 1 */
  int restart;              /* GMRES restart, 1..64 */
  double tol;               /* relative residual */
  int max_iters;
  int has_precond;          /* 0: no preconditioner */
  gs2_params precond;
  uint64_t fail_ticket;     /* fault-injection hook for tests: the request with
                               this ticket fails its admission with GS2_ERR_OOM
                               as if its allocation had failed (0 = none) */
  int64_t pack_rows;        /* requests of at most this many rows are admitted
                               together, up to pack_max of them taken in arrival
                               order from the front of the queue, and solved as
                               one pack (gs2_pack_gmres) in one slot; 0 = every
                               request alone.  Not with an AMG preconditioner. */
  int pack_max;             /* most requests in one pack (0 = 64) */
  int64_t small_rows;       /* with small_slots > 0: requests of at most this */
  int small_slots;          /* many rows are small, and small_slots of the
                               max_slots slots are kept for them -- larger
                               requests hold at most max_slots - small_slots
                               at once, and a small request is admitted before
                               larger ones that wait for their slots (arrival
                               order within each class); 0 = arrival order for
                               all.  small_slots < max_slots. */
} gs2_server_cfg;

typedef struct {
  int64_t n, nnz;
  const int64_t* rowptr; /* host CSR, copied by gs2_server_submit */
  const int32_t* col;
  const double* val;
  const double* b;  /* host, copied */
  const double* x0; /* host initial guess, copied; NULL = zero */
} gs2_request;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t pending, active, max_active;
  int64_t reserved_bytes, budget_bytes;
} gs2_server_stats;

gs2_status gs2_server_create(const gs2_server_cfg* cfg, gs2_server** out);
/* Queue a request (inputs are copied); *ticket identifies it.  OOM if it can
 * never fit the budget, INVALID_ARG for a malformed request. */
gs2_status gs2_server_submit(gs2_server* s, const gs2_request* req, uint64_t* ticket);
/* Non-blocking: BUSY while the request is queued or running, NOT_FOUND for an
 * unknown or already collected ticket; otherwise the request's status, with
 * its solve info, x (n doubles, may be NULL) and the submit-to-done latency
 * in milliseconds (may be NULL).  A collected result is released. */
gs2_status gs2_server_poll(gs2_server* s, uint64_t ticket, gs2_solve_info* info,
                           double* x_out, double* latency_ms);
/* Blocking form of poll: waits at most timeout_s seconds (TIMEOUT). */
gs2_status gs2_server_wait(gs2_server* s, uint64_t ticket, double timeout_s,
                           gs2_solve_info* info, double* x_out, double* latency_ms);
gs2_status gs2_server_get_stats(gs2_server* s, gs2_server_stats* out);
/* Device bytes the server reserves for a request of this size (the
 * admission estimate). */
int64_t gs2_server_footprint(const gs2_server_cfg* cfg, int64_t n, int64_t nnz);
/* Finish running requests, drop queued ones, release everything. */
void gs2_server_destroy(gs2_server* s);

/* ---- per-kernel device timing (CUDA events on the handle's stream) ---- */

typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double bytes; /* algorithmic bytes summed over the timed launches */
} gs2_kernel_stat;

/* enable = 1 records an event pair around every launch of the library's
 * kernels on this handle until disabled; 0 stops and keeps the totals. */
gs2_status gs2_profile_enable(gs2_handle* h, int enable);
/* Time only the kernels named `name` (as reported by gs2_profile_read);
 * NULL or "" times every kernel.  Fewer event pairs perturb a run less. */
gs2_status gs2_profile_filter(gs2_handle* h, const char* name);
/* Resolves pending events (synchronising the stream) and copies up to
 * `cap` per-kernel totals into out; *count receives the number written. */
gs2_status gs2_profile_read(gs2_handle* h, gs2_kernel_stat* out, int cap,
                            int* count);
gs2_status gs2_profile_reset(gs2_handle* h);

/* Thread-local message of the last failing call on this thread. */
const char* gs2_last_error(void);

/* Library version string. */
const char* gs2_version(void);

/* Number of CUDA kernel launches this library has made in the process
 * (all handles, all threads), for accounting of launch counts. */
int64_t gs2_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GS2_H */
