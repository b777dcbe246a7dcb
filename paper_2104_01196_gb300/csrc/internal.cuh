// Internal declarations of the GS2 library: handle layout, error plumbing,
// kernel launchers.  Not part of the public ABI (include/gs2.h is).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdint>
#include <exception>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/gs2.h"

namespace gs2 {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

void set_error(const std::string& msg);

struct Error {
  gs2_status st;
  std::string msg;
};

#define GS2_THROW(st, msg) throw ::gs2::Error{(st), (msg)}
#define GS2_CUDA(call)                                                      \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      GS2_THROW(e_ == cudaErrorMemoryAllocation ? GS2_ERR_OOM : GS2_ERR_CUDA, \
                std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)
// every kernel launch of the library is followed by this check, which also
// counts it (gs2_launch_count)
void count_launch();
void add_launches(long long delta);
#define GS2_LAUNCH_CHECK()          \
  do {                              \
    ::gs2::count_launch();          \
    GS2_CUDA(cudaGetLastError());   \
  } while (0)

// NVTX range over a library call: shows each call on the timeline of
// Nsight Systems; without a tool attached it costs a branch
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// device storage
// ---------------------------------------------------------------------------

// A CSR matrix on the device with 32-bit indices.  `va` is FP64; the
// triangles also carry FP32 values and FP16 values with an FP32 per-row
// scale (s_i = max_j |v_ij|, stored v_ij / s_i) once prepared.
struct DevCsr {
  int n = 0;
  int nnz = 0;
  int* rp = nullptr;       // n + 1
  int* ci = nullptr;       // nnz (padded)
  double* va = nullptr;    // nnz (padded)
  float* va32 = nullptr;   // FP32 copy (triangles)
  __half* va16 = nullptr;  // FP16 scaled copy (triangles)
  signed char* scale16 = nullptr;  // FP16 copy: row scale exponent e_i (scale 2^e_i)
  int tpr = 1;             // lanes per row (K) of the tile kernels
  int rpt = 1;             // rows per group of K lanes (RPT), 1 or 2 (K <= 2)
  // row tiles: desc[t] = {first row, end row, first staged entry (rowptr
  // rounded down to 8), end entry}; a tile with more than `cap` entries
  // holds exactly one (long) row and has desc.z = -1 - rowptr[first row]
  int ntiles = 0;
  int cap = 0;
  int4* desc = nullptr;  // ntiles
  double mean_row = 0.0;
  // Sliced-ELL copy (rows of similar length): chunk c holds rows 32c .. 32c+31, its
  // longest row's length L_c times 32 slots, column-major: slot k of row i
  // at sell_ptr[c] + 32 k + i % 32; padding slots have value 0 and repeat
  // a column of the row (column 0 for an empty row)
  //
  // Offset chunks: a chunk whose rows' entries lie on a few diagonals (a
  // stencil's rows: the union of the column offsets j - i over its 32 rows is
  // at most its longest row + 2, and at most 32) stores no columns: slot k of
  // row i is the entry at column i + sell_off[sell_coff[c] + k] (value 0 where
  // row i has no such entry; the column is then clamped into [0, sell_ncols)),
  // the offsets ascending.  sell_coff[c] = -1 marks a chunk with explicit
  // columns in sell_ci.
  bool sell = false;
  int sell_chunks = 0;
  int sell_slots = 0;          // length of the value and column arrays
  int* sell_ptr = nullptr;     // sell_chunks + 1
  int* sell_ci = nullptr;
  int* sell_coff = nullptr;    // sell_chunks: first offset, or -1
  int* sell_off = nullptr;     // the offset lists (chunks with equal lists share one)
  int sell_offset_chunks = 0;  // chunks without explicit columns
  int sell_ncols = 0;          // 1 + the largest column (the gathered vector's length)
  double* sell_va = nullptr;
  float* sell_va32 = nullptr;
  __half* sell_va16 = nullptr;
};

// Device-resident GMRES / CG state, one per handle.
struct KrylovState {
  int stop;      // 1: the current cycle has ended (converged/limit/breakdown)
  int status;    // gs2_status seen by the device
  int k;         // Arnoldi steps taken in the current cycle
  int iters;     // total Arnoldi steps
  int max_iters;
  int cycles;    // restart cycles started (single-launch solver)
  double tol_abs;  // tol * ||b||
  double bnorm;
  double beta;     // ||r0|| of the cycle
  double hn;       // last H(j+1, j)
  double inv_hn;
  double rz;       // CG: r.z
  double alpha;
};

struct Profiler;
struct AmgHierarchy;
struct Pack;

// Hybrid (block-Jacobi) form of the relaxations (Sec. 3): the rows in
// `parts` contiguous blocks (block p: rows [p n / P, (p+1) n / P)), A split
// into the entries inside a row's block (Aloc) and the couplings to other
// blocks (E), and the local parts of the prescaled triangles.
struct Hybrid {
  int parts = 0;
  DevCsr Aloc, E, Lloc, Uloc;
  double* c = nullptr;  // b - E x of the current exchange
  // level sets of the local triangles (local exact GS), built on first use
  bool levels_ready = false;
  std::vector<int> lev_ptr_L, lev_ptr_U;
  int* lev_rows_L = nullptr;
  int* lev_rows_U = nullptr;
};

}  // namespace gs2

struct gs2_handle {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0, nnz = 0;
  gs2::DevCsr A, L, U;  // L, U prescaled: D^{-1} L and D^{-1} U
  // D^{-1}(L + U), prescaled off-diagonal entries (whole-sweep FP32/FP16
  // precisions only: the residual of the single-precision sweep)
  gs2::DevCsr O;
  double* dinv = nullptr;
  int* dev_err = nullptr;  // sticky device error word (bounded waits)
  int64_t dev_bytes = 0;
  std::vector<void*> allocs;

  // resident temporaries (Sec. 6.2: allocated once per matrix)
  double *r = nullptr, *rhat = nullptr, *g0 = nullptr, *g1 = nullptr;
  double *z = nullptr, *t = nullptr, *bstage = nullptr, *xstage = nullptr;
  float *rhat32 = nullptr, *g32a = nullptr, *g32b = nullptr;
  // whole-sweep precisions: fl32(D^{-1} b) and the FP32 iterate
  float *bhat32 = nullptr, *x32 = nullptr;
  double* part = nullptr;  // per-block partial sums
  int nblk = 0;            // blocks of the elementwise vector kernels
  int nblk_dot = 0;        // blocks of the reduction kernels (<= nblk)
  int part_cap = 0;        // doubles in `part`

  // level sets (lazy)
  bool levels_ready = false;
  std::vector<int> lev_ptr_L, lev_ptr_U;  // host, nlev + 1
  int* lev_rows_L = nullptr;
  int* lev_rows_U = nullptr;

  // multicolour GS (lazy): colour c holds the rows color_rows[c] (ascending)
  // and their off-diagonal entries prescaled by D^{-1}, as its own matrix
  bool colors_ready = false;
  std::vector<gs2::DevCsr> colors;
  std::vector<int*> color_rows;

  // Krylov workspace (lazy, grows with restart)
  int kry_m = 0;
  double *V = nullptr, *w = nullptr, *H = nullptr, *hbuf = nullptr;
  double *gvec = nullptr, *cs = nullptr, *sn = nullptr, *y = nullptr;
  double *p = nullptr, *q = nullptr;
  gs2::KrylovState* st = nullptr;       // device
  gs2::KrylovState* st_host = nullptr;  // pinned mirror
  int* err_host = nullptr;              // pinned mirror of dev_err
  volatile int* stop_mapped = nullptr;  // pinned, device-mapped stop flag
  int* stop_mapped_dev = nullptr;

  gs2::Profiler* prof = nullptr;

  // smoothed-aggregation multigrid hierarchy (gs2_amg_setup, or built with
  // default settings on first use as a preconditioner)
  gs2::AmgHierarchy* amg = nullptr;

  // a pack of independent systems (gs2_pack_setup): the matrix is their
  // block-diagonal concatenation; null for a single system
  gs2::Pack* pack = nullptr;
  // hybrid forms built so far, one per partition (ensure_precond)
  std::vector<gs2::Hybrid*> hybrids;

  // per 32-row chunk of A's rows: 0 = the sliced-ELL kernels of A, L and U
  // skip the chunk (set by a pack's solve while some of its systems have
  // finished); null = every chunk
  const int* row_live = nullptr;

  // CUDA graph of one restart cycle's Arnoldi steps (launch-bound small
  // systems): captured on a private stream, replayed there and joined to
  // `stream` with events; re-captured when the cycle's shape changes
  int graph_mode = 0;  // 0: automatic, 1: graphs, 2: separate launches, 3: one launch,
                       // 4: one cluster
  // gs2_autotune_gmres: the automatic mode's tuned choice for (restart,
  // preconditioner) tune_key (0 = not tuned: the size rule)
  int tuned_mode = 0, tuned_candidates = 0;
  std::vector<double> tuned_key;
  double *tune_b = nullptr, *tune_x = nullptr;  // its scratch right-hand side and iterate
  unsigned* persist_bar = nullptr;  // grid barrier of the single-launch solver
  double* persist_part = nullptr;   // its partial sums
  bool stall_barrier = false;       // test hook: next one-launch solve's barrier never opens
  int cl_wa = -1, cl_wl = -1, cl_wu = -1;  // longest rows of A, L, U (longest_rows)
  void* cl_sys = nullptr;  // a pack in clusters: its per-system table (device)
  int cl_sys_cap = 0;
  // one-launch solve of a pack: per-system argument table, block -> system
  // map, barriers, partial sums and results (grown on demand)
  void* pp_args = nullptr;
  int* pp_bsys = nullptr;
  unsigned* pp_bar = nullptr;
  double* pp_part = nullptr;
  gs2::KrylovState* pp_st = nullptr;
  gs2::KrylovState* pp_st_host = nullptr;
  int pp_cap_sys = 0, pp_cap_blocks = 0;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  // CG: a chunk of iterations as one graph (same stream and events)
  cudaGraphExec_t cg_gexec = nullptr;
  std::vector<double> cg_gkey;
  int64_t cg_launches = 0;
  int64_t g_launches = 0;  // kernel launches per replay

  // stream-ordered allocation (cudaMallocAsync / cudaFreeAsync on `stream`):
  // used by server-owned handles so that freeing one request's memory never
  // synchronises the device under the other requests
  bool async_alloc = false;

  void* dalloc(size_t bytes);
  void h2d(void* dst, const void* src, size_t bytes);
  void dzero(void* dst, size_t bytes);
};

namespace gs2 {

// ---------------------------------------------------------------------------
// profiling: optional event pairs around launches
// ---------------------------------------------------------------------------

bool profiling_active(const gs2_handle* h);
// Profiling of restart cycles.  Launches are tagged with the Arnoldi step
// set by capture_step (-1 outside a cycle).  In a captured graph (between
// capture_begin and capture_end) they are bracketed by external event
// nodes; after a cycle that ran `steps` steps, harvest counts only the
// launches of those steps: from the graph's event nodes, or, for an eager
// cycle, by dropping the pending launches of later (no-op) steps.
int profile_epoch(const gs2_handle* h);
void profile_capture_begin(gs2_handle* h);
void profile_capture_step(gs2_handle* h, int step);
void profile_capture_end(gs2_handle* h);
void profile_harvest(gs2_handle* h, int steps, bool graph);

struct KernelTimer {
  gs2_handle* h;
  int id;
  double bytes;
  cudaEvent_t e0 = nullptr;
  KernelTimer(gs2_handle* h_, const char* name, double bytes_);
  ~KernelTimer();
};

// ---------------------------------------------------------------------------
// launchers (kernels.cu)
// ---------------------------------------------------------------------------

// r-hat (and optionally r) from r = b - A x in FP64; rhat written in the
// sweep precision (rhat64 or rhat32, whichever is non-null).
void launch_resid(gs2_handle* h, const double* b, const double* x,
                  double* r_out, double* rhat64, float* rhat32,
                  const int* skip);

// The same with any matrix M over the handle's rows in place of A (the
// hybrid form's local block and couplings).
void launch_resid_matrix(gs2_handle* h, const DevCsr& M, const double* b, const double* x,
                         double* r_out, double* rhat64, float* rhat32, const int* skip);

// Elementwise r-hat = D^{-1} v (v FP64) in the sweep precision.
void launch_prep_rhat(gs2_handle* h, const double* v, double* rhat64,
                      float* rhat32, const int* skip);

// INNER_MID: g' to g_out.  LAST_ADD / LAST_SET: x += omega g' / x = omega g'
// in FP64.  Whole-sweep precisions (FP32 iterate x32): LAST_ADD32 /
// LAST_SET32 write x32 + omega g' / omega g' to x32, LAST_ADD32_OUT /
// LAST_SET32_OUT write the same FP32 value, converted, to the FP64 x (the
// last half sweep of a call).
enum InnerMode {
  INNER_MID = 0,
  INNER_LAST_ADD = 1,
  INNER_LAST_SET = 2,
  INNER_LAST_ADD32 = 3,
  INNER_LAST_SET32 = 4,
  INNER_LAST_ADD32_OUT = 5,
  INNER_LAST_SET32_OUT = 6
};

// whole-sweep precisions and the value precision of their matrices
inline bool is_sweep_precision(int prec) { return prec == GS2_FP32_SWEEP || prec == GS2_FP16_SWEEP; }
inline int value_precision(int prec) {
  return prec == GS2_FP32_SWEEP ? GS2_FP32 : (prec == GS2_FP16_SWEEP ? GS2_FP16_ROWSCALED : prec);
}

// One inner JR sweep on triangle T (h->L or h->U):
//   g_out = (1-gamma) g_in + gamma (rhat - omega T g_in)
// MID writes g_out; LAST_ADD does x += omega g_out; LAST_SET does
// x = omega g_out.  Vectors are FP64 for prec == GS2_FP64, else FP32.
void launch_inner(gs2_handle* h, const DevCsr& T, int prec, const void* rhat,
                  const void* g_in, void* g_out, double* x, double omega,
                  double gamma, int mode, const int* skip);

// compact right-hand side of Eq. (9): rhat = D^{-1} b - Tother x with the
// other prescaled triangle, in the sweep precision
void launch_compact_rhs(gs2_handle* h, const DevCsr& Tother, const double* b, const double* x,
                        double* rhat64, float* rhat32, const int* skip);

// x = omega * rhat (zero inner sweeps from a zero start) or x += omega*rhat.
void launch_rhat_update(gs2_handle* h, int prec, const void* rhat, double* x,
                        double omega, bool add, const int* skip);

// Whole-sweep precisions (vprec: the value precision, GS2_FP32 or
// GS2_FP16_ROWSCALED): rhat32 = fl32(D^{-1} b) - x32 - O x32 in FP32 (bhat32
// and x32 of the handle, O = D^{-1}(L + U)); the update of a sweep with no
// inner sweep, x32 / x from rhat (mode: one of the x32 InnerModes); and the
// conversion x32 = fl32(x).
void launch_resid_sweep(gs2_handle* h, int vprec, const int* skip);
void launch_rhat_update32(gs2_handle* h, const float* rhat, double* x, double omega, int mode,
                          const int* skip);
void launch_to32(gs2_handle* h, const double* x, float* x32, const int* skip);
// M's FP64 values (the nz entries of va, padding included) to M.va32; to
// M.va16 with the per-row power-of-two scale exponents M.scale16 (the FP16
// row-scaled precision)
void launch_values_to_fp32(gs2_handle* h, const DevCsr& M, int64_t nz);
void launch_values_to_fp16(gs2_handle* h, const DevCsr& M);

void launch_spmv(gs2_handle* h, const double* x, double* y, const int* skip);
// autotuner probe: ms per launch of M's most frequent kernel (role 0: A's
// residual, 1 and 2: a triangle's inner sweep), best of reps
float time_tile_probe(gs2_handle* h, const DevCsr& M, int reps, int role);
void launch_jr(gs2_handle* h, const double* b, const double* x_in,
               double* x_out, double omega, const int* skip);
void launch_jr_matrix(gs2_handle* h, const DevCsr& M, const double* b, const double* x_in,
                      double* x_out, double omega, const int* skip);
void launch_level(gs2_handle* h, const DevCsr& T, const int* rows, int r0,
                  int r1, const double* rhat, double* g, double* x,
                  double omega, const int* skip);

// one colour of a multicolour GS sweep: for each row i of the colour matrix
// C (original row rows[i]), x_r = (1 - omega) x_r + omega (bhat_r - (C x)_i)
void launch_color(gs2_handle* h, const DevCsr& C, const int* rows, const double* bhat,
                  double* x, double omega, const int* skip);

// Fill M's sliced-ELL arrays (offsets already in M.sell_ptr, arrays zeroed)
// from its CSR arrays on the device: values from `va` into `sva`, and the
// columns too when with_ci.
void launch_to_sell(gs2_handle* h, const DevCsr& M, const double* va, double* sva, bool with_ci);
void launch_to_sell(gs2_handle* h, const DevCsr& M, const float* va, float* sva, bool with_ci);
void launch_to_sell(gs2_handle* h, const DevCsr& M, const __half* va, __half* sva, bool with_ci);

// y = M x (accumulate: y += M x) for any tiled matrix M whose columns index x
void launch_spmv_matrix(gs2_handle* h, const DevCsr& M, const double* x, double* y,
                        bool accumulate, const int* skip);

void launch_axpy(gs2_handle* h, double* y, double a, const double* x,
                 const int* skip);
void launch_copy(gs2_handle* h, double* dst, const double* src);

// Krylov kernels (krylov.cu)
void ensure_krylov(gs2_handle* h, int m);

// Preconditioner application from a zero start: z = M^{-1} v.  If
// rhat_ready, the sweep-precision D^{-1} v is already in place.
void precond_apply(gs2_handle* h, const gs2_params* p, const double* v,
                   double* z, bool rhat_ready, const int* skip);
// The buffer that must hold D^{-1} v when rhat_ready is passed.
void* precond_rhat_buffer(gs2_handle* h, const gs2_params* p);
bool precond_wants_rhat(const gs2_params* p);

// relaxations (relax.cu)
// the relaxation of p's kind (GS2, JR, exact GS, multicolour GS), global or
// in the hybrid form, from x
void gs2_relax(gs2_handle* h, const double* b, double* x, const gs2_params* p);
void gs_relax(gs2_handle* h, const double* b, double* x, int sweeps,
              double omega, int direction);
void jr_relax(gs2_handle* h, const double* b, double* x, int sweeps,
              double omega);
void mtgs_relax(gs2_handle* h, const double* b, double* x, int sweeps,
                double omega, int direction);
void ensure_levels(gs2_handle* h);
// the hybrid form with p->parts blocks (built on first use, with the
// low-precision triangles p->precision needs); null for parts <= 1
Hybrid* ensure_hybrid(gs2_handle* h, const gs2_params* p);
Hybrid* find_hybrid(gs2_handle* h, int parts);
void ensure_colors(gs2_handle* h);
// level sets or colours a preconditioner needs, built on first use
void ensure_precond(gs2_handle* h, const gs2_params* p);
// p->outer sweeps of a GS2 or JR smoother (p->kind) on A x = b from the
// current x, in direction p->direction (AMG post-smoothing)
void smooth_sweeps(gs2_handle* h, const gs2_params* p, const double* b, double* x,
                   const int* skip);

// smoothed-aggregation AMG (amg.cu)
constexpr int64_t kAmgMaxCoarse = 2048;  // rows of the exactly solved coarsest level
void amg_build(gs2_handle* h, const gs2_amg_cfg& cfg);
void amg_free(gs2_handle* h);
// build the default hierarchy if there is none, and the smoother's precision
void amg_prepare(gs2_handle* h, const gs2_params* p);
void amg_info(const gs2_handle* h, int* levels, int64_t* rows, int64_t* nnz, int64_t* pnnz);
int64_t amg_device_bytes(const gs2_handle* h);
// x = M^{-1} b: one V-cycle from zero (p->kind GS2_PC_AMG or GS2_PC_AMG_JR)
void amg_vcycle(gs2_handle* h, const gs2_params* p, const double* b, double* x,
                bool rhat_ready, const int* skip);
// a tiled CSR matrix on the device, held by h (api.cu)
void upload_matrix(gs2_handle* h, DevCsr& M, int n, const std::vector<int>& rp,
                   const std::vector<int>& ci, const std::vector<double>& va);
void ensure_precision(gs2_handle* h, int prec);

// solvers (krylov.cu)
gs2_status gmres_run(gs2_handle* h, const double* b, double* x, int m,
                     double tol, int max_iters, const gs2_params* p,
                     gs2_solve_info* info);
gs2_status cg_run(gs2_handle* h, const double* b, double* x, double tol,
                  int max_iters, const gs2_params* p, gs2_solve_info* info);
gs2_status gmres_batch(gs2_handle* const* hs, const double* const* bs,
                       double* const* xs, int count, int m, double tol,
                       int max_iters, const gs2_params* p, gs2_solve_info* infos);
void read_state(gs2_handle* h);

// GMRES(m) of a small system as one cooperative launch (persist.cu): n up
// to 65,536 rows (16,384 when chosen automatically), m <= 32, no
// preconditioner, FP64 non-compact GS2 or JR
bool persistent_eligible(const gs2_handle* h, int m, const gs2_params* p, bool automatic);
void longest_rows(gs2_handle* h);
bool cluster_eligible(gs2_handle* h, int m, const gs2_params* p);
gs2_status gmres_cluster(gs2_handle* h, const double* b, double* x, int m, double tol,
                         int max_iters, const gs2_params* p, gs2_solve_info* info);
gs2_status cg_cluster(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                      const gs2_params* p, gs2_solve_info* info);
void gmres_cluster_async(gs2_handle* h, const double* b, double* x, int m, double tol,
                         int max_iters, const gs2_params* p);
gs2_status cluster_result(gs2_handle* h, gs2_solve_info* info);
void copy_state_async(gs2_handle* h);
bool pack_cluster_eligible(gs2_handle* h, int m, const gs2_params* p);
gs2_status pack_gmres_cluster(gs2_handle* h, const double* b, double* x, int m, double tol,
                              int max_iters, const gs2_params* p, gs2_solve_info* infos);
// gs2_autotune_gmres: the fastest solve structure (1, 2, 3) for (m, p)
int autotune_gmres(gs2_handle* h, int m, const gs2_params* p);
void launch_fill_value(gs2_handle* h, double* y, double v);
// every system of a pack in one cooperative launch (per-system blocks,
// barriers and Krylov scalars); eligible like a single system, and when the
// systems' blocks fit the co-resident limit
bool pack_persistent_eligible(const gs2_handle* h, int m, const gs2_params* p, bool automatic);
gs2_status pack_gmres_persistent(gs2_handle* h, const double* b, double* x, int m, double tol,
                                 int max_iters, const gs2_params* p, gs2_solve_info* infos);
gs2_status gmres_persistent(gs2_handle* h, const double* b, double* x, int m, double tol,
                            int max_iters, const gs2_params* p, gs2_solve_info* info);
// preconditioned CG the same way (same eligibility with m = 1)
gs2_status cg_persistent(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                         const gs2_params* p, gs2_solve_info* info);
// a kernel gave up a bounded wait: clear the device error word, throw
void raise_device_error(gs2_handle* h);

// packs of independent systems (pack.cu)
// block-diagonal CSR of `count` systems; off receives the first row of each
// system (count + 1 entries)
void pack_concat(int count, const int64_t* n, const int64_t* const* rowptr,
                 const int32_t* const* col, const double* const* val, std::vector<int64_t>& off,
                 std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va);
void pack_attach(gs2_handle* h, const std::vector<int64_t>& off);
void pack_free(gs2_handle* h);
// drop the pack's captured cycle (tile shapes changed)
void pack_drop_graph(gs2_handle* h);
int pack_count(const gs2_handle* h);
const std::vector<int64_t>* pack_offsets(const gs2_handle* h);
// (system, row of that system) of a row of the pack
std::pair<int, int64_t> pack_locate(const gs2_handle* h, int64_t row);
// GMRES(m) on every system of the pack; infos[count]; returns OK if every
// system converged, else the first failing status
gs2_status pack_gmres_run(gs2_handle* h, const double* b, double* x, int m, double tol,
                          int max_iters, const gs2_params* p, gs2_solve_info* infos);
// the same as a resumable job (as GmresJob); pack_job_info gives system s's
// result once the job is done
struct PackJob;
PackJob* pack_job_start(gs2_handle* h, const double* b, double* x, int m, double tol,
                        int max_iters, const gs2_params* p);
void pack_job_prepare(PackJob* j);
bool pack_job_advance(PackJob* j);
gs2_solve_info pack_job_info(const PackJob* j, int s);
void pack_job_free(PackJob* j);

// A GMRES solve as a resumable job (used by the server): start enqueues
// the first work on the handle's stream (graph mode 4: the whole solve in
// one cluster launch); advance must be called only once that stream is idle
// and returns true when the solve has finished.
struct GmresJob;
GmresJob* gmres_job_start(gs2_handle* h, const double* b, double* x, int m, double tol,
                          int max_iters, const gs2_params* p);
bool gmres_job_advance(GmresJob* j);
// capture the job's cycle graph now (host work only) when it will use one
void gmres_job_prepare(GmresJob* j);
gs2_solve_info gmres_job_info(const GmresJob* j);
void gmres_job_free(GmresJob* j);

// host validation of a CSR matrix as gs2_setup does it (throws the first
// bad row's error); *diag receives the diagonal
void validate_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                  const double* val, std::vector<double>* diag);

// handle creation / destruction shared by gs2_setup and the server
gs2_handle* setup_handle(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                         const double* val, int on_device, unsigned precisions,
                         cudaStream_t stream, bool async_alloc);
void destroy_handle(gs2_handle* h);

// small pinned, device-mapped host buffers, recycled process-wide (freeing
// pinned memory synchronises the device)
void* pinned_get(size_t bytes);
void pinned_put(void* p, size_t bytes);

// Host setup loops run over row ranges on up to kHostThreads threads (one
// range below 64K rows per thread).  An exception thrown by f in a worker
// (a failed host allocation) is rethrown here after every worker has ended.
constexpr int kHostThreads = 16;
template <class F>
inline void parallel_ranges(int64_t n, F f) {
  const int64_t per = 65536;
  const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::max<int64_t>(
      1, std::min<int64_t>({hw, (int64_t)kHostThreads, (n + per - 1) / per}));
  if (nt == 1) {
    f(int64_t(0), n, 0);
    return;
  }
  std::vector<std::exception_ptr> err(nt);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      try {
        f(n * t / nt, n * (t + 1) / nt, t);
      } catch (...) {
        err[t] = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the previous kernel of its stream is finishing; it must
// call pdl_wait() before it touches global memory (the wait returns once the
// previous grid has completed and its writes are visible, and at once for a
// kernel launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// (No kernel triggers its dependents early: a trigger at the start of each
// kernel made the GMRES(30) solve 0.9% slower, one after each main loop
// 0.3% slower, than the implicit trigger at completion.)

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GS2_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// geometry helpers
int vec_blocks(gs2_handle* h, int64_t n);
constexpr int kVecThreads = 256;
constexpr int kRowThreads = 256;
// Mean row length up to which one lane per row is the natural width: such
// matrices always get a sliced-ELL copy (when it pads little), longer rows
// only when they stream from HBM, and then take the pipelined instantiation.
constexpr double kShortRowMean = 24.0;
constexpr int kMaxRestart = 64;

}  // namespace gs2
