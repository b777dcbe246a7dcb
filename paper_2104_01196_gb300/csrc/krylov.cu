// Krylov solvers on the device: restarted GMRES(m), right preconditioned,
// CGS2 Arnoldi, Givens rotations; preconditioned CG.
//
// All scalars stay on the device (KrylovState); the host launches a whole
// restart cycle and reads back one status word per cycle.  Every kernel of
// a step checks the device `stop` flag and returns at once after the cycle
// has ended, so the host may launch a full cycle without knowing when it
// converges.  Reductions are two-level and fixed-order (per-block partials,
// then one block per coefficient), so results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "arnoldi.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace gs2 {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// out[v] = sum over blocks of part[v * nblk + b], one block per v, fixed
// order.  mode 0: H(v, j) = s; mode 1: H(v, j) += s; both also hbuf[v] = s.
__global__ void k_reduce_cols(const double* __restrict__ part, int nblk, double* H, int ldh,
                              int j, double* hbuf, int mode, const int* skip) {
  pdl_wait();
  // the skip flag is read after the partials' loads are issued: one round trip
  const int v = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)v * nblk + b];
  if (skip && *skip) return;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  s = warp_sum(s);
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    double* hv = H + (size_t)j * ldh + v;
    if (mode == 0) *hv = t;
    else *hv += t;
    hbuf[v] = t;
  }
}

// ---------------------------------------------------------------------------
// CGS2 passes over the basis V (row-major by vector, ld = n)
//
// For j + 1 <= 32 basis vectors the kernels are instantiated for the exact
// count JC, so no predicated-off FP64 instruction takes an issue slot; larger
// restarts use the MAXK = 64 forms with a runtime bound.
// ---------------------------------------------------------------------------

// pass 1: part = V[0..JC)^T w.  (Splitting the vectors over two block
// groups, or two rows per iteration per thread, measured no faster: this
// pass wants every resident warp.)
template <int JC>
__global__ void __launch_bounds__(kVecThreads)
k_dots_x(int n, const double* __restrict__ V, const double* __restrict__ w, double* part,
         int nblk, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  double acc[JC];
#pragma unroll
  for (int k = 0; k < JC; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < JC; ++k) acc[k] = fma(__ldg(V + (size_t)k * n + i), wi, acc[k]);
  }
  block_partials_bf<JC>(acc, part, nblk);
}

// pass 2: w -= V h ; part = V^T w          (NORM = false)
// pass 3: w -= V h ; part[0] = w^T w       (NORM = true)
// (the loop bodies of these two kernels are those of dots_rows and
// update_rows, written out: through the inline functions ptxas allocates
// more registers, which lowers the resident blocks of the dot pass)
template <int JC, bool NORM>
__global__ void __launch_bounds__(kVecThreads)
k_update_x(int n, const double* __restrict__ V, const double* __restrict__ hcoef,
           double* __restrict__ w, double* part, int nblk, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  __shared__ double hneg[JC];
  for (int k = threadIdx.x; k < JC; k += blockDim.x) hneg[k] = -hcoef[k];
  __syncthreads();
  constexpr int NA = NORM ? 1 : JC;
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double wn = w[i];
#pragma unroll
    for (int k = 0; k < JC; ++k) wn = fma(__ldg(V + (size_t)k * n + i), hneg[k], wn);
    w[i] = wn;
    if (NORM) {
      acc[0] = fma(wn, wn, acc[0]);
    } else {
#pragma unroll
      for (int k = 0; k < NA; ++k) acc[k] = fma(__ldg(V + (size_t)k * n + i), wn, acc[k]);
    }
  }
  block_partials_bf<NA>(acc, part, nblk);
}

// runtime-bounded forms for 32 < j + 1 <= 64
template <int MAXK>
__global__ void __launch_bounds__(kVecThreads)
k_dots(int n, const double* __restrict__ V, int jc, const double* __restrict__ w,
       double* part, int nblk, const int* skip) {
  if (skip && *skip) return;
  double acc[MAXK];
#pragma unroll
  for (int k = 0; k < MAXK; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < MAXK; ++k)
      if (k < jc) acc[k] = fma(__ldg(V + (size_t)k * n + i), wi, acc[k]);
  }
  block_partials<MAXK>(acc, jc, part, nblk);
}

template <int MAXK, bool NORM>
__global__ void __launch_bounds__(kVecThreads)
k_update(int n, const double* __restrict__ V, int jc, const double* __restrict__ hcoef,
         double* w, double* part, int nblk, const int* skip) {
  if (skip && *skip) return;
  __shared__ double hs[MAXK];
  for (int k = threadIdx.x; k < MAXK; k += blockDim.x) hs[k] = k < jc ? hcoef[k] : 0.0;
  __syncthreads();
  constexpr int NA = NORM ? 1 : MAXK;
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < MAXK; ++k)
      if (k < jc) s = fma(__ldg(V + (size_t)k * n + i), hs[k], s);
    const double wn = w[i] - s;
    w[i] = wn;
    if (NORM) {
      acc[0] = fma(wn, wn, acc[0]);
    } else {
#pragma unroll
      for (int k = 0; k < NA; ++k)
        if (k < jc) acc[k] = fma(__ldg(V + (size_t)k * n + i), wn, acc[k]);
    }
  }
  block_partials<NA>(acc, NORM ? 1 : jc, part, nblk);
}

// Givens step j (givens_block) of the single system; a step that ends the
// cycle also raises the mapped host flag.
__global__ void k_givens(const double* __restrict__ part, int nblk, double* H, int ldh, int j,
                         double* cs, double* sn, double* gv, KrylovState* st,
                         volatile int* stop_host) {
  pdl_wait();
  if (givens_block(part, 0, nblk, H + (size_t)j * ldh, cs, sn, gv, j, st, &st->stop) &&
      threadIdx.x == 0)
    *stop_host = 1;
}

// v_{j+1} = w / H(j+1, j), and the preconditioner's D^{-1} v_{j+1}
__global__ void k_scale_next(int n, const double* __restrict__ w, double* vnext,
                             const double* __restrict__ dinv, double* rhat64, float* rhat32,
                             const KrylovState* st) {
  pdl_wait();
  if (st->stop) return;
  scale_rows(blockIdx.x * blockDim.x + threadIdx.x, n, gridDim.x * blockDim.x, st->inv_hn, w,
             vnext, dinv, rhat64, rhat32);
}

// y = R^{-1} g over the k steps of the cycle (backsolve_block)
__global__ void k_backsolve(const double* __restrict__ H, int ldh, const double* gv, double* y,
                            const KrylovState* st) {
  backsolve_block(H, ldh, gv, y, st->k);
}

// u = V[0..k) y and the preconditioner's D^{-1} u
template <int MAXK>
__global__ void __launch_bounds__(kVecThreads)
k_combine(int n, const double* __restrict__ V, const double* __restrict__ y, double* u,
          const double* __restrict__ dinv, double* rhat64, float* rhat32,
          const KrylovState* st) {
  __shared__ double ys[MAXK];
  const int k = st->k;
  for (int i = threadIdx.x; i < MAXK; i += blockDim.x) ys[i] = i < k ? y[i] : 0.0;
  __syncthreads();
  combine_rows<MAXK>(blockIdx.x * blockDim.x + threadIdx.x, n, gridDim.x * blockDim.x, n, V, ys,
                     k, u, dinv, rhat64, rhat32);
}

// per-block partial sums of x^T x
__global__ void __launch_bounds__(kVecThreads)
k_norm_part(int n, const double* __restrict__ x, double* part, int nblk) {
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc[0] = fma(x[i], x[i], acc[0]);
  block_partials<1>(acc, 1, part, nblk);
}

// beta = sqrt(sum part) into st->beta (which = 0) or st->bnorm (which = 1)
__global__ void k_norm_final(const double* __restrict__ part, int nblk, KrylovState* st,
                             int which) {
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (which == 0) st->beta = sqrt(t);
    else st->bnorm = sqrt(t);
  }
}

// cycle start: v_0 = r / beta, D^{-1} v_0, g = (beta, 0, ...), state reset
__global__ void k_cycle_start(int n, const double* __restrict__ r, double* v0,
                              const double* __restrict__ dinv, double* rhat64, float* rhat32,
                              double* gv, int m, KrylovState* st) {
  const double beta = st->beta;
  scale_rows(blockIdx.x * blockDim.x + threadIdx.x, n, gridDim.x * blockDim.x, 1.0 / beta, r, v0,
             dinv, rhat64, rhat32);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= m; i += blockDim.x) gv[i] = i == 0 ? beta : 0.0;
}

__global__ void k_state_init(KrylovState* st, double tol, int max_iters) {
  st->stop = 0;
  st->status = GS2_OK;
  st->k = 0;
  st->iters = 0;
  st->max_iters = max_iters;
  st->tol_abs = tol * st->bnorm;
}

__global__ void k_cycle_reset(KrylovState* st) {
  st->stop = 0;
  st->k = 0;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

void ensure_krylov(gs2_handle* h, int m) {
  if (!h->st) {
    h->st = (KrylovState*)h->dalloc(sizeof(KrylovState));
    h->dzero(h->st, sizeof(KrylovState));
    h->st_host = (KrylovState*)pinned_get(sizeof(KrylovState));
    h->err_host = (int*)pinned_get(sizeof(int));
    int* f = (int*)pinned_get(sizeof(int));
    h->stop_mapped = f;
    GS2_CUDA(cudaHostGetDevicePointer((void**)&h->stop_mapped_dev, f, 0));
    const size_t n = std::max<int64_t>(h->n, 1);
    h->w = (double*)h->dalloc(sizeof(double) * n);
    h->p = (double*)h->dalloc(sizeof(double) * n);
    h->q = (double*)h->dalloc(sizeof(double) * n);
  }
  if (h->kry_m >= m) return;
  const size_t n = std::max<int64_t>(h->n, 1);
  // grow: new basis and Hessenberg storage (old ones stay owned until destroy)
  h->V = (double*)h->dalloc(sizeof(double) * n * (m + 1));
  h->H = (double*)h->dalloc(sizeof(double) * (size_t)(m + 1) * m);
  h->hbuf = (double*)h->dalloc(sizeof(double) * (m + 1));
  h->gvec = (double*)h->dalloc(sizeof(double) * (m + 1));
  h->cs = (double*)h->dalloc(sizeof(double) * (m + 1));
  h->sn = (double*)h->dalloc(sizeof(double) * (m + 1));
  h->y = (double*)h->dalloc(sizeof(double) * (m + 1));
  h->kry_m = m;
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

static int maxk_for(int jc) {
  if (jc <= 8) return 8;
  if (jc <= 16) return 16;
  if (jc <= 32) return 32;
  return 64;
}

#define GS2_JC_CASES(X)                                                                  \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)  \
  X(31) X(32)

// Grid of a reduction kernel: at most `per_sm_max` blocks per SM (0 = as
// many as stay resident, queried once per instantiation), at least ~8 rows
// per thread, no more blocks than the partial-sum buffer holds, and a whole
// multiple of the SM count when there are at least that many (even load per
// SM).  The dot-product pass (one FMA per loaded value) is latency-bound and
// wants every resident warp; the update passes (two FMAs per value for
// w -= Vh, V^T w) are bound by the FP64 pipe and ran fastest at two blocks
// per SM, the update-and-norm pass at three (measured at n = 2.1M), where the
// per-block butterfly reductions stay a few percent of the work.
constexpr int kDotBlocksPerSm = 0, kUpdBlocksPerSm = 2, kNormBlocksPerSm = 3;
static int reduction_grid(gs2_handle* h, const void* fn, int per_sm_max) {
  static std::mutex mu;
  static std::map<const void*, int> occ;
  int per_sm;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = occ.find(fn);
    if (it == occ.end()) {
      int b = 0;
      GS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kVecThreads, 0));
      it = occ.emplace(fn, std::max(b, 1)).first;
    }
    per_sm = it->second;
  }
  if (per_sm_max > 0) per_sm = std::min(per_sm, per_sm_max);
  const int64_t want = (h->n + kVecThreads * 8 - 1) / (kVecThreads * 8);
  int64_t nb = std::min<int64_t>({want, (int64_t)per_sm * h->nsm, (int64_t)h->nblk});
  if (nb >= h->nsm) nb -= nb % h->nsm;
  return (int)std::max<int64_t>(1, nb);
}

// Each launcher returns the number of blocks, i.e. of partial sums per value.
static int launch_dots(gs2_handle* h, int jc, const double* w, const int* skip) {
  KernelTimer tm(h, "cgs2_dots", 8.0 * h->n * (jc + 1));
  const int n = (int)h->n;
  cudaStream_t s = h->stream;
  int nb = 1;
  switch (jc) {
#define GS2_DOTS_CASE(J)                                                          \
  case J:                                                                         \
    nb = reduction_grid(h, (const void*)k_dots_x<J>, kDotBlocksPerSm);            \
    launch_pdl(k_dots_x<J>, nb, kVecThreads, 0, s, n, (const double*)h->V, w,     \
               h->part, nb, skip);                                                \
    break;
    GS2_JC_CASES(GS2_DOTS_CASE)
#undef GS2_DOTS_CASE
    default:
      nb = reduction_grid(h, (const void*)k_dots<64>, kDotBlocksPerSm);
      k_dots<64><<<nb, kVecThreads, 0, s>>>(n, h->V, jc, w, h->part, nb, skip);
      break;
  }
  GS2_LAUNCH_CHECK();
  return nb;
}

template <bool NORM>
static int launch_update(gs2_handle* h, int jc, double* w, const int* skip) {
  KernelTimer tm(h, NORM ? "cgs2_upd_norm" : "cgs2_upd_dots", 8.0 * h->n * (jc + 2));
  const int n = (int)h->n;
  cudaStream_t s = h->stream;
  int nb = 1;
  const int cap = NORM ? kNormBlocksPerSm : kUpdBlocksPerSm;
  switch (jc) {
#define GS2_UPD_CASE(J)                                                                 \
  case J:                                                                               \
    nb = reduction_grid(h, (const void*)k_update_x<J, NORM>, cap);                      \
    launch_pdl(k_update_x<J, NORM>, nb, kVecThreads, 0, s, n, (const double*)h->V,      \
               (const double*)h->hbuf, w, h->part, nb, skip);                           \
    break;
    GS2_JC_CASES(GS2_UPD_CASE)
#undef GS2_UPD_CASE
    default:
      nb = reduction_grid(h, (const void*)k_update<64, NORM>, cap);
      k_update<64, NORM><<<nb, kVecThreads, 0, s>>>(n, h->V, jc, h->hbuf, w, h->part, nb, skip);
      break;
  }
  GS2_LAUNCH_CHECK();
  return nb;
}

static void launch_combine(gs2_handle* h, int m, double* u, double* r64, float* r32) {
  KernelTimer tm(h, "combine", 8.0 * h->n * (m + 1));
  const int n = (int)h->n, nb = h->nblk;
  switch (maxk_for(m)) {
    case 8: k_combine<8><<<nb, kVecThreads, 0, h->stream>>>(n, h->V, h->y, u, h->dinv, r64, r32, h->st); break;
    case 16: k_combine<16><<<nb, kVecThreads, 0, h->stream>>>(n, h->V, h->y, u, h->dinv, r64, r32, h->st); break;
    case 32: k_combine<32><<<nb, kVecThreads, 0, h->stream>>>(n, h->V, h->y, u, h->dinv, r64, r32, h->st); break;
    default: k_combine<64><<<nb, kVecThreads, 0, h->stream>>>(n, h->V, h->y, u, h->dinv, r64, r32, h->st); break;
  }
  GS2_LAUNCH_CHECK();
}

static void launch_norm(gs2_handle* h, const double* x, int which) {
  KernelTimer tm(h, "norm", 8.0 * h->n);
  k_norm_part<<<h->nblk_dot, kVecThreads, 0, h->stream>>>((int)h->n, x, h->part, h->nblk_dot);
  GS2_LAUNCH_CHECK();
  k_norm_final<<<1, 256, 0, h->stream>>>(h->part, h->nblk_dot, h->st, which);
  GS2_LAUNCH_CHECK();
}

// Copy the device state and the sticky error word to pinned host memory.
void copy_state_async(gs2_handle* h) {
  GS2_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KrylovState), cudaMemcpyDeviceToHost,
                           h->stream));
  GS2_CUDA(cudaMemcpyAsync(h->err_host, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream));
}

// A kernel gave up a bounded wait: clear the word and fail the call.
void raise_device_error(gs2_handle* h) {
  const int e = *h->err_host;
  *h->err_host = 0;
  GS2_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
  GS2_THROW((gs2_status)e, "a device-side bounded wait gave up (copy never completed)");
}

void read_state(gs2_handle* h) {
  copy_state_async(h);
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  if (*h->err_host) raise_device_error(h);
}

// ---------------------------------------------------------------------------
// GMRES(m)
// ---------------------------------------------------------------------------

// One GMRES solve as a resumable state machine: `launch_*` only enqueue work
// on the handle's stream and end with an asynchronous copy of the device
// state; `advance` is called after that stream has been synchronised, reads
// the state and either finishes or enqueues the next restart cycle.  Single
// solves drive one machine; the batch call drives many, one stream each.
struct GmresRun {
  gs2_handle* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int m = 0;
  double tol = 0.0;
  int max_iters = 0;
  const gs2_params* pc = nullptr;
  bool wants = false;
  double* r64 = nullptr;
  float* r32 = nullptr;
  double bnorm = 0.0;
  bool first = true;
  bool breakdown = false;
  bool done = false;
  gs2_status st = GS2_OK;
  gs2_solve_info loc{0, 0, GS2_OK, 0.0};

  void start(gs2_handle* h_, const double* b_, double* x_, int m_, double tol_, int maxit,
             const gs2_params* p) {
    h = h_; b = b_; x = x_; m = m_; tol = tol_; max_iters = maxit;
    pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
    if (h->n == 0) {
      done = true;
      return;
    }
    ensure_krylov(h, m);
    wants = precond_wants_rhat(pc);
    if (wants) {
      void* rb = precond_rhat_buffer(h, pc);
      if (rb == (void*)h->rhat32 || rb == (void*)h->bhat32) r32 = (float*)rb;
      else r64 = (double*)rb;
    }
    launch_norm(h, b, 1);
    k_state_init<<<1, 1, 0, h->stream>>>(h->st, tol, max_iters);
    GS2_LAUNCH_CHECK();
    launch_true_residual();
  }

  // r = b - A x, ||r|| -> st->beta, then the state copy to the host
  void launch_true_residual() {
    launch_resid(h, b, x, h->r, nullptr, nullptr, nullptr);
    launch_norm(h, h->r, 0);
    copy_state_async(h);
  }

  void finish(gs2_status s) {
    st = s;
    loc.status = s;
    done = true;
  }

  bool cycle_ran = false;  // a cycle was issued since the last advance
  bool graph_ran = false;  // ... as a replay of the step graph

  // Called with the stream synchronised.
  void advance() {
    if (done) return;
    const KrylovState& hs = *h->st_host;
    if (cycle_ran) {
      // before the next replay re-records the graph's events
      profile_harvest(h, hs.k, graph_ran);
      cycle_ran = graph_ran = false;
    }
    if (first) {
      first = false;
      bnorm = hs.bnorm;
      if (bnorm == 0.0) {
        GS2_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * h->n, h->stream));
        loc.true_relres = 0.0;
        finish(GS2_OK);
        return;
      }
      if (std::isnan(bnorm) || std::isinf(bnorm)) {
        loc.true_relres = NAN;
        finish(GS2_ERR_NAN);
        return;
      }
    }
    if (*h->err_host) raise_device_error(h);
    const double beta = hs.beta;
    loc.true_relres = beta / bnorm;
    loc.iters = hs.iters;
    if (std::isnan(beta) || std::isinf(beta) || hs.status == GS2_ERR_NAN)
      return finish(GS2_ERR_NAN);
    if (loc.true_relres <= tol) return finish(GS2_OK);
    if (hs.status == GS2_ERR_BREAKDOWN) breakdown = true;
    if (breakdown) return finish(GS2_ERR_BREAKDOWN);
    if (loc.iters >= max_iters) return finish(GS2_ERR_NOT_CONVERGED);
    loc.cycles++;
    launch_cycle();
  }

  // Arnoldi step j: z = M^{-1} v_j, w = A z, CGS2, Givens, v_{j+1}.  Every
  // kernel returns at once once the device has stopped the cycle.
  void enqueue_step(int j) {
    const int n = (int)h->n;
    const int ldh = m + 1;
    const int* skip = &h->st->stop;
    const double* vj = h->V + (size_t)j * n;
    precond_apply(h, pc, vj, h->z, wants, skip);
    launch_spmv(h, h->z, h->w, skip);
    const int jc = j + 1;
    // (the column reductions and the Givens step stay separate small
    // kernels: done instead by the last block of each pass, the tail work
    // serialises on one SM and the solve got 2% slower)
    int nbr = launch_dots(h, jc, h->w, skip);
    {
      KernelTimer tm(h, "reduce_cols", 8.0 * jc * nbr);
      launch_pdl(k_reduce_cols, jc, 256, 0, h->stream, (const double*)h->part, nbr, h->H, ldh, j,
                 h->hbuf, 0, skip);
      GS2_LAUNCH_CHECK();
    }
    nbr = launch_update<false>(h, jc, h->w, skip);
    {
      KernelTimer tm(h, "reduce_cols", 8.0 * jc * nbr);
      launch_pdl(k_reduce_cols, jc, 256, 0, h->stream, (const double*)h->part, nbr, h->H, ldh, j,
                 h->hbuf, 1, skip);
      GS2_LAUNCH_CHECK();
    }
    nbr = launch_update<true>(h, jc, h->w, skip);
    {
      KernelTimer tm(h, "givens", 8.0 * nbr + 8.0 * 4 * (j + 2));
      launch_pdl(k_givens, 1, 256, 0, h->stream, (const double*)h->part, nbr, h->H, ldh, j, h->cs,
                 h->sn, h->gvec, h->st, (volatile int*)h->stop_mapped_dev);
      GS2_LAUNCH_CHECK();
    }
    if (j + 1 < m) {
      // w read, v_{j+1} written, and D^{-1} v_{j+1} (D^{-1} read) when wanted
      KernelTimer tm(h, "scale_next", 16.0 * n + (r64 ? 16.0 * n : 0.0) + (r32 ? 12.0 * n : 0.0));
      launch_pdl(k_scale_next, vec_blocks(h, n), kVecThreads, 0, h->stream, n,
                 (const double*)h->w, h->V + (size_t)(j + 1) * n, (const double*)h->dinv, r64,
                 r32, (const KrylovState*)h->st);
      GS2_LAUNCH_CHECK();
    }
  }

  // Graphs by default at every size: even at n = 2.1M the launch gaps of
  // separate launches cost ~6% of a solve.
  bool use_graph() const { return h->graph_mode != 2; }

  // The m steps as one CUDA graph: captured once per cycle shape on the
  // handle's private stream, replayed there between two event joins with
  // the handle's stream.  Steps after the device-side stop run as no-ops.
  void graph_steps() {
    ensure_graph();
    GS2_CUDA(cudaEventRecord(h->gev_in, h->stream));
    GS2_CUDA(cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
    GS2_CUDA(cudaGraphLaunch(h->gexec, h->gstream));
    GS2_CUDA(cudaEventRecord(h->gev_out, h->gstream));
    GS2_CUDA(cudaStreamWaitEvent(h->stream, h->gev_out, 0));
    add_launches(h->g_launches);
  }

  // Capture (once per cycle shape) without running anything: host work
  // only, so a server can do it on a preparation thread.
  void ensure_graph() {
    std::vector<double> key = {(double)m, (double)(uintptr_t)h->V, (double)(uintptr_t)r64,
                               (double)(uintptr_t)r32, (double)(uintptr_t)h->part,
                               (double)(uintptr_t)h->amg, (double)profile_epoch(h)};
    if (pc) {
      const double pk[] = {(double)pc->kind, (double)pc->outer, (double)pc->inner, pc->omega,
                           pc->gamma, (double)pc->direction, (double)pc->precision,
                           (double)pc->form, (double)pc->parts, (double)pc->local_sweeps};
      key.insert(key.end(), pk, pk + 10);
    }
    if (!h->gstream) {
      GS2_CUDA(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
      GS2_CUDA(cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
      GS2_CUDA(cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    }
    if (!h->gexec || h->gkey != key) {
      if (h->gexec) cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
      cudaStream_t user = h->stream;
      h->stream = h->gstream;
      const long long c0 = gs2_launch_count();
      cudaGraph_t g = nullptr;
      profile_capture_begin(h);
      GS2_CUDA(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
      try {
        for (int j = 0; j < m; ++j) {
          profile_capture_step(h, j);
          enqueue_step(j);
        }
      } catch (...) {
        profile_capture_end(h);
        cudaStreamEndCapture(h->gstream, &g);
        if (g) cudaGraphDestroy(g);
        h->stream = user;
        throw;
      }
      profile_capture_end(h);
      h->stream = user;
      GS2_CUDA(cudaStreamEndCapture(h->gstream, &g));
      h->g_launches = gs2_launch_count() - c0;
      add_launches(-h->g_launches);  // captured, not run
      cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
      cudaGraphDestroy(g);
      GS2_CUDA(e);
      h->gkey = key;
    }
  }

  void launch_cycle() {
    const int n = (int)h->n;
    const int ldh = m + 1;
    *h->stop_mapped = 0;
    k_cycle_reset<<<1, 1, 0, h->stream>>>(h->st);
    GS2_LAUNCH_CHECK();
    k_cycle_start<<<vec_blocks(h, n), kVecThreads, 0, h->stream>>>(n, h->r, h->V, h->dinv, r64,
                                                                  r32, h->gvec, m, h->st);
    GS2_LAUNCH_CHECK();
    cycle_ran = true;
    if (use_graph()) {
      graph_steps();
      graph_ran = true;
    } else {
      for (int j = 0; j < m; ++j) {
        if (*h->stop_mapped) break;  // the device has already ended the cycle
        profile_capture_step(h, j);
        enqueue_step(j);
      }
      profile_capture_step(h, -1);
    }
    // x += M^{-1} V y
    k_backsolve<<<1, 64, 0, h->stream>>>(h->H, ldh, h->gvec, h->y, h->st);
    GS2_LAUNCH_CHECK();
    launch_combine(h, m, h->w, r64, r32);
    precond_apply(h, pc, h->w, h->z, wants, nullptr);
    launch_axpy(h, x, 1.0, h->z, nullptr);
    launch_true_residual();
  }
};

// the key of a tuned solve structure: restart and preconditioner
static std::vector<double> solve_key(int m, const gs2_params* p) {
  if (!p || p->kind == GS2_PC_NONE) return {(double)m, -1.0};
  return {(double)m, (double)p->kind, (double)p->outer, (double)p->inner, p->omega, p->gamma,
          (double)p->direction, (double)p->precision, (double)p->form, (double)p->parts,
          (double)p->local_sweeps};
}

static gs2_status gmres_run_mode(gs2_handle* h, const double* b, double* x, int m, double tol,
                                 int max_iters, const gs2_params* p, gs2_solve_info* info);

gs2_status gmres_run(gs2_handle* h, const double* b, double* x, int m, double tol,
                     int max_iters, const gs2_params* p, gs2_solve_info* info) {
  // automatic mode with a structure tuned for this restart and preconditioner
  // (gs2_autotune_gmres): run that structure
  if (h->graph_mode == 0 && h->tuned_mode != 0 && !profiling_active(h) &&
      h->tuned_key == solve_key(m, p)) {
    h->graph_mode = h->tuned_mode;
    gs2_status st;
    try {
      st = gmres_run_mode(h, b, x, m, tol, max_iters, p, info);
    } catch (...) {
      h->graph_mode = 0;
      throw;
    }
    h->graph_mode = 0;
    return st;
  }
  return gmres_run_mode(h, b, x, m, tol, max_iters, p, info);
}

// Time one restart cycle per candidate structure (mode 2: separate
// launches; 1: cycle graphs; 3: one launch and 4: one cluster, where
// eligible) on scratch
// vectors (b = 1, x = 0; tolerance 0 so that every cycle runs all m steps),
// best of two after one untimed run; the fastest becomes the automatic
// choice for (m, p).  Cached by matrix class and (m, p).
static std::mutex g_solve_tune_mu;
static std::map<std::vector<double>, int> g_solve_tune;

int autotune_gmres(gs2_handle* h, int m, const gs2_params* p) {
  std::vector<double> key = solve_key(m, p);
  std::vector<double> ckey = key;
  ckey.push_back(std::lround(2.0 * std::log2((double)std::max<int64_t>(h->n, 1))));
  ckey.push_back(std::lround(4.0 * h->A.mean_row));
  {
    std::lock_guard<std::mutex> g(g_solve_tune_mu);
    auto it = g_solve_tune.find(ckey);
    if (it != g_solve_tune.end()) {
      h->tuned_mode = it->second;
      h->tuned_key = key;
      return it->second;
    }
  }
  if (!h->tune_b) {
    const size_t n = std::max<int64_t>(h->n, 1);
    h->tune_b = (double*)h->dalloc(sizeof(double) * n);
    h->tune_x = (double*)h->dalloc(sizeof(double) * n);
  }
  launch_fill_value(h, h->tune_b, 1.0);
  std::vector<int> cand = {2, 1};
  if (persistent_eligible(h, m, p, false)) cand.push_back(3);
  if (cluster_eligible(h, m, p)) cand.push_back(4);
  const int saved = h->graph_mode;
  cudaEvent_t e0, e1;
  GS2_CUDA(cudaEventCreate(&e0));
  GS2_CUDA(cudaEventCreate(&e1));
  int best = 1;
  float best_ms = 0.f;
  try {
    for (int mode : cand) {
      h->graph_mode = mode;
      float ms = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        GS2_CUDA(cudaMemsetAsync(h->tune_x, 0, sizeof(double) * h->n, h->stream));
        GS2_CUDA(cudaEventRecord(e0, h->stream));
        gmres_run_mode(h, h->tune_b, h->tune_x, m, 0.0, m, p, nullptr);
        GS2_CUDA(cudaEventRecord(e1, h->stream));
        GS2_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        GS2_CUDA(cudaEventElapsedTime(&t, e0, e1));
        if (rep == 1 || (rep == 2 && t < ms)) ms = t;
      }
      if (mode == cand.front() || ms < best_ms) {
        best = mode;
        best_ms = ms;
      }
    }
  } catch (...) {
    h->graph_mode = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  h->graph_mode = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned_mode = best;
  h->tuned_candidates = (int)cand.size();
  h->tuned_key = key;
  std::lock_guard<std::mutex> g(g_solve_tune_mu);
  g_solve_tune[ckey] = best;
  return best;
}

static gs2_status gmres_run_mode(gs2_handle* h, const double* b, double* x, int m, double tol,
                                 int max_iters, const gs2_params* p, gs2_solve_info* info) {
  // small systems: the whole solve inside one cluster when its rows fit the
  // cluster's shared memory (automatic unless per-kernel profiling is on;
  // graph mode 4 asks for it), else in one cooperative launch
  const bool automatic = h->graph_mode == 0 && !profiling_active(h);
  if (h->graph_mode == 4 || (automatic && cluster_eligible(h, m, p)))
    return gmres_cluster(h, b, x, m, tol, max_iters, p, info);
  const bool forced = h->graph_mode == 3;
  if ((forced || automatic) && persistent_eligible(h, m, p, !forced))
    return gmres_persistent(h, b, x, m, tol, max_iters, p, info);
  if (h->graph_mode == 3)
    GS2_THROW(GS2_ERR_INVALID_ARG, "the one-launch solver takes n <= 65536, restart <= 32 and "
                                   "no, JR or FP64 non-compact GS2 preconditioning");
  GmresRun g;
  g.start(h, b, x, m, tol, max_iters, p);
  while (!g.done) {
    GS2_CUDA(cudaStreamSynchronize(h->stream));
    g.advance();
  }
  if (info) *info = g.loc;
  return g.st;
}

// Resumable job: owns a copy of the preconditioner parameters so that the
// caller's struct need not outlive the call that started it.
struct GmresJob {
  gs2_params params{};
  bool has_params = false;
  GmresRun run;
  // graph mode 4: the whole solve was enqueued as one cluster launch; its
  // outcome is read once the stream is idle
  gs2_handle* cluster = nullptr;
  gs2_solve_info loc{};
  bool done = false;
};

GmresJob* gmres_job_start(gs2_handle* h, const double* b, double* x, int m, double tol,
                          int max_iters, const gs2_params* p) {
  GmresJob* j = new GmresJob();
  if (p) {
    j->params = *p;
    j->has_params = true;
  }
  try {
    if (h->graph_mode == 4) {
      // the whole solve in one cluster launch, the state copied back behind it
      gmres_cluster_async(h, b, x, m, tol, max_iters, j->has_params ? &j->params : nullptr);
      j->cluster = h;
    } else {
      j->run.start(h, b, x, m, tol, max_iters, j->has_params ? &j->params : nullptr);
    }
  } catch (...) {
    delete j;
    throw;
  }
  return j;
}

void gmres_job_prepare(GmresJob* j) {
  if (!j->cluster && !j->run.done && j->run.use_graph()) j->run.ensure_graph();
}

bool gmres_job_advance(GmresJob* j) {
  if (j->cluster) {
    if (!j->done) {
      j->done = true;
      cluster_result(j->cluster, &j->loc);  // raises if a barrier gave up
    }
    return true;
  }
  if (!j->run.done) j->run.advance();
  return j->run.done;
}

gs2_solve_info gmres_job_info(const GmresJob* j) {
  if (j->cluster) return j->loc;
  gs2_solve_info i = j->run.loc;
  i.status = j->run.st;
  return i;
}

void gmres_job_free(GmresJob* j) { delete j; }

gs2_status gmres_batch(gs2_handle* const* hs, const double* const* bs, double* const* xs,
                       int count, int m, double tol, int max_iters, const gs2_params* p,
                       gs2_solve_info* infos) {
  std::vector<GmresRun> runs(count);
  for (int i = 0; i < count; ++i) runs[i].start(hs[i], bs[i], xs[i], m, tol, max_iters, p);
  for (;;) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
      if (runs[i].done) continue;
      // poll first so that finished systems are served while others run
      if (cudaStreamQuery(hs[i]->stream) == cudaErrorNotReady) {
        any = true;
        continue;
      }
      GS2_CUDA(cudaStreamSynchronize(hs[i]->stream));
      runs[i].advance();
      any = any || !runs[i].done;
    }
    if (!any) break;
    std::this_thread::yield();
  }
  gs2_status first_bad = GS2_OK;
  for (int i = 0; i < count; ++i) {
    GS2_CUDA(cudaStreamSynchronize(hs[i]->stream));
    if (infos) infos[i] = runs[i].loc;
    if (runs[i].st != GS2_OK && first_bad == GS2_OK) first_bad = runs[i].st;
  }
  return first_bad;
}

// ---------------------------------------------------------------------------
// preconditioned CG
// ---------------------------------------------------------------------------

// part = [p.q partials]
__global__ void __launch_bounds__(kVecThreads)
k_dot_part(int n, const double* __restrict__ a, const double* __restrict__ b, double* part,
           int nblk, const int* skip) {
  if (skip && *skip) return;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc[0] = fma(a[i], b[i], acc[0]);
  block_partials<1>(acc, 1, part, nblk);
}

// reduce part into a scalar: what = 0 -> alpha = rz / (p.q) (breakdown if
// p.q == 0); what = 1 -> beta_cg = rz_new / rz, rz = rz_new (stored in hn)
__global__ void k_cg_scalar(const double* __restrict__ part, int nblk, KrylovState* st,
                            int what, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  if (what == 0) {
    if (t == 0.0) {
      st->status = GS2_ERR_BREAKDOWN;
      st->stop = 1;
      return;
    }
    st->alpha = st->rz / t;
  } else if (what == 1) {
    st->hn = t / st->rz;  // beta of CG
    st->rz = t;
  } else {
    st->rz = t;
  }
}

// x += alpha p ; r -= alpha q ; part = r.r ; and the preconditioner's
// D^{-1} r in its sweep precision (whichever of rhat64, rhat32 is non-null)
__global__ void __launch_bounds__(kVecThreads)
k_cg_xr(int n, double* x, double* r, const double* __restrict__ p, const double* __restrict__ q,
        double* part, int nblk, const KrylovState* st, const int* skip,
        const double* __restrict__ dinv, double* rhat64, float* rhat32) {
  if (skip && *skip) return;
  const double a = st->alpha;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    acc[0] = fma(ri, ri, acc[0]);
    if (rhat64) rhat64[i] = dinv[i] * ri;
    if (rhat32) rhat32[i] = (float)(dinv[i] * ri);
  }
  block_partials<1>(acc, 1, part, nblk);
}

// ||r|| test after an iteration: stop the loop of launches when converged
__global__ void k_cg_check(const double* __restrict__ part, int nblk, KrylovState* st,
                           volatile int* stop_host, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  const double rn = sqrt(t);
  st->iters += 1;
  st->beta = rn;
  if (isnan(rn) || isinf(rn)) {
    st->status = GS2_ERR_NAN;
    st->stop = 1;
  } else if (rn <= st->tol_abs || st->iters >= st->max_iters) {
    st->stop = 1;
  }
  if (st->stop) *stop_host = 1;
}

// p = z + beta p
__global__ void k_cg_p(int n, double* p, const double* __restrict__ z, const KrylovState* st,
                       const int* skip) {
  if (skip && *skip) return;
  const double bt = st->hn;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = fma(bt, p[i], z[i]);
}

gs2_status cg_run(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                  const gs2_params* p, gs2_solve_info* info) {
  gs2_solve_info loc{0, 0, GS2_OK, 0.0};
  if (h->n == 0) {
    if (info) *info = loc;
    return GS2_OK;
  }
  {
    // small systems: inside one cluster where the rows fit (graph mode 4 or
    // automatic), else in one cooperative launch (graph mode 3 or automatic)
    const bool automatic = h->graph_mode == 0 && !profiling_active(h);
    if (h->graph_mode == 4 || (automatic && cluster_eligible(h, 2, p)))
      return cg_cluster(h, b, x, tol, max_iters, p, info);
    const bool forced = h->graph_mode == 3;
    if ((forced || automatic) && persistent_eligible(h, 1, p, !forced))
      return cg_persistent(h, b, x, tol, max_iters, p, info);
    if (forced)
      GS2_THROW(GS2_ERR_INVALID_ARG, "the one-launch solver takes n <= 65536 and no, JR or "
                                     "FP64 non-compact GS2 preconditioning");
  }
  ensure_krylov(h, 1);
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  const int n = (int)h->n, nb = h->nblk_dot;
  const int* skip = &h->st->stop;
  double* r = h->r;
  double* z = h->z;
  double* pv = h->p;
  double* q = h->q;

  launch_norm(h, b, 1);
  k_state_init<<<1, 1, 0, h->stream>>>(h->st, tol, max_iters);
  GS2_LAUNCH_CHECK();
  read_state(h);
  const double bnorm = h->st_host->bnorm;
  if (bnorm == 0.0) {
    GS2_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));
    if (info) *info = loc;
    return GS2_OK;
  }
  gs2_status st = GS2_OK;
  // the preconditioner's D^{-1} r comes from the kernel that updates r
  const bool wants = precond_wants_rhat(pc);
  double* r64 = nullptr;
  float* r32 = nullptr;
  if (wants) {
    void* rb = precond_rhat_buffer(h, pc);
    if (rb == (void*)h->rhat32 || rb == (void*)h->bhat32) r32 = (float*)rb;
    else r64 = (double*)rb;
  }
  // one CG iteration (every kernel a no-op once the device has stopped)
  auto enqueue_iter = [&]() {
    launch_spmv(h, pv, q, skip);
    k_dot_part<<<nb, kVecThreads, 0, h->stream>>>(n, pv, q, h->part, nb, skip);
    k_cg_scalar<<<1, 256, 0, h->stream>>>(h->part, nb, h->st, 0, skip);
    k_cg_xr<<<nb, kVecThreads, 0, h->stream>>>(n, x, r, pv, q, h->part, nb, h->st, skip,
                                               h->dinv, r64, r32);
    k_cg_check<<<1, 256, 0, h->stream>>>(h->part, nb, h->st, h->stop_mapped_dev, skip);
    precond_apply(h, pc, r, z, wants, skip);
    k_dot_part<<<nb, kVecThreads, 0, h->stream>>>(n, r, z, h->part, nb, skip);
    k_cg_scalar<<<1, 256, 0, h->stream>>>(h->part, nb, h->st, 1, skip);
    k_cg_p<<<vec_blocks(h, n), kVecThreads, 0, h->stream>>>(n, pv, z, h->st, skip);
    GS2_LAUNCH_CHECK();
  };
  constexpr int kCheckEvery = 16;
  // graphs (default): kCheckEvery iterations captured once, replayed on the
  // handle's graph stream; x is the handle's own accumulator so that the
  // graph does not depend on the caller's pointer
  const bool graph = h->graph_mode != 2;
  double* xu = x;
  if (graph) {
    x = h->w;
    launch_copy(h, x, xu);
    std::vector<double> key = {(double)(uintptr_t)x, (double)(uintptr_t)r64,
                               (double)(uintptr_t)r32, (double)(uintptr_t)h->part,
                               (double)profile_epoch(h)};
    if (pc) {
      const double pk[] = {(double)pc->kind, (double)pc->outer, (double)pc->inner, pc->omega,
                           pc->gamma, (double)pc->direction, (double)pc->precision,
                           (double)pc->form, (double)pc->parts, (double)pc->local_sweeps};
      key.insert(key.end(), pk, pk + 10);
    }
    if (!h->gstream) {
      GS2_CUDA(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
      GS2_CUDA(cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
      GS2_CUDA(cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    }
    if (!h->cg_gexec || h->cg_gkey != key) {
      if (h->cg_gexec) cudaGraphExecDestroy(h->cg_gexec);
      h->cg_gexec = nullptr;
      cudaStream_t user = h->stream;
      h->stream = h->gstream;
      const long long c0 = gs2_launch_count();
      cudaGraph_t g = nullptr;
      profile_capture_begin(h);
      GS2_CUDA(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
      try {
        for (int it = 0; it < kCheckEvery; ++it) {
          profile_capture_step(h, it);
          enqueue_iter();
        }
      } catch (...) {
        profile_capture_end(h);
        cudaStreamEndCapture(h->gstream, &g);
        if (g) cudaGraphDestroy(g);
        h->stream = user;
        throw;
      }
      profile_capture_end(h);
      h->stream = user;
      GS2_CUDA(cudaStreamEndCapture(h->gstream, &g));
      h->cg_launches = gs2_launch_count() - c0;
      add_launches(-h->cg_launches);  // captured, not run
      cudaError_t e = cudaGraphInstantiate(&h->cg_gexec, g, 0);
      cudaGraphDestroy(g);
      GS2_CUDA(e);
      h->cg_gkey = key;
    }
  }
  launch_resid(h, b, x, r, nullptr, nullptr, nullptr);
  for (;;) {
    // (re)start the search direction from the current residual
    launch_norm(h, r, 0);
    read_state(h);
    double rn = h->st_host->beta;
    loc.iters = h->st_host->iters;
    if (std::isnan(rn) || std::isinf(rn)) {
      st = GS2_ERR_NAN;
      break;
    }
    if (rn <= tol * bnorm) {
      // confirm on the true residual
      launch_resid(h, b, x, h->t, nullptr, nullptr, nullptr);
      launch_norm(h, h->t, 0);
      read_state(h);
      if (h->st_host->beta <= tol * bnorm) break;
      launch_copy(h, r, h->t);
      rn = h->st_host->beta;
    }
    if (loc.iters >= max_iters) {
      st = GS2_ERR_NOT_CONVERGED;
      break;
    }
    loc.cycles++;
    *h->stop_mapped = 0;
    k_cycle_reset<<<1, 1, 0, h->stream>>>(h->st);
    precond_apply(h, pc, r, z, false, nullptr);
    launch_copy(h, pv, z);
    k_dot_part<<<nb, kVecThreads, 0, h->stream>>>(n, r, z, h->part, nb, nullptr);
    k_cg_scalar<<<1, 256, 0, h->stream>>>(h->part, nb, h->st, 2, nullptr);
    GS2_LAUNCH_CHECK();
    for (;;) {
      const int before = h->st_host->iters;
      if (graph) {
        GS2_CUDA(cudaEventRecord(h->gev_in, h->stream));
        GS2_CUDA(cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
        GS2_CUDA(cudaGraphLaunch(h->cg_gexec, h->gstream));
        GS2_CUDA(cudaEventRecord(h->gev_out, h->gstream));
        GS2_CUDA(cudaStreamWaitEvent(h->stream, h->gev_out, 0));
        add_launches(h->cg_launches);
      } else {
        for (int it = 0; it < kCheckEvery; ++it) {
          if (*h->stop_mapped) break;
          profile_capture_step(h, it);
          enqueue_iter();
        }
        profile_capture_step(h, -1);
      }
      read_state(h);
      // launches of the iterations that ran (the rest were no-ops)
      profile_harvest(h, h->st_host->iters - before, graph);
      if (h->st_host->stop) break;
    }
    if (h->st_host->status == GS2_ERR_NAN) {
      st = GS2_ERR_NAN;
      loc.iters = h->st_host->iters;
      break;
    }
    if (h->st_host->status == GS2_ERR_BREAKDOWN) {
      st = GS2_ERR_BREAKDOWN;
      loc.iters = h->st_host->iters;
      break;
    }
  }
  launch_resid(h, b, x, h->t, nullptr, nullptr, nullptr);
  launch_norm(h, h->t, 0);
  if (x != xu) launch_copy(h, xu, x);
  read_state(h);
  loc.true_relres = h->st_host->beta / bnorm;
  loc.status = st;
  if (info) *info = loc;
  return st;
}

}  // namespace gs2
