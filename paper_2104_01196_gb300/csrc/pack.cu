// Packs: many independent systems solved together as one block-diagonal
// matrix diag(A_0, ..., A_{S-1}) held by a single handle.
//
// A GS2 sweep (and the residual, the SpMV, JR, level-scheduled and
// multicolour GS) of a block-diagonal matrix is the sweep of every block on
// its own: a row reads only columns of its own system, the triangles of the
// pack are the blocks' triangles, and its level sets and first-fit colours
// are those of the blocks side by side.  So each row kernel covers all
// systems of a pack in one launch, with the row arithmetic of a single
// system.  What is per system is the Krylov method: restarted GMRES(m) with
// CGS2 and Givens rotations (the same steps as krylov.cu) runs for every
// system at once, with per-system inner products, Hessenberg matrices,
// rotations, stopping decisions and iteration counts.  Restart cycles are in
// lockstep: each is one replay of the m captured Arnoldi steps for all
// systems; a system whose cycle has ended skips the Krylov kernels (its rows
// still pass through the row kernels, harmlessly: they read and write only
// its own part of the vectors), and a system that has finished takes no
// further cycles.  The vector kernels of the Krylov method run over a block
// table in which every block lies inside one system.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>

#include "arnoldi.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace gs2 {

struct Pack {
  int count = 0;
  std::vector<int64_t> off;  // first row of each system, count + 1
  int nb = 0;                // blocks of the per-system vector kernels
  int4* blk = nullptr;       // nb: {system, first row, end row, first block of its system}
  int* seg_blk = nullptr;    // count + 1: first block of each system
  KrylovState* st = nullptr;       // device, count
  KrylovState* st_host = nullptr;  // pinned mirror
  int* active = nullptr;           // device, count: system takes the next cycle
  int* active_host = nullptr;      // pinned
  int* nactive = nullptr;          // device: systems still in the current cycle
  int* off_dev = nullptr;          // device copy of off (int32)
  // per 32-row chunk: systems overlapping the chunk that take the current
  // cycle (live_cycle) and that are still running in it (live_run); the
  // sliced-ELL row kernels skip chunks at zero
  int nchunks = 0;
  int* live_cycle = nullptr;
  int* live_run = nullptr;
  // work lists of the systems taking the current cycle (written by the host
  // before each cycle): their block-table entries and the systems, with the
  // two counts in cnt[0], cnt[1]; grids of the kernels looping over them
  std::vector<int> seg_blk_host;
  int* items = nullptr;
  int* sys = nullptr;
  int* cnt = nullptr;
  int* items_host = nullptr;
  int* sys_host = nullptr;
  int* cnt_host = nullptr;
  int gb = 1, gs = 1;
  int m = 0;                       // restart the arrays below are sized for
  double *H = nullptr, *hbuf = nullptr, *gvec = nullptr, *cs = nullptr, *sn = nullptr,
         *y = nullptr, *part = nullptr;
  // captured Arnoldi steps of one cycle
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  int64_t g_launches = 0;

  size_t hstride() const { return (size_t)(m + 1) * m; }  // H of one system
  size_t vstride() const { return (size_t)m + 1; }        // g, cs, sn, y, hbuf
};

// ---------------------------------------------------------------------------
// kernels
//
// Work lists: the block-table entries (`items`, count at *nitems) and the
// systems (`sys`, count at *nsys) of the systems taking the current cycle,
// written by the host before each cycle.  Kernels run a fixed grid (captured
// once) and loop over the list, so a cycle in which few systems remain costs
// one short wave per kernel, not one block per entry of the table.  Whether
// a block skips an item is uniform over the block; a block that loops runs
// a barrier before it reuses shared memory.
// ---------------------------------------------------------------------------

// p = V[0..JC)^T w over an item's rows (an item of a stopped system writes
// nothing: its partial sums are never read)
template <int JC>
__global__ void __launch_bounds__(kVecThreads)
k_pdots(int ld, const int4* __restrict__ blk, const int* __restrict__ items,
        const int* __restrict__ nitems, const KrylovState* st, const double* __restrict__ V,
        const double* __restrict__ w, double* part, int nb) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int e = items[q];
    const int4 b = blk[e];
    if (st[b.x].stop) continue;
    double acc[JC];
#pragma unroll
    for (int k = 0; k < JC; ++k) acc[k] = 0.0;
    dots_rows<JC>(b.y + threadIdx.x, b.z, blockDim.x, ld, V, w, acc);
    block_partials_bf<JC>(acc, part, nb, e);
    __syncthreads();
  }
}

// w -= V h (h of the item's system); then p = V^T w or p = w^T w
template <int JC, bool NORM>
__global__ void __launch_bounds__(kVecThreads)
k_pupdate(int ld, const int4* __restrict__ blk, const int* __restrict__ items,
          const int* __restrict__ nitems, const KrylovState* st, const double* __restrict__ V,
          const double* __restrict__ hbuf, int hb_stride, double* __restrict__ w, double* part,
          int nb) {
  __shared__ double hneg[JC];
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int e = items[q];
    const int4 b = blk[e];
    if (st[b.x].stop) continue;
    for (int k = threadIdx.x; k < JC; k += blockDim.x)
      hneg[k] = -hbuf[(size_t)b.x * hb_stride + k];
    __syncthreads();
    constexpr int NA = NORM ? 1 : JC;
    double acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    update_rows<JC, NORM>(b.y + threadIdx.x, b.z, blockDim.x, ld, V, hneg, w, acc);
    block_partials_bf<NA>(acc, part, nb, e);
    __syncthreads();
  }
}

// runtime-bounded forms for 32 < jc <= 64 basis vectors
template <int MAXK>
__global__ void __launch_bounds__(kVecThreads)
k_pdots_rt(int ld, const int4* __restrict__ blk, const int* __restrict__ items,
           const int* __restrict__ nitems, const KrylovState* st, const double* __restrict__ V,
           int jc, const double* __restrict__ w, double* part, int nb) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int e = items[q];
    const int4 b = blk[e];
    if (st[b.x].stop) continue;
    double acc[MAXK];
#pragma unroll
    for (int k = 0; k < MAXK; ++k) acc[k] = 0.0;
    for (int i = b.y + threadIdx.x; i < b.z; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int k = 0; k < MAXK; ++k)
        if (k < jc) acc[k] = fma(__ldg(V + (size_t)k * ld + i), wi, acc[k]);
    }
    block_partials<MAXK>(acc, jc, part, nb, e);
    __syncthreads();
  }
}

template <int MAXK, bool NORM>
__global__ void __launch_bounds__(kVecThreads)
k_pupdate_rt(int ld, const int4* __restrict__ blk, const int* __restrict__ items,
             const int* __restrict__ nitems, const KrylovState* st,
             const double* __restrict__ V, int jc, const double* __restrict__ hbuf,
             int hb_stride, double* w, double* part, int nb) {
  __shared__ double hneg[MAXK];
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int e = items[q];
    const int4 b = blk[e];
    if (st[b.x].stop) continue;
    for (int k = threadIdx.x; k < MAXK; k += blockDim.x)
      hneg[k] = k < jc ? -hbuf[(size_t)b.x * hb_stride + k] : 0.0;
    __syncthreads();
    constexpr int NA = NORM ? 1 : MAXK;
    double acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    for (int i = b.y + threadIdx.x; i < b.z; i += blockDim.x) {
      double wn = w[i];
#pragma unroll
      for (int k = 0; k < MAXK; ++k)
        if (k < jc) wn = fma(__ldg(V + (size_t)k * ld + i), hneg[k], wn);
      w[i] = wn;
      if (NORM) {
        acc[0] = fma(wn, wn, acc[0]);
      } else {
#pragma unroll
        for (int k = 0; k < NA; ++k)
          if (k < jc) acc[k] = fma(__ldg(V + (size_t)k * ld + i), wn, acc[k]);
      }
    }
    block_partials<NA>(acc, NORM ? 1 : jc, part, nb, e);
    __syncthreads();
  }
}

// Per system: coefficient v of column j is the fixed-order sum of the
// system's block partials (warps over coefficients, lanes over blocks).
// mode 0: H(v, j) = s; mode 1: H(v, j) += s; both also hbuf[v] = s.
__global__ void k_preduce(const double* __restrict__ part, int nb, const int* __restrict__ seg_blk,
                          const int* __restrict__ sys, const int* __restrict__ nsys,
                          const KrylovState* st, double* H, size_t hstride, int ldh, int j,
                          double* hbuf, int hb_stride, int mode, int jc) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nq = *nsys;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int s = sys[q];
    if (st[s].stop) continue;
    const int b0 = seg_blk[s], b1 = seg_blk[s + 1];
    double* col = H + s * hstride + (size_t)j * ldh;
    for (int v = wid; v < jc; v += nw) {
      double t = 0.0;
      for (int b = b0 + lane; b < b1; b += 32) t += part[(size_t)v * nb + b];
      t = warp_sum(t);
      if (lane == 0) {
        if (mode == 0) col[v] = t;
        else col[v] += t;
        hbuf[(size_t)s * hb_stride + v] = t;
      }
    }
  }
}

// Per system: the Givens step (givens_block).  A system that stops takes its
// rows out of the row kernels for the rest of the cycle; the last one to
// stop stops the pack's row kernels and raises the host flag.
__global__ void k_pgivens(const double* __restrict__ part, const int* __restrict__ seg_blk,
                          const int* __restrict__ sys, const int* __restrict__ nsys,
                          KrylovState* st, double* H, size_t hstride, int ldh, int j,
                          double* cs, double* sn, double* gv, int vstride, int* nactive,
                          const int* __restrict__ off, int* live_run, KrylovState* pack_st,
                          volatile int* stop_host) {
  const int nq = *nsys;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int s = sys[q];
    if (st[s].stop) continue;
    const size_t o = (size_t)s * vstride;
    const bool ended = givens_block(part, seg_blk[s], seg_blk[s + 1],
                                    H + s * hstride + (size_t)j * ldh, cs + o, sn + o, gv + o, j,
                                    st + s);
    if (ended) {
      for (int c = off[s] / 32 + threadIdx.x; c <= (off[s + 1] - 1) / 32; c += blockDim.x)
        atomicSub(live_run + c, 1);
      if (threadIdx.x == 0 && atomicSub(nactive, 1) == 1) {
        pack_st->stop = 1;
        *stop_host = 1;
      }
    }
    __syncthreads();
  }
}

// system of row r: the last s with off[s] <= r (empty systems share their
// offset with the next one and hold no row)
__device__ __forceinline__ int system_of(const int* __restrict__ off, int count, int r) {
  int lo = 0, hi = count;  // off[lo] <= r < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= r) lo = mid;
    else hi = mid;
  }
  return lo;
}

// chunk liveness at a cycle start: the number of systems overlapping each
// 32-row chunk that take the cycle
__global__ void k_plive_init(int nchunks, int n, const int* __restrict__ off, int count,
                             const int* __restrict__ active, int* live_cycle, int* live_run) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
    const int s0 = system_of(off, count, 32 * c);
    const int s1 = system_of(off, count, min(32 * c + 31, n - 1));
    int k = 0;
    for (int s = s0; s <= s1; ++s) k += active[s] != 0;
    live_cycle[c] = k;
    live_run[c] = k;
  }
}

// x += z over the items (the systems that took the cycle)
__global__ void __launch_bounds__(kVecThreads)
k_paxpy(const int4* __restrict__ blk, const int* __restrict__ items,
        const int* __restrict__ nitems, double* x, const double* __restrict__ z) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int4 b = blk[items[q]];
    for (int i = b.y + threadIdx.x; i < b.z; i += blockDim.x) x[i] = x[i] + z[i];
  }
}

// v_{j+1} = w / H(j+1, j) of the item's system, and D^{-1} v_{j+1}
__global__ void __launch_bounds__(kVecThreads)
k_pscale_next(const int4* __restrict__ blk, const int* __restrict__ items,
              const int* __restrict__ nitems, const KrylovState* st,
              const double* __restrict__ w, double* vnext, const double* __restrict__ dinv,
              double* rhat64, float* rhat32) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int4 b = blk[items[q]];
    if (st[b.x].stop) continue;
    scale_rows(b.y + threadIdx.x, b.z, blockDim.x, st[b.x].inv_hn, w, vnext, dinv, rhat64,
               rhat32);
  }
}

// per-item partial sums of x^T x
__global__ void __launch_bounds__(kVecThreads)
k_pnorm_part(const int4* __restrict__ blk, const int* __restrict__ items,
             const int* __restrict__ nitems, const double* __restrict__ x, double* part,
             int nb) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int e = items[q];
    const int4 b = blk[e];
    double acc[1] = {0.0};
    for (int i = b.y + threadIdx.x; i < b.z; i += blockDim.x) acc[0] = fma(x[i], x[i], acc[0]);
    block_partials_bf<1>(acc, part, nb, e);
    __syncthreads();
  }
}

// per system: sqrt of the sum of its partials into st.beta (which = 0) or
// st.bnorm (which = 1)
__global__ void k_pnorm_final(const double* __restrict__ part, const int* __restrict__ seg_blk,
                              const int* __restrict__ sys, const int* __restrict__ nsys,
                              KrylovState* st, int which) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nq = *nsys;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int s = sys[q];
    double t = 0.0;
    for (int b = seg_blk[s] + threadIdx.x; b < seg_blk[s + 1]; b += blockDim.x) t += part[b];
    t = warp_sum(t);
    if (lane == 0) red[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
      if (which == 0) st[s].beta = sqrt(u);
      else st[s].bnorm = sqrt(u);
    }
    __syncthreads();
  }
}

__global__ void k_pstate_init(KrylovState* st, int count, double tol, int max_iters) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
    KrylovState& q = st[s];
    q.stop = 0;
    q.status = GS2_OK;
    q.k = 0;
    q.iters = 0;
    q.max_iters = max_iters;
    q.tol_abs = tol * q.bnorm;
  }
}

// Cycle reset (one block): systems not taking this cycle start stopped;
// nactive counts the others.
__global__ void k_pcycle_reset(KrylovState* st, const int* __restrict__ active, int count,
                               int* nactive, KrylovState* pack_st) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int s = threadIdx.x; s < count; s += blockDim.x) {
    const int a = active[s] != 0;
    st[s].stop = !a;
    st[s].k = 0;
    mine += a;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    *nactive = cnt;
    pack_st->stop = cnt == 0;
  }
}

// cycle start of the item's system: v_0 = r / beta, D^{-1} v_0, and (its
// first block) g = (beta, 0, ..., 0)
__global__ void __launch_bounds__(kVecThreads)
k_pcycle_start(const int4* __restrict__ blk, const int* __restrict__ items,
               const int* __restrict__ nitems, const KrylovState* st,
               const double* __restrict__ r, double* v0, const double* __restrict__ dinv,
               double* rhat64, float* rhat32, double* gv, int vstride, int m) {
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int4 b = blk[items[q]];
    if (st[b.x].stop) continue;
    const double beta = st[b.x].beta;
    scale_rows(b.y + threadIdx.x, b.z, blockDim.x, 1.0 / beta, r, v0, dinv, rhat64, rhat32);
    if (b.w)
      for (int i = threadIdx.x; i <= m; i += blockDim.x)
        gv[(size_t)b.x * vstride + i] = i == 0 ? beta : 0.0;
  }
}

// per system: y = R^{-1} g over the steps its cycle took
__global__ void k_pbacksolve(const double* __restrict__ H, size_t hstride, int ldh,
                             const double* gv, double* y, int vstride,
                             const int* __restrict__ sys, const int* __restrict__ nsys,
                             const KrylovState* st) {
  const int nq = *nsys;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int s = sys[q];
    backsolve_block(H + s * hstride, ldh, gv + (size_t)s * vstride, y + (size_t)s * vstride,
                    st[s].k);
    __syncthreads();
  }
}

// u = V[0..k) y of the item's system and D^{-1} u
template <int MAXK>
__global__ void __launch_bounds__(kVecThreads)
k_pcombine(int ld, const int4* __restrict__ blk, const int* __restrict__ items,
           const int* __restrict__ nitems, const KrylovState* st,
           const double* __restrict__ V, const double* __restrict__ y, int vstride, double* u,
           const double* __restrict__ dinv, double* rhat64, float* rhat32) {
  __shared__ double ys[MAXK];
  const int nq = *nitems;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int4 b = blk[items[q]];
    const int k = st[b.x].k;
    for (int i = threadIdx.x; i < MAXK; i += blockDim.x)
      ys[i] = i < k ? y[(size_t)b.x * vstride + i] : 0.0;
    __syncthreads();
    combine_rows<MAXK>(b.y + threadIdx.x, b.z, blockDim.x, ld, V, ys, k, u, dinv, rhat64,
                       rhat32);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Concatenate the systems' CSR matrices into the pack's block-diagonal CSR
// (row ranges in parallel).  Columns of system s are checked against its
// own size, so no entry can couple two systems.
void pack_concat(int count, const int64_t* n, const int64_t* const* rowptr,
                 const int32_t* const* col, const double* const* val, std::vector<int64_t>& off,
                 std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va) {
  if (count < 1) GS2_THROW(GS2_ERR_INVALID_ARG, "a pack holds at least one system");
  if (!n || !rowptr || !col || !val) GS2_THROW(GS2_ERR_INVALID_ARG, "NULL array of systems");
  off.assign(count + 1, 0);
  std::vector<int64_t> base(count + 1, 0);
  for (int s = 0; s < count; ++s) {
    const std::string who = "system " + std::to_string(s) + ": ";
    if (n[s] < 0) GS2_THROW(GS2_ERR_INVALID_ARG, who + "negative size");
    if (!rowptr[s]) GS2_THROW(GS2_ERR_INVALID_ARG, who + "NULL rowptr");
    const int64_t* R = rowptr[s];
    if (R[0] != 0) GS2_THROW(GS2_ERR_INVALID_ARG, who + "rowptr[0] must be 0");
    for (int64_t i = 0; i < n[s]; ++i)
      if (R[i + 1] < R[i]) GS2_THROW(GS2_ERR_INVALID_ARG, who + "rowptr is not monotone");
    if (R[n[s]] > 0 && (!col[s] || !val[s]))
      GS2_THROW(GS2_ERR_INVALID_ARG, who + "NULL column or value array");
    off[s + 1] = off[s] + n[s];
    base[s + 1] = base[s] + R[n[s]];
    if (off[s + 1] > std::numeric_limits<int>::max() - 1 ||
        base[s + 1] > std::numeric_limits<int>::max() - 64)
      GS2_THROW(GS2_ERR_INVALID_ARG, "the pack has more than 2^31 - 1 rows or entries");
  }
  const int64_t N = off[count];
  rp.assign(N + 1, 0);
  ci.resize(base[count]);
  va.resize(base[count]);
  rp[N] = base[count];
  std::vector<int64_t> bad(kHostThreads, std::numeric_limits<int64_t>::max());
  parallel_ranges(N, [&](int64_t g0, int64_t g1, int tid) {
    int s = (int)(std::upper_bound(off.begin(), off.end(), g0) - off.begin()) - 1;
    for (int64_t g = g0; g < g1; ++g) {
      while (g >= off[s + 1]) ++s;
      const int64_t i = g - off[s];
      const int64_t a = rowptr[s][i], e = rowptr[s][i + 1];
      const int64_t o = base[s] + a;
      rp[g] = o;
      for (int64_t k = a; k < e; ++k) {
        const int32_t c = col[s][k];
        if (c < 0 || c >= n[s]) bad[tid] = std::min(bad[tid], g);
        ci[o + (k - a)] = (int32_t)(c + off[s]);
        va[o + (k - a)] = val[s][k];
      }
    }
  });
  const int64_t g = *std::min_element(bad.begin(), bad.end());
  if (g != std::numeric_limits<int64_t>::max()) {
    const int s = (int)(std::upper_bound(off.begin(), off.end(), g) - off.begin()) - 1;
    GS2_THROW(GS2_ERR_INVALID_ARG, "system " + std::to_string(s) +
                                       ": column index out of range in row " +
                                       std::to_string(g - off[s]));
  }
}

// (system, row of the system) of a row of the pack
std::pair<int, int64_t> pack_locate(const gs2_handle* h, int64_t g) {
  const auto& off = h->pack->off;
  const int s = (int)(std::upper_bound(off.begin(), off.end(), g) - off.begin()) - 1;
  return {s, g - off[s]};
}

// The block table: every block inside one system, at least 512 rows per
// block and at most 256 blocks per system (at least one per non-empty
// system).  A system's partition depends on its own size only, so its
// reductions, and with them its whole solve, do not depend on the other
// systems of the pack.
void pack_attach(gs2_handle* h, const std::vector<int64_t>& off) {
  Pack* P = new Pack();
  h->pack = P;
  P->count = (int)off.size() - 1;
  P->off = off;
  const int64_t N = off.back();
  std::vector<int4> blk;
  std::vector<int> sb(P->count + 1, 0);
  for (int s = 0; s < P->count; ++s) {
    sb[s] = (int)blk.size();
    const int64_t r0 = off[s], ns = off[s + 1] - off[s];
    const int64_t rpb = std::max<int64_t>(2 * kVecThreads, (ns + 255) / 256);
    const int64_t k = (ns + rpb - 1) / rpb;
    for (int64_t b = 0; b < k; ++b)
      blk.push_back(make_int4(s, (int)(r0 + ns * b / k), (int)(r0 + ns * (b + 1) / k), b == 0));
  }
  sb[P->count] = (int)blk.size();
  P->nb = (int)blk.size();
  P->blk = (int4*)h->dalloc(sizeof(int4) * std::max(1, P->nb));
  P->seg_blk = (int*)h->dalloc(sizeof(int) * (P->count + 1));
  h->h2d(P->blk, blk.data(), sizeof(int4) * P->nb);
  h->h2d(P->seg_blk, sb.data(), sizeof(int) * (P->count + 1));
  P->seg_blk_host = sb;
  P->items = (int*)h->dalloc(sizeof(int) * std::max(1, P->nb));
  P->sys = (int*)h->dalloc(sizeof(int) * P->count);
  P->cnt = (int*)h->dalloc(sizeof(int) * 2);
  P->items_host = (int*)pinned_get(sizeof(int) * std::max(1, P->nb));
  P->sys_host = (int*)pinned_get(sizeof(int) * P->count);
  P->cnt_host = (int*)pinned_get(sizeof(int) * 2);
  P->gb = std::max(1, std::min(P->nb, 4 * h->nsm));
  P->gs = std::max(1, std::min(P->count, 2 * h->nsm));
  P->st = (KrylovState*)h->dalloc(sizeof(KrylovState) * P->count);
  h->dzero(P->st, sizeof(KrylovState) * P->count);
  P->st_host = (KrylovState*)pinned_get(sizeof(KrylovState) * P->count);
  P->active = (int*)h->dalloc(sizeof(int) * P->count);
  P->active_host = (int*)pinned_get(sizeof(int) * P->count);
  P->nactive = (int*)h->dalloc(sizeof(int));
  std::vector<int> off32(off.begin(), off.end());
  P->off_dev = (int*)h->dalloc(sizeof(int) * (P->count + 1));
  h->h2d(P->off_dev, off32.data(), sizeof(int) * (P->count + 1));
  P->nchunks = (int)((N + 31) / 32);
  P->live_cycle = (int*)h->dalloc(sizeof(int) * std::max(1, P->nchunks));
  P->live_run = (int*)h->dalloc(sizeof(int) * std::max(1, P->nchunks));
  GS2_CUDA(cudaStreamSynchronize(h->stream));
}

void pack_free(gs2_handle* h) {
  Pack* P = h->pack;
  if (!P) return;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  pinned_put(P->st_host, sizeof(KrylovState) * P->count);
  pinned_put(P->active_host, sizeof(int) * P->count);
  pinned_put(P->items_host, sizeof(int) * std::max(1, P->nb));
  pinned_put(P->sys_host, sizeof(int) * P->count);
  pinned_put(P->cnt_host, sizeof(int) * 2);
  delete P;
  h->pack = nullptr;
}

void pack_drop_graph(gs2_handle* h) {
  if (!h->pack || !h->pack->gexec) return;
  cudaGraphExecDestroy(h->pack->gexec);
  h->pack->gexec = nullptr;
  h->pack->gkey.clear();
}

int pack_count(const gs2_handle* h) { return h->pack ? h->pack->count : 0; }
const std::vector<int64_t>* pack_offsets(const gs2_handle* h) {
  return h->pack ? &h->pack->off : nullptr;
}

// per-system Hessenberg, rotation and right-hand-side storage for restart m
// (old arrays stay owned by the handle until it is destroyed)
static void ensure_pack_krylov(gs2_handle* h, int m) {
  Pack* P = h->pack;
  if (P->m >= m) return;
  const size_t S = (size_t)P->count;
  P->m = m;
  P->H = (double*)h->dalloc(sizeof(double) * S * P->hstride());
  P->hbuf = (double*)h->dalloc(sizeof(double) * S * P->vstride());
  P->gvec = (double*)h->dalloc(sizeof(double) * S * P->vstride());
  P->cs = (double*)h->dalloc(sizeof(double) * S * P->vstride());
  P->sn = (double*)h->dalloc(sizeof(double) * S * P->vstride());
  P->y = (double*)h->dalloc(sizeof(double) * S * P->vstride());
  P->part = (double*)h->dalloc(sizeof(double) * (size_t)(m + 2) * std::max(1, P->nb));
  h->dzero(P->H, sizeof(double) * S * P->hstride());
}


// ---------------------------------------------------------------------------
// GMRES(m) on a pack
// ---------------------------------------------------------------------------

#define GS2_PJC_CASES(X)                                                                 \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)  \
  X(31) X(32)

struct PackRun {
  gs2_handle* h = nullptr;
  Pack* P = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int m = 0;
  double tol = 0.0;
  int max_iters = 0;
  const gs2_params* pc = nullptr;
  bool wants = false;
  double* r64 = nullptr;
  float* r32 = nullptr;
  std::vector<gs2_solve_info> loc;
  std::vector<char> done;
  std::vector<double> bnorm;
  bool first = true;
  bool finished = false;
  bool cycle_ran = false, graph_ran = false;

  int ldh() const { return P->m + 1; }

  void start(gs2_handle* h_, const double* b_, double* x_, int m_, double tol_, int maxit,
             const gs2_params* p) {
    h = h_; P = h->pack; b = b_; x = x_; m = m_; tol = tol_; max_iters = maxit;
    pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
    loc.assign(P->count, gs2_solve_info{0, 0, GS2_OK, 0.0});
    done.assign(P->count, 0);
    bnorm.assign(P->count, 0.0);
    if (h->n == 0) {
      finished = true;
      return;
    }
    ensure_krylov(h, m);
    ensure_pack_krylov(h, m);
    wants = precond_wants_rhat(pc);
    if (wants) {
      void* rb = precond_rhat_buffer(h, pc);
      if (rb == (void*)h->rhat32 || rb == (void*)h->bhat32) r32 = (float*)rb;
      else r64 = (double*)rb;
    }
    upload_lists();  // every system
    launch_norms(b, 1);
    k_pstate_init<<<(P->count + 255) / 256, 256, 0, h->stream>>>(P->st, P->count, tol, max_iters);
    GS2_LAUNCH_CHECK();
    launch_true_residual();
  }

  // the work lists of the systems not done yet (all of them before the
  // first advance), copied to the device on the handle's stream
  void upload_lists() {
    int ni = 0, ns = 0;
    for (int s = 0; s < P->count; ++s) {
      if (done[s]) continue;
      P->sys_host[ns++] = s;
      for (int e = P->seg_blk_host[s]; e < P->seg_blk_host[s + 1]; ++e) P->items_host[ni++] = e;
    }
    P->cnt_host[0] = ni;
    P->cnt_host[1] = ns;
    if (ni)
      GS2_CUDA(cudaMemcpyAsync(P->items, P->items_host, sizeof(int) * ni,
                               cudaMemcpyHostToDevice, h->stream));
    if (ns)
      GS2_CUDA(cudaMemcpyAsync(P->sys, P->sys_host, sizeof(int) * ns, cudaMemcpyHostToDevice,
                               h->stream));
    GS2_CUDA(cudaMemcpyAsync(P->cnt, P->cnt_host, sizeof(int) * 2, cudaMemcpyHostToDevice,
                             h->stream));
  }

  // per-system ||v|| into st.beta (which = 0) or st.bnorm (which = 1)
  void launch_norms(const double* v, int which) {
    KernelTimer tm(h, "norm", 8.0 * h->n);
    k_pnorm_part<<<P->gb, kVecThreads, 0, h->stream>>>(P->blk, P->items, P->cnt, v, P->part,
                                                       P->nb);
    GS2_LAUNCH_CHECK();
    k_pnorm_final<<<P->gs, 256, 0, h->stream>>>(P->part, P->seg_blk, P->sys, P->cnt + 1, P->st,
                                                which);
    GS2_LAUNCH_CHECK();
  }

  // r = b - A x over the pack, per-system ||r||, and the state copy
  void launch_true_residual() {
    launch_resid(h, b, x, h->r, nullptr, nullptr, nullptr);
    launch_norms(h->r, 0);
    GS2_CUDA(cudaMemcpyAsync(P->st_host, P->st, sizeof(KrylovState) * P->count,
                             cudaMemcpyDeviceToHost, h->stream));
    GS2_CUDA(cudaMemcpyAsync(h->err_host, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
  }

  void finish(int s, gs2_status st) {
    loc[s].status = st;
    done[s] = 1;
  }

  // Called with the stream synchronised: the per-system decisions of
  // krylov.cu's single-system solve, then the next cycle for the systems
  // that continue.
  void advance() {
    if (finished) return;
    const KrylovState* hs = P->st_host;
    if (cycle_ran) {
      int steps = 0;
      for (int s = 0; s < P->count; ++s) steps = std::max(steps, hs[s].k);
      profile_harvest(h, steps, graph_ran);
      cycle_ran = graph_ran = false;
    }
    if (*h->err_host) raise_device_error(h);
    bool any = false;
    for (int s = 0; s < P->count; ++s) {
      if (done[s]) continue;
      if (first) {
        bnorm[s] = hs[s].bnorm;
        if (bnorm[s] == 0.0) {
          const int64_t n0 = P->off[s], ns = P->off[s + 1] - n0;
          if (ns) GS2_CUDA(cudaMemsetAsync(x + n0, 0, sizeof(double) * ns, h->stream));
          loc[s].true_relres = 0.0;
          finish(s, GS2_OK);
          continue;
        }
        if (std::isnan(bnorm[s]) || std::isinf(bnorm[s])) {
          loc[s].true_relres = NAN;
          finish(s, GS2_ERR_NAN);
          continue;
        }
      }
      const double beta = hs[s].beta;
      loc[s].true_relres = beta / bnorm[s];
      loc[s].iters = hs[s].iters;
      if (std::isnan(beta) || std::isinf(beta) || hs[s].status == GS2_ERR_NAN) {
        finish(s, GS2_ERR_NAN);
        continue;
      }
      if (loc[s].true_relres <= tol) {
        finish(s, GS2_OK);
        continue;
      }
      if (hs[s].status == GS2_ERR_BREAKDOWN) {
        finish(s, GS2_ERR_BREAKDOWN);
        continue;
      }
      if (loc[s].iters >= max_iters) {
        finish(s, GS2_ERR_NOT_CONVERGED);
        continue;
      }
      loc[s].cycles++;
      any = true;
    }
    first = false;
    if (!any) {
      finished = true;
      return;
    }
    for (int s = 0; s < P->count; ++s) P->active_host[s] = !done[s];
    upload_lists();
    launch_cycle();
  }

  int launch_dots(int jc) {
    KernelTimer tm(h, "cgs2_dots", 8.0 * h->n * (jc + 1));
    const int N = (int)h->n;
    switch (jc) {
#define GS2_PDOTS_CASE(J)                                                               \
  case J:                                                                               \
    k_pdots<J><<<P->gb, kVecThreads, 0, h->stream>>>(N, P->blk, P->items, P->cnt, P->st, \
                                                     h->V, h->w, P->part, P->nb);       \
    break;
      GS2_PJC_CASES(GS2_PDOTS_CASE)
#undef GS2_PDOTS_CASE
      default:
        k_pdots_rt<64><<<P->gb, kVecThreads, 0, h->stream>>>(N, P->blk, P->items, P->cnt,
                                                             P->st, h->V, jc, h->w, P->part,
                                                             P->nb);
        break;
    }
    GS2_LAUNCH_CHECK();
    return P->nb;
  }

  template <bool NORM>
  void launch_update(int jc) {
    KernelTimer tm(h, NORM ? "cgs2_upd_norm" : "cgs2_upd_dots", 8.0 * h->n * (jc + 2));
    const int N = (int)h->n, hs = (int)P->vstride();
    switch (jc) {
#define GS2_PUPD_CASE(J)                                                                \
  case J:                                                                               \
    k_pupdate<J, NORM><<<P->gb, kVecThreads, 0, h->stream>>>(                           \
        N, P->blk, P->items, P->cnt, P->st, h->V, P->hbuf, hs, h->w, P->part, P->nb);   \
    break;
      GS2_PJC_CASES(GS2_PUPD_CASE)
#undef GS2_PUPD_CASE
      default:
        k_pupdate_rt<64, NORM><<<P->gb, kVecThreads, 0, h->stream>>>(
            N, P->blk, P->items, P->cnt, P->st, h->V, jc, P->hbuf, hs, h->w, P->part, P->nb);
        break;
    }
    GS2_LAUNCH_CHECK();
  }

  void launch_reduce(int j, int jc, int mode) {
    KernelTimer tm(h, "reduce_cols", 8.0 * jc * P->nb);
    k_preduce<<<P->gs, 256, 0, h->stream>>>(P->part, P->nb, P->seg_blk, P->sys, P->cnt + 1,
                                            P->st, P->H, P->hstride(), ldh(), j, P->hbuf,
                                            (int)P->vstride(), mode, jc);
    GS2_LAUNCH_CHECK();
  }

  // the row kernels skip chunks of systems outside `live` while it lives
  struct LiveRows {
    gs2_handle* h;
    LiveRows(gs2_handle* h_, const int* live) : h(h_) { h->row_live = live; }
    ~LiveRows() { h->row_live = nullptr; }
  };

  // Arnoldi step j for every system whose cycle is still running
  void enqueue_step(int j) {
    const int N = (int)h->n;
    const int* skip = &h->st->stop;
    LiveRows lr(h, P->live_run);
    precond_apply(h, pc, h->V + (size_t)j * N, h->z, wants, skip);
    launch_spmv(h, h->z, h->w, skip);
    const int jc = j + 1;
    launch_dots(jc);
    launch_reduce(j, jc, 0);
    launch_update<false>(jc);
    launch_reduce(j, jc, 1);
    launch_update<true>(jc);
    {
      KernelTimer tm(h, "givens", 8.0 * P->nb + 8.0 * 4 * (j + 2) * P->count);
      k_pgivens<<<P->gs, 128, 0, h->stream>>>(P->part, P->seg_blk, P->sys, P->cnt + 1, P->st,
                                              P->H, P->hstride(), ldh(), j, P->cs, P->sn,
                                              P->gvec, (int)P->vstride(), P->nactive,
                                              P->off_dev, P->live_run, h->st,
                                              h->stop_mapped_dev);
      GS2_LAUNCH_CHECK();
    }
    if (j + 1 < m) {
      KernelTimer tm(h, "scale_next",
                     16.0 * N + (r64 ? 16.0 * N : 0.0) + (r32 ? 12.0 * N : 0.0));
      k_pscale_next<<<P->gb, kVecThreads, 0, h->stream>>>(P->blk, P->items, P->cnt, P->st,
                                                          h->w, h->V + (size_t)(j + 1) * N,
                                                          h->dinv, r64, r32);
      GS2_LAUNCH_CHECK();
    }
  }

  bool use_graph() const { return h->graph_mode != 2; }

  void ensure_graph() {
    std::vector<double> key = {(double)m, (double)(uintptr_t)h->V, (double)(uintptr_t)r64,
                               (double)(uintptr_t)r32, (double)(uintptr_t)P->part,
                               (double)(uintptr_t)P->H, (double)profile_epoch(h)};
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
    if (P->gexec && P->gkey == key) return;
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
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
    P->g_launches = gs2_launch_count() - c0;
    add_launches(-P->g_launches);  // captured, not run
    cudaError_t e = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    GS2_CUDA(e);
    P->gkey = key;
  }

  void launch_cycle() {
    *h->stop_mapped = 0;
    GS2_CUDA(cudaMemcpyAsync(P->active, P->active_host, sizeof(int) * P->count,
                             cudaMemcpyHostToDevice, h->stream));
    k_pcycle_reset<<<1, 1024, 0, h->stream>>>(P->st, P->active, P->count, P->nactive, h->st);
    GS2_LAUNCH_CHECK();
    k_plive_init<<<(P->nchunks + 255) / 256, 256, 0, h->stream>>>(
        P->nchunks, (int)h->n, P->off_dev, P->count, P->active, P->live_cycle, P->live_run);
    GS2_LAUNCH_CHECK();
    k_pcycle_start<<<P->gb, kVecThreads, 0, h->stream>>>(P->blk, P->items, P->cnt, P->st, h->r,
                                                         h->V, h->dinv, r64, r32, P->gvec,
                                                         (int)P->vstride(), m);
    GS2_LAUNCH_CHECK();
    cycle_ran = true;
    if (use_graph()) {
      ensure_graph();
      GS2_CUDA(cudaEventRecord(h->gev_in, h->stream));
      GS2_CUDA(cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
      GS2_CUDA(cudaGraphLaunch(P->gexec, h->gstream));
      GS2_CUDA(cudaEventRecord(h->gev_out, h->gstream));
      GS2_CUDA(cudaStreamWaitEvent(h->stream, h->gev_out, 0));
      add_launches(P->g_launches);
      graph_ran = true;
    } else {
      for (int j = 0; j < m; ++j) {
        if (*h->stop_mapped) break;  // every system has ended the cycle
        profile_capture_step(h, j);
        enqueue_step(j);
      }
      profile_capture_step(h, -1);
    }
    // x += M^{-1} V y per system (u = 0 for systems without a step)
    k_pbacksolve<<<P->gs, 64, 0, h->stream>>>(P->H, P->hstride(), ldh(), P->gvec, P->y,
                                              (int)P->vstride(), P->sys, P->cnt + 1, P->st);
    GS2_LAUNCH_CHECK();
    {
      KernelTimer tm(h, "combine", 8.0 * h->n * (m + 1));
      const int N = (int)h->n;
      const int vs = (int)P->vstride();
#define GS2_PCOMBINE(M)                                                                  \
  k_pcombine<M><<<P->gb, kVecThreads, 0, h->stream>>>(N, P->blk, P->items, P->cnt, P->st, \
                                                      h->V, P->y, vs, h->w, h->dinv, r64,  \
                                                      r32)
      if (m <= 8) GS2_PCOMBINE(8);
      else if (m <= 16) GS2_PCOMBINE(16);
      else if (m <= 32) GS2_PCOMBINE(32);
      else GS2_PCOMBINE(64);
#undef GS2_PCOMBINE
      GS2_LAUNCH_CHECK();
    }
    {
      // systems that took no part in the cycle keep their x and skip the rows
      LiveRows lr(h, P->live_cycle);
      precond_apply(h, pc, h->w, h->z, wants, nullptr);
      k_paxpy<<<P->gb, kVecThreads, 0, h->stream>>>(P->blk, P->items, P->cnt, x, h->z);
      GS2_LAUNCH_CHECK();
      launch_true_residual();
    }
  }
};

// A pack solve as a resumable job (the server's packs of small requests):
// start enqueues the first work on the handle's stream; advance is called
// only when that stream is idle and returns true once every system is done.
struct PackJob {
  gs2_params params{};
  bool has_params = false;
  PackRun run;
};

PackJob* pack_job_start(gs2_handle* h, const double* b, double* x, int m, double tol,
                        int max_iters, const gs2_params* p) {
  PackJob* j = new PackJob();
  if (p) {
    j->params = *p;
    j->has_params = true;
  }
  try {
    j->run.start(h, b, x, m, tol, max_iters, j->has_params ? &j->params : nullptr);
  } catch (...) {
    delete j;
    throw;
  }
  return j;
}

void pack_job_prepare(PackJob* j) {
  if (!j->run.finished && j->run.use_graph()) j->run.ensure_graph();
}

bool pack_job_advance(PackJob* j) {
  if (!j->run.finished) j->run.advance();
  return j->run.finished;
}

gs2_solve_info pack_job_info(const PackJob* j, int s) { return j->run.loc[s]; }

void pack_job_free(PackJob* j) { delete j; }

gs2_status pack_gmres_run(gs2_handle* h, const double* b, double* x, int m, double tol,
                          int max_iters, const gs2_params* p, gs2_solve_info* infos) {
  // one cluster per system (cluster.cu): graph mode 4, or automatically for
  // packs small enough (pack_persistent_eligible) whose systems fit a
  // cluster; else every system in one cooperative launch (persist.cu):
  // graph mode 3, or automatically for packs small enough
  if (h->graph_mode == 4) return pack_gmres_cluster(h, b, x, m, tol, max_iters, p, infos);
  if (h->graph_mode == 0 && !profiling_active(h) && pack_persistent_eligible(h, m, p, true)) {
    if (pack_cluster_eligible(h, m, p))
      return pack_gmres_cluster(h, b, x, m, tol, max_iters, p, infos);
    return pack_gmres_persistent(h, b, x, m, tol, max_iters, p, infos);
  }
  if (h->graph_mode == 3) {
    if (!pack_persistent_eligible(h, m, p, false))
      GS2_THROW(GS2_ERR_INVALID_ARG,
                "one launch: systems of at most 65,536 rows, restart <= 32, no, JR or FP64 "
                "non-compact GS2 preconditioning, and every system a co-resident block");
    return pack_gmres_persistent(h, b, x, m, tol, max_iters, p, infos);
  }
  PackRun r;
  r.start(h, b, x, m, tol, max_iters, p);
  while (!r.finished) {
    GS2_CUDA(cudaStreamSynchronize(h->stream));
    r.advance();
  }
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  gs2_status first_bad = GS2_OK;
  for (int s = 0; s < h->pack->count; ++s) {
    if (infos) infos[s] = r.loc[s];
    if (r.loc[s].status != GS2_OK && first_bad == GS2_OK) first_bad = (gs2_status)r.loc[s].status;
  }
  return first_bad;
}

}  // namespace gs2
