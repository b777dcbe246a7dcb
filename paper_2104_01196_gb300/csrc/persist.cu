// Restarted GMRES(m) for small systems as one cooperative launch.
//
// A small system (a few thousand rows) runs the multi-kernel solve at the
// launch rate: each of the ~11 kernels of an Arnoldi step costs a few
// microseconds of launch and drain however little work it holds.  Here the
// whole solve -- every restart cycle, the GS2 or JR preconditioner, the CGS2
// Arnoldi steps, the Givens rotations and the true-residual checks -- runs in
// one launch of at most 64 co-resident blocks (cooperative launch).  Rows are
// owned by threads for the whole solve, so a phase that only touches its own
// rows needs no synchronisation; a phase that gathers other rows' values
// waits at a grid barrier first.  Inner products are block partial sums
// followed by a barrier, after which every block sums all partials in the
// same fixed order, so every block holds bitwise the same scalars: the
// Hessenberg matrix, the rotations and the stopping decisions are computed
// by every block in its own shared memory, and control flow is uniform over
// the grid.  The barrier is one arrival counter in device memory that only
// grows: a block adds one with release semantics and polls it with acquire
// loads until it reaches the count the barrier completes at (1.3 us on a
// GB300, against 2.3 us for a counter that the last arrival resets and a
// generation word, which take two more dependent atomics and fences), spun
// with a bound: a block that waits too long records GS2_ERR_TIMEOUT and
// every block leaves at its next barrier.
#include <algorithm>
#include <cmath>

#include "arnoldi.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace gs2 {

// Small blocks spread the rows over many SMs: one SM issues only 2 FP64
// FMAs per clock, so rows per SM, not threads, set the time of a phase.
constexpr int kPerThreads = 128;
constexpr int kPerMaxBlocks = 128;
constexpr long long kBarrierCycles = 4LL << 30;  // ~2 s at 2.07 GHz
constexpr int64_t kPersistMaxRows = 1 << 16;
// chosen automatically up to this size: measured on the 2D Laplacian with
// GS2(1,1), GMRES(30): 4,096 rows 10.1 ms one launch vs 15.3 ms replayed
// graphs, 16,384 rows 25.7 vs 27.9 ms, 62,500 rows 82 vs 76 ms
constexpr int64_t kPersistAutoRows = 1 << 14;

struct PersistArgs {
  int n;
  const int* Arp;
  const int* Aci;
  const double* Ava;
  const int* Lrp;  // D^{-1} L
  const int* Lci;
  const double* Lva;
  const int* Urp;  // D^{-1} U
  const int* Uci;
  const double* Uva;
  const double* dinv;
  const double* b;
  double* x;
  double* V;
  double *w, *z, *r, *rh, *g0, *g1;
  double* part;  // partial sums, value v of block k at part[v * nb + k]
  int m;
  double tol;
  int max_iters;
  int kind;  // GS2_PC_NONE, GS2_PC_GS2 or GS2_PC_JR
  int outer, inner, dir;
  double omega, gamma;
  unsigned* bar;  // {arrivals, generation}
  int* err;       // device error word
  KrylovState* out;
  // the system's rows [r0, r1) of vectors of length N (a pack: one of its
  // systems; a single system: r0 = 0, r1 = N = n), and its blocks
  // [first_block, first_block + nblocks) of the launch; lb / nb: this
  // block's index among them and their number (set in the kernel)
  int r0, r1, N;
  int first_block, nblocks;
  int lb, nb;
};

// the arrival count this block's next grid barrier completes at
__shared__ unsigned s_bar_target;

// A block's arguments in shared memory: the kernel parameter (one system)
// or its system's entry of the table `sys` (a pack), with the block's index
// among its system's blocks.
__device__ __forceinline__ const PersistArgs& block_args(const PersistArgs& a0,
                                                         const PersistArgs* sys,
                                                         const int* bsys) {
  __shared__ PersistArgs sa;
  if (threadIdx.x == 0) {
    sa = sys ? sys[bsys[blockIdx.x]] : a0;
    sa.lb = blockIdx.x - sa.first_block;
    sa.nb = sa.nblocks;
    s_bar_target = 0;
  }
  __syncthreads();
  return sa;
}

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid barrier (all blocks co-resident by the cooperative launch): the
// k-th barrier completes when the counter reaches k * nb (compared as a
// signed difference, so the counter may wrap); false when this block gave
// up waiting or another block had given up before.  The block barrier
// orders the block's writes before its release add; the acquire load that
// sees the full count orders every block's writes before this block's
// reads after the barrier.
__device__ bool grid_sync(const PersistArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned target = s_bar_target + (unsigned)a.nb;
    s_bar_target = target;
    red_add_release(a.bar, 1u);
    // tight spin (a sleep between polls delays the wake-up by more than
    // the barrier itself costs), bounded by the clock
    const long long t0 = clock64();
    while ((int)(ld_acquire(a.bar) - target) < 0) {
      if (clock64() - t0 > kBarrierCycles || *(volatile int*)a.err) {
        atomicCAS(a.err, 0, (int)GS2_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// rows owned by this thread
#define FOR_ROWS(i)                                                   \
  for (int i = a.r0 + a.lb * (int)blockDim.x + (int)threadIdx.x; i < a.r1; \
       i += a.nb * (int)blockDim.x)

// The block partials of cnt consecutive values (value q at part[(slot + q)
// nb + block]) summed into out[0..cnt) (shared memory) in the same order by
// every block: warp w takes values w, w + 4, ...; lane l sums partials l,
// l + 32, ...; then a butterfly, lane 0's total.  All lanes load at once,
// where one thread summing the partials of a value in block order waited on
// its loads a few at a time (the one-launch CG solve of the 64^2 system,
// five single-value sums an iteration: 2.38 -> 2.21 ms).
__device__ void sum_partials(const PersistArgs& a, int slot, int cnt, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwp = blockDim.x >> 5;
  for (int q = w; q < cnt; q += nwp) {
    const double* p = a.part + (size_t)(slot + q) * a.nb;
    double s = 0.0;
    for (int b = lane; b < a.nb; b += 32) s += p[b];
    s = warp_sum(s);
    if (lane == 0) out[q] = s;
  }
  __syncthreads();
}

// sum over the grid of one value per thread: block partial at `slot`, a
// barrier, then every block sums the partials (sum_partials)
__device__ bool grid_sum1(const PersistArgs& a, double v, int slot, double* out) {
  __shared__ double red[kPerThreads / 32];
  __shared__ double tot;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kPerThreads / 32; ++q) s += red[q];
    a.part[(size_t)slot * a.nb + a.lb] = s;
  }
  if (!grid_sync(a)) return false;
  sum_partials(a, slot, 1, &tot);
  *out = tot;
  return true;
}

// Block sums of nv <= NV per-thread values to part[v * nb + block]
template <int NV>
__device__ __forceinline__ void block_partials_p(const double (&acc)[NV], int nv, double* part,
                                                 int nb, int lb) {
  __shared__ double red[kPerThreads / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < nv) {
      const double s = warp_sum(acc[v]);
      if (lane == 0) red[wid][v] = s;
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kPerThreads / 32; ++q) s += red[q][v];
    part[(size_t)v * nb + lb] = s;
  }
}

// y_i = sum_k M_ik u_k for a CSR row
__device__ __forceinline__ double row_dot(const int* rp, const int* ci, const double* va, int i,
                                          const double* u) {
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s = fma(va[k], u[ci[k]], s);
  return s;
}

// value slots of the partial-sum buffer
constexpr int kSlotDots1 = 0, kSlotDots2 = 32, kSlotNorm = 64, kSlotB = 65, kSlotR = 66,
              kSlotFinal = 67;
constexpr int kPerSlots = 68;

// CGS2 phases over the thread's rows, for jc <= JB basis vectors (JB a
// multiple of 8, so at most 7 predicated-off products per row and vector)
// w = A z and part = V^T w
template <int JB>
__device__ void phase_spmv_dots(const PersistArgs& a, int jc, double* part) {
  double acc[JB];
#pragma unroll
  for (int q = 0; q < JB; ++q) acc[q] = 0.0;
  FOR_ROWS(i) {
    const double wi = row_dot(a.Arp, a.Aci, a.Ava, i, a.z);
    a.w[i] = wi;
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) acc[q] = fma(a.V[(size_t)q * a.N + i], wi, acc[q]);
  }
  block_partials_p<JB>(acc, jc, part, a.nb, a.lb);
}

// w -= V h and part = V^T w
template <int JB>
__device__ void phase_update_dots(const PersistArgs& a, int jc, const double* h, double* part) {
  double acc[JB];
#pragma unroll
  for (int q = 0; q < JB; ++q) acc[q] = 0.0;
  FOR_ROWS(i) {
    double wn = a.w[i];
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) wn = fma(a.V[(size_t)q * a.N + i], -h[q], wn);
    a.w[i] = wn;
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) acc[q] = fma(a.V[(size_t)q * a.N + i], wn, acc[q]);
  }
  block_partials_p<JB>(acc, jc, part, a.nb, a.lb);
}

// w -= V h; returns this thread's sum of w_i^2
template <int JB>
__device__ double phase_update_norm(const PersistArgs& a, int jc, const double* h) {
  double t = 0.0;
  FOR_ROWS(i) {
    double wn = a.w[i];
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) wn = fma(a.V[(size_t)q * a.N + i], -h[q], wn);
    a.w[i] = wn;
    t = fma(wn, wn, t);
  }
  return t;
}

#define PHASE_JB(jc, CALL8, CALL16, CALL24, CALL32) \
  switch (((jc) + 7) >> 3) {                        \
    case 1: CALL8; break;                           \
    case 2: CALL16; break;                          \
    case 3: CALL24; break;                          \
    default: CALL32; break;                         \
  }

// z = M^{-1} v from z = 0: GS2 half sweeps (Eq. (2)-(5), damped) or JR
// sweeps, the arithmetic of the multi-kernel path row for row.  v complete
// on entry; z complete on a true return.
__device__ bool precond(const PersistArgs& a, const double* v, double* z) {
  if (a.kind == GS2_PC_NONE) {
    FOR_ROWS(i) z[i] = v[i];
    return grid_sync(a);
  }
  FOR_ROWS(i) a.rh[i] = a.dinv[i] * v[i];
  if (a.kind == GS2_PC_JR) {
    // first sweep from zero: z = omega D^{-1} v; then z + omega D^{-1} (v - A z)
    double* cur = z;
    double* nxt = a.g0;
    FOR_ROWS(i) cur[i] = a.omega * a.rh[i];
    for (int s = 1; s < a.outer; ++s) {
      if (!grid_sync(a)) return false;
      FOR_ROWS(i) {
        const double t = row_dot(a.Arp, a.Aci, a.Ava, i, cur);
        nxt[i] = cur[i] + a.omega * (a.dinv[i] * (v[i] - t));
      }
      double* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (cur != z) {
      // every block must be done gathering from z before it is overwritten
      if (!grid_sync(a)) return false;
      FOR_ROWS(i) z[i] = cur[i];
    }
    return grid_sync(a);
  }
  const bool damped = a.gamma != 1.0;
  bool zero = true;
  for (int s = 0; s < a.outer; ++s) {
    for (int half = 0; half < 2; ++half) {
      const bool fwd = half == 0;
      if (fwd && a.dir == GS2_BACKWARD) continue;
      if (!fwd && a.dir == GS2_FORWARD) continue;
      const int* Tp = fwd ? a.Lrp : a.Urp;
      const int* Tc = fwd ? a.Lci : a.Uci;
      const double* Tv = fwd ? a.Lva : a.Uva;
      if (!zero) {
        if (!grid_sync(a)) return false;  // z complete
        FOR_ROWS(i) a.rh[i] = a.dinv[i] * (v[i] - row_dot(a.Arp, a.Aci, a.Ava, i, z));
      }
      if (!grid_sync(a)) return false;  // rh complete
      if (a.inner == 0) {
        FOR_ROWS(i) z[i] = zero ? a.omega * a.rh[i] : z[i] + a.omega * a.rh[i];
      }
      const double* gin = a.rh;
      for (int k = 0; k < a.inner; ++k) {
        const bool last = k == a.inner - 1;
        double* gout = (k % 2 == 0) ? a.g0 : a.g1;
        FOR_ROWS(i) {
          const double t = row_dot(Tp, Tc, Tv, i, gin);
          double go = a.rh[i] - a.omega * t;
          if (damped) go = (1.0 - a.gamma) * gin[i] + a.gamma * go;
          if (!last) gout[i] = go;
          else z[i] = zero ? a.omega * go : z[i] + a.omega * go;
        }
        if (!last) {
          if (!grid_sync(a)) return false;
          gin = gout;
        }
      }
      zero = false;
    }
  }
  return grid_sync(a);
}

template <int MAXK>
__global__ void __launch_bounds__(kPerThreads, 4)
k_gmres_persistent(PersistArgs a0, const PersistArgs* sys, const int* bsys) {
  const PersistArgs& a = block_args(a0, sys, bsys);
  // Krylov scalars, identical in every block
  __shared__ double Hs[(MAXK + 1) * MAXK];  // column j at Hs[j * (m + 1)]
  __shared__ double cs_s[MAXK + 1], sn_s[MAXK + 1], g_s[MAXK + 1], y_s[MAXK + 1];
  __shared__ double h1[MAXK], h2[MAXK];
  __shared__ int sh_flag;
  const int n = a.N, m = a.m, ldh = m + 1;
  const int nb = a.nb;
  double* part = a.part;
  int iters = 0, cycles = 0, status = GS2_OK;
  double bnorm = 0.0, beta = 0.0;

  // ||b||
  double t = 0.0;
  FOR_ROWS(i) t = fma(a.b[i], a.b[i], t);
  if (!grid_sum1(a, t, kSlotB, &t)) return;
  bnorm = sqrt(t);
  if (bnorm == 0.0 || isnan(bnorm) || isinf(bnorm)) {
    if (bnorm == 0.0) FOR_ROWS(i) a.x[i] = 0.0;
    else status = GS2_ERR_NAN;
    if (a.lb == 0 && threadIdx.x == 0) {
      a.out->iters = 0;
      a.out->cycles = 0;
      a.out->status = status;
      a.out->bnorm = bnorm;
      a.out->beta = bnorm == 0.0 ? 0.0 : NAN;
    }
    return;
  }
  const double tol_abs = a.tol * bnorm;
  bool breakdown = false;
  for (;;) {
    // true residual r = b - A x and its norm (x complete here)
    t = 0.0;
    FOR_ROWS(i) {
      const double ri = a.b[i] - row_dot(a.Arp, a.Aci, a.Ava, i, a.x);
      a.r[i] = ri;
      t = fma(ri, ri, t);
    }
    if (!grid_sum1(a, t, kSlotR, &t)) return;
    beta = sqrt(t);
    const double relres = beta / bnorm;
    if (isnan(beta) || isinf(beta) || status == GS2_ERR_NAN) {
      status = GS2_ERR_NAN;
      break;
    }
    if (relres <= a.tol) {
      status = GS2_OK;
      break;
    }
    if (breakdown) {
      status = GS2_ERR_BREAKDOWN;
      break;
    }
    if (iters >= a.max_iters) {
      status = GS2_ERR_NOT_CONVERGED;
      break;
    }
    ++cycles;
    // cycle start: v_0 = r / beta, g = (beta, 0, ...)
    const double ib = 1.0 / beta;
    FOR_ROWS(i) a.V[i] = a.r[i] * ib;
    if (threadIdx.x <= m) g_s[threadIdx.x] = threadIdx.x == 0 ? beta : 0.0;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      const double* vj = a.V + (size_t)j * n;
      if (!precond(a, vj, a.z)) return;
      const int jc = j + 1;
      // w = A z and the first Gram-Schmidt pass V^T w
      double* p1 = part + (size_t)kSlotDots1 * nb;
      PHASE_JB(jc, phase_spmv_dots<8>(a, jc, p1), phase_spmv_dots<16>(a, jc, p1),
               phase_spmv_dots<24>(a, jc, p1), phase_spmv_dots<32>(a, jc, p1));
      if (!grid_sync(a)) return;
      // (thread q sums value q's partials in block order: for many values
      // this beats sum_partials' warp per value, 10.2 vs 10.7 ms on the 64^2
      // solve)
      if (threadIdx.x < jc) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(size_t)(kSlotDots1 + threadIdx.x) * nb + b];
        h1[threadIdx.x] = s;
      }
      __syncthreads();
      // w -= V h1 and the second pass V^T w
      double* p2 = part + (size_t)kSlotDots2 * nb;
      PHASE_JB(jc, phase_update_dots<8>(a, jc, h1, p2), phase_update_dots<16>(a, jc, h1, p2),
               phase_update_dots<24>(a, jc, h1, p2), phase_update_dots<32>(a, jc, h1, p2));
      if (!grid_sync(a)) return;
      if (threadIdx.x < jc) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(size_t)(kSlotDots2 + threadIdx.x) * nb + b];
        h2[threadIdx.x] = s;
      }
      __syncthreads();
      // w -= V h2 and ||w||^2
      PHASE_JB(jc, t = phase_update_norm<8>(a, jc, h2), t = phase_update_norm<16>(a, jc, h2),
               t = phase_update_norm<24>(a, jc, h2), t = phase_update_norm<32>(a, jc, h2));
      if (!grid_sum1(a, t, kSlotNorm, &t)) return;
      // Givens step j (every block, thread 0, on its own copies)
      if (threadIdx.x == 0) {
        double* col = Hs + (size_t)j * ldh;
        for (int q = 0; q < jc; ++q) col[q] = h1[q] + h2[q];
        const double hn = sqrt(t);
        col[j + 1] = hn;
        const double est = givens_column(col, cs_s, sn_s, g_s, j);
        int stop = 0;
        if (isnan(est) || isnan(hn) || isinf(hn)) {
          status = GS2_ERR_NAN;
          stop = 1;
        } else if (hn == 0.0) {
          breakdown = true;
          stop = 1;
        } else if (est <= tol_abs || iters + 1 >= a.max_iters) {
          stop = 1;
        }
        sh_flag = stop | (status == GS2_ERR_NAN ? 2 : 0) | (breakdown ? 4 : 0);
        y_s[0] = 1.0 / hn;  // scratch: H(j+1, j)^{-1}
      }
      __syncthreads();
      ++iters;
      k = jc;
      const int fl = sh_flag;
      if (fl & 2) status = GS2_ERR_NAN;
      if (fl & 4) breakdown = true;
      if (fl & 1) break;
      if (j + 1 < m) {
        const double ih = y_s[0];
        double* vn = a.V + (size_t)(j + 1) * n;
        FOR_ROWS(i) vn[i] = a.w[i] * ih;
      }
    }
    // x += M^{-1} V y, y = R^{-1} g over the k steps
    if (threadIdx.x == 0) {
      for (int q = 0; q < k; ++q) y_s[q] = g_s[q];
      for (int q = k - 1; q >= 0; --q) {
        const double* cq = Hs + (size_t)q * ldh;
        const double yq = y_s[q] / cq[q];
        y_s[q] = yq;
        for (int l = 0; l < q; ++l) y_s[l] -= cq[l] * yq;
      }
    }
    __syncthreads();
    FOR_ROWS(i) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = fma(a.V[(size_t)q * n + i], y_s[q], s);
      a.w[i] = s;
    }
    if (!precond(a, a.w, a.z)) return;
    FOR_ROWS(i) a.x[i] = a.x[i] + a.z[i];
    if (!grid_sync(a)) return;
  }
  if (a.lb == 0 && threadIdx.x == 0) {
    a.out->iters = iters;
    a.out->cycles = cycles;
    a.out->status = status;
    a.out->bnorm = bnorm;
    a.out->beta = beta;
  }
}


// Preconditioned CG of a small SPD system in one launch: the iteration of
// krylov.cu's cg_run (restart of the search direction when the recursive
// residual has converged but the true residual disagrees), every scalar
// summed identically by every block.
__global__ void __launch_bounds__(kPerThreads, 4)
k_cg_persistent(PersistArgs a0) {
  const PersistArgs& a = block_args(a0, nullptr, nullptr);
  double* p = a.w;           // search direction
  double* q = a.V;           // A p (first basis vector slot)
  double* t = a.V + a.N;     // true-residual scratch
  int iters = 0, cycles = 0, status = GS2_OK;
  double s = 0.0;
  FOR_ROWS(i) s = fma(a.b[i], a.b[i], s);
  if (!grid_sum1(a, s, kSlotB, &s)) return;
  const double bnorm = sqrt(s);
  double beta = 0.0;
  if (bnorm == 0.0 || isnan(bnorm) || isinf(bnorm)) {
    if (bnorm == 0.0) FOR_ROWS(i) a.x[i] = 0.0;
    if (a.lb == 0 && threadIdx.x == 0) {
      a.out->iters = 0;
      a.out->cycles = 0;
      a.out->status = bnorm == 0.0 ? GS2_OK : GS2_ERR_NAN;
      a.out->bnorm = bnorm;
      a.out->beta = bnorm == 0.0 ? 0.0 : NAN;
    }
    return;
  }
  const double tol_abs = a.tol * bnorm;
  FOR_ROWS(i) a.r[i] = a.b[i] - row_dot(a.Arp, a.Aci, a.Ava, i, a.x);
  for (;;) {
    // ||r|| of the recursive residual; confirmed on the true one
    s = 0.0;
    FOR_ROWS(i) s = fma(a.r[i], a.r[i], s);
    if (!grid_sum1(a, s, kSlotR, &s)) return;
    double rn = sqrt(s);
    beta = rn;
    if (isnan(rn) || isinf(rn)) {
      status = GS2_ERR_NAN;
      break;
    }
    if (rn <= tol_abs) {
      s = 0.0;
      FOR_ROWS(i) {
        const double ti = a.b[i] - row_dot(a.Arp, a.Aci, a.Ava, i, a.x);
        t[i] = ti;
        s = fma(ti, ti, s);
      }
      if (!grid_sum1(a, s, kSlotNorm, &s)) return;
      beta = sqrt(s);
      if (beta <= tol_abs) break;
      FOR_ROWS(i) a.r[i] = t[i];
    }
    if (iters >= a.max_iters) {
      status = GS2_ERR_NOT_CONVERGED;
      break;
    }
    ++cycles;
    // z = M^{-1} r, p = z, rz = r.z
    if (!precond(a, a.r, a.z)) return;
    s = 0.0;
    FOR_ROWS(i) {
      p[i] = a.z[i];
      s = fma(a.r[i], a.z[i], s);
    }
    double rz;
    if (!grid_sum1(a, s, kSlotDots1, &rz)) return;
    bool stop = false;
    while (!stop) {
      // q = A p (p complete: the last sum's barrier) and p.q
      s = 0.0;
      FOR_ROWS(i) {
        const double qi = row_dot(a.Arp, a.Aci, a.Ava, i, p);
        q[i] = qi;
        s = fma(p[i], qi, s);
      }
      double pq;
      if (!grid_sum1(a, s, kSlotDots2, &pq)) return;
      if (pq == 0.0) {
        status = GS2_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rz / pq;
      s = 0.0;
      FOR_ROWS(i) {
        a.x[i] = fma(alpha, p[i], a.x[i]);
        const double ri = fma(-alpha, q[i], a.r[i]);
        a.r[i] = ri;
        s = fma(ri, ri, s);
      }
      if (!grid_sum1(a, s, kSlotNorm, &s)) return;
      ++iters;
      const double rr = sqrt(s);
      if (isnan(rr) || isinf(rr)) {
        status = GS2_ERR_NAN;
        break;
      }
      if (rr <= tol_abs || iters >= a.max_iters) break;
      // z = M^{-1} r, beta = r.z / rz, p = z + beta p
      if (!precond(a, a.r, a.z)) return;
      s = 0.0;
      FOR_ROWS(i) s = fma(a.r[i], a.z[i], s);
      double rz_new;
      if (!grid_sum1(a, s, kSlotDots1 + 1, &rz_new)) return;
      const double bt = rz_new / rz;
      rz = rz_new;
      FOR_ROWS(i) p[i] = fma(bt, p[i], a.z[i]);
      if (!grid_sync(a)) return;
    }
    if (status == GS2_ERR_NAN || status == GS2_ERR_BREAKDOWN) break;
  }
  // the true residual at exit
  s = 0.0;
  FOR_ROWS(i) {
    const double ti = a.b[i] - row_dot(a.Arp, a.Aci, a.Ava, i, a.x);
    s = fma(ti, ti, s);
  }
  if (!grid_sum1(a, s, kSlotFinal, &s)) return;
  if (a.lb == 0 && threadIdx.x == 0) {
    a.out->iters = iters;
    a.out->cycles = cycles;
    a.out->status = status;
    a.out->bnorm = bnorm;
    a.out->beta = sqrt(s);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

bool persistent_eligible(const gs2_handle* h, int m, const gs2_params* p, bool automatic) {
  if (h->n == 0 || h->n > (automatic ? kPersistAutoRows : kPersistMaxRows) || m > 32)
    return false;
  if (!p || p->kind == GS2_PC_NONE) return true;
  if (p->parts > 1 || p->local_sweeps > 1) return false;
  if (p->kind == GS2_PC_JR) return true;
  return p->kind == GS2_PC_GS2 && p->precision == GS2_FP64 && p->form == GS2_NONCOMPACT;
}

template <int MAXK>
static void launch_persistent(gs2_handle* h, PersistArgs& a, int nb,
                              const PersistArgs* sys = nullptr, const int* bsys = nullptr) {
  void* args[] = {&a, &sys, &bsys};
  GS2_CUDA(cudaLaunchCooperativeKernel((const void*)k_gmres_persistent<MAXK>, nb, kPerThreads,
                                       args, 0, h->stream));
  GS2_LAUNCH_CHECK();
}

gs2_status gmres_persistent(gs2_handle* h, const double* b, double* x, int m, double tol,
                            int max_iters, const gs2_params* p, gs2_solve_info* info) {
  ensure_krylov(h, m);
  if (!h->persist_bar) {
    h->persist_bar = (unsigned*)h->dalloc(4 * sizeof(unsigned));
    // its own partial-sum buffer: kPerSlots values per block, for the most
    // blocks a launch can have (the handle's buffer is sized for the
    // multi-kernel path's grids, which a small system keeps small)
    h->persist_part = (double*)h->dalloc(sizeof(double) * kPerSlots * kPerMaxBlocks);
  }
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  const int n = (int)h->n;
  // blocks: one row per thread up to 128 blocks, at most what stays resident
  int nb = (int)std::min<int64_t>(kPerMaxBlocks, (h->n + kPerThreads - 1) / kPerThreads);
  {
    int per_sm = 0;
    const void* fn = m <= 8 ? (const void*)k_gmres_persistent<8>
                            : (m <= 16 ? (const void*)k_gmres_persistent<16>
                                       : (const void*)k_gmres_persistent<32>);
    GS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPerThreads, 0));
    nb = std::max(1, std::min(nb, per_sm * h->nsm));
  }
  PersistArgs a{};
  a.n = n;
  a.Arp = h->A.rp;
  a.Aci = h->A.ci;
  a.Ava = h->A.va;
  a.Lrp = h->L.rp;
  a.Lci = h->L.ci;
  a.Lva = h->L.va;
  a.Urp = h->U.rp;
  a.Uci = h->U.ci;
  a.Uva = h->U.va;
  a.dinv = h->dinv;
  a.b = b;
  a.x = x;
  a.V = h->V;
  a.w = h->w;
  a.z = h->z;
  a.r = h->r;
  a.rh = h->rhat;
  a.g0 = h->g0;
  a.g1 = h->g1;
  a.part = h->persist_part;
  if (nb > kPerMaxBlocks) GS2_THROW(GS2_ERR_CUDA, "one-launch grid above its partial-sum buffer");
  a.m = m;
  a.tol = tol;
  a.max_iters = max_iters;
  a.kind = pc ? pc->kind : GS2_PC_NONE;
  a.outer = pc ? std::max(1, pc->outer) : 1;
  a.inner = pc ? pc->inner : 0;
  a.dir = pc ? pc->direction : GS2_FORWARD;
  a.omega = pc ? pc->omega : 1.0;
  a.gamma = pc ? pc->gamma : 1.0;
  a.bar = h->persist_bar;
  a.err = h->dev_err;
  a.out = h->st;
  a.r0 = 0;
  a.r1 = a.N = n;
  a.first_block = 0;
  a.nblocks = nb;
  GS2_CUDA(cudaMemsetAsync(h->persist_bar, 0, 4 * sizeof(unsigned), h->stream));
  if (h->stall_barrier) {
    // test hook: a counter 2^30 arrivals short of the first barrier's count
    // (3 * 2^30 = -2^30 mod 2^32), so every block's bounded wait runs out
    // and the solve reports GS2_ERR_TIMEOUT
    h->stall_barrier = false;
    GS2_CUDA(cudaMemsetAsync((char*)h->persist_bar + 3, 0xC0, 1, h->stream));
  }
  {
    KernelTimer tm(h, "gmres_persistent", 0.0);
    if (m <= 8) launch_persistent<8>(h, a, nb);
    else if (m <= 16) launch_persistent<16>(h, a, nb);
    else launch_persistent<32>(h, a, nb);
  }
  read_state(h);  // raises GS2_ERR_TIMEOUT if a barrier gave up
  const KrylovState& st = *h->st_host;
  gs2_solve_info loc{st.iters, st.cycles, st.status, 0.0};
  loc.true_relres = st.bnorm == 0.0 ? 0.0 : st.beta / st.bnorm;
  if (info) *info = loc;
  return (gs2_status)st.status;
}

// ---------------------------------------------------------------------------
// a pack in one launch: the blocks are split among the systems in proportion
// to their rows (one row per thread while the blocks fit, at least one block
// a system, at most 128); each system's blocks run the single-system solve
// on its rows with their own barrier, partial sums and Krylov scalars, and
// leave when their system has finished, whatever the others do.
// ---------------------------------------------------------------------------

static int pack_max_blocks(const gs2_handle* h, int m) {
  int per_sm = 0;
  const void* fn = m <= 8 ? (const void*)k_gmres_persistent<8>
                          : (m <= 16 ? (const void*)k_gmres_persistent<16>
                                     : (const void*)k_gmres_persistent<32>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPerThreads, 0) != cudaSuccess)
    return 0;
  return per_sm * h->nsm;
}

// blocks per system, or an empty vector when the systems cannot all be
// co-resident with a block each
static std::vector<int> pack_blocks(const gs2_handle* h, int m) {
  const std::vector<int64_t>& off = *pack_offsets(h);
  const int S = (int)off.size() - 1;
  const int cap = pack_max_blocks(h, m);
  if (S <= 0 || S > cap) return {};
  std::vector<int> nb(S);
  int64_t want = 0;
  for (int s = 0; s < S; ++s) {
    const int64_t rows = off[s + 1] - off[s];
    nb[s] = (int)std::max<int64_t>(1, std::min<int64_t>(kPerMaxBlocks,
                                                        (rows + kPerThreads - 1) / kPerThreads));
    want += nb[s];
  }
  if (want > cap) {
    // scale down in proportion, one block at least; then trim the largest
    int64_t tot = 0;
    for (int s = 0; s < S; ++s) {
      nb[s] = (int)std::max<int64_t>(1, (int64_t)nb[s] * (cap - S) / want + 1);
      tot += nb[s];
    }
    while (tot > cap) {
      int big = (int)(std::max_element(nb.begin(), nb.end()) - nb.begin());
      if (nb[big] <= 1) return {};
      nb[big]--;
      tot--;
    }
  }
  return nb;
}

// Chosen automatically when, besides the single-system conditions, the
// whole pack gets one row per thread of the co-resident blocks: measured
// (GMRES(30) + SGS2(1,1), request-stream systems) 32 systems of 500-2,000
// rows, 35,894 rows in all: 9,971 solves/s in one launch against 8,169 with
// replayed cycle graphs; 128 systems of 1,000-31,684 rows, 1.17M rows: 1,128
// against 2,906 (a system then gets a few blocks, and tens of rows a thread).
bool pack_persistent_eligible(const gs2_handle* h, int m, const gs2_params* p, bool automatic) {
  if (!pack_offsets(h) || m > 32) return false;
  if (automatic && h->n > (int64_t)pack_max_blocks(h, m) * kPerThreads) return false;
  const std::vector<int64_t>& off = *pack_offsets(h);
  for (size_t s = 0; s + 1 < off.size(); ++s)
    if (off[s + 1] - off[s] > (automatic ? kPersistAutoRows : kPersistMaxRows)) return false;
  if (p && p->kind != GS2_PC_NONE) {
    if (p->parts > 1 || p->local_sweeps > 1) return false;
    if (p->kind != GS2_PC_JR &&
        !(p->kind == GS2_PC_GS2 && p->precision == GS2_FP64 && p->form == GS2_NONCOMPACT))
      return false;
  }
  return !pack_blocks(h, m).empty();
}

gs2_status pack_gmres_persistent(gs2_handle* h, const double* b, double* x, int m, double tol,
                                 int max_iters, const gs2_params* p, gs2_solve_info* infos) {
  const std::vector<int64_t>& off = *pack_offsets(h);
  const int S = (int)off.size() - 1;
  const std::vector<int> nbs = pack_blocks(h, m);
  if (nbs.empty()) GS2_THROW(GS2_ERR_INVALID_ARG, "the pack's systems do not fit one launch");
  ensure_krylov(h, m);
  int B = 0;
  for (int v : nbs) B += v;
  if (S > h->pp_cap_sys || B > h->pp_cap_blocks) {
    const int cs = std::max(S, h->pp_cap_sys), cb = std::max(B, h->pp_cap_blocks);
    h->pp_args = h->dalloc(sizeof(PersistArgs) * cs);
    h->pp_bsys = (int*)h->dalloc(sizeof(int) * cb);
    h->pp_bar = (unsigned*)h->dalloc(sizeof(unsigned) * 4 * cs);
    h->pp_part = (double*)h->dalloc(sizeof(double) * kPerSlots * cb);
    h->pp_st = (KrylovState*)h->dalloc(sizeof(KrylovState) * cs);
    if (h->pp_st_host) pinned_put(h->pp_st_host, sizeof(KrylovState) * h->pp_cap_sys);
    h->pp_st_host = (KrylovState*)pinned_get(sizeof(KrylovState) * cs);
    h->pp_cap_sys = cs;
    h->pp_cap_blocks = cb;
  }
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  std::vector<PersistArgs> tab(S);
  std::vector<int> bsys(B);
  int first = 0;
  for (int s = 0; s < S; ++s) {
    PersistArgs& a = tab[s];
    a = PersistArgs{};
    a.n = (int)h->n;
    a.Arp = h->A.rp;
    a.Aci = h->A.ci;
    a.Ava = h->A.va;
    a.Lrp = h->L.rp;
    a.Lci = h->L.ci;
    a.Lva = h->L.va;
    a.Urp = h->U.rp;
    a.Uci = h->U.ci;
    a.Uva = h->U.va;
    a.dinv = h->dinv;
    a.b = b;
    a.x = x;
    a.V = h->V;
    a.w = h->w;
    a.z = h->z;
    a.r = h->r;
    a.rh = h->rhat;
    a.g0 = h->g0;
    a.g1 = h->g1;
    a.part = h->pp_part + (size_t)kPerSlots * first;
    a.m = m;
    a.tol = tol;
    a.max_iters = max_iters;
    a.kind = pc ? pc->kind : GS2_PC_NONE;
    a.outer = pc ? std::max(1, pc->outer) : 1;
    a.inner = pc ? pc->inner : 0;
    a.dir = pc ? pc->direction : GS2_FORWARD;
    a.omega = pc ? pc->omega : 1.0;
    a.gamma = pc ? pc->gamma : 1.0;
    a.bar = h->pp_bar + 4 * s;
    a.err = h->dev_err;
    a.out = h->pp_st + s;
    a.r0 = (int)off[s];
    a.r1 = (int)off[s + 1];
    a.N = (int)h->n;
    a.first_block = first;
    a.nblocks = nbs[s];
    for (int k = 0; k < nbs[s]; ++k) bsys[first + k] = s;
    first += nbs[s];
  }
  h->h2d(h->pp_args, tab.data(), sizeof(PersistArgs) * S);
  h->h2d(h->pp_bsys, bsys.data(), sizeof(int) * B);
  GS2_CUDA(cudaMemsetAsync(h->pp_bar, 0, sizeof(unsigned) * 4 * S, h->stream));
  {
    KernelTimer tm(h, "gmres_persistent", 0.0);
    PersistArgs a0 = tab[0];
    const PersistArgs* sys = (const PersistArgs*)h->pp_args;
    if (m <= 8) launch_persistent<8>(h, a0, B, sys, h->pp_bsys);
    else if (m <= 16) launch_persistent<16>(h, a0, B, sys, h->pp_bsys);
    else launch_persistent<32>(h, a0, B, sys, h->pp_bsys);
  }
  GS2_CUDA(cudaMemcpyAsync(h->pp_st_host, h->pp_st, sizeof(KrylovState) * S,
                           cudaMemcpyDeviceToHost, h->stream));
  GS2_CUDA(cudaMemcpyAsync(h->err_host, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream));
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  if (*h->err_host) raise_device_error(h);  // a barrier gave up
  gs2_status first_bad = GS2_OK;
  for (int s = 0; s < S; ++s) {
    const KrylovState& st = h->pp_st_host[s];
    gs2_solve_info loc{st.iters, st.cycles, st.status, 0.0};
    loc.true_relres = st.bnorm == 0.0 ? 0.0 : st.beta / st.bnorm;
    if (infos) infos[s] = loc;
    if (loc.status != GS2_OK && first_bad == GS2_OK) first_bad = (gs2_status)loc.status;
  }
  return first_bad;
}

gs2_status cg_persistent(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                         const gs2_params* p, gs2_solve_info* info) {
  ensure_krylov(h, 2);  // V holds q and a residual scratch vector
  if (!h->persist_bar) {
    h->persist_bar = (unsigned*)h->dalloc(4 * sizeof(unsigned));
    h->persist_part = (double*)h->dalloc(sizeof(double) * kPerSlots * kPerMaxBlocks);
  }
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  int nb = (int)std::min<int64_t>(kPerMaxBlocks, (h->n + kPerThreads - 1) / kPerThreads);
  {
    int per_sm = 0;
    GS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_cg_persistent,
                                                           kPerThreads, 0));
    nb = std::max(1, std::min(nb, per_sm * h->nsm));
  }
  PersistArgs a{};
  a.n = (int)h->n;
  a.Arp = h->A.rp;
  a.Aci = h->A.ci;
  a.Ava = h->A.va;
  a.Lrp = h->L.rp;
  a.Lci = h->L.ci;
  a.Lva = h->L.va;
  a.Urp = h->U.rp;
  a.Uci = h->U.ci;
  a.Uva = h->U.va;
  a.dinv = h->dinv;
  a.b = b;
  a.x = x;
  a.V = h->V;
  a.w = h->w;
  a.z = h->z;
  a.r = h->r;
  a.rh = h->rhat;
  a.g0 = h->g0;
  a.g1 = h->g1;
  a.part = h->persist_part;
  a.m = 1;
  a.tol = tol;
  a.max_iters = max_iters;
  a.kind = pc ? pc->kind : GS2_PC_NONE;
  a.outer = pc ? std::max(1, pc->outer) : 1;
  a.inner = pc ? pc->inner : 0;
  a.dir = pc ? pc->direction : GS2_SYMMETRIC;
  a.omega = pc ? pc->omega : 1.0;
  a.gamma = pc ? pc->gamma : 1.0;
  a.bar = h->persist_bar;
  a.err = h->dev_err;
  a.out = h->st;
  a.r0 = 0;
  a.r1 = a.N = (int)h->n;
  a.first_block = 0;
  a.nblocks = nb;
  GS2_CUDA(cudaMemsetAsync(h->persist_bar, 0, 4 * sizeof(unsigned), h->stream));
  {
    KernelTimer tm(h, "cg_persistent", 0.0);
    void* args[] = {&a};
    GS2_CUDA(cudaLaunchCooperativeKernel((const void*)k_cg_persistent, nb, kPerThreads, args, 0,
                                         h->stream));
    GS2_LAUNCH_CHECK();
  }
  read_state(h);
  const KrylovState& st = *h->st_host;
  gs2_solve_info loc{st.iters, st.cycles, st.status, 0.0};
  loc.true_relres = st.bnorm == 0.0 ? 0.0 : st.beta / st.bnorm;
  if (info) *info = loc;
  return (gs2_status)st.status;
}

}  // namespace gs2
