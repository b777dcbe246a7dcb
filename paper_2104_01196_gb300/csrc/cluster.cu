// Restarted GMRES(m), or CG, of a small system inside one thread-block
// cluster.
//
// A system of a few thousand rows spends its one-launch solve (persist.cu)
// waiting: on a GB300 a grid barrier through device memory costs 1.3 us and
// a dependent L2 load 150 ns, while the arithmetic of an Arnoldi step at
// 4,096 rows is a few microseconds.  Here the system lives in the shared
// memory of the C <= 16 CTAs of one cluster: CTA k owns the rows
// [kR, kR + R) and holds their entries of every vector, of the Krylov basis
// V and of the matrices A, D^{-1}L and D^{-1}U (row-sliced ELL: slot q of
// local row l at q * Rp + l, so that a warp's lanes read consecutive words;
// rows shorter than the matrix's longest are padded with zero entries that
// point at the row itself).
// A column index is turned once, when the CTA loads its rows, into the
// distributed-shared-memory address of that row's entry of vector 0 in the
// owning CTA (mapa); the gather of any vector v is then one
// ld.shared::cluster at that address plus v's offset.  Phases meet at a
// cluster barrier made of one mbarrier per CTA: every CTA arrives on every
// CTA's barrier (release, cluster scope) and waits on its own (acquire),
// with a bound -- 0.45 us at 16 CTAs against 1.3 us for the grid barrier.
// Inner products are CTA partial sums (the warps' butterfly sums, then the
// warps as a fixed pairwise tree) that every CTA reads from all CTAs and
// adds as a fixed pairwise tree, so that every CTA holds bitwise the same
// Krylov scalars and takes the same decisions, as in the one-launch solver.
// The arithmetic of each row -- residuals, inner sweeps, the CGS2 updates --
// is that of the multi-kernel path, entry for entry in stored order (the
// padding slots add exact zeros); the grouping of the inner products'
// partial sums differs, and the Givens rotations are formed with explicit
// FMAs.  A pack gives every system a cluster of its own: a table of
// systems, cluster k solving system k with columns taken relative to the
// system's first row.
//
// The CTAs meet once with the hardware cluster barrier after loading their
// rows (so that no CTA arrives on a barrier that is not initialised yet) and
// once before they leave (so that no CTA's shared memory goes away while
// another may still read it).  Every wait between is bounded: a CTA that
// waits too long records GS2_ERR_TIMEOUT and goes straight to the final
// barrier, and so does every other CTA at its next wait.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "arnoldi.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace gs2 {

constexpr int kClMaxCtas = 16;
constexpr int kClMaxThreads = 256;
constexpr int kClMaxRestart = 32;
constexpr long long kClWaitCycles = 4LL << 30;  // ~2 s at 2.07 GHz

// vectors held per row, in this order (their offsets are the same in every
// CTA, so a gather address plus k * Rp * 8 reads vector k); the true
// residual r shares w's storage: r lives from the residual to v_0 = r / beta
// at a cycle's start, w from the first SpMV to the correction V y at its end
enum ClVec { kVX = 0, kVZ, kVRH, kVG0, kVG1, kVB, kVW, kVD, kClVecs, kVR = kVW };

// Byte offsets of a CTA's shared memory (the same in every CTA).
struct ClLayout {
  int Rp;          // per-CTA stride of vectors and ELL slices (rows, even)
  int WA, WL, WU;  // ELL widths: the longest row of A, D^{-1}L, D^{-1}U
  int m;           // restart length (basis vectors m + 1)
  unsigned vec, V, Av, Lv, Uv, Aa, La, Ua, bytes;
};

__host__ __device__ inline unsigned cl_align16(unsigned x) { return (x + 15u) & ~15u; }

__host__ __device__ inline ClLayout cl_layout(int Rp, int WA, int WL, int WU, int m) {
  ClLayout L;
  L.Rp = Rp;
  L.WA = WA;
  L.WL = WL;
  L.WU = WU;
  L.m = m;
  const unsigned r = (unsigned)Rp;
  unsigned o = 0;
  L.vec = o;
  o = cl_align16(o + 8u * r * kClVecs);
  L.V = o;
  o = cl_align16(o + 8u * r * (unsigned)(m + 1));
  L.Av = o;
  o = cl_align16(o + 8u * r * (unsigned)WA);
  L.Lv = o;
  o = cl_align16(o + 8u * r * (unsigned)WL);
  L.Uv = o;
  o = cl_align16(o + 8u * r * (unsigned)WU);
  L.Aa = o;
  o = cl_align16(o + 4u * r * (unsigned)WA);
  L.La = o;
  o = cl_align16(o + 4u * r * (unsigned)WL);
  L.Ua = o;
  o = cl_align16(o + 4u * r * (unsigned)WU);
  L.bytes = o;
  return L;
}

// One system of a pack: its rows [base, base + n) of the pack's vectors and
// block-diagonal matrix, R rows a CTA, its result slot.
struct ClSys {
  int base, n, R;
  KrylovState* out;
};

struct ClusterArgs {
  int n;     // rows
  int R;     // rows per CTA (the last CTA may hold fewer, at least one)
  int C;     // CTAs of the cluster
  int base;  // the system's first row in the vectors and the matrix
  const ClSys* sys;  // a pack: cluster k solves system sys[k] (base, n, R, out)
  ClLayout lay;
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
  double* x;  // x0 on entry, the solution on return
  int m;
  double tol;
  int max_iters;
  int kind;  // GS2_PC_NONE, GS2_PC_GS2 or GS2_PC_JR
  int outer, inner, dir;
  double omega, gamma;
  int* err;  // device error word
  KrylovState* out;
  int stall;  // test hook: the last CTA never arrives, so every wait runs out
  int cg;     // 1: preconditioned CG (basis slots 0, 1, 2: p, A p, a residual)
};

// ---------------------------------------------------------------------------
// cluster primitives (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// the address of this CTA's shared-memory word `addr` in CTA `rank`
__device__ __forceinline__ unsigned cl_map(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// a load from distributed shared memory (volatile: every gather is issued
// where it stands, never merged with one before a barrier)
__device__ __forceinline__ double ld_cl(unsigned addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ void cluster_barrier_hw() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// Per-CTA state of the bounded cluster barrier and of the partial sums.
struct ClSync {
  unsigned long long mbar;        // this CTA's barrier (C arrivals a phase)
  unsigned peer_mbar[kClMaxCtas];  // every CTA's barrier, cluster addresses
  unsigned peer_part[kClMaxCtas];  // every CTA's partial sums
  unsigned phase;                  // parity of the phase being waited for
  int pb;                          // partial-sum buffer of the next sum
  int ok;
  int mute;                        // test hook: this CTA does not arrive
  double (*red)[32];               // the warps' sums of a cluster sum (every width)
};

// Bounded cluster barrier: false when this CTA gave up waiting (it records
// GS2_ERR_TIMEOUT).  The CTA barrier orders the CTA's writes before the
// release arrivals; the acquire wait orders every CTA's writes before this
// CTA's reads after it.
__device__ bool cl_sync(ClSync& S, int C, int* err) {
  __syncthreads();
  if ((int)threadIdx.x < C && !S.mute)
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                     S.peer_mbar[threadIdx.x])
                 : "memory");
  if (threadIdx.x == 0) {
    const unsigned par = S.phase;
    const unsigned bar = smem_u32(&S.mbar);
    const long long t0 = clock64();
    int ok = 1;
    for (;;) {
      unsigned done;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar), "r"(par)
          : "memory");
      if (done) break;
      if (clock64() - t0 > kClWaitCycles) {
        atomicCAS(err, 0, (int)GS2_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    S.phase = par ^ 1u;
    S.ok = ok;
  }
  __syncthreads();
  return S.ok != 0;
}

// ---------------------------------------------------------------------------
// the CTA's view of its rows
// ---------------------------------------------------------------------------

struct ClRows {
  double* vec;  // vector k of local row l at vec[k * Rp + l]
  double* V;    // basis vector q of local row l at V[q * Rp + l]
  const double *Av, *Lv, *Uv;
  const unsigned *Aa, *La, *Ua;
  int WA, WL, WU;  // slots per row (ELL widths)
  int Rp, Rk;      // stride, rows this CTA owns
  __device__ double* v(int k) const { return vec + k * Rp; }
  __device__ unsigned off(int k) const { return 8u * (unsigned)(k * Rp); }
};

// rows owned by this thread (one at a time: unrolled, the row loops of the
// CGS2 phases would hold several rows' basis entries in registers at once)
#define CL_ROWS(l) \
  _Pragma("unroll 1") for (int l = (int)threadIdx.x; l < c.Rk; l += (int)blockDim.x)

// sum over the row's W slots of val * (vector at byte offset voff) gathered
// from the owning CTAs: the stored entries in stored order, then padding
// slots (value 0, the row's own entry).  A warp issues its loads in order
// and waits only when a result is used, so the gathers go out four at a
// time before their products (one at a time each would cost a full
// distributed-shared-memory round trip); W is the same for every row.
__device__ __forceinline__ double cl_row_dot(const double* val, const unsigned* adr, int W,
                                             int Rp, int l, unsigned voff) {
  double s = 0.0;
  int k = 0;
#pragma unroll 1
  for (; k + 4 <= W; k += 4) {
    const unsigned a0 = adr[k * Rp + l], a1 = adr[(k + 1) * Rp + l], a2 = adr[(k + 2) * Rp + l],
                   a3 = adr[(k + 3) * Rp + l];
    const double v0 = val[k * Rp + l], v1 = val[(k + 1) * Rp + l], v2 = val[(k + 2) * Rp + l],
                 v3 = val[(k + 3) * Rp + l];
    const double x0 = ld_cl(a0 + voff), x1 = ld_cl(a1 + voff), x2 = ld_cl(a2 + voff),
                 x3 = ld_cl(a3 + voff);
    s = fma(v0, x0, s);
    s = fma(v1, x1, s);
    s = fma(v2, x2, s);
    s = fma(v3, x3, s);
  }
  const int rem = W - k;
  if (rem > 0) {
    const double v0 = val[k * Rp + l];
    const double v1 = rem > 1 ? val[(k + 1) * Rp + l] : 0.0;
    const double v2 = rem > 2 ? val[(k + 2) * Rp + l] : 0.0;
    const double x0 = ld_cl(adr[k * Rp + l] + voff);
    double x1 = 0.0, x2 = 0.0;
    if (rem > 1) x1 = ld_cl(adr[(k + 1) * Rp + l] + voff);
    if (rem > 2) x2 = ld_cl(adr[(k + 2) * Rp + l] + voff);
    s = fma(v0, x0, s);
    if (rem > 1) s = fma(v1, x1, s);
    if (rem > 2) s = fma(v2, x2, s);
  }
  return s;
}

__device__ __forceinline__ double cl_dotA(const ClRows& c, int l, int k) {
  return cl_row_dot(c.Av, c.Aa, c.WA, c.Rp, l, c.off(k));
}

// Sums over the cluster of nv <= NV per-thread values into out[0 .. nv)
// (shared memory), bitwise the same in every CTA: each warp's butterfly
// sums, the warps as a fixed pairwise tree, this CTA's sums to its partial
// buffer, the barrier, then value q summed over the CTAs as a fixed
// pairwise tree in rank order.  The buffers
// alternate, so a buffer is written again only after the barrier that
// follows every CTA's reads of it.
template <int NV>
__device__ bool cl_sums(ClSync& S, const double (&acc)[NV], int nv, double* out, int C,
                        int* err, double (*part)[32]) {
  constexpr int P = Pow2<NV>::value;
  constexpr int p = Log2<P>::value;
  double (*red)[32] = S.red;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double a0 = warp_butterfly<NV>(acc);
  if ((lane & ((1 << (5 - p)) - 1)) == 0) red[wid][lane >> (5 - p)] = a0;
  __syncthreads();
  const int pb = S.pb;
  if ((int)threadIdx.x < nv) {
    // the warps' sums as a fixed pairwise tree (nw is 2, 4 or 8)
    const int v = threadIdx.x;
    double sum = red[0][v] + red[1][v];
    if (nw >= 4) sum = sum + (red[2][v] + red[3][v]);
    if (nw == 8) sum = sum + ((red[4][v] + red[5][v]) + (red[6][v] + red[7][v]));
    part[pb][v] = sum;
  }
  if (!cl_sync(S, C, err)) return false;
  if ((int)threadIdx.x < nv) {
    // all CTAs' partials in flight at once (a CTA beyond C re-reads the
    // last one), then summed
    const unsigned o = 8u * (unsigned)(pb * 32 + threadIdx.x);
    double pv[kClMaxCtas];
#pragma unroll
    for (int r = 0; r < kClMaxCtas; ++r) pv[r] = ld_cl(S.peer_part[min(r, C - 1)] + o);
    // a fixed pairwise tree over the first C: four dependent adds, not C
#pragma unroll
    for (int w = 1; w < kClMaxCtas; w *= 2)
#pragma unroll
      for (int i = 0; i + w < kClMaxCtas; i += 2 * w)
        if (i + w < C) pv[i] += pv[i + w];
    out[threadIdx.x] = pv[0];
  }
  __syncthreads();
  if (threadIdx.x == 0) S.pb = pb ^ 1;
  __syncthreads();
  return true;
}

__device__ __forceinline__ bool cl_sum1(ClSync& S, double v, double* out, int C, int* err,
                                        double (*part)[32]) {
  const double acc[1] = {v};
  return cl_sums<1>(S, acc, 1, out, C, err, part);
}

// z = M^{-1} v from z = 0 (v: this CTA's rows, complete in every CTA on
// entry, as the barrier before the call ensures for the rows it gathers):
// GS2 half sweeps (Eq. (2)-(5), damped) or JR sweeps, the arithmetic of the
// multi-kernel path row for row.  z complete in every CTA on a true return.
__device__ bool cl_precond(const ClRows& c, const ClusterArgs& a, ClSync& S, const double* v) {
  double* z = c.v(kVZ);
  double* rh = c.v(kVRH);
  const double* d = c.v(kVD);
  if (a.kind == GS2_PC_NONE) {
    CL_ROWS(l) z[l] = v[l];
    return cl_sync(S, a.C, a.err);
  }
  CL_ROWS(l) rh[l] = d[l] * v[l];
  if (a.kind == GS2_PC_JR) {
    // first sweep from zero: z = omega D^{-1} v; then z + omega D^{-1} (v - A z)
    int cur = kVZ, nxt = kVG0;
    CL_ROWS(l) z[l] = a.omega * rh[l];
    for (int s = 1; s < a.outer; ++s) {
      if (!cl_sync(S, a.C, a.err)) return false;
      double* pc = c.v(cur);
      double* pn = c.v(nxt);
      CL_ROWS(l) {
        const double t = cl_dotA(c, l, cur);
        pn[l] = pc[l] + a.omega * (d[l] * (v[l] - t));
      }
      const int tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (cur != kVZ) {
      // every CTA must be done gathering from z before it is overwritten
      if (!cl_sync(S, a.C, a.err)) return false;
      const double* pc = c.v(cur);
      CL_ROWS(l) z[l] = pc[l];
    }
    return cl_sync(S, a.C, a.err);
  }
  const bool damped = a.gamma != 1.0;
  bool zero = true;
  for (int s = 0; s < a.outer; ++s) {
    for (int half = 0; half < 2; ++half) {
      const bool fwd = half == 0;
      if (fwd && a.dir == GS2_BACKWARD) continue;
      if (!fwd && a.dir == GS2_FORWARD) continue;
      const double* Tv = fwd ? c.Lv : c.Uv;
      const unsigned* Ta = fwd ? c.La : c.Ua;
      const int TW = fwd ? c.WL : c.WU;
      if (!zero) {
        if (!cl_sync(S, a.C, a.err)) return false;  // z complete
        CL_ROWS(l) rh[l] = d[l] * (v[l] - cl_dotA(c, l, kVZ));
      }
      if (!cl_sync(S, a.C, a.err)) return false;  // rh complete
      if (a.inner == 0) {
        CL_ROWS(l) z[l] = zero ? a.omega * rh[l] : z[l] + a.omega * rh[l];
      }
      int gin = kVRH;
      for (int k = 0; k < a.inner; ++k) {
        const bool last = k == a.inner - 1;
        const int gout = (k % 2 == 0) ? kVG0 : kVG1;
        const double* pi = c.v(gin);
        double* po = c.v(gout);
        CL_ROWS(l) {
          const double t = cl_row_dot(Tv, Ta, TW, c.Rp, l, c.off(gin));
          double go = rh[l] - a.omega * t;
          if (damped) go = (1.0 - a.gamma) * pi[l] + a.gamma * go;
          if (!last) po[l] = go;
          else z[l] = zero ? a.omega * go : z[l] + a.omega * go;
        }
        if (!last) {
          if (!cl_sync(S, a.C, a.err)) return false;
          gin = gout;
        }
      }
      zero = false;
    }
  }
  return cl_sync(S, a.C, a.err);
}

// one CTA's rows of a matrix into its ELL slice: W slots a row, the stored
// entries' values and gather addresses (of vector 0 in the owning CTA) in
// stored order, then padding slots of value 0 that point at the row itself
// (W is at least the longest row; a matrix the solve does not use has
// W = 0).  row0: the CTA's first row in the matrix; base: the system's
// first row, which column numbers are taken relative to.
__device__ void cl_load_rows(const int* rp, const int* ci, const double* va, int W, int Rp,
                             int row0, int Rk, int R, int base, unsigned vec0, unsigned rank,
                             double* val, unsigned* adr) {
  for (int l = threadIdx.x; l < Rp; l += blockDim.x) {
    const bool own = l < Rk;
    const int k0 = own ? rp[row0 + l] : 0;
    const int ln = own ? min(rp[row0 + l + 1] - k0, W) : 0;
    const unsigned self = cl_map(vec0 + 8u * (unsigned)l, rank);
    for (int q = 0; q < W; ++q) {
      if (q < ln) {
        const int col = ci[k0 + q] - base;
        const int o = col / R;
        val[q * Rp + l] = va[k0 + q];
        adr[q * Rp + l] = cl_map(vec0 + 8u * (unsigned)(col - o * R), (unsigned)o);
      } else {
        val[q * Rp + l] = 0.0;
        adr[q * Rp + l] = self;
      }
    }
  }
}

// CGS2 phases over the CTA's rows for jc <= JB basis vectors (JB a multiple
// of 8): w = A z and acc = V^T w
template <int JB>
__device__ bool cl_spmv_dots(const ClRows& c, const ClusterArgs& a, ClSync& S, int jc,
                             double* h, double (*part)[32]) {
  double acc[JB];
#pragma unroll
  for (int q = 0; q < JB; ++q) acc[q] = 0.0;
  double* w = c.v(kVW);
  CL_ROWS(l) {
    const double wi = cl_dotA(c, l, kVZ);
    w[l] = wi;
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) acc[q] = fma(c.V[q * c.Rp + l], wi, acc[q]);
  }
  return cl_sums<JB>(S, acc, jc, h, a.C, a.err, part);
}

// w -= V h and acc = V^T w
template <int JB>
__device__ bool cl_update_dots(const ClRows& c, const ClusterArgs& a, ClSync& S, int jc,
                               const double* h, double* h2, double (*part)[32]) {
  double acc[JB];
#pragma unroll
  for (int q = 0; q < JB; ++q) acc[q] = 0.0;
  double* w = c.v(kVW);
  CL_ROWS(l) {
    double wn = w[l];
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) wn = fma(c.V[q * c.Rp + l], -h[q], wn);
    w[l] = wn;
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) acc[q] = fma(c.V[q * c.Rp + l], wn, acc[q]);
  }
  return cl_sums<JB>(S, acc, jc, h2, a.C, a.err, part);
}

// w -= V h; this thread's sum of w_l^2
template <int JB>
__device__ double cl_update_norm(const ClRows& c, int jc, const double* h) {
  double t = 0.0;
  double* w = c.v(kVW);
  CL_ROWS(l) {
    double wn = w[l];
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < jc) wn = fma(c.V[q * c.Rp + l], -h[q], wn);
    w[l] = wn;
    t = fma(wn, wn, t);
  }
  return t;
}

#define CL_JB(jc, CALL8, CALL16, CALL24, CALL32) \
  switch (((jc) + 7) >> 3) {                     \
    case 1: CALL8; break;                        \
    case 2: CALL16; break;                       \
    case 3: CALL24; break;                       \
    default: CALL32; break;                      \
  }

// givens_column's step on a slow FP64 pipe (a dependent FP64 operation
// takes 64 cycles on a GB300, a square root ~690 and a division ~430),
// split so that the sequential part is one FMA a rotation.  Rotation q maps
// (u_q, v_q) = (H(q, j) as rotated by rotations 0 .. q-1, H(q+1, j)) to
//   H(q, j) = c_q u_q + s_q v_q,   u_{q+1} = -s_q u_q + c_q v_q,
// so the products c_q v_q and s_q v_q do not depend on the chain: threads
// q < j form them at once (cl_givens_products), then one thread runs the
// chain of u and writes H(q, j) beside it (cl_givens_chain) while another
// forms H(j+1, j) = ||w|| (a square root and a division), and the new
// rotation's two divisions run side by side (cl_givens_rotation).
__device__ __forceinline__ void cl_givens_products(const double* col, const double* cs,
                                                   const double* sn, double* cv, double* sv,
                                                   int j) {
  const int q = threadIdx.x;
  if (q < j) {
    const double v = col[q + 1];
    cv[q] = cs[q] * v;
    sv[q] = sn[q] * v;
  }
}

// the chain: H(q, j) for q < j written back, u_j returned
__device__ __forceinline__ double cl_givens_chain(double* col, const double* cs,
                                                  const double* sn, const double* cv,
                                                  const double* sv, int j) {
  double u = col[0];
  for (int q = 0; q < j; ++q) {
    const double c = cs[q], s = sn[q], cq = cv[q], sq = sv[q];
    col[q] = fma(c, u, sq);
    u = fma(-s, u, cq);
  }
  return u;
}

// the new rotation from (f, g) = (u_j, H(j+1, j)), applied to H and to the
// right-hand side g; returns the residual estimate |g_{j+1}|
__device__ __forceinline__ double cl_givens_rotation(double* col, double* cs, double* sn,
                                                     double* g, double f, double gg, int j) {
  double c, sg, rr;
  if (gg == 0.0) {
    c = 1.0; sg = 0.0; rr = f;
  } else if (f == 0.0) {
    c = 0.0; sg = gg > 0.0 ? 1.0 : -1.0; rr = fabs(gg);
  } else {
    const double d = sqrt(fma(f, f, gg * gg));
    rr = f > 0.0 ? d : -d;
    c = fabs(f) / d;
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

// The solve on loaded rows; false when a barrier gave up (nothing more may
// be read from other CTAs then).  Writes the outcome to a.out (rank 0).
__device__ bool cl_solve(const ClRows& c, const ClusterArgs& a, ClSync& S, double (*part)[32],
                         unsigned rank) {
  __shared__ double Hs[(kClMaxRestart + 1) * kClMaxRestart];  // column j at Hs[j * (m + 1)]
  __shared__ double cs_s[kClMaxRestart + 1], sn_s[kClMaxRestart + 1];
  __shared__ double g_s[kClMaxRestart + 1], y_s[kClMaxRestart + 1];
  __shared__ double h1[kClMaxRestart], h2[kClMaxRestart];
  __shared__ double cv_s[kClMaxRestart], sv_s[kClMaxRestart];
  __shared__ double tot, hn_s, ih_s;
  __shared__ int sh_flag;
  const int m = a.m, ldh = m + 1, C = a.C;
  double* x = c.v(kVX);
  double* r = c.v(kVR);
  double* w = c.v(kVW);
  const double* z = c.v(kVZ);
  const double* bb = c.v(kVB);
  int iters = 0, cycles = 0, status = GS2_OK;
  double bnorm = 0.0, beta = 0.0;

  // ||b||
  double t = 0.0;
  CL_ROWS(l) t = fma(bb[l], bb[l], t);
  if (!cl_sum1(S, t, &tot, C, a.err, part)) return false;
  bnorm = sqrt(tot);
  if (bnorm == 0.0 || isnan(bnorm) || isinf(bnorm)) {
    if (bnorm == 0.0) CL_ROWS(l) x[l] = 0.0;
    else status = GS2_ERR_NAN;
    if (rank == 0 && threadIdx.x == 0) {
      a.out->iters = 0;
      a.out->cycles = 0;
      a.out->status = status;
      a.out->bnorm = bnorm;
      a.out->beta = bnorm == 0.0 ? 0.0 : NAN;
    }
    return true;
  }
  const double tol_abs = a.tol * bnorm;
  bool breakdown = false;
  for (;;) {
    // true residual r = b - A x and its norm (x complete here)
    t = 0.0;
    CL_ROWS(l) {
      const double ri = bb[l] - cl_dotA(c, l, kVX);
      r[l] = ri;
      t = fma(ri, ri, t);
    }
    if (!cl_sum1(S, t, &tot, C, a.err, part)) return false;
    beta = sqrt(tot);
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
    CL_ROWS(l) c.V[l] = r[l] * ib;
    if ((int)threadIdx.x <= m) g_s[threadIdx.x] = threadIdx.x == 0 ? beta : 0.0;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      if (!cl_precond(c, a, S, c.V + j * c.Rp)) return false;
      const int jc = j + 1;
      // w = A z and the first Gram-Schmidt pass V^T w
      bool ok = true;
      CL_JB(jc, ok = cl_spmv_dots<8>(c, a, S, jc, h1, part),
            ok = cl_spmv_dots<16>(c, a, S, jc, h1, part),
            ok = cl_spmv_dots<24>(c, a, S, jc, h1, part),
            ok = cl_spmv_dots<32>(c, a, S, jc, h1, part));
      if (!ok) return false;
      // w -= V h1 and the second pass V^T w
      CL_JB(jc, ok = cl_update_dots<8>(c, a, S, jc, h1, h2, part),
            ok = cl_update_dots<16>(c, a, S, jc, h1, h2, part),
            ok = cl_update_dots<24>(c, a, S, jc, h1, h2, part),
            ok = cl_update_dots<32>(c, a, S, jc, h1, h2, part));
      if (!ok) return false;
      // w -= V h2 and ||w||^2
      CL_JB(jc, t = cl_update_norm<8>(c, jc, h2), t = cl_update_norm<16>(c, jc, h2),
            t = cl_update_norm<24>(c, jc, h2), t = cl_update_norm<32>(c, jc, h2));
      if (!cl_sum1(S, t, &tot, C, a.err, part)) return false;
      // Givens step j (every CTA on its own copies): column j of H filled by
      // jc threads at once, H(j+1, j) = ||w|| and its inverse on the second
      // warp while thread 0 applies the rotations
      double* col = Hs + j * ldh;
      if ((int)threadIdx.x < jc) col[threadIdx.x] = h1[threadIdx.x] + h2[threadIdx.x];
      __syncthreads();
      double u = 0.0;  // thread 0: H(j, j) rotated by the earlier rotations
      if (threadIdx.x < 32) {
        cl_givens_products(col, cs_s, sn_s, cv_s, sv_s, j);
        __syncwarp();
        if (threadIdx.x == 0) u = cl_givens_chain(col, cs_s, sn_s, cv_s, sv_s, j);
      } else if (threadIdx.x == 32) {
        const double hn = sqrt(tot);
        hn_s = hn;
        ih_s = 1.0 / hn;  // H(j+1, j)^{-1}
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double hn = hn_s;
        const double est = cl_givens_rotation(col, cs_s, sn_s, g_s, u, hn, j);
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
      }
      __syncthreads();
      ++iters;
      k = jc;
      const int fl = sh_flag;
      if (fl & 2) status = GS2_ERR_NAN;
      if (fl & 4) breakdown = true;
      if (fl & 1) break;
      if (j + 1 < m) {
        const double ih = ih_s;
        double* vn = c.V + (j + 1) * c.Rp;
        CL_ROWS(l) vn[l] = w[l] * ih;
      }
    }
    // x += M^{-1} V y, y = R^{-1} g over the k steps
    if (threadIdx.x == 0) {
      for (int q = 0; q < k; ++q) y_s[q] = g_s[q];
      for (int q = k - 1; q >= 0; --q) {
        const double* cq = Hs + q * ldh;
        const double yq = y_s[q] / cq[q];
        y_s[q] = yq;
        for (int l = 0; l < q; ++l) y_s[l] -= cq[l] * yq;
      }
    }
    __syncthreads();
    CL_ROWS(l) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = fma(c.V[q * c.Rp + l], y_s[q], s);
      w[l] = s;
    }
    if (!cl_precond(c, a, S, w)) return false;
    CL_ROWS(l) x[l] = x[l] + z[l];
    if (!cl_sync(S, C, a.err)) return false;
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.out->iters = iters;
    a.out->cycles = cycles;
    a.out->status = status;
    a.out->bnorm = bnorm;
    a.out->beta = beta;
  }
  return true;
}

// Preconditioned CG on loaded rows: the iteration of the one-launch CG
// solver (restart of the search direction when the recursive residual has
// converged but the true residual disagrees), every scalar summed alike by
// every CTA.  p, q = A p and the true-residual scratch t are basis slots
// 0, 1, 2; r takes w's slot.  False when a barrier gave up.
__device__ bool cl_cg_solve(const ClRows& c, const ClusterArgs& a, ClSync& S,
                            double (*part)[32], unsigned rank) {
  __shared__ double tot;
  const int C = a.C;
  double* x = c.v(kVX);
  double* r = c.v(kVW);
  const double* z = c.v(kVZ);
  const double* bb = c.v(kVB);
  double* p = c.V;
  double* q = c.V + c.Rp;
  double* t = c.V + 2 * c.Rp;
  const unsigned poff = a.lay.V - a.lay.vec;  // p's offset from vector 0
  int iters = 0, cycles = 0, status = GS2_OK;
  double sm = 0.0;
  CL_ROWS(l) sm = fma(bb[l], bb[l], sm);
  if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
  const double bnorm = sqrt(tot);
  double beta = 0.0;
  if (bnorm == 0.0 || isnan(bnorm) || isinf(bnorm)) {
    if (bnorm == 0.0) CL_ROWS(l) x[l] = 0.0;
    if (rank == 0 && threadIdx.x == 0) {
      a.out->iters = 0;
      a.out->cycles = 0;
      a.out->status = bnorm == 0.0 ? GS2_OK : GS2_ERR_NAN;
      a.out->bnorm = bnorm;
      a.out->beta = bnorm == 0.0 ? 0.0 : NAN;
    }
    return true;
  }
  const double tol_abs = a.tol * bnorm;
  CL_ROWS(l) r[l] = bb[l] - cl_dotA(c, l, kVX);
  for (;;) {
    // ||r|| of the recursive residual; confirmed on the true one
    sm = 0.0;
    CL_ROWS(l) sm = fma(r[l], r[l], sm);
    if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
    const double rn = sqrt(tot);
    beta = rn;
    if (isnan(rn) || isinf(rn)) {
      status = GS2_ERR_NAN;
      break;
    }
    if (rn <= tol_abs) {
      sm = 0.0;
      CL_ROWS(l) {
        const double ti = bb[l] - cl_dotA(c, l, kVX);
        t[l] = ti;
        sm = fma(ti, ti, sm);
      }
      if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
      beta = sqrt(tot);
      if (beta <= tol_abs) break;
      CL_ROWS(l) r[l] = t[l];
    }
    if (iters >= a.max_iters) {
      status = GS2_ERR_NOT_CONVERGED;
      break;
    }
    ++cycles;
    // z = M^{-1} r, p = z, rz = r.z
    if (!cl_precond(c, a, S, r)) return false;
    sm = 0.0;
    CL_ROWS(l) {
      p[l] = z[l];
      sm = fma(r[l], z[l], sm);
    }
    if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
    double rz = tot;
    for (;;) {
      // q = A p (p complete: the last sum's barrier) and p.q
      sm = 0.0;
      CL_ROWS(l) {
        const double qi = cl_row_dot(c.Av, c.Aa, c.WA, c.Rp, l, poff);
        q[l] = qi;
        sm = fma(p[l], qi, sm);
      }
      if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
      const double pq = tot;
      if (pq == 0.0) {
        status = GS2_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rz / pq;
      sm = 0.0;
      CL_ROWS(l) {
        x[l] = fma(alpha, p[l], x[l]);
        const double ri = fma(-alpha, q[l], r[l]);
        r[l] = ri;
        sm = fma(ri, ri, sm);
      }
      if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
      ++iters;
      const double rr = sqrt(tot);
      if (isnan(rr) || isinf(rr)) {
        status = GS2_ERR_NAN;
        break;
      }
      if (rr <= tol_abs || iters >= a.max_iters) break;
      // z = M^{-1} r, beta = r.z / rz, p = z + beta p
      if (!cl_precond(c, a, S, r)) return false;
      sm = 0.0;
      CL_ROWS(l) sm = fma(r[l], z[l], sm);
      if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
      const double bt = tot / rz;
      rz = tot;
      CL_ROWS(l) p[l] = fma(bt, p[l], z[l]);
      if (!cl_sync(S, C, a.err)) return false;
    }
    if (status == GS2_ERR_NAN || status == GS2_ERR_BREAKDOWN) break;
  }
  // the true residual at exit
  sm = 0.0;
  CL_ROWS(l) {
    const double ti = bb[l] - cl_dotA(c, l, kVX);
    sm = fma(ti, ti, sm);
  }
  if (!cl_sum1(S, sm, &tot, C, a.err, part)) return false;
  if (rank == 0 && threadIdx.x == 0) {
    a.out->iters = iters;
    a.out->cycles = cycles;
    a.out->status = status;
    a.out->bnorm = bnorm;
    a.out->beta = sqrt(tot);
  }
  return true;
}

__global__ void __launch_bounds__(kClMaxThreads, 1)
    k_gmres_cluster(const __grid_constant__ ClusterArgs a0) {
  extern __shared__ __align__(16) unsigned char cl_smem[];
  __shared__ ClSync S;
  __shared__ double part[2][32];
  // one buffer for the warp sums of every width, declared here and reached
  // through S (declared at namespace scope instead, the solve went wrong)
  __shared__ double red[kClMaxThreads / 32][32];
  // the arguments and the row view in shared memory, where every phase
  // reads them (held in registers they would crowd out the row loops')
  __shared__ ClusterArgs a;
  __shared__ ClRows c;
  __shared__ int row0_s;  // this CTA's first row in the vectors and the matrix
  const unsigned rank = cl_rank();
  const ClLayout& L = a0.lay;
  if (threadIdx.x == 0) {
    a = a0;
    if (a0.sys) {
      // a pack: this cluster's system
      const ClSys q = a0.sys[blockIdx.x / a0.C];
      a.base = q.base;
      a.n = q.n;
      a.R = q.R;
      a.out = q.out;
    }
    const int r0 = (int)rank * a.R;
    row0_s = a.base + r0;
    c.vec = (double*)(cl_smem + L.vec);
    c.V = (double*)(cl_smem + L.V);
    c.Av = (const double*)(cl_smem + L.Av);
    c.Lv = (const double*)(cl_smem + L.Lv);
    c.Uv = (const double*)(cl_smem + L.Uv);
    c.Aa = (const unsigned*)(cl_smem + L.Aa);
    c.La = (const unsigned*)(cl_smem + L.La);
    c.Ua = (const unsigned*)(cl_smem + L.Ua);
    c.WA = L.WA;
    c.WL = L.WL;
    c.WU = L.WU;
    c.Rp = L.Rp;
    c.Rk = max(0, min(a.R, a.n - r0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar)), "r"(a0.C)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.phase = 0;
    S.pb = 0;
    S.ok = 1;
    S.mute = a0.stall && (int)rank == a0.C - 1;
    S.red = red;
  }
  if ((int)threadIdx.x < a0.C) {
    S.peer_mbar[threadIdx.x] = cl_map(smem_u32(&S.mbar), threadIdx.x);
    S.peer_part[threadIdx.x] = cl_map(smem_u32(&part[0][0]), threadIdx.x);
  }
  __syncthreads();
  const int row0 = row0_s;
  // this CTA's rows: x0, b, D^{-1}; the other vectors zero
  for (int l = threadIdx.x; l < L.Rp; l += blockDim.x) {
    const bool own = l < c.Rk;
    for (int k = 0; k < kClVecs; ++k) c.vec[k * L.Rp + l] = 0.0;
    if (own) {
      c.vec[kVX * L.Rp + l] = a.x[row0 + l];
      c.vec[kVB * L.Rp + l] = a.b[row0 + l];
      c.vec[kVD * L.Rp + l] = a.dinv[row0 + l];
    }
  }
  const unsigned vec0 = smem_u32(c.vec);
  cl_load_rows(a.Arp, a.Aci, a.Ava, L.WA, L.Rp, row0, c.Rk, a.R, a.base, vec0, rank,
               (double*)(cl_smem + L.Av), (unsigned*)(cl_smem + L.Aa));
  cl_load_rows(a.Lrp, a.Lci, a.Lva, L.WL, L.Rp, row0, c.Rk, a.R, a.base, vec0, rank,
               (double*)(cl_smem + L.Lv), (unsigned*)(cl_smem + L.La));
  cl_load_rows(a.Urp, a.Uci, a.Uva, L.WU, L.Rp, row0, c.Rk, a.R, a.base, vec0, rank,
               (double*)(cl_smem + L.Uv), (unsigned*)(cl_smem + L.Ua));
  // every CTA's rows loaded and barrier initialised
  cluster_barrier_hw();
  if (a.cg) cl_cg_solve(c, a, S, part, rank);
  else cl_solve(c, a, S, part, rank);
  const double* x = c.v(kVX);
  CL_ROWS(l) a.x[row0 + l] = x[l];
  // no CTA leaves while another may still read its shared memory
  cluster_barrier_hw();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct ClPlan {
  int C = 0, R = 0, T = 0;
  ClLayout lay{};
};

// the dynamic shared memory a CTA may take (the opt-in limit less the
// kernel's static shared memory), set on the kernel once per process
static size_t cl_smem_limit(gs2_handle* h) {
  static std::once_flag once;
  static size_t limit = 0;
  static cudaError_t failed = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_gmres_cluster);
    const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes
                                                          : 0;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)k_gmres_cluster,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)k_gmres_cluster,
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) limit = lim;
    else failed = e;
  });
  (void)h;
  if (failed != cudaSuccess)
    GS2_THROW(GS2_ERR_CUDA, std::string("cluster kernel setup: ") + cudaGetErrorString(failed));
  return limit;
}

// clusters of C CTAs of T threads with `bytes` of dynamic shared memory that
// fit the GPU at once (cached: the query is made once per shape)
static int cl_resident_clusters(int C, int T, unsigned bytes) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, unsigned>, int> known;
  const auto key = std::make_tuple(C, T, bytes);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = known.find(key);
    if (it != known.end()) return it->second;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)T);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  GS2_CUDA(cudaOccupancyMaxActiveClusters(&clusters, (const void*)k_gmres_cluster, &cfg));
  std::lock_guard<std::mutex> g(mu);
  known[key] = clusters;
  return clusters;
}

static bool cl_kind_ok(int m, const gs2_params* p) {
  if (m < 1 || m > kClMaxRestart) return false;
  if (!p || p->kind == GS2_PC_NONE) return true;
  if (p->parts > 1 || p->local_sweeps > 1) return false;
  if (p->kind == GS2_PC_JR) return true;
  return p->kind == GS2_PC_GS2 && p->precision == GS2_FP64 && p->form == GS2_NONCOMPACT;
}

// The cluster shape of a solve: C CTAs of T threads, R rows each (about
// 128 rows a CTA and at least 16 CTAs' worth of FP64 issue once n allows;
// more CTAs while the rows do not fit), or false when the system does not
// fit one cluster's shared memory.
static bool cluster_plan(gs2_handle* h, int m, const gs2_params* p, ClPlan* out) {
  if (h->n < 1 || h->n > (int64_t)kClMaxCtas * 4096 || !cl_kind_ok(m, p)) return false;
  const bool tri = p && p->kind == GS2_PC_GS2;
  longest_rows(h);
  const size_t limit = cl_smem_limit(h);
  const int n = (int)h->n;
  int C = (int)std::min<int64_t>(kClMaxCtas, std::max<int64_t>(1, (n + 127) / 128));
  for (; C <= kClMaxCtas; ++C) {
    const int R = (n + C - 1) / C;
    const int Cn = (n + R - 1) / R;  // every CTA holds at least one row
    const int Rp = (R + 1) & ~1;
    const ClLayout lay = cl_layout(Rp, h->cl_wa, tri ? h->cl_wl : 0, tri ? h->cl_wu : 0, m);
    if (lay.bytes > limit) continue;
    out->C = Cn;
    out->R = R;
    // one row a thread, 64 to 256 threads: every FP64 dependency costs
    // 64 cycles, so rows taken one after another by a thread cost more than
    // the extra partial sums of more threads
    out->T = R <= 64 ? 64 : (R <= 128 ? 128 : 256);
    out->lay = lay;
    // one cluster of this shape must fit the GPU (its CTAs on SMs of one
    // GPC, each with this much shared memory)
    return cl_resident_clusters(Cn, out->T, lay.bytes) >= 1;
  }
  return false;
}

bool cluster_eligible(gs2_handle* h, int m, const gs2_params* p) {
  ClPlan pl;
  return cluster_plan(h, m, p, &pl);
}

// The outcome of a one-cluster solve from the handle's host copy of the
// device state (read_state, or the asynchronous copy of gmres_cluster_async
// once the stream is idle).
gs2_status cluster_result(gs2_handle* h, gs2_solve_info* info) {
  if (*h->err_host) raise_device_error(h);  // a barrier gave up
  const KrylovState& st = *h->st_host;
  gs2_solve_info loc{st.iters, st.cycles, st.status, 0.0};
  loc.true_relres = st.bnorm == 0.0 ? 0.0 : st.beta / st.bnorm;
  if (info) *info = loc;
  return (gs2_status)st.status;
}

// GMRES(m) (cg = false) or CG (cg = true: three basis slots) in one cluster;
// with info = nullptr only enqueued (the caller copies the state back)
static gs2_status cluster_run(gs2_handle* h, const double* b, double* x, int m, double tol,
                              int max_iters, const gs2_params* p, gs2_solve_info* info,
                              bool cg) {
  ClPlan pl;
  if (!cluster_plan(h, m, p, &pl))
    GS2_THROW(GS2_ERR_INVALID_ARG, "the one-cluster solver takes restart <= 32, no, JR or FP64 "
                                   "non-compact GS2 preconditioning, and a system whose rows "
                                   "fit the shared memory of 16 CTAs");
  ensure_krylov(h, m);  // the device state the result is read from
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  ClusterArgs a{};
  a.n = (int)h->n;
  a.R = pl.R;
  a.C = pl.C;
  a.lay = pl.lay;
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
  a.m = m;
  a.tol = tol;
  a.max_iters = max_iters;
  a.kind = pc ? pc->kind : GS2_PC_NONE;
  a.outer = pc ? std::max(1, pc->outer) : 1;
  a.inner = pc ? pc->inner : 0;
  a.dir = pc ? pc->direction : (cg ? GS2_SYMMETRIC : GS2_FORWARD);
  a.omega = pc ? pc->omega : 1.0;
  a.gamma = pc ? pc->gamma : 1.0;
  a.err = h->dev_err;
  a.out = h->st;
  a.stall = h->stall_barrier ? 1 : 0;
  a.cg = cg ? 1 : 0;
  h->stall_barrier = false;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)pl.C);
  cfg.blockDim = dim3((unsigned)pl.T);
  cfg.dynamicSmemBytes = pl.lay.bytes;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    KernelTimer tm(h, cg ? "cg_cluster" : "gmres_cluster", 0.0);
    GS2_CUDA(cudaLaunchKernelEx(&cfg, k_gmres_cluster, a));
    GS2_LAUNCH_CHECK();
  }
  if (!info) return GS2_OK;  // asynchronous: cluster_result once the stream is idle
  read_state(h);             // raises GS2_ERR_TIMEOUT if a barrier gave up
  return cluster_result(h, info);
}

gs2_status gmres_cluster(gs2_handle* h, const double* b, double* x, int m, double tol,
                         int max_iters, const gs2_params* p, gs2_solve_info* info) {
  gs2_solve_info loc{};
  const gs2_status st = cluster_run(h, b, x, m, tol, max_iters, p, &loc, false);
  if (info) *info = loc;
  return st;
}

void gmres_cluster_async(gs2_handle* h, const double* b, double* x, int m, double tol,
                         int max_iters, const gs2_params* p) {
  cluster_run(h, b, x, m, tol, max_iters, p, nullptr, false);
  copy_state_async(h);
}

// ---------------------------------------------------------------------------
// a pack: one cluster per system, every cluster of the same shape (the
// largest system's rows per CTA), each solving its system's whole GMRES on
// its own -- clusters never wait for one another
// ---------------------------------------------------------------------------

static bool pack_cluster_plan(gs2_handle* h, int m, const gs2_params* p, ClPlan* out,
                              std::vector<ClSys>* sys) {
  const std::vector<int64_t>* offp = pack_offsets(h);
  if (!offp || offp->size() < 2 || !cl_kind_ok(m, p)) return false;
  const std::vector<int64_t>& off = *offp;
  const int S = (int)off.size() - 1;
  int64_t maxn = 0;
  for (int s = 0; s < S; ++s) maxn = std::max(maxn, off[s + 1] - off[s]);
  if (maxn < 1 || maxn > (int64_t)kClMaxCtas * 4096) return false;
  const bool tri = p && p->kind == GS2_PC_GS2;
  longest_rows(h);
  const size_t limit = cl_smem_limit(h);
  // The cluster shape that finishes the pack first: an Arnoldi step takes
  // about 17.4 us + 0.021 us per row of a CTA (measured from 64 to 256
  // rows a CTA), and the systems run in ceil(S / clusters resident at once)
  // waves -- more CTAs a system shorten a step but may hold fewer systems
  // on the GPU at once.
  double best = 0.0;
  bool found = false;
  for (int C = 1; C <= kClMaxCtas; ++C) {
    const int Rmax = (int)((maxn + C - 1) / C);
    const int Rp = (Rmax + 1) & ~1;
    const ClLayout lay = cl_layout(Rp, h->cl_wa, tri ? h->cl_wl : 0, tri ? h->cl_wu : 0, m);
    if (lay.bytes > limit) continue;
    const int T = Rmax <= 64 ? 64 : (Rmax <= 128 ? 128 : 256);
    const int clusters = cl_resident_clusters(C, T, lay.bytes);
    if (clusters < 1) continue;
    const double waves = std::ceil((double)S / clusters);
    const double cost = waves * (17.4 + 0.021 * Rmax);
    if (!found || cost < best) {
      found = true;
      best = cost;
      out->C = C;
      out->R = Rmax;
      out->T = T;
      out->lay = lay;
    }
  }
  if (!found) return false;
  const int C = out->C;
  sys->resize(S);
  for (int s = 0; s < S; ++s) {
    const int n = (int)(off[s + 1] - off[s]);
    (*sys)[s] = ClSys{(int)off[s], n, std::max(1, (n + C - 1) / C), nullptr};
  }
  return true;
}

bool pack_cluster_eligible(gs2_handle* h, int m, const gs2_params* p) {
  ClPlan pl;
  std::vector<ClSys> sys;
  return pack_cluster_plan(h, m, p, &pl, &sys);
}

gs2_status pack_gmres_cluster(gs2_handle* h, const double* b, double* x, int m, double tol,
                              int max_iters, const gs2_params* p, gs2_solve_info* infos) {
  ClPlan pl;
  std::vector<ClSys> sys;
  if (!pack_cluster_plan(h, m, p, &pl, &sys))
    GS2_THROW(GS2_ERR_INVALID_ARG, "one cluster per system: restart <= 32, no, JR or FP64 "
                                   "non-compact GS2 preconditioning, and systems whose rows "
                                   "fit the shared memory of 16 CTAs");
  ensure_krylov(h, m);
  const int S = (int)sys.size();
  if (S > h->pp_cap_sys || !h->cl_sys) {
    const int cs = std::max(S, h->pp_cap_sys);
    if (S > h->pp_cap_sys) {
      h->pp_st = (KrylovState*)h->dalloc(sizeof(KrylovState) * cs);
      if (h->pp_st_host) pinned_put(h->pp_st_host, sizeof(KrylovState) * h->pp_cap_sys);
      h->pp_st_host = (KrylovState*)pinned_get(sizeof(KrylovState) * cs);
      h->pp_cap_sys = cs;
    }
  }
  if (S > h->cl_sys_cap) {
    h->cl_sys = h->dalloc(sizeof(ClSys) * S);
    h->cl_sys_cap = S;
  }
  for (int s = 0; s < S; ++s) sys[s].out = h->pp_st + s;
  h->h2d(h->cl_sys, sys.data(), sizeof(ClSys) * S);
  const gs2_params* pc = (p && p->kind != GS2_PC_NONE) ? p : nullptr;
  ClusterArgs a{};
  a.C = pl.C;
  a.lay = pl.lay;
  a.sys = (const ClSys*)h->cl_sys;
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
  a.m = m;
  a.tol = tol;
  a.max_iters = max_iters;
  a.kind = pc ? pc->kind : GS2_PC_NONE;
  a.outer = pc ? std::max(1, pc->outer) : 1;
  a.inner = pc ? pc->inner : 0;
  a.dir = pc ? pc->direction : GS2_FORWARD;
  a.omega = pc ? pc->omega : 1.0;
  a.gamma = pc ? pc->gamma : 1.0;
  a.err = h->dev_err;
  a.out = h->pp_st;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(pl.C * S));
  cfg.blockDim = dim3((unsigned)pl.T);
  cfg.dynamicSmemBytes = pl.lay.bytes;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    KernelTimer tm(h, "gmres_cluster", 0.0);
    GS2_CUDA(cudaLaunchKernelEx(&cfg, k_gmres_cluster, a));
    GS2_LAUNCH_CHECK();
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

gs2_status cg_cluster(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                      const gs2_params* p, gs2_solve_info* info) {
  gs2_solve_info loc{};
  const gs2_status st = cluster_run(h, b, x, 2, tol, max_iters, p, &loc, true);
  if (info) *info = loc;
  return st;
}

}  // namespace gs2
