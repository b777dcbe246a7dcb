// Row kernels of the two-stage Gauss-Seidel library (sm_103a).
//
// Every sweep is a CSR row reduction followed by a per-row epilogue:
//   residual      r = b - A x, rhat = D^{-1} r              (Eq. 4, Eq. 5)
//   inner sweep   g' = (1-gamma) g + gamma (rhat - omega T g)  (Eq. 6-7,
//                 damped form of Sec. 3), the last one fused with
//                 x += omega g'
//   JR            x' = x + omega D^{-1} (b - A x)           (Sec. 3)
//   SpMV          y = A x
//
// Design (GB300): FP64 throughput on this part is ~2 FMA/clk/SM, so a
// warp-per-row reduction (whose shuffle-add tree runs on every lane) would
// spend more FP64 issue slots on the tree than on the products.  Rows are
// therefore reduced sequentially by one thread (or by K contiguous segments
// for long rows), with the row's values and column indices staged into
// shared memory by coalesced 128-bit streaming loads, one tile of
// consecutive rows per block iteration.  x-gathers go through the
// read-only path and stay L2-resident.
#include <cuda_fp16.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace gs2 {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

template <int K, typename T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
  for (int o = K / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, K);
  return s;
}

template <typename T>
__device__ __forceinline__ T block_sum(T s, T* red) {
  // deterministic: fixed shuffle tree inside warps, then warp 0 over warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if (lane == 0) red[wid] = s;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (wid == 0) {
    s = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

template <typename VT>
struct ValTraits;
template <>
struct ValTraits<double> {
  using AT = double;
  __device__ static double get(const double* p, int k) { return p[k]; }
};
template <>
struct ValTraits<float> {
  using AT = float;
  __device__ static float get(const float* p, int k) { return p[k]; }
};
template <>
struct ValTraits<__half> {
  using AT = float;
  __device__ static float get(const __half* p, int k) { return __half2float(p[k]); }
};

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ / sm_103a)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's (and, after a barrier, the block's) generic-proxy
// accesses of shared memory before later async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(tx)
               : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 1-D bulk copy global -> shared, completion counted on `bar` in bytes;
// src and dst 16-byte aligned, bytes a positive multiple of 16
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s of SM clock so that a wrong transaction
// count can never hang the GPU; the caller reports GS2_ERR_TIMEOUT.
constexpr long long kWaitBudgetCycles = 4LL << 30;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitBudgetCycles) return false;
  return true;
}

// ---------------------------------------------------------------------------
// tile engine
// ---------------------------------------------------------------------------

// Matrix view for the engine.  Tile t = rows [d.x, d.y) with d = desc[t];
// d.z = first staged entry (rowptr[d.x] rounded down to 8) and d.w =
// rowptr[d.y]; a tile holding one row longer than `cap` entries has
// d.z = -1 - rowptr[d.x] and is processed from global memory by the block.
template <typename VT>
struct TileMat {
  int n;
  int ntiles;
  int cap;   // max staged entries of a normal tile (multiple of 8)
  int rcap;  // max rows of a tile
  const int* __restrict__ rp;
  const int* __restrict__ ci;
  const VT* __restrict__ va;
  const int4* __restrict__ desc;
  int* err;  // set to GS2_ERR_TIMEOUT if a copy never completes
};

__host__ __device__ constexpr int round16(int b) { return (b + 15) & ~15; }

template <typename VT>
struct StageLayout {
  int rp_off, ci_off, va_off, bytes;
  __host__ __device__ StageLayout(int rcap, int cap) {
    rp_off = 0;
    ci_off = round16((rcap + 8) * 4);
    va_off = ci_off + round16((cap + 8) * 4);
    bytes = ((va_off + round16((cap + 8) * (int)sizeof(VT))) + 127) & ~127;
  }
};

// Engine: for every row i, acc_i = sum_k va[k] * epi.gather(ci[k]), then
// epi.finish(i, acc_i).  Double-buffered: while the block reduces tile t
// from one shared-memory stage, one thread has TMA fill the other stage
// with tile t + grid (its rowptr slice, columns and values), completion
// tracked by one mbarrier per stage.  Rows are reduced by one thread each
// (K = 1) or by K contiguous segments and a K-wide shuffle tree; each group
// of K lanes takes RPT rows of a tile (RPT * 256 / K rows per tile).  The
// epilogue's per-row operands are loaded before the gathers.
template <int K, int RPT, typename VT, class Epi>
__global__ void __launch_bounds__(kRowThreads)
k_tiles(TileMat<VT> M, Epi epi, const int* skip) {
  using AT = typename ValTraits<VT>::AT;
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ AT red[kRowThreads / 32];
  const StageLayout<VT> L(M.rcap, M.cap);
  const int q = threadIdx.x / K;  // row slot inside the tile
  const int l = threadIdx.x % K;  // segment of the row
  uint64_t policy = 0;

  // thread 0: describe and start the copies of tile t into stage st
  auto issue = [&](int t, int st) {
    const int4 d = M.desc[t];
    unsigned char* base = smem_raw + (size_t)st * L.bytes;
    uint32_t tx = 0;
    uint32_t brp = 0, bci = 0, bva = 0;
    if (d.z >= 0) {
      const int rpb = d.x & ~3;
      brp = (uint32_t)round16((d.y + 1 - rpb) * 4);
      const int cnt = d.w - d.z;
      bci = (uint32_t)round16(cnt * 4);
      bva = cnt > 0 ? (uint32_t)round16(cnt * (int)sizeof(VT)) : 0u;
      if (cnt == 0) bci = 0;
      tx = brp + bci + bva;
    }
    mbar_arrive_expect_tx(&bars[st], tx);
    if (d.z >= 0) {
      tma_load_1d(base + L.rp_off, M.rp + (d.x & ~3), brp, &bars[st], policy);
      if (bci) tma_load_1d(base + L.ci_off, M.ci + d.z, bci, &bars[st], policy);
      if (bva) tma_load_1d(base + L.va_off, M.va + d.z, bva, &bars[st], policy);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    policy = l2_evict_first_policy();
    if ((int)blockIdx.x < M.ntiles) issue(blockIdx.x, 0);
  }
  __syncthreads();

  int it = 0;
  for (int t = blockIdx.x; t < M.ntiles; t += gridDim.x, ++it) {
    const int st = it & 1;
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < M.ntiles) {
      fence_proxy_async_smem();
      issue(tn, st ^ 1);
    }
    const int4 d = M.desc[t];
    const bool ok = mbar_wait_bounded(&bars[st], (it >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0 && M.err) atomicExch(M.err, (int)GS2_ERR_TIMEOUT);
      return;
    }
    if (d.z < 0) {
      // one long row: whole block, straight from global memory
      const int a = -1 - d.z;
      AT s = AT(0);
      for (int k = a + threadIdx.x; k < d.w; k += blockDim.x)
        s = fma((AT)ValTraits<VT>::get(M.va, k), (AT)epi.gather(M.ci[k]), s);
      s = block_sum<AT>(s, red);
      if (threadIdx.x == 0) epi.finish(d.x, s, epi.pre(d.x));
      __syncthreads();
      continue;
    }
    const unsigned char* base = smem_raw + (size_t)st * L.bytes;
    const int* s_rp = reinterpret_cast<const int*>(base + L.rp_off);
    const int* s_ci = reinterpret_cast<const int*>(base + L.ci_off);
    const VT* s_va = reinterpret_cast<const VT*>(base + L.va_off);
    const int rpb = d.x & ~3;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int row = d.x + q + rr * (kRowThreads / K);
      AT s = AT(0);
      typename Epi::Pre pv{};
      if (row < d.y) {
        pv = epi.pre(row);
        const int rs = s_rp[row - rpb] - d.z, re = s_rp[row + 1 - rpb] - d.z;
        int ks = rs, ke = re;
        if (K > 1) {
          const int seg = (re - rs + K - 1) / K;
          ks = min(rs + l * seg, re);
          ke = min(ks + seg, re);
        }
        int k = ks;
        // groups of four: all four gathers are in flight before the FMAs
        for (; k + 4 <= ke; k += 4) {
          const AT x0 = (AT)epi.gather(s_ci[k]), x1 = (AT)epi.gather(s_ci[k + 1]);
          const AT x2 = (AT)epi.gather(s_ci[k + 2]), x3 = (AT)epi.gather(s_ci[k + 3]);
          s = fma((AT)ValTraits<VT>::get(s_va, k), x0, s);
          s = fma((AT)ValTraits<VT>::get(s_va, k + 1), x1, s);
          s = fma((AT)ValTraits<VT>::get(s_va, k + 2), x2, s);
          s = fma((AT)ValTraits<VT>::get(s_va, k + 3), x3, s);
        }
        const int rem = ke - k;
        if (rem > 0) {
          const AT x0 = (AT)epi.gather(s_ci[k]);
          const AT x1 = rem > 1 ? (AT)epi.gather(s_ci[k + 1]) : AT(0);
          const AT x2 = rem > 2 ? (AT)epi.gather(s_ci[k + 2]) : AT(0);
          s = fma((AT)ValTraits<VT>::get(s_va, k), x0, s);
          if (rem > 1) s = fma((AT)ValTraits<VT>::get(s_va, k + 1), x1, s);
          if (rem > 2) s = fma((AT)ValTraits<VT>::get(s_va, k + 2), x2, s);
        }
      }
      if (K > 1) s = group_sum<K, AT>(s);
      if (row < d.y && l == 0) epi.finish(row, s, pv);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// epilogues: pre(i) loads the row's operands before the gathers, finish(i,
// s, pre) consumes the row sum
// ---------------------------------------------------------------------------

// r = b - A x;  rhat = D^{-1} r   (Eq. 4 residual and Eq. 5 initial guess)
struct EpiResid {
  const double* __restrict__ x;
  const double* __restrict__ b;
  const double* __restrict__ dinv;
  double* __restrict__ r;
  double* __restrict__ rhat64;
  float* __restrict__ rhat32;
  struct Pre {
    double b, d;
  };
  __device__ Pre pre(int i) const { return Pre{b[i], dinv[i]}; }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s, const Pre& p) const {
    const double ri = p.b - s;
    const double rh = p.d * ri;
    if (r) r[i] = ri;
    if (rhat64) rhat64[i] = rh;
    if (rhat32) rhat32[i] = (float)rh;
  }
};

struct EpiSpmv {
  const double* __restrict__ x;
  double* __restrict__ y;
  struct Pre {};
  __device__ Pre pre(int) const { return Pre{}; }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s, const Pre&) const { y[i] = s; }
};

// y += M x (multigrid prolongation)
struct EpiSpmvAdd {
  const double* __restrict__ x;
  double* __restrict__ y;
  struct Pre {
    double y;
  };
  __device__ Pre pre(int i) const { return Pre{y[i]}; }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s, const Pre& p) const { y[i] = p.y + s; }
};

// x_out = x_in + omega D^{-1} (b - A x_in)   (damped JR, ping-pong buffers)
struct EpiJr {
  const double* __restrict__ x;
  const double* __restrict__ b;
  const double* __restrict__ dinv;
  double* __restrict__ x_out;
  double omega;
  struct Pre {
    double x, b, d;
  };
  __device__ Pre pre(int i) const { return Pre{x[i], b[i], dinv[i]}; }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s, const Pre& p) const {
    x_out[i] = p.x + omega * (p.d * (p.b - s));
  }
};

// inner JR sweep on the prescaled triangle T = D^{-1} L or D^{-1} U:
//   g' = (1-gamma) g + gamma (rhat - omega T g)
// DAMPED and SCALED (FP16 triangles with a per-row scale) are compile-time:
// a runtime flag on a uniform kernel argument is predicated, and its FP64
// instructions would then issue on every row.
template <typename GT, typename AT, bool DAMPED, bool SCALED>
struct EpiInner {
  const GT* __restrict__ g_in;
  const GT* __restrict__ rhat;
  GT* __restrict__ g_out;
  double* __restrict__ x;
  const float* __restrict__ rowscale;  // FP16 triangles only
  AT omega, gamma;
  double omega64;
  int mode;
  struct Pre {
    AT rh, gi, sc;
    double xi;
  };
  __device__ Pre pre(int i) const {
    Pre p;
    p.rh = (AT)rhat[i];
    p.gi = DAMPED ? (AT)g_in[i] : AT(0);
    p.sc = SCALED ? (AT)rowscale[i] : AT(1);
    p.xi = mode == INNER_LAST_ADD ? x[i] : 0.0;
    return p;
  }
  __device__ AT gather(int c) const { return (AT)__ldg(g_in + c); }
  __device__ void finish(int i, AT s, const Pre& p) const {
    if (SCALED) s *= p.sc;
    AT go = p.rh - omega * s;
    if (DAMPED) go = (AT(1) - gamma) * p.gi + gamma * go;
    if (mode == INNER_MID) g_out[i] = (GT)go;
    else if (mode == INNER_LAST_ADD) x[i] = p.xi + omega64 * (double)go;
    else x[i] = omega64 * (double)go;
  }
};

// one colour of multicolour GS (Sec. 5.1.2): the colour matrix holds only
// off-diagonal entries prescaled by D^{-1}, none of them inside the colour,
// so every x_j gathered here belongs to another colour and is not written
// by this launch; row i of the colour is row rows[i] of A.
//   x_r = (1 - omega) x_r + omega (bhat_r - sum_j (a_rj / a_rr) x_j)
template <bool DAMPED>
struct EpiColor {
  const int* __restrict__ rows;
  const double* __restrict__ bhat;
  double* x;
  double omega;
  struct Pre {
    int r;
    double bh, xr;
  };
  __device__ Pre pre(int i) const {
    Pre p;
    p.r = rows[i];
    p.bh = bhat[p.r];
    p.xr = DAMPED ? x[p.r] : 0.0;
    return p;
  }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int, double s, const Pre& p) const {
    const double gs = p.bh - s;
    x[p.r] = DAMPED ? p.xr + omega * (gs - p.xr) : gs;
  }
};

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------

// Resident blocks per SM of a tile kernel at a dynamic shared-memory size,
// queried once per (kernel, size) and cached (the query and the attribute
// call cost microseconds of host time per launch otherwise).  The dynamic
// shared-memory limit is one attribute per kernel, so it is only ever
// raised: matrices with smaller tiles keep launching under the larger limit.
static int blocks_per_sm(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> cache;
  static std::map<const void*, size_t> attr;
  std::lock_guard<std::mutex> g(mu);
  auto key = std::make_pair(fn, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  // the default 48 KB limit covers static + dynamic shared memory, so opt in
  // well before the dynamic part alone reaches it
  if (smem > 32 * 1024 && smem > attr[fn]) {
    GS2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[fn] = smem;
  }
  int per_sm = 0;
  GS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRowThreads, smem));
  if (per_sm < 1) per_sm = 1;
  cache[key] = per_sm;
  return per_sm;
}

template <typename VT>
static TileMat<VT> view(gs2_handle* h, const DevCsr& M, const VT* va) {
  TileMat<VT> t;
  t.n = M.n;
  t.ntiles = M.ntiles;
  t.cap = M.cap;
  t.rcap = M.rpt * kRowThreads / M.tpr;
  t.rp = M.rp;
  t.ci = M.ci;
  t.va = va;
  t.desc = M.desc;
  t.err = h->dev_err;
  return t;
}

template <int K, int RPT, typename VT, class Epi>
static void launch_k(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  if (M.n == 0 || M.ntiles == 0) return;
  const size_t smem = 2 * (size_t)StageLayout<VT>(RPT * kRowThreads / K, M.cap).bytes;
  auto fn = k_tiles<K, RPT, VT, Epi>;
  const int per_sm = blocks_per_sm((const void*)fn, smem);
  const int grid = std::min(M.ntiles, per_sm * h->nsm);
  fn<<<grid, kRowThreads, smem, h->stream>>>(view<VT>(h, M, va), epi, skip);
  GS2_LAUNCH_CHECK();
}

// (K, RPT) shapes: RPT = 2 only for short rows (K <= 2), where the per-tile
// barrier and stage overhead is largest relative to the work per row
template <typename VT, class Epi>
static void dispatch(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  switch (M.tpr * 4 + (M.rpt == 2 ? 1 : 0)) {
    case 1 * 4 + 1: launch_k<1, 2, VT, Epi>(h, M, va, epi, skip); break;
    case 2 * 4 + 1: launch_k<2, 2, VT, Epi>(h, M, va, epi, skip); break;
    case 1 * 4: launch_k<1, 1, VT, Epi>(h, M, va, epi, skip); break;
    case 2 * 4: launch_k<2, 1, VT, Epi>(h, M, va, epi, skip); break;
    case 4 * 4: launch_k<4, 1, VT, Epi>(h, M, va, epi, skip); break;
    case 8 * 4: launch_k<8, 1, VT, Epi>(h, M, va, epi, skip); break;
    default: launch_k<16, 1, VT, Epi>(h, M, va, epi, skip); break;
  }
}

static double bytes_csr(const DevCsr& M, int vbytes) {
  return (double)M.nnz * (4.0 + vbytes) + 4.0 * (M.n + 1);
}

void launch_resid(gs2_handle* h, const double* b, const double* x, double* r_out,
                  double* rhat64, float* rhat32, const int* skip) {
  // algorithmic bytes: A once, x, b, D^{-1} read, r / rhat written
  KernelTimer tm(h, "resid", bytes_csr(h->A, 8) + 24.0 * h->n + (r_out ? 8.0 * h->n : 0.0) +
                 (rhat64 ? 8.0 * h->n : 0.0) + (rhat32 ? 4.0 * h->n : 0.0));
  EpiResid e{x, b, h->dinv, r_out, rhat64, rhat32};
  dispatch<double>(h, h->A, h->A.va, e, skip);
}

void launch_spmv(gs2_handle* h, const double* x, double* y, const int* skip) {
  KernelTimer tm(h, "spmv", bytes_csr(h->A, 8) + 16.0 * h->n);
  EpiSpmv e{x, y};
  dispatch<double>(h, h->A, h->A.va, e, skip);
}

void launch_spmv_matrix(gs2_handle* h, const DevCsr& M, const double* x, double* y,
                        bool accumulate, const int* skip) {
  KernelTimer tm(h, accumulate ? "amg_prolong" : "amg_restrict",
                 bytes_csr(M, 8) + 8.0 * M.n * (accumulate ? 3.0 : 2.0));
  if (accumulate) {
    EpiSpmvAdd e{x, y};
    dispatch<double>(h, M, M.va, e, skip);
  } else {
    EpiSpmv e{x, y};
    dispatch<double>(h, M, M.va, e, skip);
  }
}

// Autotuner probe: milliseconds per launch of y = M x over M's FP64 values
// with M's current tile shape (x = h->t, y = h->z), best of `reps`.
float time_tile_probe(gs2_handle* h, const DevCsr& M, int reps) {
  EpiSpmv e{h->t, h->z};
  cudaEvent_t e0, e1;
  GS2_CUDA(cudaEventCreate(&e0));
  GS2_CUDA(cudaEventCreate(&e1));
  dispatch<double>(h, M, M.va, e, nullptr);  // warm-up (occupancy query, L2)
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    GS2_CUDA(cudaEventRecord(e0, h->stream));
    dispatch<double>(h, M, M.va, e, nullptr);
    GS2_CUDA(cudaEventRecord(e1, h->stream));
    GS2_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    GS2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void launch_jr(gs2_handle* h, const double* b, const double* x_in, double* x_out,
               double omega, const int* skip) {
  KernelTimer tm(h, "jr", bytes_csr(h->A, 8) + 32.0 * h->n);
  EpiJr e{x_in, b, h->dinv, x_out, omega};
  dispatch<double>(h, h->A, h->A.va, e, skip);
}

void launch_inner(gs2_handle* h, const DevCsr& T, int prec, const void* rhat,
                  const void* g_in, void* g_out, double* x, double omega, double gamma,
                  int mode, const int* skip) {
  const bool damped = gamma != 1.0;
  const double vb = prec == GS2_FP64 ? 8.0 : (prec == GS2_FP32 ? 4.0 : 2.0);
  const double gb = prec == GS2_FP64 ? 8.0 : 4.0;
  double bytes = bytes_csr(T, (int)vb) + gb * T.n * (2 + (damped ? 1 : 0)) +
                 (mode == INNER_MID ? gb * T.n : (mode == INNER_LAST_ADD ? 16.0 : 8.0) * T.n) +
                 (prec == GS2_FP16_ROWSCALED ? 4.0 * T.n : 0.0);
  KernelTimer tm(h, prec == GS2_FP64 ? "inner64" : (prec == GS2_FP32 ? "inner32" : "inner16"),
                 bytes);
  if (prec == GS2_FP64) {
    if (damped) {
      EpiInner<double, double, true, false> e{(const double*)g_in, (const double*)rhat,
                                              (double*)g_out, x, nullptr, omega, gamma, omega,
                                              mode};
      dispatch<double>(h, T, T.va, e, skip);
    } else {
      EpiInner<double, double, false, false> e{(const double*)g_in, (const double*)rhat,
                                               (double*)g_out, x, nullptr, omega, gamma, omega,
                                               mode};
      dispatch<double>(h, T, T.va, e, skip);
    }
  } else if (prec == GS2_FP32) {
    if (damped) {
      EpiInner<float, float, true, false> e{(const float*)g_in, (const float*)rhat,
                                            (float*)g_out, x, nullptr, (float)omega,
                                            (float)gamma, omega, mode};
      dispatch<float>(h, T, T.va32, e, skip);
    } else {
      EpiInner<float, float, false, false> e{(const float*)g_in, (const float*)rhat,
                                             (float*)g_out, x, nullptr, (float)omega,
                                             (float)gamma, omega, mode};
      dispatch<float>(h, T, T.va32, e, skip);
    }
  } else {
    if (damped) {
      EpiInner<float, float, true, true> e{(const float*)g_in, (const float*)rhat,
                                           (float*)g_out, x, T.scale16, (float)omega,
                                           (float)gamma, omega, mode};
      dispatch<__half>(h, T, T.va16, e, skip);
    } else {
      EpiInner<float, float, false, true> e{(const float*)g_in, (const float*)rhat,
                                            (float*)g_out, x, T.scale16, (float)omega,
                                            (float)gamma, omega, mode};
      dispatch<__half>(h, T, T.va16, e, skip);
    }
  }
}

void launch_color(gs2_handle* h, const DevCsr& C, const int* rows, const double* bhat,
                  double* x, double omega, const int* skip) {
  const bool damped = omega != 1.0;
  // colour matrix once; per row its index, bhat, the written x and (lower
  // bound) one gathered x of another colour; damping re-reads x_r
  KernelTimer tm(h, "color", bytes_csr(C, 8) + C.n * (28.0 + (damped ? 8.0 : 0.0)));
  if (damped) {
    EpiColor<true> e{rows, bhat, x, omega};
    dispatch<double>(h, C, C.va, e, skip);
  } else {
    EpiColor<false> e{rows, bhat, x, omega};
    dispatch<double>(h, C, C.va, e, skip);
  }
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------

__global__ void k_prep_rhat(int n, const double* __restrict__ v,
                            const double* __restrict__ dinv, double* rhat64, float* rhat32,
                            const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double rh = dinv[i] * v[i];
    if (rhat64) rhat64[i] = rh;
    if (rhat32) rhat32[i] = (float)rh;
  }
}

template <typename GT>
__global__ void k_rhat_update(int n, const GT* __restrict__ rhat, double* x, double omega,
                              int add, const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double u = omega * (double)rhat[i];
    x[i] = add ? x[i] + u : u;
  }
}

__global__ void k_axpy(int n, double* y, double a, const double* __restrict__ x,
                       const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

int vec_blocks(gs2_handle* h, int64_t n) {
  const int64_t need = (n + kVecThreads - 1) / kVecThreads;
  const int64_t cap = (int64_t)h->nsm * 8;
  return (int)std::max<int64_t>(1, std::min(need, cap));
}

void launch_prep_rhat(gs2_handle* h, const double* v, double* rhat64, float* rhat32,
                      const int* skip) {
  if (h->n == 0) return;
  KernelTimer tm(h, "prep_rhat", 16.0 * h->n + (rhat64 ? 8.0 : 4.0) * h->n);
  k_prep_rhat<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>(
      (int)h->n, v, h->dinv, rhat64, rhat32, skip);
  GS2_LAUNCH_CHECK();
}

void launch_rhat_update(gs2_handle* h, int prec, const void* rhat, double* x, double omega,
                        bool add, const int* skip) {
  if (h->n == 0) return;
  KernelTimer tm(h, "rhat_update", (prec == GS2_FP64 ? 8.0 : 4.0) * h->n +
                 (add ? 16.0 : 8.0) * h->n);
  if (prec == GS2_FP64)
    k_rhat_update<double><<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>(
        (int)h->n, (const double*)rhat, x, omega, add ? 1 : 0, skip);
  else
    k_rhat_update<float><<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>(
        (int)h->n, (const float*)rhat, x, omega, add ? 1 : 0, skip);
  GS2_LAUNCH_CHECK();
}

void launch_axpy(gs2_handle* h, double* y, double a, const double* x, const int* skip) {
  if (h->n == 0) return;
  KernelTimer tm(h, "axpy", 24.0 * h->n);
  k_axpy<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>((int)h->n, y, a, x, skip);
  GS2_LAUNCH_CHECK();
}

void launch_copy(gs2_handle* h, double* dst, const double* src) {
  if (h->n == 0 || dst == src) return;
  GS2_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * h->n, cudaMemcpyDeviceToDevice,
                           h->stream));
}

// ---------------------------------------------------------------------------
// level-scheduled triangular solve (exact GS baseline)
// ---------------------------------------------------------------------------

// Rows of one level are independent: g_i = rhat_i - omega sum_k T_ik g_k over
// dependencies k in earlier levels (final already), then x_i += omega g_i.
// This is the forward recurrence of (D + omega L) g = r scaled by D^{-1}.
template <int K>
__global__ void __launch_bounds__(kRowThreads)
k_level(const int* __restrict__ rows, int r0, int r1, const int* __restrict__ rp,
        const int* __restrict__ ci, const double* __restrict__ va,
        const double* __restrict__ rhat, double* g, double* x, double omega,
        const int* skip) {
  if (skip && *skip) return;
  const int q = threadIdx.x / K, l = threadIdx.x % K;
  constexpr int G = kRowThreads / K;
  for (int base = r0 + blockIdx.x * G; base < r1; base += gridDim.x * G) {
    const int idx = base + q;
    double s = 0.0;
    int row = -1;
    if (idx < r1) {
      row = rows[idx];
      for (int k = rp[row] + l; k < rp[row + 1]; k += K) s = fma(va[k], g[ci[k]], s);
    }
    s = group_sum<K, double>(s);
    if (row >= 0 && l == 0) {
      const double gi = rhat[row] - omega * s;
      g[row] = gi;
      x[row] += omega * gi;
    }
  }
}

void launch_level(gs2_handle* h, const DevCsr& T, const int* rows, int r0, int r1,
                  const double* rhat, double* g, double* x, double omega,
                  const int* skip) {
  const int cnt = r1 - r0;
  if (cnt <= 0) return;
  const int K = T.tpr >= 8 ? 8 : 1;
  const int G = kRowThreads / K;
  const int grid = std::max(1, std::min((cnt + G - 1) / G, h->nsm * 8));
  if (K == 8)
    k_level<8><<<grid, kRowThreads, 0, h->stream>>>(rows, r0, r1, T.rp, T.ci, T.va, rhat, g,
                                                    x, omega, skip);
  else
    k_level<1><<<grid, kRowThreads, 0, h->stream>>>(rows, r0, r1, T.rp, T.ci, T.va, rhat, g,
                                                    x, omega, skip);
  GS2_LAUNCH_CHECK();
}

}  // namespace gs2
