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

// streaming 16-byte load (read once: evict-first in L2, no L1 allocation)
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }

// ---------------------------------------------------------------------------
// tile engine
// ---------------------------------------------------------------------------

// Matrix view for the engine.  Tiles: rows [tile_row[t], tile_row[t+1]);
// a tile holding one row longer than `cap` entries is processed from global
// memory by the whole block.
template <typename VT>
struct TileMat {
  int n;
  int ntiles;
  int cap;  // max staged entries of a normal tile (multiple of 8)
  const int* __restrict__ rp;
  const int* __restrict__ ci;
  const VT* __restrict__ va;
  const int* __restrict__ tile_row;
};

// Engine: for every row i, acc_i = sum_k va[k] * epi.gather(ci[k]), then
// epi.finish(i, acc_i).  K lanes per row, each summing one contiguous
// segment of the row, combined by a K-wide shuffle tree.
template <int K, typename VT, class Epi>
__global__ void __launch_bounds__(kRowThreads)
k_tiles(TileMat<VT> M, Epi epi, const int* skip) {
  using AT = typename ValTraits<VT>::AT;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_ci = reinterpret_cast<int*>(smem_raw);
  VT* s_va = reinterpret_cast<VT*>(smem_raw + (size_t)(M.cap + 8) * sizeof(int));
  __shared__ AT red[kRowThreads / 32];

  const int q = threadIdx.x / K;  // row slot inside the tile
  const int l = threadIdx.x % K;  // segment of the row

  for (int t = blockIdx.x; t < M.ntiles; t += gridDim.x) {
    const int r0 = M.tile_row[t], r1 = M.tile_row[t + 1];
    const int a = M.rp[r0], b = M.rp[r1];
    if (b - a > M.cap) {
      // one long row: whole block, straight from global memory
      AT s = AT(0);
      for (int k = a + threadIdx.x; k < b; k += blockDim.x)
        s = fma((AT)ValTraits<VT>::get(M.va, k), (AT)epi.gather(M.ci[k]), s);
      s = block_sum<AT>(s, red);
      if (threadIdx.x == 0) epi.finish(r0, s);
      __syncthreads();
      continue;
    }
    // stage col and val of the tile, aligned down to 8 entries so that
    // every 16-byte vector load is aligned (arrays are padded at the end)
    const int a0 = a & ~7;
    const int cnt = b - a0;
    {
      const int nci = (cnt + 3) >> 2;
      const int4* src = reinterpret_cast<const int4*>(M.ci + a0);
      int4* dst = reinterpret_cast<int4*>(s_ci);
      for (int v = threadIdx.x; v < nci; v += blockDim.x) dst[v] = ld_stream(src + v);
      constexpr int per = 16 / sizeof(VT);
      const int nva = (cnt + per - 1) / per;
      const int4* srcv = reinterpret_cast<const int4*>(M.va + a0);
      int4* dstv = reinterpret_cast<int4*>(s_va);
      for (int v = threadIdx.x; v < nva; v += blockDim.x) dstv[v] = ld_stream(srcv + v);
    }
    __syncthreads();
    const int row = r0 + q;
    AT s = AT(0);
    if (row < r1) {
      const int rs = M.rp[row] - a0, re = M.rp[row + 1] - a0;
      int ks = rs, ke = re;
      if (K > 1) {
        const int seg = (re - rs + K - 1) / K;
        ks = min(rs + l * seg, re);
        ke = min(ks + seg, re);
      }
      for (int k = ks; k < ke; ++k)
        s = fma((AT)ValTraits<VT>::get(s_va, k), (AT)epi.gather(s_ci[k]), s);
    }
    if (K > 1) s = group_sum<K, AT>(s);
    if (row < r1 && l == 0) epi.finish(row, s);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// epilogues
// ---------------------------------------------------------------------------

// r = b - A x;  rhat = D^{-1} r   (Eq. 4 residual and Eq. 5 initial guess)
struct EpiResid {
  const double* __restrict__ x;
  const double* __restrict__ b;
  const double* __restrict__ dinv;
  double* __restrict__ r;
  double* __restrict__ rhat64;
  float* __restrict__ rhat32;
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s) const {
    const double ri = b[i] - s;
    const double rh = dinv[i] * ri;
    if (r) r[i] = ri;
    if (rhat64) rhat64[i] = rh;
    if (rhat32) rhat32[i] = (float)rh;
  }
};

struct EpiSpmv {
  const double* __restrict__ x;
  double* __restrict__ y;
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s) const { y[i] = s; }
};

// x_out = x_in + omega D^{-1} (b - A x_in)   (damped JR, ping-pong buffers)
struct EpiJr {
  const double* __restrict__ x;
  const double* __restrict__ b;
  const double* __restrict__ dinv;
  double* __restrict__ x_out;
  double omega;
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s) const {
    x_out[i] = x[i] + omega * (dinv[i] * (b[i] - s));
  }
};

// inner JR sweep on the prescaled triangle T = D^{-1} L or D^{-1} U:
//   g' = (1-gamma) g + gamma (rhat - omega T g)
template <typename GT, typename AT>
struct EpiInner {
  const GT* __restrict__ g_in;
  const GT* __restrict__ rhat;
  GT* __restrict__ g_out;
  double* __restrict__ x;
  const float* __restrict__ rowscale;  // FP16 triangles only
  AT omega, gamma;
  double omega64;
  int mode;
  int damped;
  __device__ AT gather(int c) const { return (AT)__ldg(g_in + c); }
  __device__ void finish(int i, AT s) const {
    if (rowscale) s *= (AT)rowscale[i];
    AT go = (AT)rhat[i] - omega * s;
    if (damped) go = (AT(1) - gamma) * (AT)g_in[i] + gamma * go;
    if (mode == INNER_MID) g_out[i] = (GT)go;
    else if (mode == INNER_LAST_ADD) x[i] += omega64 * (double)go;
    else x[i] = omega64 * (double)go;
  }
};

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------

// Resident blocks per SM of a tile kernel at a dynamic shared-memory size,
// queried once per (kernel, size) and cached (the query and the attribute
// call cost microseconds of host time per launch otherwise).
static int blocks_per_sm(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto key = std::make_pair(fn, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (smem > 48 * 1024)
    GS2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRowThreads, smem));
  if (per_sm < 1) per_sm = 1;
  cache[key] = per_sm;
  return per_sm;
}

template <typename VT>
static TileMat<VT> view(const DevCsr& M, const VT* va) {
  TileMat<VT> t;
  t.n = M.n;
  t.ntiles = M.ntiles;
  t.cap = M.cap;
  t.rp = M.rp;
  t.ci = M.ci;
  t.va = va;
  t.tile_row = M.tile_row;
  return t;
}

template <int K, typename VT, class Epi>
static void launch_k(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  if (M.n == 0 || M.ntiles == 0) return;
  const size_t smem = (size_t)(M.cap + 8) * (sizeof(int) + sizeof(VT)) + 16;
  auto fn = k_tiles<K, VT, Epi>;
  const int per_sm = blocks_per_sm((const void*)fn, smem);
  const int grid = std::min(M.ntiles, per_sm * h->nsm);
  fn<<<grid, kRowThreads, smem, h->stream>>>(view<VT>(M, va), epi, skip);
  GS2_LAUNCH_CHECK();
}

template <typename VT, class Epi>
static void dispatch(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  switch (M.tpr) {
    case 1: launch_k<1, VT, Epi>(h, M, va, epi, skip); break;
    case 2: launch_k<2, VT, Epi>(h, M, va, epi, skip); break;
    case 4: launch_k<4, VT, Epi>(h, M, va, epi, skip); break;
    case 8: launch_k<8, VT, Epi>(h, M, va, epi, skip); break;
    default: launch_k<16, VT, Epi>(h, M, va, epi, skip); break;
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
    EpiInner<double, double> e{(const double*)g_in, (const double*)rhat, (double*)g_out, x,
                               nullptr, omega, gamma, omega, mode, damped};
    dispatch<double>(h, T, T.va, e, skip);
  } else if (prec == GS2_FP32) {
    EpiInner<float, float> e{(const float*)g_in, (const float*)rhat, (float*)g_out, x,
                             nullptr, (float)omega, (float)gamma, omega, mode, damped};
    dispatch<float>(h, T, T.va32, e, skip);
  } else {
    EpiInner<float, float> e{(const float*)g_in, (const float*)rhat, (float*)g_out, x,
                             T.scale16, (float)omega, (float)gamma, omega, mode, damped};
    dispatch<__half>(h, T, T.va16, e, skip);
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
