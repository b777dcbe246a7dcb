// Row kernels of the two-stage Gauss-Seidel library (sm_103a).
//
// Every sweep is a CSR row reduction followed by a per-row epilogue:
//   residual      r = b - A x, rhat = D^{-1} r              (Eq. 2, Eq. 3)
//   inner sweep   g' = (1-gamma) g + gamma (rhat - omega T g)  (Eq. 4-5,
//                 damped form of Sec. 4), the last one fused with
//                 x += omega g'
//   JR            x' = x + omega D^{-1} (b - A x)           (Sec. 4)
//   SpMV          y = A x
//
// Design (GB300): FP64 throughput on this part is ~2 FMA/clk/SM, so a
// warp-per-row reduction (whose shuffle-add tree runs on every lane) would
// spend more FP64 issue slots on the tree than on the products.  Rows are
// therefore reduced sequentially by one thread (or by K contiguous segments
// for long rows), with each tile's row pointers, columns and values staged
// into shared memory by TMA bulk copies (tiles.cuh).  x-gathers go through
// the read-only path and stay L2-resident.  (Fusing the SpMV with the first
// Gram-Schmidt dot pass of an Arnoldi step was measured: the fused kernel
// reached only ~0.65 of both the HBM and the FP64 rate, 3% faster than the
// two kernels apart, and is not kept.)
#include "tiles.cuh"

namespace gs2 {

// ---------------------------------------------------------------------------
// epilogues: pre(i) loads the row's operands before the gathers, finish(i,
// s, pre) consumes the row sum
// ---------------------------------------------------------------------------

// r = b - A x;  rhat = D^{-1} r   (Eq. 2 residual and Eq. 3 initial guess)
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
  const signed char* __restrict__ rowscale;  // FP16 triangles only: scale 2^e_i
  AT omega, gamma;
  double omega64;
  int mode;
  float* __restrict__ x32;  // whole-sweep precisions: the FP32 iterate
  struct Pre {
    AT rh, gi, sc;
    double xi;
    float x32i;
  };
  __device__ Pre pre(int i) const {
    Pre p;
    p.rh = (AT)rhat[i];
    p.gi = DAMPED ? (AT)g_in[i] : AT(0);
    p.sc = SCALED ? (AT)__int_as_float(((int)rowscale[i] + 127) << 23) : AT(1);
    p.xi = mode == INNER_LAST_ADD ? x[i] : 0.0;
    p.x32i = (mode == INNER_LAST_ADD32 || mode == INNER_LAST_ADD32_OUT) ? x32[i] : 0.f;
    return p;
  }
  __device__ AT gather(int c) const { return (AT)__ldg(g_in + c); }
  __device__ void finish(int i, AT s, const Pre& p) const {
    if (SCALED) s *= p.sc;
    AT go = p.rh - omega * s;
    if (DAMPED) go = (AT(1) - gamma) * p.gi + gamma * go;
    if (mode == INNER_MID) {
      g_out[i] = (GT)go;
    } else if (mode == INNER_LAST_ADD) {
      x[i] = p.xi + omega64 * (double)go;
    } else if (mode == INNER_LAST_SET) {
      x[i] = omega64 * (double)go;
    } else {
      // FP32 iterate: x32 + omega g (or omega g) in FP32 arithmetic
      const float u = (float)omega * (float)go;
      const float xn = (mode == INNER_LAST_ADD32 || mode == INNER_LAST_ADD32_OUT) ? p.x32i + u : u;
      if (mode == INNER_LAST_ADD32 || mode == INNER_LAST_SET32) x32[i] = xn;
      else x[i] = (double)xn;
    }
  }
};

// residual of the whole-sweep precisions on the prescaled off-diagonal
// matrix O = D^{-1}(L + U), FP32 arithmetic:
//   rhat32 = (fl32(D^{-1} b) - x32) - O x32
template <bool SCALED>
struct EpiResidSweep {
  const float* __restrict__ bhat;
  const float* __restrict__ x32;
  const signed char* __restrict__ rowscale;
  float* __restrict__ rhat32;
  struct Pre {
    float bx, sc;
  };
  __device__ Pre pre(int i) const {
    Pre p;
    p.bx = bhat[i] - x32[i];
    p.sc = SCALED ? __int_as_float(((int)rowscale[i] + 127) << 23) : 1.f;
    return p;
  }
  __device__ float gather(int c) const { return __ldg(x32 + c); }
  __device__ void finish(int i, float s, const Pre& p) const {
    if (SCALED) s *= p.sc;
    rhat32[i] = p.bx - s;
  }
};

// compact right-hand side of Eq. (9) on the other prescaled triangle
// T' = D^{-1} U (forward) or D^{-1} L (backward):  rhat = D^{-1} b - T' x
struct EpiCompact {
  const double* __restrict__ x;
  const double* __restrict__ b;
  const double* __restrict__ dinv;
  double* __restrict__ rhat64;
  float* __restrict__ rhat32;
  struct Pre {
    double b, d;
  };
  __device__ Pre pre(int i) const { return Pre{b[i], dinv[i]}; }
  __device__ double gather(int c) const { return __ldg(x + c); }
  __device__ void finish(int i, double s, const Pre& p) const {
    const double rh = p.d * p.b - s;
    if (rhat64) rhat64[i] = rh;
    if (rhat32) rhat32[i] = (float)rh;
  }
};

// one colour of multicolour GS (Sec. 6.1.2): the colour matrix holds only
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
int blocks_per_sm(const void* fn, size_t smem) {
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



void launch_resid(gs2_handle* h, const double* b, const double* x, double* r_out,
                  double* rhat64, float* rhat32, const int* skip) {
  launch_resid_matrix(h, h->A, b, x, r_out, rhat64, rhat32, skip);
}

void launch_resid_matrix(gs2_handle* h, const DevCsr& M, const double* b, const double* x,
                         double* r_out, double* rhat64, float* rhat32, const int* skip) {
  // algorithmic bytes: M once, x, b, D^{-1} read, r / rhat written
  KernelTimer tm(h, "resid", bytes_csr(M, 8) + 24.0 * h->n + (r_out ? 8.0 * h->n : 0.0) +
                 (rhat64 ? 8.0 * h->n : 0.0) + (rhat32 ? 4.0 * h->n : 0.0));
  EpiResid e{x, b, h->dinv, r_out, rhat64, rhat32};
  dispatch<double>(h, M, M.va, e, skip);
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

__device__ __forceinline__ void add_to(double* p, double v) { *p += v; }
__device__ __forceinline__ void add_to(float* p, float v) { *p += v; }
__device__ __forceinline__ void add_to(__half* p, __half v) {
  *p = __float2half(__half2float(*p) + __half2float(v));
}

// CSR rows into the sliced-ELL layout, one thread per row (c = i / 32).
// Explicit chunk: slot k of row i goes to cptr[c] + 32 k + i % 32; value
// slots past the row's end keep their zero, column slots repeat the row's
// last column (column 0 for an empty row, whose slots stay zero).  Offset
// chunk: the entry at column j goes to the slot of offset j - i in the
// chunk's offset list (added, so duplicate entries of an unvalidated matrix
// sum as in an SpMV); the other slots keep their zero, and no column is
// stored.
template <typename T>
__global__ void k_to_sell(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                          const T* __restrict__ va, const int* __restrict__ cptr,
                          const int* __restrict__ coff, const int* __restrict__ offs, int* sci,
                          T* sva) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = i >> 5, lane = i & 31;
    const int L = (cptr[c + 1] - cptr[c]) >> 5;
    const int a = rp[i], len = rp[i + 1] - a;
    const int ob = coff[c];
    if (ob >= 0) {
      for (int k = 0; k < len; ++k) {
        const int o = ci[a + k] - i;
        int p = 0;
        while (p < L && offs[ob + p] != o) ++p;  // present by construction
        if (p < L) add_to(sva + cptr[c] + (p << 5) + lane, va[a + k]);
      }
      continue;
    }
    for (int k = 0; k < L; ++k) {
      const int slot = cptr[c] + (k << 5) + lane;
      if (k < len) {
        sva[slot] = va[a + k];
        if (sci) sci[slot] = ci[a + k];
      } else if (sci && len > 0) {
        sci[slot] = ci[a + len - 1];
      }
    }
  }
}

template <typename T>
static void to_sell(gs2_handle* h, const DevCsr& M, const T* va, T* sva, bool with_ci) {
  k_to_sell<T><<<vec_blocks(h, M.n), kVecThreads, 0, h->stream>>>(
      M.n, M.rp, M.ci, va, M.sell_ptr, M.sell_coff, M.sell_off, with_ci ? M.sell_ci : nullptr,
      sva);
  GS2_LAUNCH_CHECK();
}
void launch_to_sell(gs2_handle* h, const DevCsr& M, const double* va, double* sva, bool with_ci) {
  to_sell(h, M, va, sva, with_ci);
}
void launch_to_sell(gs2_handle* h, const DevCsr& M, const float* va, float* sva, bool with_ci) {
  to_sell(h, M, va, sva, with_ci);
}
void launch_to_sell(gs2_handle* h, const DevCsr& M, const __half* va, __half* sva, bool with_ci) {
  to_sell(h, M, va, sva, with_ci);
}

// Autotuner probe: milliseconds per launch of M's most frequent kernel with
// M's current tile shape, best of `reps`: the residual for A (role 0), the
// inner sweep with the x update for a triangle (roles 1, 2).  The operands
// are the handle's temporaries (their values do not matter for the timing).
template <class Epi>
static float time_epilogue(gs2_handle* h, const DevCsr& M, const Epi& e, int reps) {
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

float time_tile_probe(gs2_handle* h, const DevCsr& M, int reps, int role) {
  if (role == 0) {
    EpiResid e{h->t, h->g1, h->dinv, nullptr, h->rhat, nullptr};
    return time_epilogue(h, M, e, reps);
  }
  EpiInner<double, double, false, false> e{h->g0, h->rhat, nullptr, h->z, nullptr,
                                           1.0, 1.0, 1.0, INNER_LAST_ADD};
  return time_epilogue(h, M, e, reps);
}

void launch_compact_rhs(gs2_handle* h, const DevCsr& Tother, const double* b, const double* x,
                        double* rhat64, float* rhat32, const int* skip) {
  KernelTimer tm(h, "compact_rhs", bytes_csr(Tother, 8) + 24.0 * h->n +
                                       (rhat64 ? 8.0 : 4.0) * h->n);
  EpiCompact e{x, b, h->dinv, rhat64, rhat32};
  dispatch<double>(h, Tother, Tother.va, e, skip);
}

void launch_jr(gs2_handle* h, const double* b, const double* x_in, double* x_out,
               double omega, const int* skip) {
  launch_jr_matrix(h, h->A, b, x_in, x_out, omega, skip);
}

void launch_jr_matrix(gs2_handle* h, const DevCsr& M, const double* b, const double* x_in,
                      double* x_out, double omega, const int* skip) {
  KernelTimer tm(h, "jr", bytes_csr(M, 8) + 32.0 * h->n);
  EpiJr e{x_in, b, h->dinv, x_out, omega};
  dispatch<double>(h, M, M.va, e, skip);
}

void launch_inner(gs2_handle* h, const DevCsr& T, int prec, const void* rhat,
                  const void* g_in, void* g_out, double* x, double omega, double gamma,
                  int mode, const int* skip) {
  const bool damped = gamma != 1.0;
  const double vb = prec == GS2_FP64 ? 8.0 : (prec == GS2_FP32 ? 4.0 : 2.0);
  const double gb = prec == GS2_FP64 ? 8.0 : 4.0;
  double bytes = bytes_csr(T, (int)vb) + gb * T.n * (2 + (damped ? 1 : 0)) +
                 (mode == INNER_MID ? gb * T.n : (mode == INNER_LAST_ADD ? 16.0 : 8.0) * T.n) +
                 (prec == GS2_FP16_ROWSCALED ? 1.0 * T.n : 0.0);
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
                                            (float)gamma, omega, mode, h->x32};
      dispatch<float>(h, T, T.va32, e, skip);
    } else {
      EpiInner<float, float, false, false> e{(const float*)g_in, (const float*)rhat,
                                             (float*)g_out, x, nullptr, (float)omega,
                                             (float)gamma, omega, mode, h->x32};
      dispatch<float>(h, T, T.va32, e, skip);
    }
  } else {
    if (damped) {
      EpiInner<float, float, true, true> e{(const float*)g_in, (const float*)rhat,
                                           (float*)g_out, x, T.scale16, (float)omega,
                                           (float)gamma, omega, mode, h->x32};
      dispatch<__half>(h, T, T.va16, e, skip);
    } else {
      EpiInner<float, float, false, true> e{(const float*)g_in, (const float*)rhat,
                                            (float*)g_out, x, T.scale16, (float)omega,
                                            (float)gamma, omega, mode, h->x32};
      dispatch<__half>(h, T, T.va16, e, skip);
    }
  }
}

void launch_resid_sweep(gs2_handle* h, int vprec, const int* skip) {
  const DevCsr& O = h->O;
  if (O.n == 0) return;
  // O once (FP32 or FP16 values and a one-byte row scale), bhat32 and x32
  // read, rhat32 written
  const bool half = vprec == GS2_FP16_ROWSCALED;
  KernelTimer tm(h, half ? "resid16" : "resid32",
                 bytes_csr(O, half ? 2 : 4) + 12.0 * O.n + (half ? 1.0 * O.n : 0.0));
  if (half) {
    EpiResidSweep<true> e{h->bhat32, h->x32, O.scale16, h->rhat32};
    dispatch<__half>(h, O, O.va16, e, skip);
  } else {
    EpiResidSweep<false> e{h->bhat32, h->x32, nullptr, h->rhat32};
    dispatch<float>(h, O, O.va32, e, skip);
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

// update of a whole-sweep-precision sweep without inner sweeps: the FP32
// iterate x32 + omega rhat (or omega rhat), to x32 or converted to x
__global__ void k_rhat_update32(int n, const float* __restrict__ rhat, float* x32, double* x,
                                float omega, int mode, const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float u = omega * rhat[i];
    const bool add = mode == INNER_LAST_ADD32 || mode == INNER_LAST_ADD32_OUT;
    const float xn = add ? x32[i] + u : u;
    if (mode == INNER_LAST_ADD32 || mode == INNER_LAST_SET32) x32[i] = xn;
    else x[i] = (double)xn;
  }
}

__global__ void k_to32(int n, const double* __restrict__ x, float* x32, const int* skip) {
  if (skip && *skip) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x32[i] = (float)x[i];
}

__global__ void k_values_to_fp32(int64_t nz, const double* __restrict__ va, float* va32) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nz;
       k += (int64_t)gridDim.x * blockDim.x)
    va32[k] = (float)va[k];
}

// Row i: e_i such that max_j |v_ij| = f 2^e_i with f in [1/2, 1) (e_i = 0 for a
// row of zeros; clamped to [-126, 127]), read off the exponent field of the
// maximum; q_ij = fl16(v_ij 2^-e_i), the power of two applied exactly.
__global__ void k_values_to_fp16(int n, const int* __restrict__ rp, const double* __restrict__ va,
                                 __half* va16, signed char* scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double m = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) m = fmax(m, fabs(va[k]));
    int e = 0;
    if (m > 0.0) {
      const int E = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
      e = E == 0 ? -1022 : E - 1022;
      e = min(127, max(-126, e));
    }
    scale[i] = (signed char)e;
    const double inv = __longlong_as_double((long long)(1023 - e) << 52);  // 2^-e
    for (int k = rp[i]; k < rp[i + 1]; ++k) va16[k] = __double2half(va[k] * inv);
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

void launch_rhat_update32(gs2_handle* h, const float* rhat, double* x, double omega, int mode,
                          const int* skip) {
  if (h->n == 0) return;
  const bool add = mode == INNER_LAST_ADD32 || mode == INNER_LAST_ADD32_OUT;
  const bool out = mode == INNER_LAST_ADD32_OUT || mode == INNER_LAST_SET32_OUT;
  KernelTimer tm(h, "rhat_update", 4.0 * h->n + (add ? 4.0 : 0.0) * h->n +
                 (out ? 8.0 : 4.0) * h->n);
  k_rhat_update32<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>(
      (int)h->n, rhat, h->x32, x, (float)omega, mode, skip);
  GS2_LAUNCH_CHECK();
}

void launch_values_to_fp32(gs2_handle* h, const DevCsr& M, int64_t nz) {
  k_values_to_fp32<<<vec_blocks(h, nz), kVecThreads, 0, h->stream>>>(nz, M.va, M.va32);
  GS2_LAUNCH_CHECK();
}

void launch_values_to_fp16(gs2_handle* h, const DevCsr& M) {
  if (M.n == 0) return;
  k_values_to_fp16<<<vec_blocks(h, M.n), kVecThreads, 0, h->stream>>>(M.n, M.rp, M.va, M.va16,
                                                                      M.scale16);
  GS2_LAUNCH_CHECK();
}

void launch_to32(gs2_handle* h, const double* x, float* x32, const int* skip) {
  if (h->n == 0) return;
  KernelTimer tm(h, "to32", 12.0 * h->n);
  k_to32<<<vec_blocks(h, h->n), kVecThreads, 0, h->stream>>>((int)h->n, x, x32, skip);
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
  // launched with programmatic dependent launch: the next level's launch
  // overlaps this one; its rows wait here for the previous level's results
  pdl_wait();
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
    launch_pdl(k_level<8>, grid, kRowThreads, 0, h->stream, rows, r0, r1, (const int*)T.rp,
               (const int*)T.ci, (const double*)T.va, rhat, g, x, omega, skip);
  else
    launch_pdl(k_level<1>, grid, kRowThreads, 0, h->stream, rows, r0, r1, (const int*)T.rp,
               (const int*)T.ci, (const double*)T.va, rhat, g, x, omega, skip);
  GS2_LAUNCH_CHECK();
}

}  // namespace gs2
