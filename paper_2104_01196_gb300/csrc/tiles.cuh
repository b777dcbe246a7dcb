// The row-tile engine of the sweep kernels: TMA bulk copies of row tiles
// into double-buffered shared memory, mbarrier completion with bounded
// waits, one thread (or K lanes) per row, and a per-row epilogue.
#pragma once

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
  pdl_wait();
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
      if (threadIdx.x == 0) {
        if (M.err) atomicExch(M.err, (int)GS2_ERR_TIMEOUT);
        // let the copies still in flight (the late tile's and the next
        // one's) land before the block exits; each wait is bounded too
        mbar_wait_bounded(&bars[st], (it >> 1) & 1);
        if (tn < M.ntiles) mbar_wait_bounded(&bars[st ^ 1], ((it + 1) >> 1) & 1);
      }
      __syncthreads();
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
// launch plumbing
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// sliced-ELL rows (one thread per row, one warp per chunk of 32
// rows): slot k of the warp's rows is one coalesced 32-wide load of columns
// and one of values, streamed with evict-first hints so the gathered vector
// stays in L2; no shared memory and no block barrier.  Rows are reduced in
// CSR order, as by the row-tile engine with one lane per row.
// ---------------------------------------------------------------------------

template <typename VT>
__device__ __forceinline__ typename ValTraits<VT>::AT stream_val(const VT* p);
template <>
__device__ __forceinline__ double stream_val<double>(const double* p) { return __ldcs(p); }
template <>
__device__ __forceinline__ float stream_val<float>(const float* p) { return __ldcs(p); }
template <>
__device__ __forceinline__ float stream_val<__half>(const __half* p) {
  return __half2float(__ushort_as_half(__ldcs(reinterpret_cast<const unsigned short*>(p))));
}

// LONG (matrices with long rows): the next group's slots are loaded while
// the current group's gathers are in flight, one dependent round trip per
// group of four instead of two.  Its extra registers would cost short-row
// matrices occupancy, so it is a separate instantiation.
//
// Offset chunks (stencil rows) store no columns: the warp reads the chunk's
// offset list (one broadcast load per slot) and forms column row + o, so a
// slot moves only its value; the gathers of consecutive rows are contiguous.

// Two consecutive offset chunks of the same short width (<= 8 slots) at once,
// one row of each per lane: with FP32 / FP16 values a single chunk leaves
// too few bytes in flight per warp (the inner sweeps were latency-bound, 20
// long-scoreboard stalls per issue at 92% of the maximum warps), so both
// chunks' slots and gathers are issued before their FMAs.  Rows are reduced
// in the same slot order as one chunk at a time.  False (nothing done) when
// the pair does not qualify.
template <typename VT, class Epi>
__device__ __forceinline__ bool sell_pair(int n, int c, const int* __restrict__ cptr,
                                          const VT* __restrict__ va, const Epi& epi,
                                          const int* __restrict__ live,
                                          const int* __restrict__ coff,
                                          const int* __restrict__ offs, int cmax, int lane) {
  using AT = typename ValTraits<VT>::AT;
  const int ob0 = __ldg(coff + c), ob1 = __ldg(coff + c + 1);
  if (ob0 < 0 || ob1 < 0) return false;
  const int b0 = cptr[c], b1 = cptr[c + 1], b2 = cptr[c + 2];
  const int L = (b1 - b0) >> 5;
  if (L > 8 || ((b2 - b1) >> 5) != L) return false;
  if (live && (live[c] == 0 || live[c + 1] == 0)) return false;
  const int r0 = c * 32 + lane, r1 = r0 + 32;
  typename Epi::Pre p0{}, p1{};
  if (r0 < n) p0 = epi.pre(r0);
  if (r1 < n) p1 = epi.pre(r1);
  const VT* v0 = va + b0 + lane;
  const VT* v1 = va + b1 + lane;
  const int* o0 = offs + ob0;
  const int* o1 = offs + ob1;
  AT s0 = AT(0), s1 = AT(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < L) {
      const int ca = min(max(r0 + __ldg(o0 + k), 0), cmax);
      const int cb = min(max(r1 + __ldg(o1 + k), 0), cmax);
      const AT a = stream_val<VT>(v0 + 32 * k), b = stream_val<VT>(v1 + 32 * k);
      const AT xa = (AT)epi.gather(ca), xb = (AT)epi.gather(cb);
      s0 = fma(a, xa, s0);
      s1 = fma(b, xb, s1);
    }
  }
  if (r0 < n) epi.finish(r0, s0, p0);
  if (r1 < n) epi.finish(r1, s1, p1);
  return true;
}

template <typename VT, class Epi, bool LONG, bool PAIR>
__global__ void __launch_bounds__(kRowThreads)
k_sell(int n, int nchunks, const int* __restrict__ cptr, const int* __restrict__ ci,
       const VT* __restrict__ va, Epi epi, const int* skip, const int* __restrict__ live,
       const int* __restrict__ coff, const int* __restrict__ offs, int ncols) {
  using AT = typename ValTraits<VT>::AT;
  pdl_wait();
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int cmax = ncols - 1;
  // PAIR: a warp takes two chunks per iteration (sell_pair)
  constexpr int STEP = PAIR ? 2 : 1;
  for (int cw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cw * STEP < nchunks; cw += nw) {
  if (STEP == 2 && cw * 2 + 1 < nchunks &&
      sell_pair<VT, Epi>(n, cw * 2, cptr, va, epi, live, coff, offs, cmax, lane))
    continue;
  for (int c = cw * STEP; c < min(cw * STEP + STEP, nchunks); ++c) {
    // a chunk whose rows belong only to finished systems of a pack
    if (live && live[c] == 0) continue;
    const int row = c * 32 + lane;
    const int base = cptr[c], L = (cptr[c + 1] - base) >> 5;
    typename Epi::Pre pv{};
    if (row < n) pv = epi.pre(row);
    const VT* vv = va + base + lane;
    AT s = AT(0);
    int k = 0;
    const int ob = __ldg(coff + c);
    if (ob >= 0) {
      // columns row + o, clamped into [0, ncols) for the zero slots of rows
      // at a boundary (and the rows past n of the last chunk)
      const int* oo = offs + ob;
      for (; k + 4 <= L; k += 4, vv += 128) {
        const int c0 = min(max(row + __ldg(oo + k), 0), cmax);
        const int c1 = min(max(row + __ldg(oo + k + 1), 0), cmax);
        const int c2 = min(max(row + __ldg(oo + k + 2), 0), cmax);
        const int c3 = min(max(row + __ldg(oo + k + 3), 0), cmax);
        const AT a0 = stream_val<VT>(vv), a1 = stream_val<VT>(vv + 32);
        const AT a2 = stream_val<VT>(vv + 64), a3 = stream_val<VT>(vv + 96);
        const AT x0 = (AT)epi.gather(c0), x1 = (AT)epi.gather(c1);
        const AT x2 = (AT)epi.gather(c2), x3 = (AT)epi.gather(c3);
        s = fma(a0, x0, s);
        s = fma(a1, x1, s);
        s = fma(a2, x2, s);
        s = fma(a3, x3, s);
      }
      const int rem = L - k;
      if (rem > 0) {
        const int c0 = min(max(row + __ldg(oo + k), 0), cmax);
        const int c1 = rem > 1 ? min(max(row + __ldg(oo + k + 1), 0), cmax) : c0;
        const int c2 = rem > 2 ? min(max(row + __ldg(oo + k + 2), 0), cmax) : c0;
        const AT a0 = stream_val<VT>(vv);
        const AT a1 = rem > 1 ? stream_val<VT>(vv + 32) : AT(0);
        const AT a2 = rem > 2 ? stream_val<VT>(vv + 64) : AT(0);
        const AT x0 = (AT)epi.gather(c0);
        const AT x1 = rem > 1 ? (AT)epi.gather(c1) : AT(0);
        const AT x2 = rem > 2 ? (AT)epi.gather(c2) : AT(0);
        s = fma(a0, x0, s);
        if (rem > 1) s = fma(a1, x1, s);
        if (rem > 2) s = fma(a2, x2, s);
      }
      if (row < n) epi.finish(row, s, pv);
      continue;
    }
    const int* cc = ci + base + lane;
    if (LONG && L >= 8) {
      int c0 = __ldcs(cc), c1 = __ldcs(cc + 32), c2 = __ldcs(cc + 64), c3 = __ldcs(cc + 96);
      AT a0 = stream_val<VT>(vv), a1 = stream_val<VT>(vv + 32);
      AT a2 = stream_val<VT>(vv + 64), a3 = stream_val<VT>(vv + 96);
      for (; k + 8 <= L; k += 4) {
        cc += 128;
        vv += 128;
        const AT x0 = (AT)epi.gather(c0), x1 = (AT)epi.gather(c1);
        const AT x2 = (AT)epi.gather(c2), x3 = (AT)epi.gather(c3);
        const int n0 = __ldcs(cc), n1 = __ldcs(cc + 32), n2 = __ldcs(cc + 64), n3 = __ldcs(cc + 96);
        const AT b0 = stream_val<VT>(vv), b1 = stream_val<VT>(vv + 32);
        const AT b2 = stream_val<VT>(vv + 64), b3 = stream_val<VT>(vv + 96);
        s = fma(a0, x0, s);
        s = fma(a1, x1, s);
        s = fma(a2, x2, s);
        s = fma(a3, x3, s);
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        a0 = b0; a1 = b1; a2 = b2; a3 = b3;
      }
      // the last preloaded group
      const AT x0 = (AT)epi.gather(c0), x1 = (AT)epi.gather(c1);
      const AT x2 = (AT)epi.gather(c2), x3 = (AT)epi.gather(c3);
      s = fma(a0, x0, s);
      s = fma(a1, x1, s);
      s = fma(a2, x2, s);
      s = fma(a3, x3, s);
      k += 4;
      cc += 128;
      vv += 128;
    }
    // groups of four: all loads and gathers are in flight before the FMAs
    for (; k + 4 <= L; k += 4, cc += 128, vv += 128) {
      const int c0 = __ldcs(cc), c1 = __ldcs(cc + 32), c2 = __ldcs(cc + 64), c3 = __ldcs(cc + 96);
      const AT a0 = stream_val<VT>(vv), a1 = stream_val<VT>(vv + 32);
      const AT a2 = stream_val<VT>(vv + 64), a3 = stream_val<VT>(vv + 96);
      const AT x0 = (AT)epi.gather(c0), x1 = (AT)epi.gather(c1);
      const AT x2 = (AT)epi.gather(c2), x3 = (AT)epi.gather(c3);
      s = fma(a0, x0, s);
      s = fma(a1, x1, s);
      s = fma(a2, x2, s);
      s = fma(a3, x3, s);
    }
    // the last one to three slots, also issued together
    const int rem = L - k;
    if (rem > 0) {
      const int c0 = __ldcs(cc);
      const int c1 = rem > 1 ? __ldcs(cc + 32) : c0;
      const int c2 = rem > 2 ? __ldcs(cc + 64) : c0;
      const AT a0 = stream_val<VT>(vv);
      const AT a1 = rem > 1 ? stream_val<VT>(vv + 32) : AT(0);
      const AT a2 = rem > 2 ? stream_val<VT>(vv + 64) : AT(0);
      const AT x0 = (AT)epi.gather(c0);
      const AT x1 = rem > 1 ? (AT)epi.gather(c1) : AT(0);
      const AT x2 = rem > 2 ? (AT)epi.gather(c2) : AT(0);
      s = fma(a0, x0, s);
      if (rem > 1) s = fma(a1, x1, s);
      if (rem > 2) s = fma(a2, x2, s);
    }
    if (row < n) epi.finish(row, s, pv);
  }
  }
}

inline const double* sell_values(const DevCsr& M, const double*) { return M.sell_va; }
inline const float* sell_values(const DevCsr& M, const float*) { return M.sell_va32; }
inline const __half* sell_values(const DevCsr& M, const __half*) { return M.sell_va16; }

// Resident blocks per SM of a tile kernel at a dynamic shared-memory size
// (kernels.cu; cached per kernel and size, the attribute only ever raised).
int blocks_per_sm(const void* fn, size_t smem);

template <typename VT>
inline TileMat<VT> view(gs2_handle* h, const DevCsr& M, const VT* va) {
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
inline void launch_k(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  if (M.n == 0 || M.ntiles == 0) return;
  const size_t smem = 2 * (size_t)StageLayout<VT>(RPT * kRowThreads / K, M.cap).bytes;
  auto fn = k_tiles<K, RPT, VT, Epi>;
  const int per_sm = blocks_per_sm((const void*)fn, smem);
  const int grid = std::min(M.ntiles, per_sm * h->nsm);
  launch_pdl(fn, grid, kRowThreads, smem, h->stream, view<VT>(h, M, va), epi, skip);
  GS2_LAUNCH_CHECK();
}

template <typename VT, class Epi>
inline void launch_sell(gs2_handle* h, const DevCsr& M, const VT* sv, const Epi& epi,
                        const int* skip) {
  if (M.n == 0 || M.sell_chunks == 0) return;
  // mean rows longer than 24 entries take the software-pipelined form
  // (Q1 elasticity, 77 per row: GMRES+SGS2(1,2) 90.3 -> 81.8 ms per 120
  // iterations; on 7-entry rows it was 2% slower)
  // FP32 / FP16 values on rows of 5-8 entries (the whole-sweep residual's
  // off-diagonal matrix): two chunks per warp iteration (FP32 residual on
  // the 192^3 convection-diffusion matrix 59 -> 51 us).  Rows of 3 entries
  // (the inner sweeps' triangles) lost occupancy to it (51 -> 57 us), and
  // FP64 rows are bound by the FP64 pipe, so they keep one chunk.
  bool pair = false;
  auto fn = M.mean_row > kShortRowMean ? k_sell<VT, Epi, true, false> : k_sell<VT, Epi, false, false>;
  if constexpr (sizeof(VT) < sizeof(double)) {
    if (M.mean_row >= 4.5 && M.mean_row <= 8.0) {
      pair = true;
      fn = k_sell<VT, Epi, false, true>;
    }
  }
  const int per_sm = blocks_per_sm((const void*)fn, 0);
  const int warps = kRowThreads / 32;
  // (FP32 / FP16 values: a warp takes chunks in pairs)
  const int tasks = pair ? (M.sell_chunks + 1) / 2 : M.sell_chunks;
  const int grid = std::max(1, std::min((tasks + warps - 1) / warps, per_sm * h->nsm));
  // chunk liveness applies to the matrices whose rows are the handle's rows
  const int* live =
      (h->row_live && (&M == &h->A || &M == &h->L || &M == &h->U)) ? h->row_live : nullptr;
  launch_pdl(fn, grid, kRowThreads, 0, h->stream, M.n, M.sell_chunks,
             (const int*)M.sell_ptr, (const int*)M.sell_ci, sv, epi, skip, live,
             (const int*)M.sell_coff, (const int*)M.sell_off, M.sell_ncols);
  GS2_LAUNCH_CHECK();
}

// (K, RPT) shapes: RPT = 2 only for short rows (K <= 2), where the per-tile
// barrier and stage overhead is largest relative to the work per row
template <typename VT, class Epi>
inline void dispatch(gs2_handle* h, const DevCsr& M, const VT* va, const Epi& epi,
                     const int* skip) {
  const VT* sv = M.sell ? sell_values(M, va) : nullptr;
  if (sv) {
    launch_sell<VT, Epi>(h, M, sv, epi, skip);
    return;
  }
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

inline double bytes_csr(const DevCsr& M, int vbytes) {
  return (double)M.nnz * (4.0 + vbytes) + 4.0 * (M.n + 1);
}

}  // namespace gs2
