// Fixed-order block reductions of per-thread FP64 partial sums used by the
// Krylov kernels.  Deterministic: the same shuffle pattern and the same
// summation order on every run.
#pragma once

#include "internal.cuh"

namespace gs2 {

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <int N>
struct Pow2 {
  static constexpr int value = N <= 1 ? 1 : 2 * Pow2<(N + 1) / 2>::value;
};
template <>
struct Pow2<1> {
  static constexpr int value = 1;
};
template <int P>
struct Log2 {
  static constexpr int value = P <= 1 ? 0 : 1 + Log2<P / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

// Warp sums of NV <= 32 per-thread values.  A butterfly transpose-reduction
// halves the values each lane holds at every exchange, P - 1 adds per lane
// for P = NV rounded up to a power of two, instead of 5 adds per value of a
// shuffle tree -- the FP64 pipe is the bottleneck of these kernels.  Returns
// this lane's share: the lanes whose low 5 - p bits are zero (p = log2 P)
// hold the warp's sum of value lane >> (5 - p).
template <int NV>
__device__ __forceinline__ double warp_butterfly(const double (&acc)[NV]) {
  constexpr int P = Pow2<NV>::value;
  constexpr int p = Log2<P>::value;
  static_assert(P <= 32, "butterfly reduction holds at most 32 values");
  const int lane = threadIdx.x & 31;
  double a[P];
#pragma unroll
  for (int k = 0; k < P; ++k) a[k] = k < NV ? acc[k] : 0.0;
#pragma unroll
  for (int s = 0; s < p; ++s) {
    const int off = 16 >> s;
    const int half = (P >> s) / 2;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const double send = upper ? a[j] : a[j + half];
      const double recv = __shfl_xor_sync(0xffffffffu, send, off);
      a[j] = (upper ? a[j + half] : a[j]) + recv;
    }
  }
  // lanes that differ only in their low 5 - p bits hold parts of the same
  // value: finish with a plain tree over those bits
#pragma unroll
  for (int o = 16 >> p; o > 0; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
  return a[0];
}

// Block-wide sums of NV <= 32 per-thread values (warp_butterfly, then the
// warps' sums in warp order).  The block's sums go to column `col` of part
// (the block index by default; a block that loops over several work items
// passes the item).
template <int NV>
__device__ __forceinline__ void block_partials_bf(const double (&acc)[NV], double* part,
                                                  int nblk, int col) {
  constexpr int P = Pow2<NV>::value;
  constexpr int p = Log2<P>::value;
  __shared__ double red[kVecThreads / 32][P];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double a0 = warp_butterfly<NV>(acc);
  const int k = lane >> (5 - p);
  if ((lane & ((1 << (5 - p)) - 1)) == 0) red[wid][k] = a0;
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kVecThreads / 32; ++w) s += red[w][threadIdx.x];
    part[(size_t)threadIdx.x * nblk + col] = s;
  }
}

template <int NV>
__device__ __forceinline__ void block_partials_bf(const double (&acc)[NV], double* part,
                                                  int nblk) {
  block_partials_bf<NV>(acc, part, nblk, (int)blockIdx.x);
}

// Block-wide sums of NV per-thread values, written to part[v * nblk + blk]
// (general form: one shuffle tree per value; used for NV > 32).
template <int NV>
__device__ __forceinline__ void block_partials(const double (&acc)[NV], int nv, double* part,
                                               int nblk, int col) {
  __shared__ double red[kVecThreads / 32][NV];
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
    for (int w = 0; w < kVecThreads / 32; ++w) s += red[w][v];
    part[(size_t)v * nblk + col] = s;
  }
}

template <int NV>
__device__ __forceinline__ void block_partials(const double (&acc)[NV], int nv, double* part,
                                               int nblk) {
  block_partials<NV>(acc, nv, part, nblk, (int)blockIdx.x);
}

}  // namespace gs2
