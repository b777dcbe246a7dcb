// gs2_apply_noalloc: the GS2 relaxation for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc: a plugin whose host application owns
// every byte of GPU memory through its own allocator, code that runs after a
// service has frozen its memory footprint, or a real-time loop where an
// allocation (and the synchronisation it can imply) is not allowed.  They
// still own their inputs and outputs; what they cannot provide is the
// solver's working memory.  This entry point keeps that working memory in a
// fixed array in the library's own device image, so a call allocates
// nothing: no cudaMalloc, no cudaFree, no library routine that allocates.
//
// Limits and sharing:
//  - at most kNoAllocMaxRows rows (262,144); larger systems are rejected
//    with GS2_ERR_INVALID_ARG;
//  - the array (4 x 262,144 doubles = 8 MiB) is part of the library image:
//    every GPU that loads the library holds it until the process exits;
//  - all calls share it and it keeps the last call's contents.  Every value a
//    sweep reads from it is written earlier in the same call, so nothing has
//    to start at zero, but calls that overlap on the GPU (different streams,
//    or different host threads on one device) race on it: serialise them;
//  - every call outside stream capture looks the array's device address up
//    with cudaGetSymbolAddress on the current device (cheap) and remembers it
//    per device; a call made while its stream is being captured uses the
//    remembered address, so make one call on that device before capturing
//    (a capture with none before it is refused).  Looking the address up
//    again on every uncaptured call keeps it right after a device reset.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace gs2 {

constexpr int64_t kNoAllocMaxRows = 1 << 18;
constexpr int kNoAllocMaxDevices = 64;

// D^{-1}, r-hat, g_a, g_b: four slices of kNoAllocMaxRows doubles
static __device__ __align__(256) double g_noalloc_scratch[4 * kNoAllocMaxRows];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with the device current.  Outside capture it is
// looked up on every call (and remembered); inside a capture the remembered
// address of an earlier call on this device is used.
static double* noalloc_scratch(cudaStream_t stream) {
  int dev = 0;
  GS2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    GS2_THROW(GS2_ERR_INVALID_ARG, "device index out of range for the no-allocation path");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GS2_CUDA(cudaStreamIsCapturing(stream, &cap));
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    GS2_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  } else if (!g_noalloc_ptr[dev]) {
    GS2_THROW(GS2_ERR_INVALID_ARG,
              "the no-allocation path needs one uncaptured call on this device before a "
              "stream capture");
  }
  return g_noalloc_ptr[dev];
}

// dinv_i = 1 / a_ii, a_ii the sum of the row's stored diagonal entries (as
// an SpMV would use them; a missing or zero diagonal gives inf, and the
// sweep then produces inf / NaN in x)
__global__ void k_na_diag(int64_t n, const int64_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const double* __restrict__ va,
                          double* dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d += va[k];
    dinv[i] = 1.0 / d;
  }
}

// rhat = D^{-1} (b - A x)   (Eq. 2 residual, Eq. 3 initial guess)
__global__ void k_na_resid(int64_t n, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const double* __restrict__ va,
                           const double* __restrict__ b, const double* __restrict__ x,
                           const double* __restrict__ dinv, double* rhat) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s = fma(va[k], x[ci[k]], s);
    rhat[i] = dinv[i] * (b[i] - s);
  }
}

// g_out = rhat - omega D^{-1} T g_in over the strict triangle T of A
// (Eq. 4-5 with the outer damping); the last sweep adds omega g to x
__global__ void k_na_inner(int64_t n, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const double* __restrict__ va,
                           const double* __restrict__ dinv, const double* __restrict__ rhat,
                           const double* __restrict__ g_in, double* g_out, double* x,
                           double omega, int lower, int last) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = ci[k];
      if (lower ? j < i : j > i) s = fma(va[k], g_in[j], s);
    }
    const double g = rhat[i] - omega * (dinv[i] * s);
    if (last) x[i] += omega * g;
    else g_out[i] = g;
  }
}

__global__ void k_na_update(int64_t n, const double* __restrict__ rhat, double* x,
                            double omega) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += omega * rhat[i];
}

}  // namespace gs2

using namespace gs2;

extern "C" gs2_status gs2_apply_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                        const double* val, const double* b, double* x,
                                        int outer_sweeps, int inner_sweeps, double damping,
                                        int direction, void* stream) {
  try {
    // the bounds gs2_apply checks: 0..1000 outer and 0..100000 inner sweeps,
    // a finite positive damping, a known direction
    if (n < 0 || outer_sweeps < 0 || outer_sweeps > 1000 || inner_sweeps < 0 ||
        inner_sweeps > 100000 || !(damping > 0.0) || !std::isfinite(damping) ||
        direction < 0 || direction > 2)
      GS2_THROW(GS2_ERR_INVALID_ARG, "bad size, sweep count, damping or direction");
    if (n > kNoAllocMaxRows)
      GS2_THROW(GS2_ERR_INVALID_ARG,
                "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                    std::to_string(kNoAllocMaxRows) + " rows");
    if (n == 0 || outer_sweeps == 0) return GS2_OK;
    if (!rowptr || !col || !val || !b || !x) GS2_THROW(GS2_ERR_INVALID_ARG, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* base = noalloc_scratch(s);
    double* dinv = base;
    double* rhat = base + kNoAllocMaxRows;
    double* ga = base + 2 * kNoAllocMaxRows;
    double* gb = base + 3 * kNoAllocMaxRows;
    int dev = 0, nsm = 0;
    GS2_CUDA(cudaGetDevice(&dev));
    GS2_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    const int grid = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)nsm * 8);
    k_na_diag<<<grid, threads, 0, s>>>(n, rowptr, col, val, dinv);
    GS2_LAUNCH_CHECK();
    for (int sweep = 0; sweep < outer_sweeps; ++sweep) {
      for (int half = 0; half < 2; ++half) {
        const int lower = half == 0;
        if (lower && direction == GS2_BACKWARD) continue;
        if (!lower && direction == GS2_FORWARD) continue;
        k_na_resid<<<grid, threads, 0, s>>>(n, rowptr, col, val, b, x, dinv, rhat);
        GS2_LAUNCH_CHECK();
        if (inner_sweeps == 0) {
          k_na_update<<<grid, threads, 0, s>>>(n, rhat, x, damping);
          GS2_LAUNCH_CHECK();
          continue;
        }
        const double* gin = rhat;  // g_0 = D^{-1} r
        for (int j = 0; j < inner_sweeps; ++j) {
          const int last = j == inner_sweeps - 1;
          double* gout = last ? nullptr : (j % 2 == 0 ? ga : gb);
          k_na_inner<<<grid, threads, 0, s>>>(n, rowptr, col, val, dinv, rhat, gin, gout, x,
                                             damping, lower, last);
          GS2_LAUNCH_CHECK();
          gin = gout;
        }
      }
    }
    return GS2_OK;
  } catch (const gs2::Error& e) {
    gs2::set_error(e.msg);
    return e.st;
  } catch (...) {
    gs2::set_error("unexpected C++ exception");
    return GS2_ERR_CUDA;
  }
}
