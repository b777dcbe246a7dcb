// Host runtime of the GS2 library: handle setup (validation, the A = L + D + U
// split with prescaled triangles, row tiles, precision copies), the C ABI
// entry points, host-vector staging and per-kernel event timing.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace gs2 {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// profiler
// ---------------------------------------------------------------------------

struct Profiler {
  bool enabled = false;
  std::string only;  // non-empty: time only kernels of this name
  std::vector<std::string> names;
  std::unordered_map<std::string, int> ids;
  std::vector<gs2_kernel_stat> stats;
  struct Pending {
    int id;
    cudaEvent_t a, b;
    double bytes;
    int step;  // Arnoldi step of an eager cycle, -1 outside one
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // Event pairs captured into an Arnoldi-step graph: recorded as external
  // event nodes at every replay and read after each replay of a cycle,
  // counting only the steps the cycle ran (later steps are no-ops).
  struct Captured {
    int id;
    cudaEvent_t a, b;
    double bytes;
    int step;
  };
  std::vector<Captured> captured;
  bool capturing = false;
  int cap_step = -1;  // step of the launches being issued (graph or eager), or -1
  int epoch = 0;  // changes with enable/filter, so graphs are re-captured

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  int id_of(const char* name) {
    auto it = ids.find(name);
    if (it != ids.end()) return it->second;
    const int id = (int)stats.size();
    ids[name] = id;
    gs2_kernel_stat s{};
    std::strncpy(s.name, name, sizeof(s.name) - 1);
    stats.push_back(s);
    return id;
  }
  void resolve(cudaStream_t st) {
    if (pending.empty()) return;
    cudaStreamSynchronize(st);
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        stats[p.id].launches += 1;
        stats[p.id].total_ms += ms;
        stats[p.id].bytes += p.bytes;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void clear_captured() {
    for (auto& c : captured) {
      cudaEventDestroy(c.a);
      cudaEventDestroy(c.b);
    }
    captured.clear();
  }
  // after an eager cycle that ran `steps` steps: launches of later steps
  // (issued before the host saw the device stop) ran as no-ops
  void settle(int steps) {
    std::vector<Pending> keep;
    keep.reserve(pending.size());
    for (auto& p : pending) {
      if (p.step >= steps) {
        pool.push_back(p.a);
        pool.push_back(p.b);
      } else {
        p.step = -1;
        keep.push_back(p);
      }
    }
    pending.swap(keep);
  }
  void harvest(int steps) {
    for (auto& c : captured) {
      if (c.step >= steps) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c.a, c.b) == cudaSuccess) {
        stats[c.id].launches += 1;
        stats[c.id].total_ms += ms;
        stats[c.id].bytes += c.bytes;
      }
    }
  }
  ~Profiler() {
    clear_captured();
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

bool profiling_active(const gs2_handle* h) { return h->prof && h->prof->enabled; }

int profile_epoch(const gs2_handle* h) {
  return profiling_active(h) ? h->prof->epoch : -1;
}

void profile_capture_begin(gs2_handle* h) {
  if (!profiling_active(h)) return;
  h->prof->clear_captured();
  h->prof->capturing = true;
}

void profile_capture_step(gs2_handle* h, int step) {
  if (profiling_active(h)) h->prof->cap_step = step;
}

void profile_capture_end(gs2_handle* h) {
  if (!h->prof) return;
  h->prof->capturing = false;
  h->prof->cap_step = -1;
}

void profile_harvest(gs2_handle* h, int steps, bool graph) {
  if (!profiling_active(h)) return;
  if (graph) h->prof->harvest(steps);
  else h->prof->settle(steps);
}

KernelTimer::KernelTimer(gs2_handle* h_, const char* name, double bytes_)
    : h(h_), id(-1), bytes(bytes_) {
  if (h->prof && h->prof->enabled && (h->prof->only.empty() || h->prof->only == name)) {
    id = h->prof->id_of(name);
    if (h->prof->capturing) {
      cudaEventCreate(&e0);
      cudaEventRecordWithFlags(e0, h->stream, cudaEventRecordExternal);
    } else {
      e0 = h->prof->get();
      cudaEventRecord(e0, h->stream);
    }
  }
}

KernelTimer::~KernelTimer() {
  if (id >= 0 && e0) {
    if (h->prof->capturing) {
      cudaEvent_t e1 = nullptr;
      cudaEventCreate(&e1);
      cudaEventRecordWithFlags(e1, h->stream, cudaEventRecordExternal);
      h->prof->captured.push_back({id, e0, e1, bytes, h->prof->cap_step});
      return;
    }
    cudaEvent_t e1 = h->prof->get();
    cudaEventRecord(e1, h->stream);
    h->prof->pending.push_back({id, e0, e1, bytes, h->prof->cap_step});
    // keep the pending list bounded on long runs (never inside a cycle,
    // whose trailing launches are settled when it ends)
    if (h->prof->cap_step < 0 && h->prof->pending.size() > 16384)
      h->prof->resolve(h->stream);
  }
}

// ---------------------------------------------------------------------------
// setup helpers
// ---------------------------------------------------------------------------

constexpr int kHardCap = 6144;  // staged entries per tile at most
constexpr int kPad = 16;        // padding entries after every CSR array

static int choose_lanes(double mean) {
  int K = 1;
  while (K < 16 && mean / K > 24.0) K *= 2;
  return K;
}

static void build_tiles(const std::vector<int>& rp, int n, int K, int RPT,
                        std::vector<int>& tiles, int& cap) {
  const int R = RPT * kRowThreads / K;
  tiles.clear();
  tiles.push_back(0);
  int maxnz = 0;
  int r = 0;
  while (r < n) {
    int len = rp[r + 1] - rp[r];
    if (len > kHardCap) {
      ++r;
      tiles.push_back(r);
      continue;
    }
    int cnt = 0, nz = 0;
    while (r < n && cnt < R) {
      len = rp[r + 1] - rp[r];
      if (len > kHardCap || nz + len > kHardCap) break;
      nz += len;
      ++cnt;
      ++r;
    }
    maxnz = std::max(maxnz, nz);
    tiles.push_back(r);
  }
  cap = ((maxnz + 7) / 8) * 8;
  if (cap < 8) cap = 8;
}

void retile(gs2_handle* h, DevCsr& M, const std::vector<int>& rp, int K, int RPT);

// ---------------------------------------------------------------------------
// sliced-ELL copies
// ---------------------------------------------------------------------------

// A matrix whose sliced-ELL layout pads by at most 20% gets the copy when
// its rows are short (one lane per row is the natural width) or when it is
// streamed from HBM (its CSR larger than the 129 MB L2): there one lane per
// row issues only the row's FMAs, with no segment reduction and no idle
// lanes, which matters on this part's FP64 pipe (on the 81-entry rows of Q1
// elasticity the residual went from 2.8 to 5.0 TB/s against the best
// row-tile shape, 8 lanes per row).  Smaller long-row matrices (coarse
// multigrid levels) are latency-bound and keep the row tiles, whose K lanes
// per row shorten each row's chain of dependent gathers.
constexpr int kSellC = 32;                       // rows per chunk (one warp)
constexpr double kSellMaxPadding = 1.2;          // slots / entries
constexpr double kSellStreamBytes = 128.0 * (1 << 20);  // CSR bytes beyond L2

// Chunk layout: chunk c takes width_c x 32 slots, width_c its longest row
// (explicit columns) or, for an offset chunk, the number of distinct column
// offsets j - i over its rows.  A chunk is an offset chunk when that union is
// at most its longest row + kOffsetSlack and at most 32 (stencil rows: the
// rows at a grid boundary miss some offsets and get zero slots there).
// Consecutive chunks with the same offset list share one copy.  Returns
// false when the slots would not fit 32-bit offsets.
constexpr int kOffsetSlack = 2;
constexpr int kOffsetMax = 32;

struct SellLayout {
  std::vector<int> cptr, coff, offs;
  int offset_chunks = 0;
};

static bool sell_layout(const std::vector<int>& rp, const int* ci, int n, SellLayout& out) {
  const int nc = (n + kSellC - 1) / kSellC;
  out.cptr.assign(nc + 1, 0);
  out.coff.assign(nc, -1);
  out.offs.clear();
  out.offset_chunks = 0;
  int64_t total = 0;
  std::vector<int> u;
  int prev = -1, prev_len = 0;
  for (int c = 0; c < nc; ++c) {
    int L = 0;
    u.clear();
    bool regular = true;
    for (int i = c * kSellC; i < std::min(n, (c + 1) * kSellC); ++i) {
      L = std::max(L, rp[i + 1] - rp[i]);
      for (int k = rp[i]; regular && k < rp[i + 1]; ++k) {
        const int o = ci[k] - i;
        if (std::find(u.begin(), u.end(), o) == u.end()) {
          u.push_back(o);
          if ((int)u.size() > kOffsetMax) regular = false;
        }
      }
    }
    int width = L;
    if (regular && L > 0 && (int)u.size() <= L + kOffsetSlack) {
      std::sort(u.begin(), u.end());
      width = (int)u.size();
      if (prev >= 0 && prev_len == width &&
          std::equal(u.begin(), u.end(), out.offs.begin() + prev)) {
        out.coff[c] = prev;
      } else {
        prev = (int)out.offs.size();
        prev_len = width;
        out.offs.insert(out.offs.end(), u.begin(), u.end());
        out.coff[c] = prev;
      }
      out.offset_chunks++;
    }
    total += (int64_t)width * kSellC;
    if (total > INT32_MAX) return false;
    out.cptr[c + 1] = (int)total;
  }
  return true;
}

// The sliced-ELL arrays are filled on the device from the CSR arrays already
// there (launch_to_sell); only the chunk layout is computed here.
static void upload_sell(gs2_handle* h, DevCsr& M, const std::vector<int>& rp, const int* ci) {
  const int n = M.n;
  if (n == 0 || M.nnz == 0) return;
  if (M.mean_row > kShortRowMean && 12.0 * M.nnz < kSellStreamBytes) return;
  SellLayout lay;
  if (!sell_layout(rp, ci, n, lay) || lay.cptr.back() > kSellMaxPadding * M.nnz) return;
  const std::vector<int>& cptr = lay.cptr;
  const size_t slots = std::max(cptr.back(), 1);
  int ncols = 1;
  for (int k = 0; k < M.nnz; ++k) ncols = std::max(ncols, ci[k] + 1);
  M.sell_chunks = (int)cptr.size() - 1;
  M.sell_slots = (int)slots;
  M.sell_ncols = ncols;
  M.sell_offset_chunks = lay.offset_chunks;
  M.sell_ptr = (int*)h->dalloc(sizeof(int) * cptr.size());
  M.sell_ci = (int*)h->dalloc(sizeof(int) * slots);
  M.sell_va = (double*)h->dalloc(sizeof(double) * slots);
  M.sell_coff = (int*)h->dalloc(sizeof(int) * std::max<size_t>(lay.coff.size(), 1));
  M.sell_off = (int*)h->dalloc(sizeof(int) * std::max<size_t>(lay.offs.size(), 1));
  h->dzero(M.sell_ci, sizeof(int) * slots);
  h->dzero(M.sell_va, sizeof(double) * slots);
  h->h2d(M.sell_ptr, cptr.data(), sizeof(int) * cptr.size());
  h->h2d(M.sell_coff, lay.coff.data(), sizeof(int) * lay.coff.size());
  if (!lay.offs.empty()) h->h2d(M.sell_off, lay.offs.data(), sizeof(int) * lay.offs.size());
  launch_to_sell(h, M, M.va, M.sell_va, true);
  M.sell = true;
}

static void upload_csr(gs2_handle* h, DevCsr& M, int n, const std::vector<int>& rp,
                       const int* ci, const double* va, int nnz) {
  M.n = n;
  M.nnz = nnz;
  M.mean_row = n ? (double)M.nnz / n : 0.0;
  M.tpr = choose_lanes(M.mean_row);
  // every array is padded by kPad entries so that the 16-byte-rounded bulk
  // copies of a tile's slices never leave the allocation
  const size_t nz = (size_t)M.nnz + kPad;
  M.rp = (int*)h->dalloc(sizeof(int) * (n + 1 + kPad));
  M.ci = (int*)h->dalloc(sizeof(int) * nz);
  M.va = (double*)h->dalloc(sizeof(double) * nz);
  h->dzero(M.rp, sizeof(int) * (n + 1 + kPad));
  h->h2d(M.rp, rp.data(), sizeof(int) * (n + 1));
  h->dzero(M.ci, sizeof(int) * nz);
  h->dzero(M.va, sizeof(double) * nz);
  h->h2d(M.ci, ci, sizeof(int) * M.nnz);
  h->h2d(M.va, va, sizeof(double) * M.nnz);
  retile(h, M, rp, M.tpr, 1);
  upload_sell(h, M, rp, ci);
}

// (Re)build the row tiles of M for K lanes per row and RPT rows per lane
// group, and upload their descriptors.
void retile(gs2_handle* h, DevCsr& M, const std::vector<int>& rp, int K, int RPT) {
  std::vector<int> tiles;
  build_tiles(rp, M.n, K, RPT, tiles, M.cap);
  M.tpr = K;
  M.rpt = RPT;
  M.ntiles = (int)tiles.size() - 1;
  std::vector<int4> desc(std::max(M.ntiles, 1));
  for (int t = 0; t < M.ntiles; ++t) {
    const int r0 = tiles[t], r1 = tiles[t + 1];
    const int a = rp[r0], b = rp[r1];
    const bool longrow = (r1 - r0 == 1) && (b - a > kHardCap);
    desc[t] = make_int4(r0, r1, longrow ? -1 - a : (a & ~7), b);
  }
  M.desc = (int4*)h->dalloc(sizeof(int4) * desc.size());
  h->h2d(M.desc, desc.data(), sizeof(int4) * desc.size());
}

// FP32 copy and FP16 copy with per-row scale s_i = max_j |v_ij| of a
// triangle (Sec. 10 single-precision preconditioner; FP16 with row scale
// is an extension of it).
struct HostTri {
  std::vector<int> rp, ci;
  std::vector<double> va;
};

static void prepare_lowprec(gs2_handle* h, DevCsr& M, const HostTri&, int prec) {
  const size_t nz = (size_t)M.nnz + kPad;
  if (prec == GS2_FP32 && !M.va32) {
    // converted on the device from the resident FP64 values (the host loop
    // and the upload were most of a lower-precision request's setup)
    M.va32 = (float*)h->dalloc(sizeof(float) * nz);
    launch_values_to_fp32(h, M, (int64_t)nz);
    if (M.sell_chunks > 0) {  // the layout exists (the autotuner may turn it off and on)
      const size_t slots = M.sell_slots;
      M.sell_va32 = (float*)h->dalloc(sizeof(float) * slots);
      h->dzero(M.sell_va32, sizeof(float) * slots);
      launch_to_sell(h, M, M.va32, M.sell_va32, false);
    }
  }
  if (prec == GS2_FP16_ROWSCALED && !M.va16) {
    // row scale 2^e_i with max_j |v_ij| / 2^e_i in [1/2, 1): scaling by a
    // power of two is exact, so q_ij = fl16(v_ij 2^-e_i) is the only rounding
    // and the row keeps binary16's full precision at any magnitude; e_i is
    // stored in one byte (clamped to [-126, 127], the exponents of a normal
    // FP32 power of two); converted on the device
    M.va16 = (__half*)h->dalloc(sizeof(__half) * nz);
    M.scale16 = (signed char*)h->dalloc(sizeof(signed char) * std::max(M.n, 1));
    h->dzero(M.va16, sizeof(__half) * nz);
    launch_values_to_fp16(h, M);
    if (M.sell_chunks > 0) {  // the layout exists (the autotuner may turn it off and on)
      const size_t slots = M.sell_slots;
      M.sell_va16 = (__half*)h->dalloc(sizeof(__half) * slots);
      h->dzero(M.sell_va16, sizeof(__half) * slots);
      launch_to_sell(h, M, M.va16, M.sell_va16, false);
    }
  }
}

}  // namespace gs2

// host copies of the triangles, kept for lazy precision / level setup
struct gs2_host_side {
  gs2::HostTri L, U;
  gs2::HostTri O;  // D^{-1}(L + U): row i's L entries, then its U entries (built lazily)
  std::vector<int> Arp;  // rowptr of A (re-tiling)
  // local triangles of each hybrid form (low-precision copies), by parts
  std::map<int, std::pair<gs2::HostTri, gs2::HostTri>> hyb;
};
static std::mutex g_host_mu;
static std::unordered_map<const gs2_handle*, gs2_host_side*> g_host;

void* gs2_handle::dalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = async_alloc ? cudaMallocAsync(&p, bytes, stream) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    GS2_THROW(e == cudaErrorMemoryAllocation ? GS2_ERR_OOM : GS2_ERR_CUDA,
              std::string("device allocation of ") + std::to_string(bytes) +
                  " bytes: " + cudaGetErrorString(e));
  }
  allocs.push_back(p);
  dev_bytes += (int64_t)bytes;
  return p;
}

// setup copies are ordered on the handle's stream (pageable sources are
// staged by the CUDA driver before the call returns)
void gs2_handle::h2d(void* dst, const void* src, size_t bytes) {
  if (bytes) GS2_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream));
}

void gs2_handle::dzero(void* dst, size_t bytes) {
  if (bytes) GS2_CUDA(cudaMemsetAsync(dst, 0, bytes, stream));
}

namespace gs2 {

static std::mutex g_pinned_mu;
static std::unordered_map<size_t, std::vector<void*>> g_pinned_free;

void* pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> g(g_pinned_mu);
    auto& v = g_pinned_free[bytes];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      std::memset(p, 0, bytes);
      return p;
    }
  }
  void* p = nullptr;
  GS2_CUDA(cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset(p, 0, bytes);
  return p;
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pinned_mu);
  g_pinned_free[bytes].push_back(p);
}

}  // namespace gs2

namespace gs2 {

static gs2_host_side* host_side(const gs2_handle* h) {
  std::lock_guard<std::mutex> g(g_host_mu);
  auto it = g_host.find(h);
  return it == g_host.end() ? nullptr : it->second;
}

// the longest rows of A, D^{-1}L and D^{-1}U, from the host copies of their
// row pointers (cached in the handle)
void longest_rows(gs2_handle* h) {
  if (h->cl_wa >= 0) return;
  const gs2_host_side* hs = host_side(h);
  auto widest = [](const std::vector<int>& rp) {
    int w = 0;
    for (size_t i = 0; i + 1 < rp.size(); ++i) w = std::max(w, rp[i + 1] - rp[i]);
    return w;
  };
  h->cl_wa = widest(hs->Arp);
  h->cl_wl = widest(hs->L.rp);
  h->cl_wu = widest(hs->U.rp);
}

void ensure_precision(gs2_handle* h, int prec) {
  if (prec == GS2_FP64) return;
  if (prec != GS2_FP32 && prec != GS2_FP16_ROWSCALED && !is_sweep_precision(prec))
    GS2_THROW(GS2_ERR_INVALID_ARG, "unknown precision");
  gs2_host_side* hs = host_side(h);
  const int vprec = value_precision(prec);
  prepare_lowprec(h, h->L, hs->L, vprec);
  prepare_lowprec(h, h->U, hs->U, vprec);
  const size_t n = std::max<int64_t>(h->n, 1);
  if (!h->rhat32) {
    h->rhat32 = (float*)h->dalloc(sizeof(float) * n);
    h->g32a = (float*)h->dalloc(sizeof(float) * n);
    h->g32b = (float*)h->dalloc(sizeof(float) * n);
  }
  if (!is_sweep_precision(prec)) return;
  // the whole-sweep precisions: the prescaled off-diagonal matrix O =
  // D^{-1}(L + U) in the value precision, fl32(D^{-1} b) and the FP32 iterate
  if (h->O.rp == nullptr) {
    HostTri& O = hs->O;
    const int nn = (int)h->n;
    O.rp.assign(nn + 1, 0);
    for (int i = 0; i < nn; ++i)
      O.rp[i + 1] = O.rp[i] + (hs->L.rp[i + 1] - hs->L.rp[i]) + (hs->U.rp[i + 1] - hs->U.rp[i]);
    O.ci.resize(O.rp[nn]);
    O.va.resize(O.rp[nn]);
    for (int i = 0; i < nn; ++i) {
      int k = O.rp[i];
      for (int q = hs->L.rp[i]; q < hs->L.rp[i + 1]; ++q, ++k) {
        O.ci[k] = hs->L.ci[q];
        O.va[k] = hs->L.va[q];
      }
      for (int q = hs->U.rp[i]; q < hs->U.rp[i + 1]; ++q, ++k) {
        O.ci[k] = hs->U.ci[q];
        O.va[k] = hs->U.va[q];
      }
    }
    upload_csr(h, h->O, nn, O.rp, O.ci.data(), O.va.data(), (int)O.ci.size());
  }
  prepare_lowprec(h, h->O, hs->O, vprec);
  if (!h->bhat32) {
    h->bhat32 = (float*)h->dalloc(sizeof(float) * n);
    h->x32 = (float*)h->dalloc(sizeof(float) * n);
  }
}

// Level sets of the triangles (level-set scheduling, Sec. 3): level(i) =
// 1 + max level over row i's dependencies; rows are grouped by level.
// Level sets of a strict triangle: level(i) = 1 + the largest level of the
// rows row i depends on (0 without any); rows grouped by level on the device.
static void build_levels(gs2_handle* h, const HostTri& T, bool lower, std::vector<int>& ptr,
                         int*& rows_dev) {
  const int n = (int)h->n;
  std::vector<int> lev(n, 0);
  int nlev = n ? 1 : 0;
  for (int s = 0; s < n; ++s) {
    const int i = lower ? s : n - 1 - s;
    int lv = 0;
    for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) lv = std::max(lv, lev[T.ci[k]] + 1);
    lev[i] = lv;
    nlev = std::max(nlev, lv + 1);
  }
  ptr.assign(nlev + 1, 0);
  for (int i = 0; i < n; ++i) ptr[lev[i] + 1]++;
  for (int l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1), rows(std::max(n, 1));
  for (int i = 0; i < n; ++i) rows[fill[lev[i]]++] = i;
  rows_dev = (int*)h->dalloc(sizeof(int) * std::max(n, 1));
  h->h2d(rows_dev, rows.data(), sizeof(int) * std::max(n, 1));
}

void ensure_levels(gs2_handle* h) {
  if (h->levels_ready) return;
  gs2_host_side* hs = host_side(h);
  build_levels(h, hs->L, true, h->lev_ptr_L, h->lev_rows_L);
  build_levels(h, hs->U, false, h->lev_ptr_U, h->lev_rows_U);
  h->levels_ready = true;
}

// First-fit colouring in natural row order of the symmetrised pattern
// (rows i, j adjacent if a_ij or a_ji is stored, i != j), then one matrix
// per colour: its rows ascending, their off-diagonal entries prescaled by
// D^{-1} (the L part, then the U part of each row).  Only neighbours j < i
// are coloured when row i is, so the earlier neighbours are the columns of
// row i of L and the rows j < i whose U row holds column i.
void ensure_colors(gs2_handle* h) {
  if (h->colors_ready) return;
  gs2_host_side* hs = host_side(h);
  const int n = (int)h->n;
  const HostTri& L = hs->L;
  const HostTri& U = hs->U;
  std::vector<int> utp(n + 1, 0), uti(U.ci.size());
  for (int k = 0; k < (int)U.ci.size(); ++k) utp[U.ci[k] + 1]++;
  for (int i = 0; i < n; ++i) utp[i + 1] += utp[i];
  {
    std::vector<int> fill(utp.begin(), utp.end() - 1);
    for (int j = 0; j < n; ++j)
      for (int k = U.rp[j]; k < U.rp[j + 1]; ++k) uti[fill[U.ci[k]]++] = j;
  }
  std::vector<int> color(n, -1), mark(n + 1, -1);
  int nc = 0;
  for (int i = 0; i < n; ++i) {
    for (int k = L.rp[i]; k < L.rp[i + 1]; ++k) mark[color[L.ci[k]]] = i;
    for (int k = utp[i]; k < utp[i + 1]; ++k) mark[color[uti[k]]] = i;
    int c = 0;
    while (mark[c] == i) ++c;
    color[i] = c;
    nc = std::max(nc, c + 1);
  }
  h->colors.assign(nc, DevCsr{});
  h->color_rows.assign(nc, nullptr);
  std::vector<std::vector<int>> rows(nc);
  for (int i = 0; i < n; ++i) rows[color[i]].push_back(i);
  for (int c = 0; c < nc; ++c) {
    const std::vector<int>& rr = rows[c];
    std::vector<int> rp(rr.size() + 1, 0), ci;
    std::vector<double> va;
    for (size_t q = 0; q < rr.size(); ++q) {
      const int i = rr[q];
      for (int k = L.rp[i]; k < L.rp[i + 1]; ++k) {
        ci.push_back(L.ci[k]);
        va.push_back(L.va[k]);
      }
      for (int k = U.rp[i]; k < U.rp[i + 1]; ++k) {
        ci.push_back(U.ci[k]);
        va.push_back(U.va[k]);
      }
      rp[q + 1] = (int)ci.size();
    }
    upload_csr(h, h->colors[c], (int)rr.size(), rp, ci.data(), va.data(), (int)ci.size());
    h->color_rows[c] = (int*)h->dalloc(sizeof(int) * std::max<size_t>(rr.size(), 1));
    h->h2d(h->color_rows[c], rr.data(), sizeof(int) * rr.size());
  }
  h->colors_ready = true;
}

Hybrid* find_hybrid(gs2_handle* h, int parts) {
  for (Hybrid* y : h->hybrids)
    if (y->parts == parts) return y;
  return nullptr;
}

// Build the hybrid form with P = min(parts, n) blocks: A's entries split by
// whether the column lies in the row's block (A is read back from the
// device once), the prescaled triangles filtered the same way.
Hybrid* ensure_hybrid(gs2_handle* h, const gs2_params* p) {
  if (!p || p->parts <= 1 || h->n == 0) return nullptr;
  const int n = (int)h->n;
  const int P = (int)std::min<int64_t>(p->parts, n);
  gs2_host_side* hs = host_side(h);
  Hybrid* y = find_hybrid(h, P);
  if (!y) {
    std::vector<int> blk(n);
    for (int q = 0; q < P; ++q)
      for (int64_t i = (int64_t)q * n / P; i < (int64_t)(q + 1) * n / P; ++i) blk[i] = q;
    std::vector<int> rp(n + 1), ci(h->A.nnz);
    std::vector<double> va(h->A.nnz);
    GS2_CUDA(cudaStreamSynchronize(h->stream));
    GS2_CUDA(cudaMemcpy(rp.data(), h->A.rp, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
    if (h->A.nnz) {
      GS2_CUDA(cudaMemcpy(ci.data(), h->A.ci, sizeof(int) * h->A.nnz, cudaMemcpyDeviceToHost));
      GS2_CUDA(cudaMemcpy(va.data(), h->A.va, sizeof(double) * h->A.nnz,
                          cudaMemcpyDeviceToHost));
    }
    std::vector<int> lrp(n + 1, 0), erp(n + 1, 0), lci, eci;
    std::vector<double> lva, eva;
    for (int i = 0; i < n; ++i) {
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        if (blk[ci[k]] == blk[i]) {
          lci.push_back(ci[k]);
          lva.push_back(va[k]);
        } else {
          eci.push_back(ci[k]);
          eva.push_back(va[k]);
        }
      }
      lrp[i + 1] = (int)lci.size();
      erp[i + 1] = (int)eci.size();
    }
    auto local_tri = [&](const HostTri& T) {
      HostTri o;
      o.rp.assign(n + 1, 0);
      for (int i = 0; i < n; ++i) {
        for (int k = T.rp[i]; k < T.rp[i + 1]; ++k)
          if (blk[T.ci[k]] == blk[i]) {
            o.ci.push_back(T.ci[k]);
            o.va.push_back(T.va[k]);
          }
        o.rp[i + 1] = (int)o.ci.size();
      }
      return o;
    };
    auto& tris = hs->hyb[P];
    tris.first = local_tri(hs->L);
    tris.second = local_tri(hs->U);
    y = new Hybrid();
    y->parts = P;
    h->hybrids.push_back(y);
    upload_matrix(h, y->Aloc, n, lrp, lci, lva);
    upload_matrix(h, y->E, n, erp, eci, eva);
    upload_matrix(h, y->Lloc, n, tris.first.rp, tris.first.ci, tris.first.va);
    upload_matrix(h, y->Uloc, n, tris.second.rp, tris.second.ci, tris.second.va);
    y->c = (double*)h->dalloc(sizeof(double) * n);
  }
  if (p->kind == GS2_PC_GS2 && p->precision != GS2_FP64) {
    auto& tris = hs->hyb[P];
    prepare_lowprec(h, y->Lloc, tris.first, p->precision);
    prepare_lowprec(h, y->Uloc, tris.second, p->precision);
  }
  if (p->kind == GS2_PC_GS && !y->levels_ready) {
    // local exact GS: level sets of the local triangles (each block's own
    // dependency chains side by side)
    auto& tris = hs->hyb[P];
    build_levels(h, tris.first, true, y->lev_ptr_L, y->lev_rows_L);
    build_levels(h, tris.second, false, y->lev_ptr_U, y->lev_rows_U);
    y->levels_ready = true;
  }
  return y;
}

void ensure_precond(gs2_handle* h, const gs2_params* p) {
  if (!p) return;
  ensure_hybrid(h, p);
  if (p->kind == GS2_PC_GS) ensure_levels(h);
  if (p->kind == GS2_PC_MTGS) ensure_colors(h);
  if (p->kind == GS2_PC_AMG || p->kind == GS2_PC_AMG_JR) amg_prepare(h, p);
}

void upload_matrix(gs2_handle* h, DevCsr& M, int n, const std::vector<int>& rp,
                   const std::vector<int>& ci, const std::vector<double>& va) {
  upload_csr(h, M, n, rp, ci.data(), va.data(), (int)ci.size());
}

// ---------------------------------------------------------------------------
// autotuner: tile shape (lanes per row K, rows per lane group RPT) per matrix
// ---------------------------------------------------------------------------

// Best choices found so far -- row-tile shape (K, RPT) and whether the
// sliced-ELL layout is used -- by (matrix role, n to a factor sqrt(2), mean
// row length to a quarter): matrices of the same class reuse a measurement.
struct TuneChoice {
  int K, RPT;
  bool sell;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, TuneChoice> g_tune;

static void tune_matrix(gs2_handle* h, DevCsr& M, const std::vector<int>& rp, int role) {
  if (M.n == 0 || M.nnz == 0) return;
  const auto key = std::make_tuple(role, (int)std::lround(2.0 * std::log2((double)M.n)),
                                   (int)std::lround(4.0 * M.mean_row));
  // whether M has a sliced-ELL copy at all (padding of at most 20%)
  const bool has_sell = M.sell_chunks > 0;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const TuneChoice& c = it->second;
      if (c.K != M.tpr || c.RPT != M.rpt) retile(h, M, rp, c.K, c.RPT);
      M.sell = has_sell && c.sell;
      return;
    }
  }
  // the sliced-ELL layout against the best row-tile shape: SELL is kept
  // unless the tiles are at least 2% faster
  float sell_ms = 0.f;
  if (has_sell) {
    M.sell = true;
    sell_ms = time_tile_probe(h, M, 5, role);
    M.sell = false;
  }
  // candidates around the mean-row-length heuristic
  const int kh = choose_lanes(M.mean_row);
  std::vector<std::pair<int, int>> cand;
  for (int K : {1, 2, 4, 8, 16}) {
    if (2 * K < kh || K > 2 * kh) continue;
    cand.emplace_back(K, 1);
    if (K <= 2) cand.emplace_back(K, 2);
  }
  // the heuristic shape is timed first; another shape must beat it by 2%,
  // so timing noise does not flip the choice between near-equal shapes
  std::pair<int, int> best{M.tpr, M.rpt};
  float best_ms = time_tile_probe(h, M, 5, role);
  for (const auto& c : cand) {
    if (c == best) continue;
    retile(h, M, rp, c.first, c.second);
    const float ms = time_tile_probe(h, M, 5, role);
    if (ms < 0.98f * best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  retile(h, M, rp, best.first, best.second);
  M.sell = has_sell && !(best_ms < 0.98f * sell_ms);
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[key] = TuneChoice{best.first, best.second, M.sell};
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host-vector staging: device pointers pass through; host vectors are
// copied to the handle's staging buffers and x is copied back at the end.
struct Staged {
  gs2_handle* h;
  const double* b;
  double* x;
  double* x_user;
  bool host_x = false;
  Staged(gs2_handle* h_, const double* b_user, double* x_user_, bool x_in)
      : h(h_), b(b_user), x(x_user_), x_user(x_user_) {
    const size_t bytes = sizeof(double) * h->n;
    if (b_user && !is_device_ptr(b_user)) {
      GS2_CUDA(cudaMemcpyAsync(h->bstage, b_user, bytes, cudaMemcpyHostToDevice, h->stream));
      b = h->bstage;
    }
    if (x_user_ && !is_device_ptr(x_user_)) {
      host_x = true;
      if (x_in)
        GS2_CUDA(cudaMemcpyAsync(h->xstage, x_user_, bytes, cudaMemcpyHostToDevice,
                                 h->stream));
      x = h->xstage;
    }
  }
  void finish() {
    if (host_x) {
      GS2_CUDA(cudaMemcpyAsync(x_user, h->xstage, sizeof(double) * h->n,
                               cudaMemcpyDeviceToHost, h->stream));
      GS2_CUDA(cudaStreamSynchronize(h->stream));
    } else if (b != nullptr && b == h->bstage) {
      GS2_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
};

static void check_params(const gs2_params* p) {
  if (!p) return;
  if (p->kind < GS2_PC_NONE || p->kind > GS2_PC_AMG_JR)
    GS2_THROW(GS2_ERR_INVALID_ARG, "unknown preconditioner kind");
  if (p->kind == GS2_PC_NONE) return;
  if (p->outer < 1 || p->outer > 1000) GS2_THROW(GS2_ERR_INVALID_ARG, "outer sweeps < 1");
  if (p->inner < 0 || p->inner > 100000) GS2_THROW(GS2_ERR_INVALID_ARG, "inner sweeps < 0");
  if (!(p->omega > 0.0) || !std::isfinite(p->omega))
    GS2_THROW(GS2_ERR_INVALID_ARG, "omega must be > 0");
  if (!(p->gamma > 0.0) || !std::isfinite(p->gamma))
    GS2_THROW(GS2_ERR_INVALID_ARG, "gamma must be > 0");
  if (p->direction < 0 || p->direction > 2) GS2_THROW(GS2_ERR_INVALID_ARG, "direction");
  if (p->precision < 0 || p->precision > 4) GS2_THROW(GS2_ERR_INVALID_ARG, "precision");
  if (is_sweep_precision(p->precision) &&
      (p->kind != GS2_PC_GS2 || p->form != GS2_NONCOMPACT || p->parts > 1))
    GS2_THROW(GS2_ERR_INVALID_ARG,
              "the whole-sweep precisions are for non-compact, non-hybrid GS2");
  if (p->form != GS2_NONCOMPACT && p->form != GS2_COMPACT)
    GS2_THROW(GS2_ERR_INVALID_ARG, "form");
  if (p->form == GS2_COMPACT && (p->kind != GS2_PC_GS2 || p->omega != 1.0 || p->gamma != 1.0))
    GS2_THROW(GS2_ERR_INVALID_ARG, "the compact form is undamped GS2 (omega = gamma = 1)");
  if (p->parts < 0 || p->local_sweeps < 0 || p->local_sweeps > 1000)
    GS2_THROW(GS2_ERR_INVALID_ARG, "parts and local_sweeps must be >= 0");
  if ((p->parts > 1 || p->local_sweeps > 1) && p->kind != GS2_PC_GS2 && p->kind != GS2_PC_JR &&
      p->kind != GS2_PC_GS)
    GS2_THROW(GS2_ERR_INVALID_ARG, "the hybrid form and local sweeps are for GS2, JR and GS");
  if (p->parts > 1 && p->form == GS2_COMPACT)
    GS2_THROW(GS2_ERR_INVALID_ARG, "the hybrid form is non-compact");
}

}  // namespace gs2

using namespace gs2;

#define API_BEGIN try {
#define API_END                                        \
  }                                                    \
  catch (const gs2::Error& e) {                        \
    gs2::set_error(e.msg);                             \
    return e.st;                                       \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    gs2::set_error("host allocation failed");          \
    return GS2_ERR_OOM;                                \
  }                                                    \
  catch (...) {                                        \
    gs2::set_error("unexpected C++ exception");        \
    return GS2_ERR_CUDA;                               \
  }

// Release a handle.  Stream-ordered handles free their device memory on
// their own stream (no device-wide synchronisation); the small pinned
// mirrors go back to the process-wide pool.
void gs2::destroy_handle(gs2_handle* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gstream) cudaStreamSynchronize(h->gstream);
  if (h->amg) amg_free(h);
  if (h->pack) pack_free(h);
  for (Hybrid* y : h->hybrids) delete y;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cg_gexec) cudaGraphExecDestroy(h->cg_gexec);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->gev_in) cudaEventDestroy(h->gev_in);
  if (h->gev_out) cudaEventDestroy(h->gev_out);
  delete h->prof;
  for (void* p : h->allocs) {
    if (h->async_alloc) cudaFreeAsync(p, h->stream);
    else cudaFree(p);
  }
  pinned_put(h->st_host, sizeof(KrylovState));
  pinned_put(h->err_host, sizeof(int));
  pinned_put((void*)h->stop_mapped, sizeof(int));
  {
    std::lock_guard<std::mutex> g(g_host_mu);
    auto it = g_host.find(h);
    if (it != g_host.end()) {
      delete it->second;
      g_host.erase(it);
    }
  }
  delete h;
  cudaSetDevice(cur);
}

static void destroy_impl(gs2_handle* h) { gs2::destroy_handle(h); }

extern "C" {

const char* gs2_last_error(void) { return g_last_error.c_str(); }

const char* gs2_version(void) { return "gs2-gb300 0.1 (sm_103a)"; }

int64_t gs2_launch_count(void) { return (int64_t)g_launches.load(); }

gs2_status gs2_setup(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                     const double* val, int on_device, unsigned precisions, void* stream,
                     gs2_handle** out) {
  if (!out) {
    set_error("out is NULL");
    return GS2_ERR_INVALID_ARG;
  }
  *out = nullptr;
  API_BEGIN
  NvtxRange nvtx_("gs2_setup");
  *out = setup_handle(n, nnz, rowptr, col, val, on_device, precisions, (cudaStream_t)stream,
                      false);
  return GS2_OK;
  API_END
}

}  // extern "C"

// Validate a host CSR matrix (rowptr, column range, duplicates, nonzero
// finite diagonal) over parallel row ranges and return its diagonal; the
// first bad row in row order is reported.
void gs2::validate_csr(int64_t n, int64_t nnz, const int64_t* RP, const int32_t* CI,
                       const double* VA, std::vector<double>* diag_out) {
  if (RP[0] != 0 || RP[n] != nnz)
    GS2_THROW(GS2_ERR_INVALID_ARG, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  for (int64_t i = 0; i < n; ++i)
    if (RP[i + 1] < RP[i]) GS2_THROW(GS2_ERR_INVALID_ARG, "rowptr is not monotone");
  std::vector<double>& diag = *diag_out;
  diag.assign(n, 0.0);
  struct RowError {
    int64_t row = std::numeric_limits<int64_t>::max();
    gs2_status st = GS2_OK;
    const char* what = "";
  };
  std::vector<RowError> errs(kHostThreads);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int tid) {
    std::vector<int32_t> cols;
    for (int64_t i = i0; i < i1; ++i) {
      const int64_t a = RP[i], e = RP[i + 1];
      const char* what = nullptr;
      gs2_status st = GS2_ERR_INVALID_ARG;
      for (int64_t k = a; k < e && !what; ++k)
        if (CI[k] < 0 || CI[k] >= n) what = "column index out of range in row ";
      if (!what) {
        if (e - a <= 32) {
          for (int64_t k = a; k < e && !what; ++k)
            for (int64_t q = k + 1; q < e; ++q)
              if (CI[q] == CI[k]) {
                what = "duplicate entry in row ";
                break;
              }
        } else {
          cols.assign(CI + a, CI + e);
          std::sort(cols.begin(), cols.end());
          if (std::adjacent_find(cols.begin(), cols.end()) != cols.end())
            what = "duplicate entry in row ";
        }
      }
      if (!what) {
        bool has_diag = false;
        for (int64_t k = a; k < e; ++k)
          if (CI[k] == i) {
            has_diag = true;
            diag[i] = VA[k];
          }
        if (!has_diag || diag[i] == 0.0 || !std::isfinite(diag[i])) {
          what = "zero or missing diagonal in row ";
          st = GS2_ERR_ZERO_DIAGONAL;
        }
      }
      if (what) {
        errs[tid] = RowError{i, st, what};
        return;
      }
    }
  });
  const RowError* first = &errs[0];
  for (const RowError& e : errs)
    if (e.row < first->row) first = &e;
  if (first->st != GS2_OK) GS2_THROW(first->st, first->what + std::to_string(first->row));
}

// Validate A, split it, upload everything and allocate the resident
// temporaries.  Throws gs2::Error; a partly built handle is released.
gs2_handle* gs2::setup_handle(int64_t n, int64_t nnz, const int64_t* rowptr,
                              const int32_t* col, const double* val, int on_device,
                              unsigned precisions, cudaStream_t stream, bool async_alloc) {
  gs2_handle* h = nullptr;
  try {
  if (n < 0 || nnz < 0) GS2_THROW(GS2_ERR_INVALID_ARG, "negative size");
  if (n > std::numeric_limits<int>::max() - 1 || nnz > std::numeric_limits<int>::max() - 64)
    GS2_THROW(GS2_ERR_INVALID_ARG, "n or nnz above 2^31 - 1");
  if (!rowptr || (nnz > 0 && (!col || !val)))
    GS2_THROW(GS2_ERR_INVALID_ARG, "NULL CSR array");
  // the input on the host: the caller's arrays, or copies of device arrays
  std::vector<int64_t> rp_copy;
  std::vector<int32_t> ci_copy;
  std::vector<double> va_copy;
  const int64_t* RP = rowptr;
  const int32_t* CI = col;
  const double* VA = val;
  if (on_device) {
    rp_copy.resize(n + 1);
    ci_copy.resize(nnz);
    va_copy.resize(nnz);
    GS2_CUDA(cudaMemcpy(rp_copy.data(), rowptr, sizeof(int64_t) * (n + 1),
                        cudaMemcpyDeviceToHost));
    if (nnz) {
      GS2_CUDA(cudaMemcpy(ci_copy.data(), col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
      GS2_CUDA(cudaMemcpy(va_copy.data(), val, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    }
    RP = rp_copy.data();
    CI = ci_copy.data();
    VA = va_copy.data();
  }
  // validation, row ranges in parallel; the first bad row (in row order) is
  // reported
  std::vector<double> diag;
  validate_csr(n, nnz, RP, CI, VA, &diag);
  // split A = L + D + U, triangles prescaled by D^{-1} (Sec. 6.1.3): count
  // per row, prefix sums, fill, row ranges in parallel
  std::vector<int> rp32(n + 1);
  for (int64_t i = 0; i <= n; ++i) rp32[i] = (int)RP[i];
  auto* hs = new gs2_host_side();
  HostTri& L = hs->L;
  HostTri& U = hs->U;
  L.rp.assign(n + 1, 0);
  U.rp.assign(n + 1, 0);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t k = RP[i]; k < RP[i + 1]; ++k) {
        if (CI[k] < i) L.rp[i + 1]++;
        else if (CI[k] > i) U.rp[i + 1]++;
      }
  });
  for (int64_t i = 0; i < n; ++i) {
    L.rp[i + 1] += L.rp[i];
    U.rp[i + 1] += U.rp[i];
  }
  L.ci.resize(L.rp[n]);
  L.va.resize(L.rp[n]);
  U.ci.resize(U.rp[n]);
  U.va.resize(U.rp[n]);
  std::vector<double> dinv(n);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i) {
      const double di = 1.0 / diag[i];
      dinv[i] = di;
      int ql = L.rp[i], qu = U.rp[i];
      for (int64_t k = RP[i]; k < RP[i + 1]; ++k) {
        const int j = CI[k];
        if (j < i) {
          L.ci[ql] = j;
          L.va[ql++] = VA[k] * di;
        } else if (j > i) {
          U.ci[qu] = j;
          U.va[qu++] = VA[k] * di;
        }
      }
    }
  });
  h = new gs2_handle();
  {
    std::lock_guard<std::mutex> g(g_host_mu);
    g_host[h] = hs;
  }
  GS2_CUDA(cudaGetDevice(&h->device));
  GS2_CUDA(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
  h->stream = stream;
  h->async_alloc = async_alloc;
  h->n = n;
  h->nnz = nnz;
  upload_csr(h, h->A, (int)n, rp32, CI, VA, (int)nnz);
  hs->Arp = rp32;
  upload_csr(h, h->L, (int)n, L.rp, L.ci.data(), L.va.data(), (int)L.ci.size());
  upload_csr(h, h->U, (int)n, U.rp, U.ci.data(), U.va.data(), (int)U.ci.size());
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  h->dinv = (double*)h->dalloc(sizeof(double) * nv);
  h->dev_err = (int*)h->dalloc(sizeof(int));
  h->dzero(h->dev_err, sizeof(int));
  h->h2d(h->dinv, dinv.data(), sizeof(double) * n);
  h->r = (double*)h->dalloc(sizeof(double) * nv);
  h->rhat = (double*)h->dalloc(sizeof(double) * nv);
  h->g0 = (double*)h->dalloc(sizeof(double) * nv);
  h->g1 = (double*)h->dalloc(sizeof(double) * nv);
  h->z = (double*)h->dalloc(sizeof(double) * nv);
  h->t = (double*)h->dalloc(sizeof(double) * nv);
  h->bstage = (double*)h->dalloc(sizeof(double) * nv);
  h->xstage = (double*)h->dalloc(sizeof(double) * nv);
  h->nblk = vec_blocks(h, n);
  // reductions: at least ~16 rows per thread and one block per SM (the
  // widest CGS2 kernels hold ~150 registers per thread, one 256-thread block
  // per SM), so the per-block reduction stays small next to the FP64 work
  h->nblk_dot = (int)std::max<int64_t>(
      1, std::min<int64_t>((n + kVecThreads * 16 - 1) / (kVecThreads * 16), h->nsm));
  h->part_cap = h->nblk * (kMaxRestart + 2);
  h->part = (double*)h->dalloc(sizeof(double) * h->part_cap);
  for (int p = 1; p <= 4; ++p)
    if (precisions & (1u << p)) ensure_precision(h, p);
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  return h;
  } catch (...) {
    destroy_handle(h);
    throw;
  }
}

extern "C" {

void gs2_destroy(gs2_handle* h) { destroy_impl(h); }

gs2_status gs2_set_stream(gs2_handle* h, void* stream) {
  if (!h) return GS2_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return GS2_OK;
}

gs2_status gs2_get_stats(const gs2_handle* h, gs2_handle_stats* out) {
  if (!h || !out) return GS2_ERR_INVALID_ARG;
  out->n = h->n;
  out->nnz = h->nnz;
  out->nnz_lower = h->L.nnz;
  out->nnz_upper = h->U.nnz;
  out->levels_lower = h->levels_ready ? (int)h->lev_ptr_L.size() - 1 : 0;
  out->levels_upper = h->levels_ready ? (int)h->lev_ptr_U.size() - 1 : 0;
  out->device_bytes = h->dev_bytes + amg_device_bytes(h);
  out->tpr_a = h->A.tpr;
  out->tpr_tri = h->L.tpr;
  out->rpt_a = h->A.rpt;
  out->rpt_tri = h->L.rpt;
  out->colors = h->colors_ready ? (int)h->colors.size() : 0;
  out->sell_a = h->A.sell ? 1 : 0;
  out->sell_tri = h->L.sell ? 1 : 0;
  out->offset_frac_a =
      h->A.sell_chunks ? (double)h->A.sell_offset_chunks / h->A.sell_chunks : 0.0;
  out->offset_frac_tri =
      h->L.sell_chunks ? (double)h->L.sell_offset_chunks / h->L.sell_chunks : 0.0;
  out->solve_mode = h->tuned_mode;
  out->solve_modes_timed = h->tuned_candidates;
  return GS2_OK;
}

gs2_status gs2_apply_ex(gs2_handle* h, const double* b, double* x, const gs2_params* p) {
  if (!h || !p || (h->n && (!b || !x))) {
    set_error("NULL argument");
    return GS2_ERR_INVALID_ARG;
  }
  API_BEGIN
  NvtxRange nvtx_("gs2_apply_ex");
  gs2_params q = *p;
  q.kind = GS2_PC_GS2;
  check_params(&q);
  if (q.outer == 0 || h->n == 0) return GS2_OK;
  ensure_precision(h, q.precision);
  Staged s(h, b, x, true);
  gs2_relax(h, s.b, s.x, &q);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status gs2_apply(gs2_handle* h, const double* b, double* x, int outer_sweeps,
                     int inner_sweeps, double damping, int direction) {
  if (outer_sweeps == 0) return h ? GS2_OK : GS2_ERR_INVALID_ARG;
  gs2_params p{GS2_PC_GS2, outer_sweeps, inner_sweeps, damping, 1.0, direction,
               GS2_FP64, GS2_NONCOMPACT};
  return gs2_apply_ex(h, b, x, &p);
}

gs2_status relax_apply(gs2_handle* h, const double* b, double* x, const gs2_params* p) {
  if (!h || !p || (h->n && (!b || !x))) {
    set_error("NULL argument");
    return GS2_ERR_INVALID_ARG;
  }
  API_BEGIN
  NvtxRange nvtx_("relax_apply");
  check_params(p);
  if (p->kind != GS2_PC_GS2 && p->kind != GS2_PC_JR && p->kind != GS2_PC_GS &&
      p->kind != GS2_PC_MTGS)
    GS2_THROW(GS2_ERR_INVALID_ARG, "relax_apply takes kinds GS2, JR, GS and MTGS");
  if (h->n == 0) return GS2_OK;
  if (p->kind == GS2_PC_GS2) ensure_precision(h, p->precision);
  ensure_precond(h, p);
  Staged s(h, b, x, true);
  gs2_relax(h, s.b, s.x, p);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status gs_apply(gs2_handle* h, const double* b, double* x, int sweeps, double omega,
                    int direction) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs_apply");
  if (sweeps < 0 || !(omega > 0.0) || direction < 0 || direction > 2)
    GS2_THROW(GS2_ERR_INVALID_ARG, "bad sweeps/omega/direction");
  if (sweeps == 0 || h->n == 0) return GS2_OK;
  ensure_levels(h);
  Staged s(h, b, x, true);
  gs_relax(h, s.b, s.x, sweeps, omega, direction);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status mtgs_apply(gs2_handle* h, const double* b, double* x, int sweeps, double omega,
                      int direction) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("mtgs_apply");
  if (sweeps < 0 || !(omega > 0.0) || direction < 0 || direction > 2)
    GS2_THROW(GS2_ERR_INVALID_ARG, "bad sweeps/omega/direction");
  if (sweeps == 0 || h->n == 0) return GS2_OK;
  ensure_colors(h);
  Staged s(h, b, x, true);
  mtgs_relax(h, s.b, s.x, sweeps, omega, direction);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status gs2_amg_setup(gs2_handle* h, const gs2_amg_cfg* cfg) {
  if (!h) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_amg_setup");
  gs2_amg_cfg c{0.25, 10, 64};
  if (cfg) c = *cfg;
  if (h->n == 0) GS2_THROW(GS2_ERR_INVALID_ARG, "AMG of an empty matrix");
  amg_build(h, c);
  return GS2_OK;
  API_END
}

gs2_status gs2_amg_info(const gs2_handle* h, int* levels, int64_t* rows, int64_t* nnz,
                        int64_t* pnnz) {
  if (!h || !levels) return GS2_ERR_INVALID_ARG;
  amg_info(h, levels, rows, nnz, pnnz);
  return GS2_OK;
}

gs2_status gs2_amg_vcycle(gs2_handle* h, const double* b, double* x, const gs2_params* p) {
  if (!h || !p || (h->n && (!b || !x))) {
    set_error("NULL argument");
    return GS2_ERR_INVALID_ARG;
  }
  API_BEGIN
  NvtxRange nvtx_("gs2_amg_vcycle");
  if (p->kind != GS2_PC_AMG && p->kind != GS2_PC_AMG_JR)
    GS2_THROW(GS2_ERR_INVALID_ARG, "kind must be GS2_PC_AMG or GS2_PC_AMG_JR");
  check_params(p);
  if (h->n == 0) return GS2_OK;
  amg_prepare(h, p);
  Staged s(h, b, x, false);
  amg_vcycle(h, p, s.b, s.x, false, nullptr);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status jr_apply(gs2_handle* h, const double* b, double* x, int sweeps, double omega) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("jr_apply");
  if (sweeps < 0 || !(omega > 0.0)) GS2_THROW(GS2_ERR_INVALID_ARG, "bad sweeps/omega");
  if (sweeps == 0 || h->n == 0) return GS2_OK;
  Staged s(h, b, x, true);
  jr_relax(h, s.b, s.x, sweeps, omega);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status gs2_spmv(gs2_handle* h, const double* x, double* y) {
  if (!h || (h->n && (!x || !y))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_spmv");
  if (h->n == 0) return GS2_OK;
  Staged s(h, x, y, false);
  launch_spmv(h, s.b, s.x, nullptr);
  s.finish();
  return GS2_OK;
  API_END
}

gs2_status gmres_solve(gs2_handle* h, const double* b, double* x, int restart, double tol,
                       int max_iters, const gs2_params* precond, gs2_solve_info* info) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gmres_solve");
  if (restart < 1 || restart > kMaxRestart || !(tol >= 0.0) || max_iters < 0)
    GS2_THROW(GS2_ERR_INVALID_ARG, "restart must be in [1, 64], tol >= 0, max_iters >= 0");
  check_params(precond);
  if (precond && precond->kind == GS2_PC_GS2) ensure_precision(h, precond->precision);
  ensure_precond(h, precond);
  Staged s(h, b, x, true);
  gs2_status st = gmres_run(h, s.b, s.x, restart, tol, max_iters, precond, info);
  s.finish();
  return st;
  API_END
}

gs2_status cg_solve(gs2_handle* h, const double* b, double* x, double tol, int max_iters,
                    const gs2_params* precond, gs2_solve_info* info) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("cg_solve");
  if (!(tol >= 0.0) || max_iters < 0) GS2_THROW(GS2_ERR_INVALID_ARG, "tol/max_iters");
  check_params(precond);
  if (precond && precond->kind == GS2_PC_GS2) ensure_precision(h, precond->precision);
  ensure_precond(h, precond);
  Staged s(h, b, x, true);
  gs2_status st = cg_run(h, s.b, s.x, tol, max_iters, precond, info);
  s.finish();
  return st;
  API_END
}

gs2_status gs2_batch_solve(gs2_handle* const* hs, const double* const* bs, double* const* xs,
                           int count, int restart, double tol, int max_iters,
                           const gs2_params* precond, gs2_solve_info* infos) {
  if (count < 0 || (count > 0 && (!hs || !bs || !xs))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_batch_solve");
  if (restart < 1 || restart > kMaxRestart || !(tol >= 0.0) || max_iters < 0)
    GS2_THROW(GS2_ERR_INVALID_ARG, "restart must be in [1, 64], tol >= 0, max_iters >= 0");
  check_params(precond);
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) GS2_THROW(GS2_ERR_INVALID_ARG, "NULL handle in batch");
    if (hs[i]->n && (!is_device_ptr(bs[i]) || !is_device_ptr(xs[i])))
      GS2_THROW(GS2_ERR_INVALID_ARG, "batch vectors must be device pointers");
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) GS2_THROW(GS2_ERR_INVALID_ARG, "a handle appears twice in a batch");
    if (precond && precond->kind == GS2_PC_GS2) ensure_precision(hs[i], precond->precision);
    ensure_precond(hs[i], precond);
  }
  return gmres_batch(hs, bs, xs, count, restart, tol, max_iters, precond, infos);
  API_END
}

gs2_status gs2_pack_setup(int count, const int64_t* n, const int64_t* const* rowptr,
                          const int32_t* const* col, const double* const* val,
                          unsigned precisions, void* stream, gs2_handle** out) {
  if (!out) {
    set_error("out is NULL");
    return GS2_ERR_INVALID_ARG;
  }
  *out = nullptr;
  API_BEGIN
  NvtxRange nvtx_("gs2_pack_setup");
  std::vector<int64_t> off, rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
  pack_concat(count, n, rowptr, col, val, off, rp, ci, va);
  gs2_handle* h = nullptr;
  try {
    h = setup_handle(off.back(), (int64_t)ci.size(), rp.data(), ci.data(), va.data(), 0,
                     precisions, (cudaStream_t)stream, false);
  } catch (const gs2::Error& e) {
    // "... in row <g>": name the system and its own row
    const size_t sp = e.msg.find_last_of(' ');
    if (sp != std::string::npos && e.msg.find(" in row ") != std::string::npos) {
      const int64_t g = std::stoll(e.msg.substr(sp + 1));
      const int sys = (int)(std::upper_bound(off.begin(), off.end(), g) - off.begin()) - 1;
      GS2_THROW(e.st, "system " + std::to_string(sys) + ": " + e.msg.substr(0, sp + 1) +
                          std::to_string(g - off[sys]));
    }
    throw;
  }
  try {
    pack_attach(h, off);
  } catch (...) {
    destroy_handle(h);
    throw;
  }
  *out = h;
  return GS2_OK;
  API_END
}

gs2_status gs2_pack_info(const gs2_handle* h, int* count, int64_t* offsets) {
  if (!h || !count) return GS2_ERR_INVALID_ARG;
  *count = pack_count(h);
  if (offsets && *count) {
    const std::vector<int64_t>& off = *pack_offsets(h);
    std::copy(off.begin(), off.end(), offsets);
  }
  return GS2_OK;
}

gs2_status gs2_pack_gmres(gs2_handle* h, const double* b, double* x, int restart, double tol,
                          int max_iters, const gs2_params* precond, gs2_solve_info* infos) {
  if (!h || (h->n && (!b || !x))) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_pack_gmres");
  if (!h->pack) GS2_THROW(GS2_ERR_INVALID_ARG, "the handle is not a pack (gs2_pack_setup)");
  if (restart < 1 || restart > kMaxRestart || !(tol >= 0.0) || max_iters < 0)
    GS2_THROW(GS2_ERR_INVALID_ARG, "restart must be in [1, 64], tol >= 0, max_iters >= 0");
  check_params(precond);
  if (precond && (precond->kind == GS2_PC_AMG || precond->kind == GS2_PC_AMG_JR))
    GS2_THROW(GS2_ERR_INVALID_ARG, "a pack takes no AMG preconditioner");
  if (precond && precond->parts > 1)
    GS2_THROW(GS2_ERR_INVALID_ARG, "a pack takes no hybrid preconditioner (its blocks would "
                                   "cut across the systems)");
  if (precond && precond->kind == GS2_PC_GS2) ensure_precision(h, precond->precision);
  ensure_precond(h, precond);
  Staged s(h, b, x, true);
  gs2_status st = pack_gmres_run(h, s.b, s.x, restart, tol, max_iters, precond, infos);
  s.finish();
  return st;
  API_END
}

gs2_status gs2_profile_enable(gs2_handle* h, int enable) {
  if (!h) return GS2_ERR_INVALID_ARG;
  if (!h->prof) h->prof = new gs2::Profiler();
  h->prof->enabled = enable != 0;
  h->prof->epoch++;
  return GS2_OK;
}

gs2_status gs2_autotune(gs2_handle* h) {
  if (!h) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_autotune");
  if (h->n == 0) return GS2_OK;
  gs2_host_side* hs = host_side(h);
  h->dzero(h->t, sizeof(double) * h->n);
  h->dzero(h->z, sizeof(double) * h->n);
  tune_matrix(h, h->A, hs->Arp, 0);
  tune_matrix(h, h->L, hs->L.rp, 1);
  tune_matrix(h, h->U, hs->U.rp, 2);
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  // cached CUDA graphs hold the old tile shapes
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gkey.clear();
  }
  if (h->cg_gexec) {
    cudaGraphExecDestroy(h->cg_gexec);
    h->cg_gexec = nullptr;
    h->cg_gkey.clear();
  }
  pack_drop_graph(h);
  return GS2_OK;
  API_END
}

gs2_status gs2_autotune_gmres(gs2_handle* h, int restart, const gs2_params* precond,
                              int* mode_out) {
  if (!h) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  NvtxRange nvtx_("gs2_autotune_gmres");
  if (restart < 1 || restart > kMaxRestart)
    GS2_THROW(GS2_ERR_INVALID_ARG, "restart must be in [1, 64]");
  check_params(precond);
  if (precond && precond->kind == GS2_PC_GS2) ensure_precision(h, precond->precision);
  ensure_precond(h, precond);
  const int mode = h->n ? autotune_gmres(h, restart, precond) : 1;
  if (mode_out) *mode_out = mode;
  return GS2_OK;
  API_END
}

gs2_status gs2_set_graph_mode(gs2_handle* h, int mode) {
  if (!h || mode < 0 || mode > 4) return GS2_ERR_INVALID_ARG;
  h->graph_mode = mode;
  return GS2_OK;
}

gs2_status gs2_test_stall_barrier(gs2_handle* h) {
  if (!h) return GS2_ERR_INVALID_ARG;
  h->stall_barrier = true;
  return GS2_OK;
}

gs2_status gs2_check(gs2_handle* h) {
  if (!h) return GS2_ERR_INVALID_ARG;
  API_BEGIN
  GS2_CUDA(cudaStreamSynchronize(h->stream));
  int e = 0;
  GS2_CUDA(cudaMemcpy(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    GS2_CUDA(cudaMemset(h->dev_err, 0, sizeof(int)));
    GS2_THROW((gs2_status)e, "a device-side bounded wait gave up (copy never completed)");
  }
  return GS2_OK;
  API_END
}

gs2_status gs2_profile_filter(gs2_handle* h, const char* name) {
  if (!h) return GS2_ERR_INVALID_ARG;
  if (!h->prof) h->prof = new gs2::Profiler();
  h->prof->only = name ? name : "";
  h->prof->epoch++;
  return GS2_OK;
}

gs2_status gs2_profile_read(gs2_handle* h, gs2_kernel_stat* out, int cap, int* count) {
  if (!h || !count || (cap > 0 && !out)) return GS2_ERR_INVALID_ARG;
  *count = 0;
  if (!h->prof) return GS2_OK;
  h->prof->resolve(h->stream);
  const int m = std::min<int>(cap, (int)h->prof->stats.size());
  for (int i = 0; i < m; ++i) out[i] = h->prof->stats[i];
  *count = m;
  return GS2_OK;
}

gs2_status gs2_profile_reset(gs2_handle* h) {
  if (!h) return GS2_ERR_INVALID_ARG;
  if (!h->prof) return GS2_OK;
  h->prof->resolve(h->stream);
  for (auto& s : h->prof->stats) {
    s.launches = 0;
    s.total_ms = 0;
    s.bytes = 0;
  }
  return GS2_OK;
}

}  // extern "C"
