// Smoothed-aggregation algebraic multigrid with GS2 (or JR) as the smoother
// of a V-cycle -- the second role the paper gives the two-stage iteration
// (its Nalu-Wind runs, Sec. 11.2, smooth an AMG V-cycle with one GS2 sweep
// per level).
//
// Setup runs on the host once per matrix: classical strength of connection
// (j is strong for i if |a_ij| >= theta max_{k != i} |a_ik|, theta = 0.25 as
// in the paper's C-AMG runs), symmetrised; greedy aggregation in natural row
// order (seed aggregates from rows whose neighbourhood is free, attach the
// rest to a neighbouring seed aggregate, seed new aggregates from what is
// left); unit-norm constant tentative prolongator P0; smoothed prolongator
// P = (I - w D^{-1} A) P0 with w = 4 / (3 rho), rho the Gershgorin bound of
// rho(D^{-1} A); Galerkin coarse operator A_c = P^T A P.  Every coarse level
// becomes a full library handle (row tiles, prescaled triangles, resident
// temporaries), so the smoother is the same GS2 kernel path as on the fine
// level; P and R = P^T are tiled matrices of the same engine.  The coarsest
// level is solved exactly with its inverse, formed on the host by
// Gauss-Jordan elimination with partial pivoting and applied by a dense
// matrix-vector kernel.
//
// A V-cycle from a zero start on level l with right-hand side b_l:
//   x_l = S_pre(b_l) from zero;  r_l = b_l - A_l x_l;  b_{l+1} = R_l r_l;
//   x_{l+1} = V-cycle(l + 1);  x_l += P_l x_{l+1};  x_l = S_post(b_l, x_l),
// with S forward before and backward after for a symmetric smoother.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.cuh"

namespace gs2 {

// ---------------------------------------------------------------------------
// host sparse matrices
// ---------------------------------------------------------------------------

struct HCsr {
  int64_t n = 0, m = 0;  // rows, columns
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
  int64_t nnz() const { return rp.empty() ? 0 : rp[n]; }
};

static HCsr transpose(const HCsr& a) {
  HCsr t;
  t.n = a.m;
  t.m = a.n;
  t.rp.assign(t.n + 1, 0);
  t.ci.resize(a.nnz());
  t.va.resize(a.nnz());
  for (int64_t k = 0; k < a.nnz(); ++k) t.rp[a.ci[k] + 1]++;
  std::partial_sum(t.rp.begin(), t.rp.end(), t.rp.begin());
  std::vector<int64_t> pos(t.rp.begin(), t.rp.end() - 1);
  for (int64_t i = 0; i < a.n; ++i)
    for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      const int64_t q = pos[a.ci[k]]++;
      t.ci[q] = (int32_t)i;
      t.va[q] = a.va[k];
    }
  return t;
}

// C = A B by rows (Gustavson): a dense accumulator indexed by column and a
// list of the columns a row touched; columns of each row sorted.  Row
// ranges run on parallel host threads (a symbolic pass counts each row's
// columns, a numeric pass fills them); every row is summed in the same order
// as a sequential product.
static HCsr multiply(const HCsr& a, const HCsr& b) {
  HCsr c;
  c.n = a.n;
  c.m = b.m;
  c.rp.assign(c.n + 1, 0);
  parallel_ranges(a.n, [&](int64_t i0, int64_t i1, int) {
    std::vector<int64_t> seen(b.m, -1);
    for (int64_t i = i0; i < i1; ++i) {
      int64_t cnt = 0;
      for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
        const int64_t r = a.ci[k];
        for (int64_t q = b.rp[r]; q < b.rp[r + 1]; ++q)
          if (seen[b.ci[q]] != i) {
            seen[b.ci[q]] = i;
            ++cnt;
          }
      }
      c.rp[i + 1] = cnt;
    }
  });
  for (int64_t i = 0; i < c.n; ++i) c.rp[i + 1] += c.rp[i];
  c.ci.resize(c.rp[c.n]);
  c.va.resize(c.rp[c.n]);
  parallel_ranges(a.n, [&](int64_t i0, int64_t i1, int) {
    std::vector<int64_t> seen(b.m, -1);
    std::vector<double> acc(b.m, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = i0; i < i1; ++i) {
      cols.clear();
      for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
        const int64_t r = a.ci[k];
        const double av = a.va[k];
        for (int64_t q = b.rp[r]; q < b.rp[r + 1]; ++q) {
          const int32_t j = b.ci[q];
          if (seen[j] != i) {
            seen[j] = i;
            acc[j] = 0.0;
            cols.push_back(j);
          }
          acc[j] += av * b.va[q];
        }
      }
      std::sort(cols.begin(), cols.end());
      int64_t o = c.rp[i];
      for (int32_t j : cols) {
        c.ci[o] = j;
        c.va[o++] = acc[j];
      }
    }
  });
  return c;
}

// ---------------------------------------------------------------------------
// aggregation
// ---------------------------------------------------------------------------

// Symmetrised strength graph as sorted adjacency lists: the directed strong
// entries (S), their transpose, and per row the sorted union of both, each
// step over parallel row ranges except the transpose's counting.
static void strength(const HCsr& a, double theta, std::vector<int64_t>& gp,
                     std::vector<int32_t>& gi) {
  const int64_t n = a.n;
  HCsr S;
  S.n = S.m = n;
  S.rp.assign(n + 1, 0);
  std::vector<double> big(n, 0.0);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i) {
      double m = 0.0;
      for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k)
        if (a.ci[k] != i) m = std::max(m, std::fabs(a.va[k]));
      big[i] = m;
      int64_t cnt = 0;
      if (m > 0.0)
        for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k)
          if (a.ci[k] != i && std::fabs(a.va[k]) >= theta * m) ++cnt;
      S.rp[i + 1] = cnt;
    }
  });
  for (int64_t i = 0; i < n; ++i) S.rp[i + 1] += S.rp[i];
  S.ci.resize(S.rp[n]);
  S.va.assign(S.rp[n], 1.0);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i) {
      int64_t o = S.rp[i];
      if (big[i] > 0.0)
        for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k)
          if (a.ci[k] != i && std::fabs(a.va[k]) >= theta * big[i]) S.ci[o++] = a.ci[k];
    }
  });
  const HCsr St = transpose(S);
  gp.assign(n + 1, 0);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    std::vector<int32_t> v;
    for (int64_t i = i0; i < i1; ++i) {
      v.assign(S.ci.begin() + S.rp[i], S.ci.begin() + S.rp[i + 1]);
      v.insert(v.end(), St.ci.begin() + St.rp[i], St.ci.begin() + St.rp[i + 1]);
      std::sort(v.begin(), v.end());
      gp[i + 1] = std::unique(v.begin(), v.end()) - v.begin();
    }
  });
  for (int64_t i = 0; i < n; ++i) gp[i + 1] += gp[i];
  gi.resize(gp[n]);
  parallel_ranges(n, [&](int64_t i0, int64_t i1, int) {
    std::vector<int32_t> v;
    for (int64_t i = i0; i < i1; ++i) {
      v.assign(S.ci.begin() + S.rp[i], S.ci.begin() + S.rp[i + 1]);
      v.insert(v.end(), St.ci.begin() + St.rp[i], St.ci.begin() + St.rp[i + 1]);
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      std::copy(v.begin(), v.end(), gi.begin() + gp[i]);
    }
  });
}

static int64_t aggregate(const std::vector<int64_t>& gp, const std::vector<int32_t>& gi,
                         std::vector<int32_t>& agg) {
  const int64_t n = (int64_t)gp.size() - 1;
  agg.assign(n, -1);
  int32_t na = 0;
  // 1: rows with an entirely free neighbourhood seed an aggregate
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool ok = true;
    for (int64_t k = gp[i]; k < gp[i + 1] && ok; ++k) ok = agg[gi[k]] < 0;
    if (!ok) continue;
    agg[i] = na;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k) agg[gi[k]] = na;
    ++na;
  }
  // 2: free rows join the seed aggregate of their first seeded neighbour
  const std::vector<int32_t> seeded(agg);
  for (int64_t i = 0; i < n; ++i) {
    if (seeded[i] >= 0) continue;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k)
      if (seeded[gi[k]] >= 0) {
        agg[i] = seeded[gi[k]];
        break;
      }
  }
  // 3: what is left seeds aggregates with its free neighbours
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int64_t k = gp[i]; k < gp[i + 1]; ++k)
      if (agg[gi[k]] < 0) agg[gi[k]] = na;
    ++na;
  }
  return na;
}

// P = (I - w D^{-1} A) P0 of one level
static HCsr prolongator(const HCsr& a, double theta, std::vector<int32_t>& agg, int64_t& na) {
  std::vector<int64_t> gp;
  std::vector<int32_t> gi;
  strength(a, theta, gp, gi);
  na = aggregate(gp, gi, agg);
  std::vector<int64_t> size(na, 0);
  for (int32_t g : agg) size[g]++;
  HCsr p0;
  p0.n = a.n;
  p0.m = na;
  p0.rp.resize(a.n + 1);
  p0.ci.resize(a.n);
  p0.va.resize(a.n);
  for (int64_t i = 0; i < a.n; ++i) {
    p0.rp[i] = i;
    p0.ci[i] = agg[i];
    p0.va[i] = 1.0 / std::sqrt((double)size[agg[i]]);
  }
  p0.rp[a.n] = a.n;
  std::vector<double> d(a.n, 0.0);
  double rho = 0.0;
  for (int64_t i = 0; i < a.n; ++i) {
    double row = 0.0;
    for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      if (a.ci[k] == i) d[i] = a.va[k];
      row += std::fabs(a.va[k]);
    }
    rho = std::max(rho, row / std::fabs(d[i]));
  }
  const double w = 4.0 / (3.0 * rho);
  HCsr p = multiply(a, p0);  // A P0, whose pattern holds that of P0
  for (int64_t i = 0; i < a.n; ++i) {
    const double s = w / d[i];
    for (int64_t k = p.rp[i]; k < p.rp[i + 1]; ++k) {
      const double base = p.ci[k] == agg[i] ? p0.va[i] : 0.0;
      p.va[k] = base - s * p.va[k];
    }
  }
  return p;
}

// inverse of a small dense matrix (row-major) by Gauss-Jordan elimination
// with partial pivoting; false if singular
static bool invert(int64_t n, std::vector<double>& a, std::vector<double>& inv) {
  inv.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t pr = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[pr * n + c])) pr = r;
    if (a[pr * n + c] == 0.0) return false;
    if (pr != c)
      for (int64_t j = 0; j < n; ++j) {
        std::swap(a[c * n + j], a[pr * n + j]);
        std::swap(inv[c * n + j], inv[pr * n + j]);
      }
    const double piv = a[c * n + c];
    for (int64_t j = 0; j < n; ++j) {
      a[c * n + j] /= piv;
      inv[c * n + j] /= piv;
    }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < n; ++j) {
        a[r * n + j] -= f * a[c * n + j];
        inv[r * n + j] -= f * inv[c * n + j];
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// hierarchy on the device
// ---------------------------------------------------------------------------

struct AmgLevel {
  gs2_handle* h = nullptr;  // level 0: the owning handle (not owned here)
  DevCsr P, R;              // to and from level l + 1, tiled for h's engine
  double* b = nullptr;      // right-hand side (levels >= 1)
  double* x = nullptr;      // solution (levels >= 1)
  double* r = nullptr;      // residual
  int64_t n = 0, nnz = 0, pnnz = 0;
};

struct AmgHierarchy {
  gs2_amg_cfg cfg{};
  std::vector<AmgLevel> lv;
  double* cinv = nullptr;  // inverse of the coarsest matrix, row-major
  int64_t nc = 0;
  std::vector<void*> own;  // device memory not held by a level handle
  int64_t own_bytes = 0;
};

// stream-ordered like the owner's own memory when the owner is (server
// handles), so building or freeing a hierarchy never synchronises the device
static void* own_alloc(AmgHierarchy* H, gs2_handle* h, size_t bytes) {
  void* p = nullptr;
  bytes = std::max<size_t>(bytes, 16);
  GS2_CUDA(h->async_alloc ? cudaMallocAsync(&p, bytes, h->stream) : cudaMalloc(&p, bytes));
  H->own.push_back(p);
  H->own_bytes += (int64_t)bytes;
  return p;
}

static void free_hierarchy(AmgHierarchy* H, gs2_handle* h) {
  if (!H) return;
  for (size_t l = 1; l < H->lv.size(); ++l) destroy_handle(H->lv[l].h);
  for (void* p : H->own) {
    if (h->async_alloc) cudaFreeAsync(p, h->stream);
    else cudaFree(p);
  }
  delete H;
}

void amg_free(gs2_handle* h) {
  if (!h->amg) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  // a captured cycle may hold the hierarchy's buffers
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gkey.clear();
  }
  free_hierarchy(h->amg, h);
  h->amg = nullptr;
}

static std::vector<int> to_int(const std::vector<int64_t>& v) {
  return std::vector<int>(v.begin(), v.end());
}

void amg_build(gs2_handle* h, const gs2_amg_cfg& cfg) {
  if (!(cfg.theta >= 0.0 && cfg.theta <= 1.0) || cfg.max_levels < 1 ||
      cfg.max_levels > GS2_AMG_MAX_LEVELS || cfg.coarse_size < 1)
    GS2_THROW(GS2_ERR_INVALID_ARG, "AMG: theta in [0, 1], 1 <= max_levels <= 16, coarse_size >= 1");
  amg_free(h);
  // level 0 from the handle's device copy of A
  HCsr a;
  a.n = a.m = h->n;
  {
    std::vector<int> rp(h->n + 1);
    a.ci.resize(h->nnz);
    a.va.resize(h->nnz);
    GS2_CUDA(cudaMemcpy(rp.data(), h->A.rp, sizeof(int) * (h->n + 1), cudaMemcpyDeviceToHost));
    GS2_CUDA(cudaMemcpy(a.ci.data(), h->A.ci, sizeof(int) * h->nnz, cudaMemcpyDeviceToHost));
    GS2_CUDA(cudaMemcpy(a.va.data(), h->A.va, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost));
    a.rp.assign(rp.begin(), rp.end());
  }
  auto* H = new AmgHierarchy();
  H->cfg = cfg;
  try {
    AmgLevel top;
    top.h = h;
    top.n = a.n;
    top.nnz = a.nnz();
    H->lv.push_back(top);
    while ((int)H->lv.size() < cfg.max_levels && a.n > cfg.coarse_size) {
      std::vector<int32_t> agg;
      int64_t na = 0;
      HCsr p = prolongator(a, cfg.theta, agg, na);
      if (na >= a.n || na == 0) break;
      HCsr r = transpose(p);
      HCsr ac = multiply(r, multiply(a, p));
      AmgLevel lvl;
      lvl.h = setup_handle(ac.n, ac.nnz(), ac.rp.data(), ac.ci.data(), ac.va.data(), 0, 0u,
                           h->stream, h->async_alloc);
      lvl.h->dev_err = h->dev_err;  // timeouts of coarse kernels reach the owner
      lvl.n = ac.n;
      lvl.nnz = ac.nnz();
      H->lv.push_back(lvl);
      AmgLevel& fine = H->lv[H->lv.size() - 2];
      gs2_handle* ch = H->lv.back().h;
      // the transfer operators and the fine residual live with the coarse
      // handle, so replacing or freeing the hierarchy releases them
      upload_matrix(ch, fine.P, (int)p.n, to_int(p.rp), std::vector<int>(p.ci.begin(), p.ci.end()),
                    p.va);
      upload_matrix(ch, fine.R, (int)r.n, to_int(r.rp), std::vector<int>(r.ci.begin(), r.ci.end()),
                    r.va);
      fine.pnnz = p.nnz();
      fine.r = (double*)ch->dalloc(sizeof(double) * std::max<int64_t>(fine.n, 1));
      AmgLevel& coarse = H->lv.back();
      coarse.b = (double*)ch->dalloc(sizeof(double) * std::max<int64_t>(coarse.n, 1));
      coarse.x = (double*)ch->dalloc(sizeof(double) * std::max<int64_t>(coarse.n, 1));
      a = std::move(ac);
    }
    // the coarsest level is solved exactly
    if (a.n > kAmgMaxCoarse)
      GS2_THROW(GS2_ERR_INVALID_ARG,
                "AMG: coarsest level has " + std::to_string(a.n) + " rows (at most " +
                    std::to_string(kAmgMaxCoarse) + " are solved exactly); raise max_levels");
    std::vector<double> dense(a.n * a.n, 0.0), inv;
    for (int64_t i = 0; i < a.n; ++i)
      for (int64_t k = a.rp[i]; k < a.rp[i + 1]; ++k) dense[i * a.n + a.ci[k]] += a.va[k];
    if (!invert(a.n, dense, inv))
      GS2_THROW(GS2_ERR_INVALID_ARG, "AMG: the coarsest matrix is singular");
    H->nc = a.n;
    H->cinv = (double*)own_alloc(H, h, sizeof(double) * inv.size());
    GS2_CUDA(cudaMemcpyAsync(H->cinv, inv.data(), sizeof(double) * inv.size(),
                             cudaMemcpyHostToDevice, h->stream));
    GS2_CUDA(cudaStreamSynchronize(h->stream));
  } catch (...) {
    free_hierarchy(H, h);
    throw;
  }
  h->amg = H;
}

void amg_info(const gs2_handle* h, int* levels, int64_t* rows, int64_t* nnz, int64_t* pnnz) {
  const AmgHierarchy* H = h->amg;
  *levels = H ? (int)H->lv.size() : 0;
  for (int l = 0; l < GS2_AMG_MAX_LEVELS; ++l) {
    const bool on = H && l < (int)H->lv.size();
    if (rows) rows[l] = on ? H->lv[l].n : 0;
    if (nnz) nnz[l] = on ? H->lv[l].nnz : 0;
    if (pnnz) pnnz[l] = on ? H->lv[l].pnnz : 0;
  }
}

int64_t amg_device_bytes(const gs2_handle* h) {
  const AmgHierarchy* H = h->amg;
  if (!H) return 0;
  int64_t b = H->own_bytes;
  for (size_t l = 1; l < H->lv.size(); ++l) b += H->lv[l].h->dev_bytes;
  return b;
}

void amg_prepare(gs2_handle* h, const gs2_params* p) {
  if (!h->amg) {
    gs2_amg_cfg cfg{};
    cfg.theta = 0.25;
    cfg.max_levels = 10;
    cfg.coarse_size = 64;
    amg_build(h, cfg);
  }
  if (p->kind == GS2_PC_AMG && p->precision != GS2_FP64)
    for (AmgLevel& l : h->amg->lv) ensure_precision(l.h, p->precision);
}

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------

// x = C b for the dense coarsest inverse: one warp per row
__global__ void k_dense_mv(int n, const double* __restrict__ c, const double* __restrict__ b,
                           double* x, const int* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(c[(size_t)row * n + j], b[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = s;
}

static void cycle(AmgHierarchy* H, size_t l, const gs2_params& sp, const double* b, double* x,
                  bool rhat_ready, const int* skip) {
  AmgLevel& L = H->lv[l];
  gs2_handle* hl = L.h;
  if (l + 1 == H->lv.size()) {
    KernelTimer tm(hl, "amg_coarse", 8.0 * H->nc * (H->nc + 2));
    k_dense_mv<<<(int)((H->nc + 7) / 8), 256, 0, hl->stream>>>((int)H->nc, H->cinv, b, x, skip);
    GS2_LAUNCH_CHECK();
    return;
  }
  gs2_params pre = sp, post = sp;
  if (sp.direction == GS2_SYMMETRIC) {
    pre.direction = GS2_FORWARD;
    post.direction = GS2_BACKWARD;
  }
  AmgLevel& C = H->lv[l + 1];
  precond_apply(hl, &pre, b, x, rhat_ready, skip);           // x = S_pre(b) from zero
  launch_resid(hl, b, x, L.r, nullptr, nullptr, skip);       // r = b - A x
  launch_spmv_matrix(hl, L.R, L.r, C.b, false, skip);        // b_c = R r
  cycle(H, l + 1, sp, C.b, C.x, false, skip);                // x_c
  launch_spmv_matrix(hl, L.P, C.x, x, true, skip);           // x += P x_c
  smooth_sweeps(hl, &post, b, x, skip);                      // x = S_post(b, x)
}

// Coarse handles launch on the owner's current stream (also while it is
// being captured into a graph) and report to its profiler.
struct LevelBinding {
  AmgHierarchy* H;
  explicit LevelBinding(gs2_handle* h) : H(h->amg) {
    for (size_t l = 1; l < H->lv.size(); ++l) {
      H->lv[l].h->stream = h->stream;
      H->lv[l].h->prof = h->prof;
    }
  }
  ~LevelBinding() {
    for (size_t l = 1; l < H->lv.size(); ++l) H->lv[l].h->prof = nullptr;
  }
};

void amg_vcycle(gs2_handle* h, const gs2_params* p, const double* b, double* x,
                bool rhat_ready, const int* skip) {
  if (!h->amg) GS2_THROW(GS2_ERR_INVALID_ARG, "no AMG hierarchy on this handle");
  LevelBinding bind(h);
  gs2_params sp = *p;
  sp.kind = p->kind == GS2_PC_AMG ? GS2_PC_GS2 : GS2_PC_JR;
  cycle(h->amg, 0, sp, b, x, rhat_ready, skip);
}

}  // namespace gs2
