// Solve server: continuous batching of independent systems on one GPU.
//
// Requests are queued on submission and admitted in arrival order as soon as
// a slot is free and their estimated device footprint fits the server's
// budget (by default 90% of the device memory free when the server starts;
// optionally some slots kept for small requests).  A preparation thread
// builds an admitted request's handle on a stream of its own, with
// stream-ordered allocations, and starts its GMRES job: a system that fits
// one cluster's shared memory is solved by one cluster launch, any other by
// one replayed graph per restart cycle.  The progress thread polls every
// running job's stream and advances the job by one restart cycle (or reads
// the cluster solve's outcome) whenever that stream is idle.  Requests that
// arrive while others run are therefore admitted as slots and memory free
// up, and their kernels overlap on the GPU.  Every request runs the same
// kernels with the same launch geometry as a lone gmres_solve in the same
// graph mode (4 or 1), so its result is bitwise the same alone and in the
// mix.  With packing enabled,
// small requests at the front of the queue are admitted together and solved
// as one pack (pack.cu) in one slot: one set of launches for all of them,
// each result independent of its pack-mates.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace gs2 {

using Clock = std::chrono::steady_clock;

enum ReqState { REQ_PENDING = 0, REQ_PREPARING = 1, REQ_ACTIVE = 2, REQ_DONE = 3 };

struct Request {
  uint64_t ticket = 0;
  int state = REQ_PENDING;
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va, b, x0;
  int64_t footprint = 0;
  bool large = false;  // holds one of the slots not reserved for small requests
  Clock::time_point t_submit, t_done;
  cudaStream_t stream = nullptr;
  gs2_handle* h = nullptr;
  GmresJob* job = nullptr;
  gs2_solve_info info{0, 0, GS2_OK, 0.0};
  gs2_status status = GS2_OK;
  std::vector<double> x;
};

// Small requests admitted together and solved as one pack in one slot.
struct Group {
  std::vector<Request*> members;  // in pack order
  bool large = false;             // its slot is one of the large requests'
  cudaStream_t stream = nullptr;
  gs2_handle* h = nullptr;
  PackJob* job = nullptr;
};

// Bytes of the sliced-ELL copy of a matrix with this many entries (at most
// 1.2 slots per entry, else no copy is made) holding vbytes-byte values, with
// its chunk offsets.
static int64_t sell_bytes(int64_t entries, int64_t n, int vbytes) {
  return (entries * 6 / 5 + 1) * (4 + vbytes) + 4 * (n / 32 + 2);
}

// Device bytes a request of this size holds once admitted: the matrix, its
// two prescaled triangles, their sliced-ELL copies, the resident vectors,
// the Krylov basis and the optional lower-precision, level-set and colour
// storage (mirrors setup_handle, upload_sell, ensure_precision,
// ensure_levels, ensure_colors and ensure_krylov).
static int64_t footprint(const gs2_server_cfg& c, int64_t n, int64_t nnz) {
  const int64_t off = std::max<int64_t>(nnz - n, 0);
  const int64_t m = std::max(c.restart, 1);
  int64_t b = 12 * nnz + 12 * off + 3 * 4 * (n + 17) + 3 * (n / 16 + 16) * 16;
  b += sell_bytes(nnz, n, 8) + 2 * sell_bytes(off / 2 + 1, n, 8);
  b += 8 * n * 9;                     // D^{-1} and eight resident temporaries
  b += 8 * (int64_t)8 * 152 * 66;     // per-block partial sums (upper bound)
  b += 8 * n * (m + 1) + 3 * 8 * n;   // Krylov basis, w, p, q
  b += 8 * (m + 1) * (m + 6);         // Hessenberg, rotations, y
  if (c.has_precond && c.precond.kind == GS2_PC_GS2) {
    const int vp = value_precision(c.precond.precision);
    if (vp == GS2_FP32) b += 4 * off + 12 * n + 4 * (off * 6 / 5 + 2);
    if (vp == GS2_FP16_ROWSCALED) b += 2 * off + 8 * n + 12 * n + 2 * (off * 6 / 5 + 2);
    // whole-sweep precisions: the off-diagonal matrix O (its CSR, its
    // sliced-ELL copy, its value-precision copies) and two FP32 vectors
    if (is_sweep_precision(c.precond.precision))
      b += 12 * off + 4 * (n + 17) + (n / 16 + 16) * 16 + sell_bytes(off, n, 8) +
           (vp == GS2_FP32 ? 8 : 4) * off + 2 * n + 8 * n + 4 * (n / 32 + 2);
  }
  if (c.has_precond && c.precond.kind == GS2_PC_GS) b += 8 * n;
  // hybrid form: the local block of A, the couplings, the local triangles
  // (with their low-precision copies) and the exchange vector
  if (c.has_precond && c.precond.parts > 1) {
    b += 12 * nnz + 12 * off + 4 * 4 * (n + 17) + 8 * n;
    b += sell_bytes(nnz, n, 8) + 2 * sell_bytes(off / 2 + 1, n, 8) + 4 * (n / 32 + 2);
    if (c.precond.precision == GS2_FP32) b += 4 * off + 4 * (off * 6 / 5 + 2);
    if (c.precond.precision == GS2_FP16_ROWSCALED) b += 2 * off + 4 * n + 2 * (off * 6 / 5 + 2);
  }
  // colour matrices: the off-diagonal entries again, row lists, row
  // pointers and tile descriptors, plus per-colour allocation slack
  if (c.has_precond && c.precond.kind == GS2_PC_MTGS)
    b += 12 * off + 8 * n + 4 * (n / 16 + 16) * 16 + (1 << 18) + sell_bytes(off, n, 8);
  // multigrid hierarchy: coarse matrices with their triangles and resident
  // vectors (operator complexity below ~1.6 for the model problems), the
  // transfer operators P and R (about 6 entries per fine row each), level
  // vectors and the coarsest inverse
  if (c.has_precond && (c.precond.kind == GS2_PC_AMG || c.precond.kind == GS2_PC_AMG_JR))
    b += 60 * nnz + 160 * n + (64 << 20);
  return b + (1 << 20);
}

}  // namespace gs2

struct gs2_server {
  gs2_server_cfg cfg{};
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_prep;  // preparation threads wait for admissible work
  std::condition_variable cv_done;  // gs2_server_wait callers
  std::condition_variable cv_loop;  // the progress thread, when idle
  std::deque<gs2::Request*> pending;
  std::vector<gs2::Request*> active;
  std::vector<gs2::Group*> groups;  // packs on the GPU
  std::unordered_map<uint64_t, gs2::Request*> table;
  uint64_t next_ticket = 1;
  int64_t reserved = 0;
  int64_t slots_used = 0;  // preparing + active
  int64_t large_used = 0;  // of them, slots held by large requests (small_slots > 0)
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, max_active = 0;
  bool stopping = false;
  std::vector<std::thread> prep;
  std::thread loop;
};

using namespace gs2;

// A request is large when small_slots slots are reserved for requests of at
// most small_rows rows and it has more; large requests hold at most
// max_slots - small_slots slots at once.
static bool is_large(const gs2_server* s, const Request* r) {
  return s->cfg.small_slots > 0 && r->n > s->cfg.small_rows;
}

// The queue position of the request to admit next, or -1: the first request
// in arrival order that may take a slot -- every request without reserved
// slots, else large ones only while their slots are not all taken, so that a
// small request passes the large ones waiting for those -- provided it fits
// the memory budget (a request that does not fit holds the queue, as it
// would in arrival order).
static int next_admissible(gs2_server* s) {
  if (s->slots_used >= s->cfg.max_slots) return -1;
  const int64_t large_cap = s->cfg.max_slots - s->cfg.small_slots;
  for (size_t k = 0; k < s->pending.size(); ++k) {
    const Request* r = s->pending[k];
    if (is_large(s, r) && s->large_used >= large_cap) continue;
    return s->reserved + r->footprint <= s->budget ? (int)k : -1;
  }
  return -1;
}

static bool packable(const gs2_server* s, const Request* r) {
  const bool amg = s->cfg.has_precond &&
                   (s->cfg.precond.kind == GS2_PC_AMG || s->cfg.precond.kind == GS2_PC_AMG_JR);
  const bool hybrid = s->cfg.has_precond && s->cfg.precond.parts > 1;
  return s->cfg.pack_rows > 0 && r->n <= s->cfg.pack_rows && !amg && !hybrid;
}

// Called with the lock held: release the request's reservation (and its
// slot, unless it was one of a pack's), record its end and wake everybody
// who may be waiting on it or on free capacity.
static void retire_locked(gs2_server* s, Request* r, bool ok, bool frees_slot = true) {
  r->state = REQ_DONE;
  r->t_done = Clock::now();
  s->reserved -= r->footprint;
  if (frees_slot) {
    s->slots_used -= 1;
    if (r->large) s->large_used -= 1;
  }
  if (ok) s->completed += 1;
  else s->failed += 1;
  s->cv_done.notify_all();
  s->cv_prep.notify_all();
}

// Release the device resources of a request (its stream-ordered memory is
// freed on its own stream; the stream goes once its work has drained).
static void release_device(Request* r) {
  if (r->job) gmres_job_free(r->job);
  r->job = nullptr;
  if (r->h) destroy_handle(r->h);
  r->h = nullptr;
  if (r->stream) cudaStreamDestroy(r->stream);
  r->stream = nullptr;
}

// Build the handle and start the GMRES job of an admitted request.
static void prepare(gs2_server* s, Request* r) {
  gs2_status st = GS2_OK;
  try {
    if (s->cfg.fail_ticket && r->ticket == s->cfg.fail_ticket)
      GS2_THROW(GS2_ERR_OOM, "injected allocation failure");
    GS2_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
    unsigned prec = 0;
    const gs2_params* pc = s->cfg.has_precond ? &s->cfg.precond : nullptr;
    if (pc && pc->kind == GS2_PC_GS2) prec = 1u << pc->precision;
    r->h = setup_handle(r->n, r->nnz, r->rp.data(), r->ci.data(), r->va.data(), 0, prec,
                        r->stream, true);
    ensure_precond(r->h, pc);
    // a request whose rows fit one cluster's shared memory is solved by one
    // cluster launch (clusters never wait for one another, so requests on
    // other streams cannot hold it up); every other request replays its
    // cycles as a graph captured by this thread, so the single progress
    // thread only ever launches whole cycles
    r->h->graph_mode = cluster_eligible(r->h, s->cfg.restart, pc) ? 4 : 1;
    r->h->h2d(r->h->bstage, r->b.data(), sizeof(double) * r->n);
    if (r->x0.empty()) r->h->dzero(r->h->xstage, sizeof(double) * r->n);
    else r->h->h2d(r->h->xstage, r->x0.data(), sizeof(double) * r->n);
    r->job = gmres_job_start(r->h, r->h->bstage, r->h->xstage, s->cfg.restart, s->cfg.tol,
                             s->cfg.max_iters, pc);
    // capture the cycle graph here, off the progress thread
    gmres_job_prepare(r->job);
  } catch (const Error& e) {
    st = e.st;
  } catch (const std::bad_alloc&) {
    st = GS2_ERR_OOM;
  } catch (...) {
    st = GS2_ERR_CUDA;
  }
  // the host copies of the matrix are no longer needed
  std::vector<int64_t>().swap(r->rp);
  std::vector<int32_t>().swap(r->ci);
  std::vector<double>().swap(r->va);
  std::lock_guard<std::mutex> g(s->mu);
  if (st != GS2_OK) {
    release_device(r);
    r->status = st;
    r->info.status = st;
    retire_locked(s, r, false);
    return;
  }
  r->state = REQ_ACTIVE;
  s->active.push_back(r);
  s->cv_loop.notify_one();
}

// Build one pack from the group's requests and start its job.  Each request
// is validated on its own first, so a malformed one fails alone.
static void prepare_group(gs2_server* s, Group* g) {
  std::vector<std::pair<Request*, gs2_status>> failed;
  std::vector<Request*> ok;
  for (Request* r : g->members) {
    gs2_status st = GS2_OK;
    try {
      if (s->cfg.fail_ticket && r->ticket == s->cfg.fail_ticket)
        GS2_THROW(GS2_ERR_OOM, "injected allocation failure");
      std::vector<double> d;
      validate_csr(r->n, r->nnz, r->rp.data(), r->ci.data(), r->va.data(), &d);
    } catch (const Error& e) {
      st = e.st;
    } catch (const std::bad_alloc&) {
      st = GS2_ERR_OOM;
    }
    if (st == GS2_OK) ok.push_back(r);
    else failed.push_back({r, st});
  }
  g->members = ok;
  gs2_status st = GS2_OK;
  if (!ok.empty()) {
    try {
      GS2_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
      const int cnt = (int)ok.size();
      std::vector<int64_t> n(cnt);
      std::vector<const int64_t*> rp(cnt);
      std::vector<const int32_t*> ci(cnt);
      std::vector<const double*> va(cnt);
      std::vector<double> b, x0;
      for (int k = 0; k < cnt; ++k) {
        Request* r = ok[k];
        n[k] = r->n;
        rp[k] = r->rp.data();
        ci[k] = r->ci.data();
        va[k] = r->va.data();
        b.insert(b.end(), r->b.begin(), r->b.end());
        if (r->x0.empty()) x0.insert(x0.end(), r->n, 0.0);
        else x0.insert(x0.end(), r->x0.begin(), r->x0.end());
      }
      std::vector<int64_t> off, crp;
      std::vector<int32_t> cci;
      std::vector<double> cva;
      pack_concat(cnt, n.data(), rp.data(), ci.data(), va.data(), off, crp, cci, cva);
      unsigned prec = 0;
      const gs2_params* pc = s->cfg.has_precond ? &s->cfg.precond : nullptr;
      if (pc && pc->kind == GS2_PC_GS2) prec = 1u << pc->precision;
      g->h = setup_handle(off.back(), (int64_t)cci.size(), crp.data(), cci.data(), cva.data(), 0,
                          prec, g->stream, true);
      pack_attach(g->h, off);
      ensure_precond(g->h, pc);
      g->h->graph_mode = 1;
      if (!b.empty()) {
        g->h->h2d(g->h->bstage, b.data(), sizeof(double) * b.size());
        g->h->h2d(g->h->xstage, x0.data(), sizeof(double) * x0.size());
      }
      g->job = pack_job_start(g->h, g->h->bstage, g->h->xstage, s->cfg.restart, s->cfg.tol,
                              s->cfg.max_iters, pc);
      pack_job_prepare(g->job);
      // the pageable staging copies above have been taken by the CUDA driver
    } catch (const Error& e) {
      st = e.st;
    } catch (const std::bad_alloc&) {
      st = GS2_ERR_OOM;
    } catch (...) {
      st = GS2_ERR_CUDA;
    }
  }
  for (Request* r : g->members) {
    std::vector<int64_t>().swap(r->rp);
    std::vector<int32_t>().swap(r->ci);
    std::vector<double>().swap(r->va);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& f : failed) {
    f.first->status = f.second;
    f.first->info.status = f.second;
    retire_locked(s, f.first, false, false);
  }
  if (ok.empty() || st != GS2_OK) {
    if (g->job) pack_job_free(g->job);
    if (g->h) destroy_handle(g->h);
    if (g->stream) cudaStreamDestroy(g->stream);
    for (Request* r : g->members) {
      r->status = st;
      r->info.status = st;
      retire_locked(s, r, false, false);
    }
    s->slots_used -= 1;
    if (g->large) s->large_used -= 1;
    s->cv_prep.notify_all();
    delete g;
    return;
  }
  for (Request* r : g->members) r->state = REQ_ACTIVE;
  s->groups.push_back(g);
  s->cv_loop.notify_one();
}

static void prep_thread(gs2_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    Group* g = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int k = -1;
      s->cv_prep.wait(lk, [&] { return s->stopping || (k = next_admissible(s)) >= 0; });
      if (s->stopping) return;
      r = s->pending[k];
      s->pending.erase(s->pending.begin() + k);
      r->state = REQ_PREPARING;
      r->large = is_large(s, r);
      s->reserved += r->footprint;
      s->slots_used += 1;
      if (r->large) s->large_used += 1;
      s->admitted += 1;
      s->max_active = std::max(s->max_active, s->slots_used);
      if (packable(s, r)) {
        // the small requests behind it join its pack while they fit: the
        // next ones in arrival order, or with reserved small slots the next
        // ones of its own size class, passing the others
        g = new Group();
        g->large = r->large;
        g->members.push_back(r);
        const int cap = s->cfg.pack_max > 0 ? s->cfg.pack_max : 64;
        for (size_t q = k; (int)g->members.size() < cap && q < s->pending.size();) {
          Request* c = s->pending[q];
          if (!packable(s, c) || is_large(s, c) != r->large) {
            if (s->cfg.small_slots == 0) break;
            ++q;
            continue;
          }
          if (s->reserved + c->footprint > s->budget) break;
          s->pending.erase(s->pending.begin() + q);
          c->state = REQ_PREPARING;
          s->reserved += c->footprint;
          s->admitted += 1;
          g->members.push_back(c);
        }
      }
    }
    if (g) prepare_group(s, g);
    else prepare(s, r);
  }
}

// Copy the solution back and retire a finished request.
static void finish(gs2_server* s, Request* r, gs2_status err) {
  bool ok = err == GS2_OK;
  if (ok) {
    r->info = gmres_job_info(r->job);
    r->status = (gs2_status)r->info.status;
    r->x.resize(r->n);
    if (r->n &&
        cudaMemcpyAsync(r->x.data(), r->h->xstage, sizeof(double) * r->n,
                        cudaMemcpyDeviceToHost, r->stream) != cudaSuccess) {
      cudaGetLastError();
      r->status = GS2_ERR_CUDA;
    }
    cudaStreamSynchronize(r->stream);
  } else {
    r->status = err;
    r->info.status = err;
  }
  release_device(r);
  std::lock_guard<std::mutex> g(s->mu);
  s->active.erase(std::find(s->active.begin(), s->active.end(), r));
  retire_locked(s, r, ok && r->status == GS2_OK);
}

// Copy a finished pack's solutions back and retire its requests (one slot).
static void finish_group(gs2_server* s, Group* g, gs2_status err) {
  std::vector<double> xall;
  if (err == GS2_OK) {
    xall.resize(g->h->n);
    if (g->h->n &&
        cudaMemcpyAsync(xall.data(), g->h->xstage, sizeof(double) * g->h->n,
                        cudaMemcpyDeviceToHost, g->stream) != cudaSuccess) {
      cudaGetLastError();
      err = GS2_ERR_CUDA;
    }
    cudaStreamSynchronize(g->stream);
  }
  int64_t o = 0;
  for (size_t k = 0; k < g->members.size(); ++k) {
    Request* r = g->members[k];
    if (err == GS2_OK) {
      r->info = pack_job_info(g->job, (int)k);
      r->status = (gs2_status)r->info.status;
      r->x.assign(xall.begin() + o, xall.begin() + o + r->n);
    } else {
      r->status = err;
      r->info.status = err;
    }
    o += r->n;
  }
  pack_job_free(g->job);
  destroy_handle(g->h);
  cudaStreamDestroy(g->stream);
  std::lock_guard<std::mutex> lk(s->mu);
  s->groups.erase(std::find(s->groups.begin(), s->groups.end(), g));
  for (Request* r : g->members) retire_locked(s, r, err == GS2_OK && r->status == GS2_OK, false);
  s->slots_used -= 1;
  if (g->large) s->large_used -= 1;
  s->cv_prep.notify_all();
  delete g;
}

static void progress_thread(gs2_server* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> snap;
  std::vector<Group*> gsnap;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty() && s->groups.empty()) {
        if (s->stopping && s->slots_used == 0) return;
        s->cv_loop.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      snap = s->active;
      gsnap = s->groups;
    }
    bool progressed = false;
    for (Group* g : gsnap) {
      const cudaError_t q = cudaStreamQuery(g->stream);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      if (q != cudaSuccess) {
        cudaGetLastError();
        finish_group(s, g, GS2_ERR_CUDA);
        continue;
      }
      gs2_status err = GS2_OK;
      bool done = false;
      try {
        done = pack_job_advance(g->job);
      } catch (const Error& e) {
        err = e.st;
        done = true;
      } catch (...) {
        err = GS2_ERR_CUDA;
        done = true;
      }
      if (done) finish_group(s, g, err);
    }
    for (Request* r : snap) {
      const cudaError_t q = cudaStreamQuery(r->stream);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      if (q != cudaSuccess) {
        cudaGetLastError();
        finish(s, r, GS2_ERR_CUDA);
        continue;
      }
      gs2_status err = GS2_OK;
      bool done = false;
      try {
        done = gmres_job_advance(r->job);
      } catch (const Error& e) {
        err = e.st;
        done = true;
      } catch (...) {
        err = GS2_ERR_CUDA;
        done = true;
      }
      if (done) finish(s, r, err);
    }
    if (!progressed) std::this_thread::yield();
  }
}

static gs2_status collect_locked(gs2_server* s, Request* r, gs2_solve_info* info, double* x_out,
                                 double* latency_ms) {
  if (info) *info = r->info;
  if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), sizeof(double) * r->x.size());
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const gs2_status st = r->status;
  s->table.erase(r->ticket);
  delete r;
  return st;
}

extern "C" {

int64_t gs2_server_footprint(const gs2_server_cfg* cfg, int64_t n, int64_t nnz) {
  if (!cfg || n < 0 || nnz < 0) return -1;
  return footprint(*cfg, n, nnz);
}

gs2_status gs2_server_create(const gs2_server_cfg* cfg, gs2_server** out) {
  if (!cfg || !out) return GS2_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->restart < 1 || cfg->restart > kMaxRestart ||
      !(cfg->tol >= 0.0) || cfg->max_iters < 0 || cfg->hbm_budget_bytes < 0 ||
      cfg->pack_rows < 0 || cfg->pack_max < 0 || cfg->small_rows < 0 || cfg->small_slots < 0 ||
      cfg->small_slots >= cfg->max_slots) {
    set_error("bad server configuration");
    return GS2_ERR_INVALID_ARG;
  }
  if (cfg->has_precond) {
    const gs2_params& p = cfg->precond;
    if (p.kind < GS2_PC_NONE || p.kind > GS2_PC_AMG_JR || p.outer < 1 || p.inner < 0 ||
        !(p.omega > 0.0) || !(p.gamma > 0.0) || p.direction < 0 || p.direction > 2 ||
        p.precision < 0 || p.precision > 4 || p.parts < 0 || p.local_sweeps < 0 ||
        (is_sweep_precision(p.precision) &&
         (p.kind != GS2_PC_GS2 || p.form != GS2_NONCOMPACT || p.parts > 1)) ||
        ((p.parts > 1 || p.local_sweeps > 1) && p.kind != GS2_PC_GS2 && p.kind != GS2_PC_JR &&
         p.kind != GS2_PC_GS) ||
        (p.parts > 1 && p.form == GS2_COMPACT)) {
      set_error("bad preconditioner parameters");
      return GS2_ERR_INVALID_ARG;
    }
  }
  auto* s = new gs2_server();
  s->cfg = *cfg;
  if (s->cfg.prep_threads < 1) s->cfg.prep_threads = 1;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_error("no CUDA device");
    return GS2_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_error("cudaMemGetInfo failed");
    return GS2_ERR_CUDA;
  }
  s->budget = cfg->hbm_budget_bytes > 0 ? cfg->hbm_budget_bytes : (int64_t)(0.9 * (double)fr);
  for (int i = 0; i < s->cfg.prep_threads; ++i) s->prep.emplace_back(prep_thread, s);
  s->loop = std::thread(progress_thread, s);
  *out = s;
  return GS2_OK;
}

gs2_status gs2_server_submit(gs2_server* s, const gs2_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket || q->n < 0 || q->nnz < 0 || !q->rowptr || !q->b ||
      (q->nnz > 0 && (!q->col || !q->val))) {
    set_error("bad request");
    return GS2_ERR_INVALID_ARG;
  }
  if (q->rowptr[0] != 0 || q->rowptr[q->n] != q->nnz) {
    set_error("rowptr[0] must be 0 and rowptr[n] must be nnz");
    return GS2_ERR_INVALID_ARG;
  }
  const int64_t fp = footprint(s->cfg, q->n, q->nnz);
  if (fp > s->budget) {
    set_error("request needs " + std::to_string(fp) + " device bytes, budget is " +
              std::to_string(s->budget));
    return GS2_ERR_OOM;
  }
  auto* r = new Request();
  try {
    r->n = q->n;
    r->nnz = q->nnz;
    r->rp.assign(q->rowptr, q->rowptr + q->n + 1);
    r->ci.assign(q->col, q->col + q->nnz);
    r->va.assign(q->val, q->val + q->nnz);
    r->b.assign(q->b, q->b + q->n);
    if (q->x0) r->x0.assign(q->x0, q->x0 + q->n);
  } catch (const std::bad_alloc&) {
    delete r;
    set_error("host allocation failed");
    return GS2_ERR_OOM;
  }
  r->footprint = fp;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stopping) {
    delete r;
    return GS2_ERR_BUSY;
  }
  r->ticket = s->next_ticket++;
  s->table[r->ticket] = r;
  s->pending.push_back(r);
  s->submitted += 1;
  *ticket = r->ticket;
  s->cv_prep.notify_one();
  return GS2_OK;
}

gs2_status gs2_server_poll(gs2_server* s, uint64_t ticket, gs2_solve_info* info, double* x_out,
                           double* latency_ms) {
  if (!s) return GS2_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return GS2_ERR_NOT_FOUND;
  if (it->second->state != REQ_DONE) return GS2_ERR_BUSY;
  return collect_locked(s, it->second, info, x_out, latency_ms);
}

gs2_status gs2_server_wait(gs2_server* s, uint64_t ticket, double timeout_s, gs2_solve_info* info,
                           double* x_out, double* latency_ms) {
  if (!s) return GS2_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return GS2_ERR_NOT_FOUND;
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(std::max(timeout_s, 0.0));
  if (!s->cv_done.wait_until(lk, deadline, [&] { return r->state == REQ_DONE; }))
    return GS2_ERR_TIMEOUT;
  return collect_locked(s, r, info, x_out, latency_ms);
}

gs2_status gs2_server_get_stats(gs2_server* s, gs2_server_stats* out) {
  if (!s || !out) return GS2_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->pending = (int64_t)s->pending.size();
  out->active = s->slots_used;
  out->max_active = s->max_active;
  out->reserved_bytes = s->reserved;
  out->budget_bytes = s->budget;
  return GS2_OK;
}

void gs2_server_destroy(gs2_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stopping = true;
    for (Request* r : s->pending) {
      s->table.erase(r->ticket);
      delete r;
    }
    s->pending.clear();
    s->cv_prep.notify_all();
    s->cv_loop.notify_all();
  }
  for (auto& t : s->prep) t.join();
  s->loop.join();
  for (auto& kv : s->table) delete kv.second;
  delete s;
}

}  // extern "C"
