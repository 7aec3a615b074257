// serve.cu -- the serving form: factorizations kept resident on the device and
// a request loop around them.  Factorizations are admitted by an HBM budget,
// `workers` threads execute requests at once, and the solves queued against
// one factor are merged into one multi-column GMRES (continuous batching).
// Host code only: the device work is lrs_factor / lrs_solve (or the caller's
// executor hooks).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "lrs_internal.h"

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  bool is_factor = false;
  // factorization
  const lrs_plan* plan = nullptr;
  const double* val = nullptr;
  double eps = 0.0;
  int precision = LRS_PREC_FP64;
  size_t reserve = 0;
  // solve
  int64_t factor = 0;
  const double* b = nullptr;
  double* x = nullptr;
  int nrhs = 0;
  lrs_solve_opts so{};
  // outcome
  bool done = false;
  double t_submit = 0.0, t_start = 0.0;
  lrs_request_info info{};
  // a factorization holds a reference to its plan from submission until the
  // request is forgotten (the factor built from it takes its own)
  ~Request() { lrs::unref_plan(plan); }
};

struct Resident {
  void* handle = nullptr;     // the executor's factor, once built
  int64_t n = 0;
  size_t bytes = 0;           // held bytes once built
  bool admitted = false, built = false, failed = false, busy = false, evicting = false;
  int status = LRS_OK;
  int pending = 0;            // solves queued or running against it
};

// The library's executor: every factor on its own CUDA stream, with
// stream-ordered allocations (cudaFree would synchronise the whole device
// and serialise the workers).
struct GpuFactor {
  lrs_factor_t* f = nullptr;
  cudaStream_t st = nullptr;
};

void* gpu_alloc(size_t bytes, void* stream, void*) {
  void* p = nullptr;
  return cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(stream)) == cudaSuccess ? p : nullptr;
}

void gpu_free(void* p, size_t, void* stream, void*) { cudaFreeAsync(p, static_cast<cudaStream_t>(stream)); }

// Factorizations run one at a time (process-wide): their dense kernels are
// cooperative launches whose CTAs wait on one another, and two of them must
// not share the GPU.  Solves have no such kernels and overlap freely.
std::mutex factor_mu;

int gpu_factor(void*, const lrs_plan* plan, const double* val, double eps, int precision, void** out,
               size_t* bytes) {
  std::lock_guard<std::mutex> one_at_a_time(factor_mu);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LRS_ERR_CUDA;
  lrs_factor_opts o{};
  o.eps = eps;
  o.stream = st;
  o.alloc = gpu_alloc;
  o.free = gpu_free;
  o.precision = precision;
  lrs_factor_t* f = nullptr;
  const int code = lrs_factor(plan, val, 0, &o, &f);
  if (code != LRS_OK) {
    cudaStreamDestroy(st);
    return code;
  }
  lrs_stats stv{};
  lrs_factor_stats(f, &stv);
  GpuFactor* g = new (std::nothrow) GpuFactor{f, st};
  if (!g) {
    lrs_factor_destroy(f);
    cudaStreamDestroy(st);
    return LRS_ERR_OOM;
  }
  *out = g;
  *bytes = (size_t)stv.factor_bytes;
  return LRS_OK;
}

int gpu_solve(void*, void* h, const double* b, double* x, int nrhs, const lrs_solve_opts* o, lrs_solve_info* info) {
  return lrs_solve(static_cast<GpuFactor*>(h)->f, b, x, nrhs, 0, o, info);
}

void gpu_release(void*, void* h) {
  GpuFactor* g = static_cast<GpuFactor*>(h);
  lrs_factor_destroy(g->f);
  cudaStreamDestroy(g->st);
  delete g;
}

bool same_opts(const lrs_solve_opts& a, const lrs_solve_opts& b) {
  return a.restart == b.restart && a.maxit == b.maxit && a.tol == b.tol && a.side == b.side &&
         (a.precond_residual != 0) == (b.precond_residual != 0);
}

}  // namespace

struct lrs_server {
  lrs_server_opts o{};
  bool gpu = true;                  // the library's executor (else the caller's hooks)
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int64_t, std::unique_ptr<Request>> reqs;   // submitted and not yet waited for
  std::deque<int64_t> q_solve, q_factor;              // queued, in submission order
  std::map<int64_t, Resident> res;                    // factors by their ticket
  std::vector<void*> release_later;                   // handles to release outside the lock
  size_t held = 0;                                    // built bytes + admitted reservations
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;

  void finish(Request* r, int status) {
    r->info.status = status;
    r->info.queue_ms = (r->t_start > 0.0 ? r->t_start : now_ms()) - r->t_submit;
    r->done = true;
  }

  // Solves queued against factor id fail with `status` (its factorization
  // failed, or it was evicted before it was built).
  void fail_solves_of(int64_t id, int status) {
    for (auto it = q_solve.begin(); it != q_solve.end();) {
      Request* r = reqs.at(*it).get();
      if (r->factor == id) {
        finish(r, status);
        res.at(id).pending--;
        it = q_solve.erase(it);
      } else {
        ++it;
      }
    }
  }

  // A factor marked for eviction goes once nothing runs or waits on it.
  void maybe_release(int64_t id) {
    auto it = res.find(id);
    if (it == res.end()) return;
    Resident& f = it->second;
    if (!f.evicting || f.busy || f.pending > 0 || (f.admitted && !f.built && !f.failed)) return;
    if (f.built) {
      release_later.push_back(f.handle);
      held -= f.bytes;
    }
    res.erase(it);
  }

  // Under the lock: the next work, solves first.  Returns false when none.
  bool pick(std::vector<Request*>& batch, Request*& fac) {
    for (size_t i = 0; i < q_solve.size(); ++i) {
      Request* r = reqs.at(q_solve[i]).get();
      Resident& f = res.at(r->factor);
      if (!f.built || f.busy) continue;
      batch.push_back(r);
      int total = r->nrhs;
      std::vector<size_t> take = {i};
      for (size_t j = i + 1; j < q_solve.size(); ++j) {
        Request* q = reqs.at(q_solve[j]).get();
        if (q->factor != r->factor || !same_opts(q->so, r->so) || total + q->nrhs > o.max_batch_rhs) continue;
        batch.push_back(q);
        total += q->nrhs;
        take.push_back(j);
      }
      for (size_t k = take.size(); k-- > 0;) q_solve.erase(q_solve.begin() + (std::ptrdiff_t)take[k]);
      f.busy = true;
      const double t = now_ms();
      for (Request* q : batch) q->t_start = t;
      return true;
    }
    if (!q_factor.empty()) {
      Request* r = reqs.at(q_factor.front()).get();
      if (held + r->reserve <= o.hbm_budget) {
        q_factor.pop_front();
        held += r->reserve;
        res.at(r->id).admitted = true;
        r->t_start = now_ms();
        fac = r;
        return true;
      }
    }
    return false;
  }

  void run_factor(Request* r) {
    void* h = nullptr;
    size_t bytes = 0;
    const int code = o.factor_fn(o.exec_ctx, r->plan, r->val, r->eps, r->precision, &h, &bytes);
    const double t_end = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    Resident& f = res.at(r->id);
    held -= r->reserve;
    if (code == LRS_OK) {
      f.handle = h;
      f.bytes = bytes;
      f.built = true;
      held += bytes;
    } else {
      f.failed = true;
      f.status = code;
      fail_solves_of(r->id, code);
    }
    r->info.bytes = code == LRS_OK ? bytes : 0;
    r->info.run_ms = t_end - r->t_start;
    finish(r, code);
    maybe_release(r->id);
  }

  void run_solves(const std::vector<Request*>& batch) {
    Request* r0 = batch.front();
    const int64_t id = r0->factor;
    void* h;
    int64_t n;
    {
      std::lock_guard<std::mutex> lk(mu);
      const Resident& f = res.at(id);
      h = f.handle;
      n = f.n;
    }
    int total = 0;
    for (Request* r : batch) total += r->nrhs;
    lrs_solve_info info{};
    int code;
    if (batch.size() == 1) {
      code = o.solve_fn(o.exec_ctx, h, r0->b, r0->x, r0->nrhs, &r0->so, &info);
    } else {
      // the requests' columns side by side (column-major n x total), one GMRES
      std::vector<double> B, X;
      try {
        B.resize((size_t)n * total);
        X.resize((size_t)n * total);
      } catch (...) {
        B.clear();
      }
      if (B.empty()) {
        code = LRS_ERR_OOM;
      } else {
        size_t c = 0;
        for (Request* r : batch) {
          std::memcpy(B.data() + c * n, r->b, sizeof(double) * (size_t)n * r->nrhs);
          c += r->nrhs;
        }
        code = o.solve_fn(o.exec_ctx, h, B.data(), X.data(), total, &r0->so, &info);
        c = 0;
        for (Request* r : batch) {
          std::memcpy(r->x, X.data() + c * n, sizeof(double) * (size_t)n * r->nrhs);
          c += r->nrhs;
        }
      }
    }
    const double t_end = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    Resident& f = res.at(id);
    f.busy = false;
    for (Request* r : batch) {
      r->info.iters = info.iters;
      r->info.rel_res = info.rel_res;
      r->info.batch_rhs = total;
      r->info.run_ms = t_end - r->t_start;
      finish(r, code);
      f.pending--;
    }
    maybe_release(id);
  }

  void worker() {
    if (gpu) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      std::vector<Request*> batch;
      Request* fac = nullptr;
      cv_work.wait(lk, [&] { return stop || pick(batch, fac); });
      if (batch.empty() && !fac) break;
      lk.unlock();
      if (fac) run_factor(fac);
      else run_solves(batch);
      lk.lock();
      std::vector<void*> rel;
      rel.swap(release_later);
      cv_done.notify_all();
      cv_work.notify_all();
      if (!rel.empty()) {
        lk.unlock();
        for (void* p : rel) o.release_fn(o.exec_ctx, p);
        lk.lock();
      }
    }
  }
};

extern "C" {

int lrs_server_create(const lrs_server_opts* opts, lrs_server** out) {
  if (!opts || !out || opts->hbm_budget == 0 || opts->workers < 1 || opts->max_batch_rhs < 1)
    return LRS_ERR_INVALID_ARG;
  const int hooks = (opts->factor_fn != nullptr) + (opts->solve_fn != nullptr) + (opts->release_fn != nullptr);
  if (hooks != 0 && hooks != 3) return LRS_ERR_INVALID_ARG;
  lrs_server* s = new (std::nothrow) lrs_server();
  if (!s) return LRS_ERR_OOM;
  s->o = *opts;
  s->gpu = hooks == 0;
  if (s->gpu) {
    if (cudaGetDevice(&s->device) != cudaSuccess) {
      delete s;
      return LRS_ERR_CUDA;
    }
    s->o.factor_fn = gpu_factor;
    s->o.solve_fn = gpu_solve;
    s->o.release_fn = gpu_release;
  }
  try {
    for (int w = 0; w < opts->workers; ++w) s->workers.emplace_back([s] { s->worker(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers) t.join();
    delete s;
    return LRS_ERR_OOM;
  }
  *out = s;
  return LRS_OK;
}

int lrs_server_factor(lrs_server* s, const lrs_plan* plan, const double* val, double eps, int precision,
                      size_t reserve_bytes, int64_t* ticket) {
  if (!s || !plan || !val || !ticket || !(eps >= 0.0)) return LRS_ERR_INVALID_ARG;
  if (precision != LRS_PREC_FP64 && precision != LRS_PREC_FP32) return LRS_ERR_INVALID_ARG;
  const size_t reserve = reserve_bytes ? reserve_bytes : (size_t)65536 * (size_t)plan->n;
  if (reserve > s->o.hbm_budget) return LRS_ERR_OOM;
  try {
    std::lock_guard<std::mutex> lk(s->mu);
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->is_factor = true;
    plan->refs.fetch_add(1, std::memory_order_relaxed);
    r->plan = plan;
    r->val = val;
    r->eps = eps;
    r->precision = precision;
    r->reserve = reserve;
    r->t_submit = now_ms();
    Resident f;
    f.n = plan->n;
    s->res[r->id] = f;
    s->q_factor.push_back(r->id);
    *ticket = r->id;
    s->reqs[r->id] = std::move(r);
  } catch (...) {
    return LRS_ERR_OOM;
  }
  s->cv_work.notify_one();
  return LRS_OK;
}

int lrs_server_solve(lrs_server* s, int64_t factor_ticket, const double* b, double* x, int nrhs,
                     const lrs_solve_opts* opts, int64_t* ticket) {
  if (!s || !b || !x || nrhs < 1 || !opts || !ticket) return LRS_ERR_INVALID_ARG;
  if (opts->restart < 1 || opts->maxit < 1 || !(opts->tol > 0.0)) return LRS_ERR_INVALID_ARG;
  if (opts->side != LRS_GMRES_RIGHT && opts->side != LRS_GMRES_LEFT) return LRS_ERR_INVALID_ARG;
  try {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->res.find(factor_ticket);
    if (it == s->res.end()) return LRS_ERR_INVALID_ARG;
    Resident& f = it->second;
    if (f.evicting) return LRS_ERR_STATE;
    if (f.failed) return f.status;
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->factor = factor_ticket;
    r->b = b;
    r->x = x;
    r->nrhs = nrhs;
    r->so = *opts;
    r->t_submit = now_ms();
    f.pending++;
    s->q_solve.push_back(r->id);
    *ticket = r->id;
    s->reqs[r->id] = std::move(r);
  } catch (...) {
    return LRS_ERR_OOM;
  }
  s->cv_work.notify_one();
  return LRS_OK;
}

int lrs_server_wait(lrs_server* s, int64_t ticket, lrs_request_info* info) {
  if (!s || !info) return LRS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->reqs.find(ticket) == s->reqs.end()) return LRS_ERR_INVALID_ARG;
  // looked up again after every wake-up: another waiter may have taken it
  s->cv_done.wait(lk, [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second->done;
  });
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LRS_ERR_INVALID_ARG;
  *info = it->second->info;
  s->reqs.erase(it);
  return LRS_OK;
}

int lrs_server_evict(lrs_server* s, int64_t factor_ticket) {
  if (!s) return LRS_ERR_INVALID_ARG;
  std::vector<void*> rel;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->res.find(factor_ticket);
    if (it == s->res.end()) return LRS_ERR_INVALID_ARG;
    Resident& f = it->second;
    f.evicting = true;
    if (!f.admitted) {
      // still queued: never built; it and the solves waiting for it end here
      auto q = std::find(s->q_factor.begin(), s->q_factor.end(), factor_ticket);
      if (q != s->q_factor.end()) {
        s->q_factor.erase(q);
        s->fail_solves_of(factor_ticket, LRS_ERR_STATE);
        s->finish(s->reqs.at(factor_ticket).get(), LRS_ERR_STATE);
      }
    }
    s->maybe_release(factor_ticket);
    rel.swap(s->release_later);
  }
  for (void* p : rel) s->o.release_fn(s->o.exec_ctx, p);
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return LRS_OK;
}

int lrs_server_stats(lrs_server* s, size_t* held_bytes, int* resident, int* queued) {
  if (!s) return LRS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (held_bytes) *held_bytes = s->held;
  if (resident) {
    int k = 0;
    for (const auto& kv : s->res) k += kv.second.built && !kv.second.evicting;
    *resident = k;
  }
  if (queued) *queued = (int)(s->q_solve.size() + s->q_factor.size());
  return LRS_OK;
}

void lrs_server_destroy(lrs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (std::thread& t : s->workers) t.join();
  for (void* p : s->release_later) s->o.release_fn(s->o.exec_ctx, p);
  for (auto& kv : s->res)
    if (kv.second.built) s->o.release_fn(s->o.exec_ctx, kv.second.handle);
  delete s;
}

}  // extern "C"
