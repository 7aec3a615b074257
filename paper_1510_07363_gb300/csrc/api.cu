// api.cu -- the extern "C" entry points declared in include/lrs.h.  Each one
// validates its arguments, runs the C++ runtime and turns internal errors
// into status codes; no exception leaves this file.
#include <algorithm>
#include <new>
#include <vector>

#include "runtime.h"

namespace {

template <class Fn>
int guarded(Fn&& fn) {
  try {
    fn();
    return LRS_OK;
  } catch (const lrs::Error& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    return LRS_ERR_OOM;
  } catch (...) {
    return LRS_ERR_CUDA;
  }
}

void release(lrs_factor_t* f) {
  if (!f) return;
  cudaStreamSynchronize(f->stream);
  if (f->side) cudaStreamSynchronize(f->side);    // inverses of a batch an error interrupted
  if (f->prog.graph) cudaGraphExecDestroy(f->prog.graph);
  f->persist.release();
  f->store32.release();
  f->emu_ws.release();
  f->trans[0].release();
  f->trans[1].release();
  f->scratch.release();
  f->workspace.release();
  f->stager.release();
  f->prof.release();
  if (f->side) cudaStreamDestroy(f->side);
  if (f->ev_fork) cudaEventDestroy(f->ev_fork);
  if (f->ev_join) cudaEventDestroy(f->ev_join);
  f->al.put(f->status, sizeof(lrs::DeviceStatus));
  f->al.put(f->d_perm, f->plan->n * sizeof(int32_t));
  f->al.put(f->d_rowptr, (f->plan->n + 1) * sizeof(int64_t));
  f->al.put(f->d_colind, f->plan->nnz * sizeof(int32_t));
  f->al.put(f->d_val, f->plan->nnz * sizeof(double));
  f->al.put(const_cast<int64_t*>(f->segs.seg_off), f->plan->inst_row_off.size() * sizeof(int64_t));
  f->al.put(const_cast<int32_t*>(f->segs.seg), f->plan->n * sizeof(int32_t));
  const lrs_plan* plan = f->plan;
  delete f;
  lrs::unref_plan(plan);
}

int export_vec(const std::vector<int32_t>& v, int32_t* out, int64_t* count) {
  *count = (int64_t)v.size();
  if (out) std::copy(v.begin(), v.end(), out);
  return LRS_OK;
}

// Copy a host multi-vector to the device (or pass a device one through).
struct DevVec {
  lrs_factor_t* f;
  double* p = nullptr;
  size_t bytes = 0;
  bool owned = false;
  DevVec(lrs_factor_t* f_, const double* src, size_t count, int on_device, bool copy_in) : f(f_) {
    bytes = count * sizeof(double);
    if (on_device) { p = const_cast<double*>(src); return; }
    p = static_cast<double*>(f->al.get(bytes ? bytes : 8));
    owned = true;
    if (copy_in && bytes)
      lrs::cuda_check(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, f->stream), "vector in");
  }
  void copy_out(double* dst) {
    if (owned && bytes)
      lrs::cuda_check(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyDeviceToHost, f->stream), "vector out");
  }
  ~DevVec() {
    if (owned) {
      cudaStreamSynchronize(f->stream);
      f->al.put(p, bytes ? bytes : 8);
    }
  }
};

}  // namespace

extern "C" {

int lrs_analyze(const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out) {
  int st = LRS_OK;
  int g = guarded([&] { st = lrs::analyze(A, opts, out); });
  return g != LRS_OK ? g : st;
}

int lrs_analyze_batch(int count, const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out) {
  int st = LRS_OK;
  int g = guarded([&] { st = lrs::analyze_batch(count, A, opts, out); });
  return g != LRS_OK ? g : st;
}

int lrs_plan_export(const lrs_plan* plan, int what, int32_t* out, int64_t* count) {
  if (!plan || !count || what < 0 || what > 5) return LRS_ERR_INVALID_ARG;
  return guarded([&] {
    std::vector<int32_t> v;
    lrs::export_plan(*plan, what, v);
    export_vec(v, out, count);
  });
}

void lrs_plan_destroy(lrs_plan* plan) { lrs::unref_plan(plan); }

int lrs_factor(const lrs_plan* plan, const double* val, int val_on_device, const lrs_factor_opts* opts,
               lrs_factor_t** out) {
  if (!plan || !val || !opts || !out || !(opts->eps >= 0.0)) return LRS_ERR_INVALID_ARG;
  if ((opts->alloc == nullptr) != (opts->free == nullptr)) return LRS_ERR_INVALID_ARG;
  if (opts->symmetry < LRS_SYM_DETECT || opts->symmetry > LRS_SYM_SYMMETRIC) return LRS_ERR_INVALID_ARG;
  if (opts->precision != LRS_PREC_FP64 && opts->precision != LRS_PREC_FP32) return LRS_ERR_INVALID_ARG;
  if (opts->trunc_rule != LRS_TRUNC_CUTOFF1 && opts->trunc_rule != LRS_TRUNC_CUROFF6) return LRS_ERR_INVALID_ARG;
  if (opts->gemm != LRS_GEMM_AUTO && opts->gemm != LRS_GEMM_FP64 && opts->gemm != LRS_GEMM_EMU) return LRS_ERR_INVALID_ARG;
  lrs_factor_t* f = new (std::nothrow) struct lrs_factor();
  if (!f) return LRS_ERR_OOM;
  f->plan = plan;
  plan->refs.fetch_add(1, std::memory_order_relaxed);
  f->stream = static_cast<cudaStream_t>(opts->stream);
  f->eps = opts->eps;
  f->symmetry = opts->symmetry;
  f->precision = opts->precision;
  f->trunc_rule = opts->trunc_rule;
  f->gemm_emu = opts->gemm != LRS_GEMM_FP64;
  f->al.alloc = opts->alloc;
  f->al.free = opts->free;
  f->al.ctx = opts->alloc_ctx;
  f->al.stream = f->stream;
  f->prof.on = opts->profile != 0;
  f->prof.stream = f->stream;
  if (f->prof.on) {
    const char* path = std::getenv("LRS_TRACE");   // optional per-launch trace (class,ms,flops,bytes,m,kind,ntask)
    if (path && *path) f->prof.trace = std::fopen(path, "a");
  }
  for (lrs::Arena* a : {&f->persist, &f->trans[0], &f->trans[1], &f->scratch, &f->workspace, &f->store32,
                        &f->emu_ws})
    a->al = &f->al;
  int st = guarded([&] {
    lrs::cuda_check(cudaGetDevice(&f->device), "device");
    lrs::cuda_check(cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking), "side stream");
    lrs::cuda_check(cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming), "event");
    lrs::cuda_check(cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming), "event");
    f->stager.init(&f->al, f->stream, size_t(8) << 20);
    f->status = static_cast<lrs::DeviceStatus*>(f->al.get(sizeof(lrs::DeviceStatus)));
    lrs::cuda_check(cudaMemsetAsync(f->status, 0, sizeof(lrs::DeviceStatus), f->stream), "status");
    const lrs_plan& P = *plan;
    f->d_perm = static_cast<int32_t*>(f->al.get(P.n * sizeof(int32_t)));
    f->d_rowptr = static_cast<int64_t*>(f->al.get((P.n + 1) * sizeof(int64_t)));
    f->d_colind = static_cast<int32_t*>(f->al.get(std::max<int64_t>(P.nnz, 1) * sizeof(int32_t)));
    lrs::cuda_check(cudaMemcpyAsync(f->d_perm, P.perm.data(), P.n * sizeof(int32_t), cudaMemcpyHostToDevice, f->stream), "perm");
    lrs::cuda_check(cudaMemcpyAsync(f->d_rowptr, P.rowptr.data(), (P.n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, f->stream), "rowptr");
    lrs::cuda_check(cudaMemcpyAsync(f->d_colind, P.colind.data(), P.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, f->stream), "colind");
    const int nseg = (int)P.inst_row_off.size() - 1;
    if (nseg > 1) {
      // segment tables of a batched plan: instance row ranges, instance of each row
      int64_t* off = static_cast<int64_t*>(f->al.get((nseg + 1) * sizeof(int64_t)));
      f->segs.seg_off = off;
      int32_t* seg = static_cast<int32_t*>(f->al.get(P.n * sizeof(int32_t)));
      f->segs.seg = seg;
      f->segs.nseg = nseg;
      f->seg_host.assign(P.n, 0);
      for (int k = 0; k < nseg; ++k)
        std::fill(f->seg_host.begin() + P.inst_row_off[k], f->seg_host.begin() + P.inst_row_off[k + 1], k);
      lrs::cuda_check(cudaMemcpyAsync(off, P.inst_row_off.data(), (nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, f->stream), "segments");
      lrs::cuda_check(cudaMemcpyAsync(seg, f->seg_host.data(), P.n * sizeof(int32_t), cudaMemcpyHostToDevice, f->stream), "segments");
    }
    lrs::run_factor(f, val, val_on_device);
    if (f->precision == LRS_PREC_FP32) lrs::move_factor_to_f32(f);
    lrs::cuda_check(cudaStreamSynchronize(f->stream), "factor");
    std::vector<int32_t>().swap(f->seg_host);
  });
  if (st != LRS_OK) {
    release(f);
    return st;
  }
  *out = f;
  return LRS_OK;
}

int lrs_apply(lrs_factor_t* f, const double* b, double* x, int nrhs, int on_device) {
  if (!f || !b || !x || nrhs < 1 || b == x) return LRS_ERR_INVALID_ARG;
  return guarded([&] {
    const size_t count = (size_t)f->plan->n * nrhs;
    DevVec db(f, b, count, on_device, true), dx(f, x, count, on_device, false);
    lrs::run_apply_device(f, db.p, dx.p, nrhs);
    dx.copy_out(x);
    lrs::cuda_check(cudaStreamSynchronize(f->stream), "apply");
    f->prof.collect();
  });
}

int lrs_solve(lrs_factor_t* f, const double* b, double* x, int nrhs, int on_device, const lrs_solve_opts* opts,
              lrs_solve_info* info) {
  if (info) {
    info->iters = 0;
    info->status = LRS_ERR_INVALID_ARG;
    info->rel_res = -1.0;
    info->rel_res_precond = -1.0;
  }
  if (!f || !b || !x || !opts || !info || nrhs < 1 || b == x) return LRS_ERR_INVALID_ARG;
  if (opts->restart < 1 || opts->maxit < 1 || !(opts->tol >= 0.0)) return LRS_ERR_INVALID_ARG;
  if (opts->side != LRS_GMRES_RIGHT && opts->side != LRS_GMRES_LEFT) return LRS_ERR_INVALID_ARG;
  int st = guarded([&] {
    const size_t count = (size_t)f->plan->n * nrhs;
    DevVec db(f, b, count, on_device, true), dx(f, x, count, on_device, false);
    lrs::run_gmres_device(f, db.p, dx.p, nrhs, *opts, info);
    dx.copy_out(x);
    lrs::cuda_check(cudaStreamSynchronize(f->stream), "solve");
    f->prof.collect();
  });
  if (st != LRS_OK) {
    info->status = st;
    return st;
  }
  return info->status;
}

int lrs_factor_export(const lrs_factor_t* f, int what, int32_t* out, int64_t* count) {
  if (!f || !count) return LRS_ERR_INVALID_ARG;
  if (what == 5) return export_vec(f->ranks, out, count);
  if (what == 6) return export_vec(f->pivots, out, count);
  if (what == 7) return export_vec(f->last_iters, out, count);
  return LRS_ERR_INVALID_ARG;
}

int lrs_factor_sigma(const lrs_factor_t* f, int64_t k, double* out, int64_t* count) {
  if (!f || !count || k < 0 || k >= (int64_t)f->sigma_off.size()) return LRS_ERR_INVALID_ARG;
  const int64_t b = f->sigma_off[k];
  const int64_t e = (k + 1 < (int64_t)f->sigma_off.size()) ? f->sigma_off[k + 1] : (int64_t)f->sigma_all.size();
  *count = e - b;
  if (out) std::copy(f->sigma_all.begin() + b, f->sigma_all.begin() + e, out);
  return LRS_OK;
}

int lrs_factor_stats(const lrs_factor_t* f, lrs_stats* out) {
  if (!f || !out) return LRS_ERR_INVALID_ARG;
  *out = f->stats;
  return LRS_OK;
}

int lrs_factor_profile(lrs_factor_t* f, lrs_prof_entry* out, int reset) {
  if (!f || !out) return LRS_ERR_INVALID_ARG;
  return guarded([&] {
    lrs::cuda_check(cudaStreamSynchronize(f->stream), "profile");
    f->prof.collect();
    for (int c = 0; c < LRS_PROF_CLASSES; ++c) out[c] = f->prof.acc[c];
    if (reset)
      for (int c = 0; c < LRS_PROF_CLASSES; ++c) f->prof.acc[c] = lrs_prof_entry{};
  });
}

void lrs_factor_destroy(lrs_factor_t* f) { release(f); }

const char* lrs_status_string(int status) {
  switch (status) {
    case LRS_OK: return "ok";
    case LRS_ERR_INVALID_ARG: return "invalid argument";
    case LRS_ERR_OOM: return "out of memory";
    case LRS_ERR_SINGULAR_PIVOT: return "singular pivot block";
    case LRS_ERR_NOT_CONVERGED: return "GMRES did not converge";
    case LRS_ERR_TIMEOUT: return "device wait timed out";
    case LRS_ERR_CUDA: return "CUDA error";
    case LRS_ERR_NUMERIC: return "NaN or Inf in the factorization";
    case LRS_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

int lrs_selftest_bounded_wait(double* waited_ms) {
  using namespace lrs;
  if (!waited_ms) return LRS_ERR_INVALID_ARG;
  unsigned long long* words = nullptr;
  DeviceStatus* st = nullptr;
  if (cudaMalloc(&words, 4 * sizeof(unsigned long long)) != cudaSuccess) return LRS_ERR_OOM;
  if (cudaMalloc(&st, sizeof(DeviceStatus)) != cudaSuccess) {
    cudaFree(words);
    return LRS_ERR_OOM;
  }
  int code = LRS_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMemset(words, 0, 4 * sizeof(unsigned long long)) == cudaSuccess &&
      cudaMemset(st, 0, sizeof(DeviceStatus)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    cudaEventRecord(e0, 0);
    if (launch_bounded_wait_selftest(words, st, 0) == cudaSuccess) {
      cudaEventRecord(e1, 0);
      DeviceStatus hs{};
      unsigned long long hw[4] = {0, 0, 0, 0};
      float ms = 0.f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
          cudaMemcpy(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost) == cudaSuccess &&
          cudaMemcpy(hw, words, sizeof(hw), cudaMemcpyDeviceToHost) == cudaSuccess) {
        *waited_ms = ms;
        // the expected outcome: the wait gave up (0), set the abort word and the status
        code = (hw[2] == 0 && hw[1] == 1 && hs.wait_timeout == 1) ? LRS_ERR_TIMEOUT : LRS_ERR_STATE;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(words);
  cudaFree(st);
  return code;
}

}  // extern "C"

namespace {
// The emulated product of lrs_block_gemm: its plan, a workspace and the task
// arrays from cudaMalloc (freed after the synchronous call), on stream 0.
cudaError_t run_emu(const std::vector<lrs::GemmTask>& tasks, const lrs::GemmTerm& term, const lrs::GemmTask* d_tasks,
                    lrs::DeviceStatus* d_st, cudaEvent_t e0, cudaEvent_t e1) {
  using namespace lrs;
  EmuPlan plan = plan_gemm_emu(tasks.data(), (int)tasks.size(), &term, 1);
  uint8_t* work = nullptr;
  EmuSplitTask* d_split = nullptr;
  EmuTerm* d_eterm = nullptr;
  cudaError_t e = cudaMalloc(&work, std::max<size_t>(plan.bytes, 256));
  if (e == cudaSuccess) e = cudaMalloc(&d_split, std::max<size_t>(1, plan.split.size()) * sizeof(EmuSplitTask));
  if (e == cudaSuccess) e = cudaMalloc(&d_eterm, sizeof(EmuTerm));
  if (e == cudaSuccess) {
    plan.bind(work);
    e = cudaMemcpy(d_split, plan.split.data(), plan.split.size() * sizeof(EmuSplitTask), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_eterm, plan.eterms.data(), sizeof(EmuTerm), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && plan.bad_bytes) e = cudaMemset(work + plan.bad_off, 0, plan.bad_bytes);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    cudaEventRecord(e0, 0);                           // the split and product kernels only
    if (e == cudaSuccess) e = launch_gemm_emu(plan, d_split, d_tasks, (int)tasks.size(), d_eterm, d_st, 0);
    cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  }
  cudaFree(work);
  cudaFree(d_split);
  cudaFree(d_eterm);
  return e;
}
}  // namespace

extern "C" {

int lrs_block_gemm(int engine, int rows, int cols, int k, const double* A, int lda, int transa, const double* B,
                   int ldb, int transb, double* C, int ldc, int accumulate, int subtract, double* ms) {
  using namespace lrs;
  if (engine != LRS_GEMM_FP64 && engine != LRS_GEMM_EMU && engine != LRS_GEMM_TF32) return LRS_ERR_INVALID_ARG;
  if (rows < 0 || cols < 0 || k < 0 || !C || ldc < std::max(1, rows)) return LRS_ERR_INVALID_ARG;
  if (k > 0 && (!A || !B)) return LRS_ERR_INVALID_ARG;
  if (k > 0 && lda < std::max(1, transa ? k : rows)) return LRS_ERR_INVALID_ARG;
  if (k > 0 && ldb < std::max(1, transb ? cols : k)) return LRS_ERR_INVALID_ARG;
  if (engine == LRS_GEMM_EMU && k > kEmuChunk * kEmuMaxChunks) return LRS_ERR_INVALID_ARG;
  if (ms) *ms = 0.0;
  if (rows == 0 || cols == 0) return LRS_OK;
  const int tm = engine == LRS_GEMM_EMU ? kEmuTileM : engine == LRS_GEMM_TF32 ? kTcTile : kTile;
  const int tn = engine == LRS_GEMM_EMU ? kEmuTileN : engine == LRS_GEMM_TF32 ? kTcTile : kTile;
  const GemmTerm term{A, B, lda, ldb, k, (transa ? 1 : 0) | (transb ? 2 : 0)};
  const int mode = (accumulate ? kAccumulate : 0) | (subtract ? kSubtract : 0);
  std::vector<GemmTask> tasks;
  for (int tj = 0; tj < (cols + tn - 1) / tn; ++tj)
    for (int ti = 0; ti < (rows + tm - 1) / tm; ++ti)
      tasks.push_back(GemmTask{C, nullptr, ldc, 0, rows, cols, ti, tj, 0, k > 0 ? 1 : 0, mode});
  GemmTask* d_tasks = nullptr;
  GemmTerm* d_term = nullptr;
  DeviceStatus* d_st = nullptr;
  int code = LRS_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&d_tasks, tasks.size() * sizeof(GemmTask)) == cudaSuccess &&
      cudaMalloc(&d_term, sizeof(GemmTerm)) == cudaSuccess &&
      cudaMalloc(&d_st, sizeof(DeviceStatus)) == cudaSuccess) {
    code = LRS_ERR_CUDA;
    if (cudaMemcpy(d_tasks, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice) == cudaSuccess &&
        cudaMemcpy(d_term, &term, sizeof(GemmTerm), cudaMemcpyHostToDevice) == cudaSuccess &&
        cudaMemset(d_st, 0, sizeof(DeviceStatus)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
      cudaError_t le = cudaSuccess;
      if (engine != LRS_GEMM_EMU) cudaEventRecord(e0, 0);
      if (engine == LRS_GEMM_EMU) le = run_emu(tasks, term, d_tasks, d_st, e0, e1);
      else if (engine == LRS_GEMM_TF32) le = launch_gemm_tc(d_tasks, (int)tasks.size(), d_term, d_st, 0);
      else {
        launch_gemm(d_tasks, (int)tasks.size(), d_term, 0);
        le = cudaGetLastError();
      }
      if (engine != LRS_GEMM_EMU) cudaEventRecord(e1, 0);
      DeviceStatus hs{};
      float t = 0.f;
      if (le == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
          cudaMemcpy(&hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost) == cudaSuccess) {
        if (ms) *ms = t;
        code = hs.wait_timeout ? LRS_ERR_TIMEOUT : LRS_OK;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_tasks);
  cudaFree(d_term);
  cudaFree(d_st);
  return code;
}

}  // extern "C"
