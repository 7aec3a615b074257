// runtime.h -- device memory, task staging and the factor object of liblrs.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "lrs_internal.h"

namespace lrs {

// Internal error carrier; converted to a status code at the ABI boundary.
struct Error {
  int code;
  const char* what;
};
[[noreturn]] inline void fail(int code, const char* what) { throw Error{code, what}; }
inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(e == cudaErrorMemoryAllocation ? LRS_ERR_OOM : LRS_ERR_CUDA, what);
}

// Device allocations through the caller's hooks (or cudaMalloc).
struct Allocator {
  lrs_alloc_fn alloc = nullptr;
  lrs_free_fn free = nullptr;
  void* ctx = nullptr;
  cudaStream_t stream = nullptr;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (alloc) p = alloc(bytes, (void*)stream, ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
    if (!p) fail(LRS_ERR_OOM, "device allocation");
    return p;
  }
  void put(void* p, size_t bytes) {
    if (!p) return;
    if (free) free(p, bytes, (void*)stream, ctx);
    else cudaFree(p);
  }
};

// Bump allocator over device chunks; reset() keeps the chunks for reuse.
// Every block starts on a 256-byte boundary.
struct Arena {
  struct Chunk { char* p; size_t size, used; };
  Allocator* al = nullptr;
  std::vector<Chunk> chunks;
  size_t cur = 0;
  size_t chunk_bytes = size_t(256) << 20;
  double* take(size_t count) {
    const size_t bytes = ((count * sizeof(double)) + 255) & ~size_t(255);
    if (bytes == 0) return nullptr;
    while (cur < chunks.size()) {
      Chunk& c = chunks[cur];
      if (c.size - c.used >= bytes) {
        double* p = reinterpret_cast<double*>(c.p + c.used);
        c.used += bytes;
        return p;
      }
      ++cur;
    }
    const size_t sz = bytes > chunk_bytes ? bytes : chunk_bytes;
    chunks.push_back({static_cast<char*>(al->get(sz)), sz, bytes});
    cur = chunks.size() - 1;
    return reinterpret_cast<double*>(chunks.back().p);
  }
  void reset() {
    for (auto& c : chunks) c.used = 0;
    cur = 0;
  }
  size_t held() const {
    size_t s = 0;
    for (auto& c : chunks) s += c.size;
    return s;
  }
  void release() {
    for (auto& c : chunks) al->put(c.p, c.size);
    chunks.clear();
    cur = 0;
  }
};

// Host -> device staging of task arrays: pinned host ring plus a device
// mirror; flush() waits for the stream before the ring is reused.
struct Stager {
  // Chunks of pinned host memory, each with a device mirror.  Space handed
  // out by put() is never reused before the next flush(), so a launch may
  // take several puts (tasks and terms) and a later put can neither move nor
  // overwrite an earlier one; flush() waits for the stream and recycles all.
  struct Chunk {
    char* host = nullptr;
    char* dev = nullptr;
    size_t cap = 0;
  };
  Allocator* al = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<Chunk> chunks;
  size_t chunk_bytes = 0, cur = 0, used = 0;
  void init(Allocator* a, cudaStream_t s, size_t bytes) {
    al = a;
    stream = s;
    chunk_bytes = bytes;
    add(bytes);
  }
  void add(size_t bytes) {
    Chunk c;
    c.cap = std::max(bytes, chunk_bytes);
    cuda_check(cudaMallocHost(&c.host, c.cap), "pinned staging");
    c.dev = static_cast<char*>(al->get(c.cap));
    chunks.push_back(c);
  }
  void flush() {
    cuda_check(cudaStreamSynchronize(stream), "stream sync");
    cur = 0;
    used = 0;
  }
  template <class T>
  const T* put(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    const size_t bytes = ((v.size() * sizeof(T)) + 255) & ~size_t(255);
    while (cur < chunks.size() && used + bytes > chunks[cur].cap) {
      ++cur;
      used = 0;
    }
    if (cur == chunks.size()) add(bytes);
    Chunk& c = chunks[cur];
    std::memcpy(c.host + used, v.data(), v.size() * sizeof(T));
    cuda_check(cudaMemcpyAsync(c.dev + used, c.host + used, v.size() * sizeof(T), cudaMemcpyHostToDevice, stream),
               "stage tasks");
    const T* p = reinterpret_cast<const T*>(c.dev + used);
    used += bytes;
    return p;
  }
  void release() {
    for (Chunk& c : chunks) {
      if (c.host) cudaFreeHost(c.host);
      if (c.dev) al->put(c.dev, c.cap);
    }
    chunks.clear();
    cur = used = 0;
  }
};

// Optional per-launch timing: an event pair around every kernel launch,
// resolved (and summed per kernel class) after the stream has synchronised.
struct Profiler {
  bool on = false;
  cudaStream_t stream = nullptr;
  FILE* trace = nullptr;            // per-launch CSV when LRS_TRACE names a file
  struct Pending { int cls; cudaEvent_t a, b; double flops, bytes; int tag, kind, ntask, kernels; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  lrs_prof_entry acc[LRS_PROF_CLASSES] = {};
  cudaEvent_t take() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "profiler event");
    return e;
  }
  cudaEvent_t start(cudaStream_t s = nullptr) {
    if (!on) return nullptr;
    cudaEvent_t e = take();
    cudaEventRecord(e, s ? s : stream);
    return e;
  }
  // tag: largest block size of the launch; kind: 0 one CTA, 1 cluster, 2 grid
  // kernels: the kernel launches the timed region holds (a CUDA graph holds many)
  void stop(int cls, cudaEvent_t a, double flops, double bytes, int tag = 0, int kind = 0, int ntask = 0,
            cudaStream_t s = nullptr, int kernels = 1) {
    if (!on || !a) return;
    cudaEvent_t b = take();
    cudaEventRecord(b, s ? s : stream);
    pending.push_back({cls, a, b, flops, bytes, tag, kind, ntask, kernels});
  }
  void collect() {                  // call after the stream has synchronised
    for (const Pending& p : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      lrs_prof_entry& e = acc[p.cls];
      e.launches += p.kernels;
      e.ms += ms;
      e.flops += p.flops;
      e.bytes += p.bytes;
      if (trace) fprintf(trace, "%d,%.6f,%.6e,%.6e,%d,%d,%d\n", p.cls, ms, p.flops, p.bytes, p.tag, p.kind, p.ntask);
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void release() {
    if (trace) { fclose(trace); trace = nullptr; }
    for (const Pending& p : pending) { pool.push_back(p.a); pool.push_back(p.b); }
    pending.clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// One eliminated node as the solve sees it (Alg. 3, 4): the inverse of its
// pivot block and, per neighbour q eliminated later, L = A_{q,p} and
// T = A_pp^{-1} A_{p,q}.
struct ElimRecord {
  int level;
  int32_t node;                  // local name at its level
  int m;
  const double* inv;
  std::vector<int32_t> nbr;      // local names at the same level
  std::vector<int> nbr_m;
  std::vector<const double*> L, T;
  // the same blocks in FP32 once the precision form's factor has moved to
  // FP32 storage (the FP64 pointers above are then null)
  const float* inv32 = nullptr;
  std::vector<const float*> L32, T32;
};

struct ApplyProgram {
  int nrhs = 0;
  double *y = nullptr, *f = nullptr, *x = nullptr;   // ext_n x nrhs each
  const GemmTask* tasks = nullptr;
  const GemmTerm* terms = nullptr;
  // per phase: [fwd diag, fwd update, bwd] task ranges into `tasks`
  std::vector<int> fd0, fdn, fu0, fun, bw0, bwn;
  // per phase: algorithmic flops and bytes of the three launches
  std::vector<double> fd_flops, fu_flops, bw_flops, fd_bytes, fu_bytes, bw_bytes;
  // per phase: contraction split of the three launches (<= 16 right-hand
  // sides), and the partial-tile buffer they share
  std::vector<int> fds, fus, bws;
  double* part = nullptr;
  // the FP32 traversal (a factor in FP32 storage): FP32 extended vectors,
  // tasks of 64 x 16 tiles, and its partial-tile buffer
  float *y32 = nullptr, *f32 = nullptr, *x32 = nullptr;
  const GemmTask32* tasks32 = nullptr;
  const GemmTerm32* terms32 = nullptr;
  float* part32 = nullptr;
  // the traversal's kernels captured once into a CUDA graph (per nrhs), with
  // their number and algorithmic flops / bytes
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
  double graph_flops = 0.0, graph_bytes = 0.0;
};

}  // namespace lrs

struct lrs_factor {
  const lrs_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;                  // second stream: pivot inverses overlap compression
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0;
  double eps = 0.0;
  int symmetry = LRS_SYM_DETECT;   // option; stats.symmetric says which path was taken
  int precision = LRS_PREC_FP64;
  int trunc_rule = LRS_TRUNC_CUTOFF1;
  bool gemm_emu = true;                         // FP64 products emulated on the tensor cores
  lrs::Allocator al;
  lrs::Arena persist, trans[2], scratch, workspace;
  lrs::Arena store32;                           // the precision form's factor blocks in FP32
  lrs::Arena emu_ws;                            // digit slices of one emulated-product launch
  bool apply32 = false;                         // the traversal reads store32 in FP32 arithmetic
  lrs::Stager stager;
  lrs::DeviceStatus* status = nullptr;          // device
  lrs::Profiler prof;
  // results of the factorization
  std::vector<lrs::ElimRecord> recs;
  std::vector<std::pair<int, int>> phases;      // record ranges eliminated together
  std::vector<std::vector<int64_t>> off_red;    // x_e offsets of red-nodes per level
  std::vector<std::vector<int64_t>> off_black;  // x_e offsets of black-nodes per level
  int64_t ext_n = 0;
  std::vector<int32_t> ranks;                   // per compression, in order
  std::vector<int32_t> pivots;                  // per elimination, in order
  std::vector<int64_t> sigma_off;               // per compression into sigma_all
  std::vector<double> sigma_all;
  std::vector<int32_t> last_iters;
  lrs_stats stats{};
  // solve state
  int32_t* d_perm = nullptr;
  int64_t* d_rowptr = nullptr;
  int32_t* d_colind = nullptr;
  double* d_val = nullptr;
  lrs::Segments segs;                           // GMRES segments: the plan's instances
  std::vector<int32_t> seg_host;                // host copy source of segs.seg
  lrs::ApplyProgram prog;
  std::vector<lrs::GemmTask> prog_tasks;
  std::vector<lrs::GemmTerm> prog_terms;
  std::vector<lrs::GemmTask32> prog_tasks32;
  std::vector<lrs::GemmTerm32> prog_terms32;
  int64_t node_offset(int level, int32_t local) const;
};

namespace lrs {
void run_factor(lrs_factor_t* F, const double* val, int val_on_device);
// The precision form's factor to FP32 storage: every stored block (A_pp^{-1},
// A_qp, T_pq) rounded into store32, the FP64 blocks released; the traversal
// then runs in FP32 (apply32).
void move_factor_to_f32(lrs_factor_t* F);
void build_apply(lrs_factor_t* F, int nrhs);
void run_apply_device(lrs_factor_t* F, const double* b, double* x, int nrhs);
void run_gmres_device(lrs_factor_t* F, const double* b, double* x, int nrhs, const lrs_solve_opts& o,
                      lrs_solve_info* info);
}  // namespace lrs
