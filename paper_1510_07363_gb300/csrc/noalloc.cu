// noalloc.cu -- lrs_apply_static: the same preconditioner apply as lrs_apply,
// for callers that cannot allocate device memory at apply time (code that
// runs inside another library's fixed memory pool, under a strict memory
// budget, or from a context where cudaMalloc is forbidden).  Its scratch --
// the three extended vectors of the traversal and the traversal's task tables
// -- lives in the file-scope array below instead of being allocated.
#include <map>
#include <mutex>

#include "runtime.h"

namespace {

// Static scratch: 2^21 doubles (16 MiB), held by every GPU that loads this
// library until the process exits.
constexpr size_t kStaticScratchDoubles = size_t(1) << 21;
__device__ __align__(256) double g_apply_scratch[kStaticScratchDoubles];

// Device address of g_apply_scratch, looked up once per device.  In host code
// the symbol is only a host-side stand-in; the address must come from
// cudaGetSymbolAddress with the device current.
struct ScratchSlot {
  bool ready = false;
  double* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
ScratchSlot g_slots[kMaxDevices];
std::mutex g_slots_mutex;

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LRS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LRS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_slots_mutex);
  if (!g_slots[dev].ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess) return LRS_ERR_CUDA;
    g_slots[dev].ptr = static_cast<double*>(p);
    g_slots[dev].ready = true;
  }
  *out = g_slots[dev].ptr;
  return LRS_OK;
}

inline size_t round256(size_t doubles) { return (doubles + 31) & ~size_t(31); }

}  // namespace

extern "C" int lrs_apply_static(lrs_factor_t* f, const double* b, double* x, int nrhs) {
  using namespace lrs;
  if (!f || !b || !x || nrhs < 1 || b == x) return LRS_ERR_INVALID_ARG;
  if (f->apply32) return LRS_ERR_INVALID_ARG;    // FP32 storage: its traversal is lrs_apply's
  try {
    // the array's address is per device: a call made with another device
    // current would copy into that device's array, so it is refused first
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return LRS_ERR_CUDA;
    if (cur != f->device) return LRS_ERR_INVALID_ARG;
    double* base = nullptr;
    int st = scratch_address(&base);
    if (st != LRS_OK) return st;
    const int64_t ext = f->ext_n;
    const size_t vec = round256((size_t)ext * nrhs);
    if ((size_t)ext * nrhs > kStaticScratchDoubles / 3) return LRS_ERR_INVALID_ARG;
    double* y = base;
    double* fv = base + vec;
    double* xe = base + 2 * vec;
    // task tables of the traversal, pointing into the static vectors
    std::vector<GemmTerm> terms;
    std::vector<GemmTask> tasks;
    std::vector<int> fd0, fdn, fu0, fun, bw0, bwn;
    auto add = [&](double* C, const double* D, int rows, int mode, const std::vector<GemmTerm>& tm) {
      if (rows <= 0) return;
      const int t0 = (int)terms.size();
      terms.insert(terms.end(), tm.begin(), tm.end());
      for (int tj = 0; tj * kTile < nrhs; ++tj)
        for (int ti = 0; ti * kTile < rows; ++ti)
          tasks.push_back(GemmTask{C, D, (int)ext, (int)ext, rows, nrhs, ti, tj, t0, (int)tm.size(), mode});
    };
    for (auto [r0, cnt] : f->phases) {
      fd0.push_back((int)tasks.size());
      for (int r = r0; r < r0 + cnt; ++r) {
        const ElimRecord& rec = f->recs[r];
        if (rec.m == 0) continue;
        const int64_t op = f->node_offset(rec.level, rec.node);
        add(fv + op, nullptr, rec.m, 0, {GemmTerm{rec.inv, y + op, rec.m, (int)ext, rec.m, 0}});
      }
      fdn.push_back((int)tasks.size() - fd0.back());
      fu0.push_back((int)tasks.size());
      std::map<int64_t, std::pair<int, std::vector<GemmTerm>>> upd;
      for (int r = r0; r < r0 + cnt; ++r) {
        const ElimRecord& rec = f->recs[r];
        if (rec.m == 0) continue;
        const int64_t op = f->node_offset(rec.level, rec.node);
        for (size_t v = 0; v < rec.nbr.size(); ++v) {
          if (rec.nbr_m[v] == 0) continue;
          auto& e = upd[f->node_offset(rec.level, rec.nbr[v])];
          e.first = rec.nbr_m[v];
          e.second.push_back(GemmTerm{rec.L[v], fv + op, rec.nbr_m[v], (int)ext, rec.m, 0});
        }
      }
      for (auto& kv : upd) add(y + kv.first, nullptr, kv.second.first, kAccumulate | kSubtract, kv.second.second);
      fun.push_back((int)tasks.size() - fu0.back());
      bw0.push_back((int)tasks.size());
      for (int r = r0; r < r0 + cnt; ++r) {
        const ElimRecord& rec = f->recs[r];
        if (rec.m == 0) continue;
        const int64_t op = f->node_offset(rec.level, rec.node);
        std::vector<GemmTerm> tm;
        for (size_t v = 0; v < rec.nbr.size(); ++v)
          if (rec.nbr_m[v])
            tm.push_back(GemmTerm{rec.T[v], xe + f->node_offset(rec.level, rec.nbr[v]), rec.m, (int)ext,
                                  rec.nbr_m[v], 0});
        if (tm.empty()) add(xe + op, fv + op, rec.m, 0, {GemmTerm{nullptr, nullptr, 1, 1, 0, 0}});
        else add(xe + op, fv + op, rec.m, kSubtract, tm);
      }
      bwn.push_back((int)tasks.size() - bw0.back());
    }
    const size_t term_d = round256((terms.size() * sizeof(GemmTerm) + 7) / 8);
    const size_t task_d = round256((tasks.size() * sizeof(GemmTask) + 7) / 8);
    if (3 * vec + term_d + task_d > kStaticScratchDoubles) return LRS_ERR_INVALID_ARG;
    GemmTerm* dterms = reinterpret_cast<GemmTerm*>(base + 3 * vec);
    GemmTask* dtasks = reinterpret_cast<GemmTask*>(base + 3 * vec + term_d);
    cudaStream_t s = f->stream;
    const lrs_plan& P = *f->plan;
    if (!terms.empty())
      cuda_check(cudaMemcpyAsync(dterms, terms.data(), terms.size() * sizeof(GemmTerm), cudaMemcpyHostToDevice, s),
                 "static terms");
    if (!tasks.empty())
      cuda_check(cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, s),
                 "static tasks");
    // the array keeps the previous call's contents: y must start at zero
    cuda_check(cudaMemsetAsync(y, 0, (size_t)ext * nrhs * sizeof(double), s), "static zero");
    launch_permute_in(b, P.n, nrhs, f->d_perm, y, ext, s);
    const size_t nph = f->phases.size();
    for (size_t k = 0; k < nph; ++k) {
      launch_gemm(dtasks + fd0[k], fdn[k], dterms, s);
      launch_gemm(dtasks + fu0[k], fun[k], dterms, s);
    }
    for (size_t k = nph; k-- > 0;) launch_gemm(dtasks + bw0[k], bwn[k], dterms, s);
    launch_permute_out(xe, ext, P.n, nrhs, f->d_perm, x, s);
    cuda_check(cudaGetLastError(), "static apply launch");
    cuda_check(cudaStreamSynchronize(s), "static apply");
    return LRS_OK;
  } catch (const lrs::Error& e) {
    return e.code;
  } catch (...) {
    return LRS_ERR_CUDA;
  }
}
