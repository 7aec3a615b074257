// Test doubles for the CUDA runtime and the library's kernel launches, so that
// the factorization's and the traversal's host planning (factor.cu, solve.cu,
// emu_plan.cpp) run on a machine without a GPU.  Device memory is a fake
// address range that is never dereferenced; host-to-device copies keep a host
// shadow, so that every launch double can read the task arrays it is given and
// check them against what its kernel reads: tiles inside their blocks, term
// ranges inside the launch's terms, and for the emulated products every digit,
// exponent and flag the product kernel addresses inside the split that wrote
// it and inside the launch's workspace.  Ranks and singular values read back
// from the "device" are a constant rank (the scenario sets it), so the symbolic
// program runs with blocks of realistic sizes.  Test infrastructure only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "host_doubles.h"

namespace hp {
int rank_value = 16;
Checks checks;
std::map<uintptr_t, std::vector<char>> shadow;   // host copies of uploaded arrays, by device address
uint64_t digest = 1469598103934665603ull;        // FNV-1a over every checked task array, in launch order

void fail(const char* what, int line) {
  if (checks.failures++ < 20) std::fprintf(stderr, "host planning check failed: %s (device_doubles.cpp:%d)\n", what, line);
}

// the host copy of [p, p + bytes) if one upload holds it
const void* host_of(const void* p, size_t bytes) {
  if (!p) return nullptr;
  auto it = shadow.upper_bound((uintptr_t)p);
  if (it == shadow.begin()) return nullptr;
  --it;
  const uintptr_t off = (uintptr_t)p - it->first;
  if (off + bytes > it->second.size()) return nullptr;
  return it->second.data() + off;
}

void mix(const void* data, size_t bytes) {
  const unsigned char* c = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) digest = (digest ^ c[i]) * 1099511628211ull;
}
template <class T>
void mix_value(const T& v) {
  mix(&v, sizeof(v));
}
// field by field: the structs' padding bytes hold whatever was there before
template <class Task>
void mix_tasks(const Task* t, int n) {
  for (int i = 0; i < n; ++i) {
    mix_value(t[i].C), mix_value(t[i].D), mix_value(t[i].ldc), mix_value(t[i].ldd), mix_value(t[i].rows);
    mix_value(t[i].cols), mix_value(t[i].ti), mix_value(t[i].tj), mix_value(t[i].term0), mix_value(t[i].nterm);
    mix_value(t[i].mode);
  }
}
}  // namespace hp

#define CHECK(c)                       \
  do {                                 \
    if (!(c)) hp::fail(#c, __LINE__);  \
  } while (0)

// ---------------------------------------------------------------- runtime
namespace {
char* fake_next = reinterpret_cast<char*>(0x100000000000ull);
}
extern "C" {
cudaError_t cudaMalloc(void** p, size_t b) {
  *p = fake_next;
  fake_next += (b + 4095) & ~size_t(4095);
  return cudaSuccess;
}
cudaError_t cudaFree(void*) { return cudaSuccess; }
cudaError_t cudaHostAlloc(void** p, size_t b, unsigned int) {
  *p = std::malloc(b);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaMallocHost(void** p, size_t b) { return cudaHostAlloc(p, b, 0); }
cudaError_t cudaFreeHost(void* p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t b, cudaMemcpyKind k, cudaStream_t) {
  if (k == cudaMemcpyDeviceToHost) {
    // ranks (int) and singular values: the constant rank, word by word
    int* q = static_cast<int*>(d);
    for (size_t i = 0; i < b / sizeof(int); ++i) q[i] = hp::rank_value;
  } else if (k == cudaMemcpyHostToDevice && b > 0) {
    hp::shadow[(uintptr_t)d].assign(static_cast<const char*>(s), static_cast<const char*>(s) + b);
  }
  return cudaSuccess;
}
cudaError_t cudaMemcpy(void* d, const void*, size_t b, cudaMemcpyKind k) {
  if (k == cudaMemcpyDeviceToHost) std::memset(d, 0, b);   // the status word: no error
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void*, int, size_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t* e) {
  *e = reinterpret_cast<cudaEvent_t>(1);
  return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) {
  *ms = 0.f;
  return cudaSuccess;
}
cudaError_t cudaGetLastError() { return cudaSuccess; }
cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) { return cudaSuccess; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t* g) {
  *g = reinterpret_cast<cudaGraph_t>(1);
  return cudaSuccess;
}
cudaError_t cudaGraphInstantiate(cudaGraphExec_t* e, cudaGraph_t, unsigned long long) {
  *e = reinterpret_cast<cudaGraphExec_t>(1);
  return cudaSuccess;
}
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaSuccess; }
}

// ---------------------------------------------------------------- launches
namespace lrs {
namespace {

// bytes of the upload that holds p, from p on (0 if none does)
size_t avail(const void* p) {
  if (!p) return 0;
  auto it = hp::shadow.upper_bound((uintptr_t)p);
  if (it == hp::shadow.begin()) return 0;
  --it;
  const uintptr_t off = (uintptr_t)p - it->first;
  return off < it->second.size() ? it->second.size() - off : 0;
}

// A launch of tiles tm x tn: every tile inside its block (rows x cols at C,
// leading dimension ldc), its terms inside the launch's term array, every
// term's operands stored with leading dimensions that hold op(A) (rows x k)
// and op(B) (k x cols).
template <class Task, class Term>
void check_tiles(const Task* d_tasks, int n, const Term* d_terms, int tm, int tn) {
  if (n <= 0) return;
  const Task* t = static_cast<const Task*>(hp::host_of(d_tasks, (size_t)n * sizeof(Task)));
  CHECK(t != nullptr);
  if (!t) return;
  hp::mix_tasks(t, n);
  const size_t nterm = avail(d_terms) / sizeof(Term);
  const Term* tm_h = static_cast<const Term*>(hp::host_of(d_terms, nterm * sizeof(Term)));
  for (int i = 0; i < n; ++i) {
    const Task& g = t[i];
    CHECK(g.C != nullptr && g.rows > 0 && g.cols > 0 && g.ldc >= g.rows);
    CHECK(g.D == nullptr || g.ldd >= g.rows);
    CHECK(g.ti >= 0 && g.tj >= 0 && (int64_t)g.ti * tm < g.rows && (int64_t)g.tj * tn < g.cols);
    CHECK(g.term0 >= 0 && g.nterm >= 1 && (size_t)g.term0 + g.nterm <= nterm);
    if (!tm_h || g.term0 < 0 || (size_t)g.term0 + g.nterm > nterm) continue;
    for (int q = 0; q < g.nterm; ++q) {
      const Term& e = tm_h[g.term0 + q];
      CHECK(e.k >= 0);
      if (e.k == 0) continue;
      CHECK(e.A != nullptr && e.B != nullptr);
      CHECK(e.lda >= ((e.trans & 1) ? e.k : g.rows));
      CHECK(e.ldb >= ((e.trans & 2) ? g.cols : e.k));
    }
  }
}

}  // namespace

void launch_gemm(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t) {
  ++hp::checks.gemm_launches;
  hp::checks.gemm_tiles += ntask;
  check_tiles(tasks, ntask, terms, kTile, kTile);
}
void launch_gemm_narrow(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t, int split, double*,
                        bool) {
  ++hp::checks.gemm_launches;
  hp::checks.gemm_tiles += ntask;
  CHECK(split >= 1);
  check_tiles(tasks, ntask, terms, kTile, kTile);
}
void launch_gemv(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t, int split, double*, bool) {
  ++hp::checks.gemm_launches;
  hp::checks.gemm_tiles += ntask;
  CHECK(split >= 1);
  check_tiles(tasks, ntask, terms, kTile, kTile);
}
void launch_gemm_narrow32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t, int split, float*,
                          bool) {
  ++hp::checks.gemm_launches;
  hp::checks.gemm_tiles += ntask;
  CHECK(split >= 1);
  check_tiles(tasks, ntask, terms, kTile, 16);
}
void launch_gemv32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t, int split, float*, bool) {
  ++hp::checks.gemm_launches;
  hp::checks.gemm_tiles += ntask;
  CHECK(split >= 1);
  check_tiles(tasks, ntask, terms, kTile, 16);
}
cudaError_t launch_gemm_tc(const GemmTask* tasks, int ntask, const GemmTerm* terms, DeviceStatus*, cudaStream_t) {
  ++hp::checks.tc_launches;
  hp::checks.tc_tiles += ntask;
  check_tiles(tasks, ntask, terms, kTcTile, kTcTile);
  return cudaSuccess;
}

// The emulated products: the split tasks fill the launch's workspace without
// overlap and in CTA order, and every tile reads digit blocks, exponents and
// flags only inside the split of its own operand, within at most
// kEmuMaxChunks chunks.
cudaError_t launch_gemm_emu(const EmuPlan& plan, const EmuSplitTask* d_split, const GemmTask* d_tasks, int ntask,
                            const EmuTerm* d_eterms, DeviceStatus*, cudaStream_t) {
  ++hp::checks.emu_launches;
  hp::checks.emu_tiles += ntask;
  if (ntask <= 0) return cudaSuccess;
  const size_t nsplit = plan.split.size(), nterm = plan.eterms.size();
  hp::checks.emu_splits += (long long)nsplit;
  const GemmTask* t = static_cast<const GemmTask*>(hp::host_of(d_tasks, (size_t)ntask * sizeof(GemmTask)));
  const EmuTerm* et = static_cast<const EmuTerm*>(hp::host_of(d_eterms, nterm * sizeof(EmuTerm)));
  const EmuSplitTask* sp =
      nsplit ? static_cast<const EmuSplitTask*>(hp::host_of(d_split, nsplit * sizeof(EmuSplitTask))) : nullptr;
  CHECK(t != nullptr && et != nullptr && (nsplit == 0 || sp != nullptr));
  if (!t || !et || (nsplit && !sp)) return cudaSuccess;
  hp::mix_tasks(t, ntask);
  const uint8_t* base = nsplit ? sp[0].dig : nullptr;     // the first split starts the workspace
  const uint8_t* end = base + plan.bytes;
  int cta = 0;
  for (size_t i = 0; i < nsplit; ++i) {
    const EmuSplitTask& s = sp[i];
    const size_t nch = (size_t)(s.k + kEmuChunk - 1) / kEmuChunk;
    const size_t ngr = (size_t)(s.k + kEmuChunk * kEmuGroup - 1) / (kEmuChunk * kEmuGroup);
    CHECK(s.cta0 == cta);
    CHECK(s.tile == kEmuTileM || s.tile == kEmuTileN);
    CHECK(s.rows <= s.rows_pad && s.rows_pad % s.tile == 0 && s.rows_pad % kEmuSplitRows == 0);
    CHECK(((uintptr_t)s.dig & 15) == 0);
    CHECK(s.dig >= base && s.dig + (size_t)s.rows_pad * nch * kEmuChunk * 16 <= end);
    CHECK((const uint8_t*)s.ex >= base && (const uint8_t*)(s.ex + (size_t)s.rows_pad * ngr) <= end);
    CHECK((const uint8_t*)s.bad >= base + plan.bad_off &&
          (const uint8_t*)(s.bad + s.rows_pad) <= base + plan.bad_off + plan.bad_bytes);
    if (i > 0) CHECK(s.dig >= sp[i - 1].dig + (size_t)sp[i - 1].rows_pad * ((sp[i - 1].k + 63) / 64) * 1024);
    cta += (s.rows_pad / kEmuSplitRows) * (int)ngr;
  }
  CHECK(cta == plan.split_ctas);
  auto split_of = [&](const uint8_t* dig) -> const EmuSplitTask* {
    for (size_t i = 0; i < nsplit; ++i)
      if (sp[i].dig == dig) return &sp[i];
    return nullptr;
  };
  for (int i = 0; i < ntask; ++i) {
    const GemmTask& g = t[i];
    CHECK(g.C != nullptr && g.rows > 0 && g.cols > 0 && g.ldc >= g.rows);
    CHECK(g.ti >= 0 && g.tj >= 0 && g.ti * kEmuTileM < g.rows && g.tj * kEmuTileN < g.cols);
    CHECK(g.term0 >= 0 && g.nterm >= 1 && (size_t)g.term0 + g.nterm <= nterm);
    if (g.term0 < 0 || (size_t)g.term0 + g.nterm > nterm) continue;
    int chunks = 0;
    for (int q = 0; q < g.nterm; ++q) {
      const EmuTerm& e = et[g.term0 + q];
      const size_t nch = (size_t)(e.k + kEmuChunk - 1) / kEmuChunk;
      chunks += (int)nch;
      if (e.k == 0) continue;
      const EmuSplitTask* a = split_of(e.a_dig);
      const EmuSplitTask* b = split_of(e.b_dig);
      CHECK(a != nullptr && b != nullptr);
      if (!a || !b) continue;
      CHECK(a->k == e.k && b->k == e.k && a->tile == kEmuTileM && b->tile == kEmuTileN);
      CHECK(e.a_tiles * kEmuTileM == a->rows_pad && e.b_tiles * kEmuTileN == b->rows_pad);
      CHECK(e.a_rows_pad == a->rows_pad && e.b_rows_pad == b->rows_pad);
      CHECK(e.a_ex == a->ex && e.b_ex == b->ex && e.a_bad == a->bad && e.b_bad == b->bad);
      CHECK(g.ti < e.a_tiles && g.tj < e.b_tiles && g.rows <= a->rows_pad && g.cols <= b->rows_pad);
      // the product kernel's last bulk copies: K step (nch 4 - 1), this tile
      CHECK(e.a_dig + ((nch * 4 - 1) * e.a_tiles + g.ti + 1) * (size_t)(kEmuTileM * 16 * 16) <=
            a->dig + (size_t)a->rows_pad * nch * kEmuChunk * 16);
      CHECK(e.b_dig + ((nch * 4 - 1) * e.b_tiles + g.tj + 1) * (size_t)(kEmuTileN * 16 * 16) <=
            b->dig + (size_t)b->rows_pad * nch * kEmuChunk * 16);
    }
    CHECK(chunks <= kEmuMaxChunks);
  }
  return cudaSuccess;
}

// Copies: mode 0 copy, 1 transpose, 2 alpha I (or zero), 3 in-place mirror of
// a square block, 4 one diagonal piece of alpha I.
void launch_copy(const CopyTask* tasks, int ntask, cudaStream_t) {
  ++hp::checks.copy_launches;
  hp::checks.copy_tasks += ntask;
  if (ntask <= 0) return;
  const CopyTask* t = static_cast<const CopyTask*>(hp::host_of(tasks, (size_t)ntask * sizeof(CopyTask)));
  CHECK(t != nullptr);
  if (!t) return;
  for (int i = 0; i < ntask; ++i) {
    hp::mix_value(t[i].src), hp::mix_value(t[i].dst), hp::mix_value(t[i].lds), hp::mix_value(t[i].ldd);
    hp::mix_value(t[i].rows), hp::mix_value(t[i].cols), hp::mix_value(t[i].mode), hp::mix_value(t[i].alpha);
  }
  for (int i = 0; i < ntask; ++i) {
    const CopyTask& c = t[i];
    CHECK(c.mode >= 0 && c.mode <= 4 && c.rows >= 0 && c.cols >= 0);
    if (c.rows == 0 || c.cols == 0) continue;
    CHECK(c.dst != nullptr && c.ldd >= c.rows);
    if (c.mode == 0) CHECK(c.src != nullptr && c.lds >= c.rows);
    if (c.mode == 1) CHECK(c.src != nullptr && c.lds >= c.cols);
    if (c.mode == 3) CHECK(c.src == c.dst && c.rows == c.cols);
  }
}

#define OTHER ++hp::checks.other_launches
cudaError_t launch_eig(const EigTask*, int, int, TeamKind, int, DeviceStatus*, cudaStream_t) { OTHER; return cudaSuccess; }
cudaError_t launch_invert(const InvTask*, int, int, TeamKind, int, DeviceStatus*, cudaStream_t) { OTHER; return cudaSuccess; }
cudaError_t launch_invert_resident(const InvTask*, const InvTask*, int, DeviceStatus*, cudaStream_t) { OTHER; return cudaSuccess; }
cudaError_t launch_tridiag_resident(const EigTask*, const EigTask*, int, DeviceStatus*, cudaStream_t) { OTHER; return cudaSuccess; }
cudaError_t launch_resident_mix(const InvTask*, const InvTask*, int, const EigTask*, const EigTask*, int, DeviceStatus*,
                                cudaStream_t) { OTHER; return cudaSuccess; }
void launch_amax(const double*, int64_t, DeviceStatus*, cudaStream_t) { OTHER; }
void launch_asymmetry(const double*, const int64_t*, int64_t, DeviceStatus*, cudaStream_t) { OTHER; }
void launch_scatter(const double*, const int64_t*, int64_t, double*, cudaStream_t) { OTHER; }
void launch_sumsq(const SumSqTask*, int, double*, double*, cudaStream_t) { OTHER; }
void launch_to_f32(const ConvTask*, int, cudaStream_t) { OTHER; }
void launch_permute_in(const double*, int64_t, int, const int32_t*, double*, int64_t, cudaStream_t) { OTHER; }
void launch_permute_out(const double*, int64_t, int64_t, int, const int32_t*, double*, cudaStream_t) { OTHER; }
void launch_permute_in32(const double*, int64_t, int, const int32_t*, float*, int64_t, cudaStream_t) { OTHER; }
void launch_permute_out32(const float*, int64_t, int64_t, int, const int32_t*, double*, cudaStream_t) { OTHER; }
void launch_spmv(int64_t, const int64_t*, const int32_t*, const double*, const double*, double*, int, cudaStream_t) { OTHER; }
void launch_dot(const double*, const double*, int64_t, int, const Segments&, double*, double*, cudaStream_t) { OTHER; }
void launch_axpy_col(const double*, double, const double*, double*, int64_t, int, const Segments&, cudaStream_t) { OTHER; }
void launch_scale_col(const double*, const int*, const double*, double*, int64_t, int, const Segments&, cudaStream_t) { OTHER; }
void launch_combine(const double*, int, const double*, int64_t, double*, int64_t, int, const Segments&, cudaStream_t) { OTHER; }
void launch_residual(const double*, double*, int64_t, cudaStream_t) { OTHER; }

// ---------------------------------------------------------------- dense-kernel planners
// Simple stand-ins with the library's workspace sizes: one resident block per
// wave, resident up to m = 2400, sub-teams of one CTA.
int grid_team_size(int m, bool eig) { return eig ? 152 : std::min(256, std::max(8, (m + 15) / 16)); }
int sub_team_capacity(int) { return 304; }
std::vector<std::pair<int, int>> plan_sub_teams(const int*, int n, int capacity, int* team0, int* size) {
  std::vector<std::pair<int, int>> waves;
  capacity = std::max(capacity, 1);
  for (int b = 0; b < n; b += capacity) {
    const int e = std::min(n, b + capacity);
    for (int i = b; i < e; ++i) {
      team0[i] = i - b;
      size[i] = 1;
    }
    waves.emplace_back(b, e);
  }
  return waves;
}
size_t inv_resident_workspace(int m) { return (size_t)m * m + m + 8; }
size_t tridiag_resident_workspace(int m) { return (size_t)m * (m + 4) + (size_t)m * m + 2 * (size_t)m + 8; }
bool resident_fits(int m, bool) { return m >= 1 && m <= 2400; }
std::vector<std::pair<int, int>> plan_mixed_waves(const int* m, const char*, int n, int* cta0, int* cw, int) {
  std::vector<std::pair<int, int>> waves;
  for (int i = 0; i < n; ++i) {
    if (!resident_fits(m[i], false)) return {};
    cta0[i] = 0;
    cw[i] = std::max(1, (m[i] + 151) / 152);
    waves.emplace_back(i, i + 1);
  }
  return waves;
}
std::vector<std::pair<int, int>> plan_resident_waves(const int* m, int n, bool eig, int* cta0, int* cw, int sms) {
  std::vector<char> kinds((size_t)n, eig ? 1 : 0);
  return plan_mixed_waves(m, kinds.data(), n, cta0, cw, sms);
}
}  // namespace lrs
