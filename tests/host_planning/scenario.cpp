// Scenario runner of the host-planning test: builds a stencil matrix (or a batch of
// them), runs lrs::analyze / analyze_batch, the factorization's host program
// (Algorithm 1's launches, recorded and checked by device_doubles.cpp) and the
// traversal's with 1 and 16 right-hand sides, then prints one line of counts
// and the digest of every checked task array.  Exit status 1 if any check
// failed.  Test infrastructure only.
//
//   scenario <grid> <nx> <ny> <nz> <leaf> <rank> <sym 0/1> <fp32 0/1> <emu 0/1>
//            [<instances> [<separation 2/3> [<curoff6 0/1>]]]
//
// grid: 5/7-point Poisson pattern on nx x ny (x nz) points (nz = 1: 2D);
// instances > 1: that many matrices with nx + 8 k columns, as one batched plan;
// separation 3: the stronger well-separation (Sec. 7); curoff6: eq. curOff6's
// truncation (its level norms are launched at every level).
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "host_doubles.h"
#include "runtime.h"

namespace {
struct Matrix {
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<double> val, xyz;
  int64_t n = 0;
  int dim = 2;
};

Matrix stencil(int nx, int ny, int nz) {
  Matrix a;
  a.n = (int64_t)nx * ny * nz;
  a.dim = nz > 1 ? 3 : 2;
  a.rowptr.push_back(0);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t r = ((int64_t)z * ny + y) * nx + x;
        auto add = [&](int64_t c, double v) {
          a.colind.push_back((int32_t)c);
          a.val.push_back(v);
        };
        if (z > 0) add(r - (int64_t)nx * ny, -1.0);
        if (y > 0) add(r - nx, -1.0);
        if (x > 0) add(r - 1, -1.0);
        add(r, 2.0 * a.dim);
        if (x + 1 < nx) add(r + 1, -1.0);
        if (y + 1 < ny) add(r + nx, -1.0);
        if (z + 1 < nz) add(r + (int64_t)nx * ny, -1.0);
        a.rowptr.push_back((int64_t)a.colind.size());
        a.xyz.push_back(x);
        a.xyz.push_back(y);
        if (a.dim == 3) a.xyz.push_back(z);
      }
  return a;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc < 10) {
    std::fprintf(stderr, "usage: scenario grid nx ny nz leaf rank sym fp32 emu [instances [separation [curoff6]]]\n");
    return 2;
  }
  const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]);
  const int leaf = std::atoi(argv[5]);
  hp::rank_value = std::atoi(argv[6]);
  const bool sym = std::atoi(argv[7]) != 0, fp32 = std::atoi(argv[8]) != 0, emu = std::atoi(argv[9]) != 0;
  const int count = argc > 10 ? std::atoi(argv[10]) : 1;
  const int separation = argc > 11 ? std::atoi(argv[11]) : 0;
  const bool curoff6 = argc > 12 && std::atoi(argv[12]) != 0;

  std::vector<Matrix> mats;
  for (int k = 0; k < count; ++k) mats.push_back(stencil(nx + 8 * k, ny, nz));
  std::vector<lrs_csr> csr;
  for (const Matrix& m : mats)
    csr.push_back(lrs_csr{m.n, m.rowptr.data(), m.colind.data(), m.val.data(), m.dim, m.xyz.data()});
  lrs_analyze_opts ao{leaf, 0, separation};
  lrs_plan* plan = nullptr;
  const int st = count > 1 ? lrs::analyze_batch(count, csr.data(), &ao, &plan) : lrs::analyze(csr.data(), &ao, &plan);
  if (st != LRS_OK || !plan) {
    std::fprintf(stderr, "analysis failed: %d\n", st);
    return 2;
  }

  // a factor as lrs_factor sets it up (device pointers from the doubles)
  lrs_factor_t* f = new lrs_factor_t();
  f->plan = plan;
  f->eps = 1e-2;
  f->symmetry = sym ? LRS_SYM_SYMMETRIC : LRS_SYM_GENERAL;
  f->precision = fp32 ? LRS_PREC_FP32 : LRS_PREC_FP64;
  f->gemm_emu = emu;
  f->trunc_rule = curoff6 ? LRS_TRUNC_CUROFF6 : LRS_TRUNC_CUTOFF1;
  for (lrs::Arena* a : {&f->persist, &f->trans[0], &f->trans[1], &f->scratch, &f->workspace, &f->store32, &f->emu_ws})
    a->al = &f->al;
  try {
    f->stager.init(&f->al, f->stream, size_t(8) << 20);
    f->status = static_cast<lrs::DeviceStatus*>(f->al.get(sizeof(lrs::DeviceStatus)));
    f->d_perm = static_cast<int32_t*>(f->al.get(plan->n * sizeof(int32_t)));
    const double* d_val = static_cast<const double*>(f->al.get(plan->nnz * sizeof(double)));
    lrs::run_factor(f, d_val, 1);
    if (fp32) lrs::move_factor_to_f32(f);
    for (int nrhs : {1, 16}) {
      const double* b = static_cast<const double*>(f->al.get(plan->n * nrhs * sizeof(double)));
      double* x = static_cast<double*>(f->al.get(plan->n * nrhs * sizeof(double)));
      lrs::run_apply_device(f, b, x, nrhs);
    }
  } catch (const lrs::Error& e) {
    std::fprintf(stderr, "library error %d: %s\n", e.code, e.what);
    return 2;
  }
  const hp::Checks& c = hp::checks;
  std::printf(
      "n=%lld ext_n=%lld eliminations=%zu phases=%zu max_rank=%d gemm_launches=%lld gemm_tiles=%lld "
      "emu_launches=%lld emu_tiles=%lld emu_splits=%lld tc_launches=%lld tc_tiles=%lld copy_launches=%lld "
      "copy_tasks=%lld other_launches=%lld failures=%lld digest=%016llx\n",
      (long long)plan->n, (long long)f->ext_n, f->recs.size(), f->phases.size(), f->stats.max_rank, c.gemm_launches,
      c.gemm_tiles, c.emu_launches, c.emu_tiles, c.emu_splits, c.tc_launches, c.tc_tiles, c.copy_launches,
      c.copy_tasks, c.other_launches, c.failures, (unsigned long long)hp::digest);
  return c.failures ? 1 : 0;
}
