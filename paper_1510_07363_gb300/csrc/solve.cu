// solve.cu -- Algorithms 2-4 (forward and backward traversal of the stored
// factor) and right-preconditioned restarted GMRES on the GPU.
//
// The extended vector x_e (Sec. 4.5) holds the leaf red-nodes in bisection
// order followed, per level, by the black-nodes and the red-nodes of the level
// above; the two red-nodes of a super-node are adjacent, so concatenation
// (eq. concatRHS) and SplitVar cost nothing.  Nodes eliminated together (one
// phase: the super-nodes or the black-nodes of one batch) are independent, so
// each traversal step is one launch per phase:
//   forward  f_p = A_pp^{-1} y_p ; y_q -= sum_p A_{q,p} f_p        (SolveL)
//   backward x_p = f_p - sum_q (A_pp^{-1} A_{p,q}) x_q              (SolveU)
// which is Alg. 4's x_p = A_pp^{-1} (y_p - sum_q A_{p,q} x_q) regrouped.
#include <algorithm>
#include <cmath>
#include <map>

#include "runtime.h"

namespace lrs {

// The FP32 traversal of a factor in FP32 storage: the same phases and tasks
// as build_apply's below, on FP32 blocks and FP32 extended vectors, with tiles
// of 64 rows x 16 columns (tj counts 16-column slices, any nrhs).
static void build_apply32(lrs_factor_t* F, int nrhs) {
  ApplyProgram& pg = F->prog;
  const int64_t ext = F->ext_n;
  pg.nrhs = nrhs;
  pg.y32 = reinterpret_cast<float*>(F->workspace.take(((size_t)ext * nrhs + 1) / 2));
  pg.f32 = reinterpret_cast<float*>(F->workspace.take(((size_t)ext * nrhs + 1) / 2));
  pg.x32 = reinterpret_cast<float*>(F->workspace.take(((size_t)ext * nrhs + 1) / 2));
  std::vector<GemmTask32>& tasks = F->prog_tasks32;
  std::vector<GemmTerm32>& terms = F->prog_terms32;
  tasks.clear();
  terms.clear();
  size_t part_tiles = 0;
  auto split_of = [&](int t0) -> int {
    const int nt = (int)tasks.size() - t0;
    if (nt <= 0 || nt >= kSplitTarget / 2) return 1;
    int chunks = 0;
    for (int i = t0; i < (int)tasks.size(); ++i) {
      int c = 0;
      for (int q = 0; q < tasks[i].nterm; ++q) c += (terms[tasks[i].term0 + q].k + kTileK - 1) / kTileK;
      chunks = std::max(chunks, c);
    }
    const int S = std::max(1, std::min({(kSplitTarget + nt - 1) / nt, chunks / 4, 32}));
    if (S > 1) part_tiles = std::max(part_tiles, (size_t)S * nt);
    return S;
  };
  const int tn = nrhs == 1 ? 1 : 16;
  double cur_flops = 0.0, cur_bytes = 0.0;
  auto add = [&](float* C, const float* D, int rows, int mode, const std::vector<GemmTerm32>& tm) {
    if (rows <= 0) return;
    for (const GemmTerm32& t : tm) {
      cur_flops += 2.0 * rows * nrhs * t.k;
      cur_bytes += 4.0 * ((double)rows * t.k + (double)t.k * nrhs);
    }
    cur_bytes += 4.0 * rows * nrhs * ((D || (mode & kAccumulate)) ? 2 : 1);
    const int t0 = (int)terms.size();
    terms.insert(terms.end(), tm.begin(), tm.end());
    for (int tj = 0; tj * tn < nrhs; ++tj)
      for (int ti = 0; ti * kTile < rows; ++ti)
        tasks.push_back(GemmTask32{C, D, (int)ext, (int)ext, rows, nrhs, ti, tj, t0, (int)tm.size(), mode});
  };
  int64_t bytes = 0;
  for (auto [r0, cnt] : F->phases) {
    pg.fd0.push_back((int)tasks.size());
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      add(pg.f32 + op, nullptr, rec.m, 0, {GemmTerm32{rec.inv32, pg.y32 + op, rec.m, (int)ext, rec.m, 0}});
      bytes += (int64_t)rec.m * rec.m * 4;
    }
    pg.fdn.push_back((int)tasks.size() - pg.fd0.back());
    pg.fds.push_back(split_of(pg.fd0.back()));
    pg.fd_flops.push_back(cur_flops); pg.fd_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
    pg.fu0.push_back((int)tasks.size());
    std::map<int64_t, std::pair<int, std::vector<GemmTerm32>>> upd;
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      for (size_t v = 0; v < rec.nbr.size(); ++v) {
        const int mq = rec.nbr_m[v];
        if (mq == 0) continue;
        auto& e = upd[F->node_offset(rec.level, rec.nbr[v])];
        e.first = mq;
        e.second.push_back(GemmTerm32{rec.L32[v], pg.f32 + op, mq, (int)ext, rec.m, 0});
        bytes += (int64_t)rec.m * mq * 4;
      }
    }
    for (auto& kv : upd) add(pg.y32 + kv.first, nullptr, kv.second.first, kAccumulate | kSubtract, kv.second.second);
    pg.fun.push_back((int)tasks.size() - pg.fu0.back());
    pg.fus.push_back(split_of(pg.fu0.back()));
    pg.fu_flops.push_back(cur_flops); pg.fu_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
    pg.bw0.push_back((int)tasks.size());
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      std::vector<GemmTerm32> tm;
      for (size_t v = 0; v < rec.nbr.size(); ++v) {
        const int mq = rec.nbr_m[v];
        if (mq == 0) continue;
        tm.push_back(GemmTerm32{rec.T32[v], pg.x32 + F->node_offset(rec.level, rec.nbr[v]), rec.m, (int)ext, mq, 0});
        bytes += (int64_t)rec.m * mq * 4;
      }
      if (tm.empty()) add(pg.x32 + op, pg.f32 + op, rec.m, 0, {GemmTerm32{nullptr, nullptr, 1, 1, 0, 0}});
      else add(pg.x32 + op, pg.f32 + op, rec.m, kSubtract, tm);
    }
    pg.bwn.push_back((int)tasks.size() - pg.bw0.back());
    pg.bws.push_back(split_of(pg.bw0.back()));
    pg.bw_flops.push_back(cur_flops); pg.bw_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
  }
  F->stats.apply_bytes = bytes;
  pg.part32 = part_tiles ? reinterpret_cast<float*>(F->workspace.take(part_tiles * kTile * 16 / 2 + 1)) : nullptr;
  GemmTerm32* dterms = reinterpret_cast<GemmTerm32*>(F->workspace.take((terms.size() * sizeof(GemmTerm32) + 7) / 8 + 1));
  GemmTask32* dtasks = reinterpret_cast<GemmTask32*>(F->workspace.take((tasks.size() * sizeof(GemmTask32) + 7) / 8 + 1));
  if (!terms.empty())
    cuda_check(cudaMemcpyAsync(dterms, terms.data(), terms.size() * sizeof(GemmTerm32), cudaMemcpyHostToDevice,
                               F->stream), "apply terms");
  if (!tasks.empty())
    cuda_check(cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(GemmTask32), cudaMemcpyHostToDevice,
                               F->stream), "apply tasks");
  cuda_check(cudaStreamSynchronize(F->stream), "apply program");
  pg.terms32 = dterms;
  pg.tasks32 = dtasks;
}

void build_apply(lrs_factor_t* F, int nrhs) {
  ApplyProgram& pg = F->prog;
  if (pg.nrhs == nrhs) return;
  cuda_check(cudaStreamSynchronize(F->stream), "apply rebuild");
  if (pg.graph) {
    cudaGraphExecDestroy(pg.graph);
    pg.graph = nullptr;
  }
  F->workspace.reset();
  const int64_t ext = F->ext_n;
  pg.nrhs = nrhs;
  std::vector<GemmTask>& tasks = F->prog_tasks;
  std::vector<GemmTerm>& terms = F->prog_terms;
  tasks.clear();
  terms.clear();
  pg.fd0.clear(); pg.fdn.clear(); pg.fu0.clear(); pg.fun.clear(); pg.bw0.clear(); pg.bwn.clear();
  pg.fd_flops.clear(); pg.fu_flops.clear(); pg.bw_flops.clear();
  pg.fd_bytes.clear(); pg.fu_bytes.clear(); pg.bw_bytes.clear();
  pg.fds.clear(); pg.fus.clear(); pg.bws.clear();
  if (F->apply32) {
    build_apply32(F, nrhs);
    return;
  }
  pg.y = F->workspace.take((size_t)ext * nrhs);
  pg.f = F->workspace.take((size_t)ext * nrhs);
  pg.x = F->workspace.take((size_t)ext * nrhs);
  // contraction split of a launch of tasks [t0, end): phases with few tiles
  // but long contractions (the top of the tree) spread each tile over
  // several CTAs, so that about 4 CTAs per SM have work
  size_t part_tiles = 0;
  auto split_of = [&](int t0) -> int {
    const int nt = (int)tasks.size() - t0;
    if (nrhs > 16 || nt <= 0 || nt >= kSplitTarget / 2) return 1;
    int chunks = 0;
    for (int i = t0; i < (int)tasks.size(); ++i) {
      int c = 0;
      for (int q = 0; q < tasks[i].nterm; ++q) c += (terms[tasks[i].term0 + q].k + kTileK - 1) / kTileK;
      chunks = std::max(chunks, c);
    }
    const int S = std::max(1, std::min({(kSplitTarget + nt - 1) / nt, chunks / 4, 32}));
    if (S > 1) part_tiles = std::max(part_tiles, (size_t)S * nt);
    return S;
  };
  double cur_flops = 0.0, cur_bytes = 0.0;
  auto add = [&](double* C, const double* D, int rows, int mode, const std::vector<GemmTerm>& tm) {
    if (rows <= 0) return;
    for (const GemmTerm& t : tm) {
      cur_flops += 2.0 * rows * nrhs * t.k;
      cur_bytes += 8.0 * ((double)rows * t.k + (double)t.k * nrhs);   // block + input vector
    }
    cur_bytes += 8.0 * rows * nrhs * ((D || (mode & kAccumulate)) ? 2 : 1);
    const int t0 = (int)terms.size();
    terms.insert(terms.end(), tm.begin(), tm.end());
    for (int tj = 0; tj * kTile < nrhs; ++tj)
      for (int ti = 0; ti * kTile < rows; ++ti)
        tasks.push_back(GemmTask{C, D, (int)ext, (int)ext, rows, nrhs, ti, tj, t0, (int)tm.size(), mode});
  };
  int64_t bytes = 0;
  for (auto [r0, cnt] : F->phases) {
    // forward: diagonal solves
    pg.fd0.push_back((int)tasks.size());
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      add(pg.f + op, nullptr, rec.m, 0, {GemmTerm{rec.inv, pg.y + op, rec.m, (int)ext, rec.m, 0}});
      bytes += (int64_t)rec.m * rec.m * 8;
    }
    pg.fdn.push_back((int)tasks.size() - pg.fd0.back());
    pg.fds.push_back(split_of(pg.fd0.back()));
    pg.fd_flops.push_back(cur_flops); pg.fd_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
    // forward: updates of later nodes, gathered per target
    pg.fu0.push_back((int)tasks.size());
    std::map<int64_t, std::pair<int, std::vector<GemmTerm>>> upd;
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      for (size_t v = 0; v < rec.nbr.size(); ++v) {
        const int mq = rec.nbr_m[v];
        if (mq == 0) continue;
        const int64_t oq = F->node_offset(rec.level, rec.nbr[v]);
        auto& e = upd[oq];
        e.first = mq;
        e.second.push_back(GemmTerm{rec.L[v], pg.f + op, mq, (int)ext, rec.m, 0});
        bytes += (int64_t)rec.m * mq * 8;
      }
    }
    for (auto& kv : upd) add(pg.y + kv.first, nullptr, kv.second.first, kAccumulate | kSubtract, kv.second.second);
    pg.fun.push_back((int)tasks.size() - pg.fu0.back());
    pg.fus.push_back(split_of(pg.fu0.back()));
    pg.fu_flops.push_back(cur_flops); pg.fu_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
    // backward
    pg.bw0.push_back((int)tasks.size());
    for (int r = r0; r < r0 + cnt; ++r) {
      const ElimRecord& rec = F->recs[r];
      if (rec.m == 0) continue;
      const int64_t op = F->node_offset(rec.level, rec.node);
      std::vector<GemmTerm> tm;
      for (size_t v = 0; v < rec.nbr.size(); ++v) {
        const int mq = rec.nbr_m[v];
        if (mq == 0) continue;
        const int64_t oq = F->node_offset(rec.level, rec.nbr[v]);
        tm.push_back(GemmTerm{rec.T[v], pg.x + oq, rec.m, (int)ext, mq, 0});
        bytes += (int64_t)rec.m * mq * 8;
      }
      if (tm.empty()) add(pg.x + op, pg.f + op, rec.m, 0, {GemmTerm{nullptr, nullptr, 1, 1, 0, 0}});
      else add(pg.x + op, pg.f + op, rec.m, kSubtract, tm);
    }
    pg.bwn.push_back((int)tasks.size() - pg.bw0.back());
    pg.bws.push_back(split_of(pg.bw0.back()));
    pg.bw_flops.push_back(cur_flops); pg.bw_bytes.push_back(cur_bytes); cur_flops = cur_bytes = 0.0;
  }
  F->stats.apply_bytes = bytes;
  pg.part = part_tiles ? F->workspace.take(part_tiles * kTile * 16) : nullptr;
  GemmTerm* dterms = reinterpret_cast<GemmTerm*>(F->workspace.take((terms.size() * sizeof(GemmTerm) + 7) / 8 + 1));
  GemmTask* dtasks = reinterpret_cast<GemmTask*>(F->workspace.take((tasks.size() * sizeof(GemmTask) + 7) / 8 + 1));
  if (!terms.empty())
    cuda_check(cudaMemcpyAsync(dterms, terms.data(), terms.size() * sizeof(GemmTerm), cudaMemcpyHostToDevice, F->stream), "apply terms");
  if (!tasks.empty())
    cuda_check(cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, F->stream), "apply tasks");
  cuda_check(cudaStreamSynchronize(F->stream), "apply program");
  pg.terms = dterms;
  pg.tasks = dtasks;
}

// x = M b for device column-major n x nrhs arrays (b, x may not alias).
void run_apply_device(lrs_factor_t* F, const double* b, double* x, int nrhs) {
  build_apply(F, nrhs);
  ApplyProgram& pg = F->prog;
  const lrs_plan& P = *F->plan;
  const int64_t ext = F->ext_n;
  cudaStream_t st = F->stream;
  Profiler& pf = F->prof;
  const bool f32 = F->apply32;
  if (f32) cuda_check(cudaMemsetAsync(pg.y32, 0, (size_t)ext * nrhs * sizeof(float), st), "apply zero");
  else cuda_check(cudaMemsetAsync(pg.y, 0, (size_t)ext * nrhs * sizeof(double), st), "apply zero");
  const double vbytes = 8.0 * P.n * nrhs;
  cudaEvent_t e = pf.start();
  if (f32) launch_permute_in32(b, P.n, nrhs, F->d_perm, pg.y32, ext, st);
  else launch_permute_in(b, P.n, nrhs, F->d_perm, pg.y, ext, st);
  pf.stop(LRS_PROF_VECTOR, e, 0.0, 2 * vbytes + 4.0 * P.n);
  // the traversal: one launch per phase and step, captured once into a CUDA
  // graph on the side stream (the caller's stream may be the legacy default
  // stream, which cannot capture) and replayed on the factor's stream.  The
  // FP32 traversal's launches are programmatic dependent launches (10% faster
  // applications measured); the FP64 one's are not (its FP64-pipe-bound
  // 16-column kernels measured 28% slower with them)
  if (!pg.graph) {
    cudaStream_t cs = F->side;
    const size_t nph = F->phases.size();
    int kernels = 0;
    double flops = 0.0, bytes = 0.0;
    auto gemm = [&](int t0, int n, int split) {
      kernels += split > 1 ? 2 : 1;
      if (f32) {
        if (nrhs == 1) launch_gemv32(pg.tasks32 + t0, n, pg.terms32, cs, split, pg.part32, true);
        else launch_gemm_narrow32(pg.tasks32 + t0, n, pg.terms32, cs, split, pg.part32, true);
      } else if (nrhs == 1) {
        launch_gemv(pg.tasks + t0, n, pg.terms, cs, split, pg.part);
      } else if (nrhs <= 16) {
        launch_gemm_narrow(pg.tasks + t0, n, pg.terms, cs, split, pg.part);
      } else {
        kernels -= split > 1 ? 1 : 0;
        launch_gemm(pg.tasks + t0, n, pg.terms, cs);
      }
    };
    cudaGraph_t g = nullptr;
    cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "apply capture");
    for (size_t k = 0; k < nph; ++k) {
      if (pg.fdn[k]) { gemm(pg.fd0[k], pg.fdn[k], pg.fds[k]); flops += pg.fd_flops[k]; bytes += pg.fd_bytes[k]; }
      if (pg.fun[k]) { gemm(pg.fu0[k], pg.fun[k], pg.fus[k]); flops += pg.fu_flops[k]; bytes += pg.fu_bytes[k]; }
    }
    for (size_t k = nph; k-- > 0;) {
      if (!pg.bwn[k]) continue;
      gemm(pg.bw0[k], pg.bwn[k], pg.bws[k]);
      flops += pg.bw_flops[k];
      bytes += pg.bw_bytes[k];
    }
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cuda_check(ce, "apply capture");
    const cudaError_t ie = cudaGraphInstantiate(&pg.graph, g, 0);
    cudaGraphDestroy(g);
    cuda_check(ie, "apply graph");
    pg.graph_kernels = kernels;
    pg.graph_flops = flops;
    pg.graph_bytes = bytes;
  }
  e = pf.start();
  cuda_check(cudaGraphLaunch(pg.graph, st), "apply graph launch");
  pf.stop(LRS_PROF_APPLY_GEMM, e, pg.graph_flops, pg.graph_bytes, 0, 0, 0, nullptr, pg.graph_kernels);
  e = pf.start();
  if (f32) launch_permute_out32(pg.x32, ext, P.n, nrhs, F->d_perm, x, st);
  else launch_permute_out(pg.x, ext, P.n, nrhs, F->d_perm, x, st);
  pf.stop(LRS_PROF_VECTOR, e, 0.0, 2 * vbytes + 4.0 * P.n);
  cuda_check(cudaGetLastError(), "apply launch");
}

// Restarted GMRES(restart) on A x = b preconditioned by the factor, x0 = 0,
// modified Gram-Schmidt Arnoldi and Givens rotations per group (the right
// form flexible: z_k = M v_k kept, x += Z y); all groups
// advance in lock step and a group stops once its own residual estimate
// reaches tol (then the residual is recomputed at the end of the cycle, as in
// Saad & Schultz's algorithm).  Right preconditioning (A M y = b, x = M y)
// iterates on the true residual b - A x (eq. accres); left preconditioning,
// the form of Sec. 5.2, iterates on M (b - A x) and stops on eq.
// GMRES_residual.  A group is one column, or on a batched plan one (column,
// instance) pair: the preconditioner and A are block diagonal over the
// instances, so each instance's rows of a column carry a Krylov process of
// their own, and only the inner products and the coefficients are per group.
void run_gmres_device(lrs_factor_t* F, const double* b, double* x, int nrhs, const lrs_solve_opts& o,
                      lrs_solve_info* info) {
  const lrs_plan& P = *F->plan;
  const int64_t n = P.n;
  const int kr = o.restart;
  const Segments& sg = F->segs;
  const int G = nrhs * sg.nseg;                     // groups
  cudaStream_t st = F->stream;
  build_apply(F, nrhs);
  Arena& ws = F->scratch;
  ws.reset();
  Profiler& pf = F->prof;
  const double vb = 8.0 * n * nrhs;                 // bytes of one multi-vector
  auto timed = [&](int cls, double flops, double bytes, auto&& launch) {
    cudaEvent_t e = pf.start();
    launch();
    pf.stop(cls, e, flops, bytes);
  };
  const double spmv_flops = 2.0 * P.nnz * nrhs;
  const double spmv_bytes = 12.0 * P.nnz + 8.0 * (P.n + 1) + 2 * vb;
  const size_t nn = (size_t)n * nrhs;
  double* V = ws.take(nn * (kr + 1));
  // right preconditioning is flexible (Saad 1993): z_k = M v_k is kept and the
  // update is x += Z y, so a traversal in FP32 arithmetic (the precision
  // form's FP32 storage), whose rounding makes M slightly input-dependent,
  // still gives GMRES's minimal residual over span(Z); for an exact M this is
  // right-preconditioned GMRES, one application of M per cycle cheaper
  const bool left = o.side == LRS_GMRES_LEFT;
  double* Z = left ? nullptr : ws.take(nn * kr);
  double* w = ws.take(nn);
  double* z = ws.take(nn);
  double* r = ws.take(nn);
  double* h = ws.take((size_t)(kr + 2) * G);
  double* partial = ws.take(dot_partials(sg.nseg) * nrhs);
  double* dcoef = ws.take((size_t)(kr + 1) * G);
  int* dmask = reinterpret_cast<int*>(ws.take(G));
  std::vector<double> hh((size_t)(kr + 2) * G), coef((size_t)(kr + 1) * G), nrm(G), bnorm(G);
  std::vector<int> mask(G), iters(G, 0), active(G, 0), conv(G, 0);
  std::vector<double> relres(G, 1.0);
  auto col_norms = [&](const double* v, std::vector<double>& out) {
    timed(LRS_PROF_VECTOR, 2.0 * n * nrhs, vb, [&] { launch_dot(v, v, n, nrhs, sg, partial, h, st); });
    cuda_check(cudaMemcpyAsync(hh.data(), h, G * sizeof(double), cudaMemcpyDeviceToHost, st), "norms");
    cuda_check(cudaStreamSynchronize(st), "norms");
    for (int c = 0; c < G; ++c) out[c] = std::sqrt(hh[c]);
  };
  col_norms(b, bnorm);
  cuda_check(cudaMemsetAsync(x, 0, nn * sizeof(double), st), "x0");
  // the residual GMRES works on: b - A x0 = b (right), M b (left)
  std::vector<double> ref = bnorm;                  // its norm at x0: the denominator of relres
  if (left) {
    run_apply_device(F, b, r, nrhs);
    col_norms(r, ref);
  } else {
    cuda_check(cudaMemcpyAsync(r, b, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "r0");
  }
  std::vector<double> beta = ref;
  for (int c = 0; c < G; ++c) {
    active[c] = ref[c] > 0.0;
    if (!active[c]) { relres[c] = 0.0; conv[c] = 1; }
  }
  const int ld = kr + 1;
  while (true) {
    bool any = false;
    for (int c = 0; c < G; ++c) any |= active[c] && iters[c] < o.maxit;
    if (!any) break;
    // V_0 = r / beta on the groups still running
    for (int c = 0; c < G; ++c) {
      mask[c] = active[c] && iters[c] < o.maxit;
      nrm[c] = beta[c] * beta[c];
    }
    cuda_check(cudaMemcpyAsync(dmask, mask.data(), G * sizeof(int), cudaMemcpyHostToDevice, st), "mask");
    cuda_check(cudaMemcpyAsync(h, nrm.data(), G * sizeof(double), cudaMemcpyHostToDevice, st), "beta");
    timed(LRS_PROF_VECTOR, n * nrhs, 2 * vb, [&] { launch_scale_col(h, dmask, r, V, n, nrhs, sg, st); });
    std::vector<std::vector<double>> H(G, std::vector<double>((size_t)ld * kr, 0.0));
    std::vector<std::vector<double>> cs(G), sn(G), g(G);
    std::vector<int> kc(G, 0), running(mask);
    for (int c = 0; c < G; ++c) g[c].assign(kr + 1, 0.0), g[c][0] = beta[c];
    for (int k = 0; k < kr; ++k) {
      bool go = false;
      for (int c = 0; c < G; ++c) go |= running[c];
      if (!go) break;
      if (left) {                                   // w = M A v_k
        timed(LRS_PROF_SPMV, spmv_flops, spmv_bytes,
              [&] { launch_spmv(n, F->d_rowptr, F->d_colind, F->d_val, V + (size_t)k * nn, z, nrhs, st); });
        run_apply_device(F, z, w, nrhs);
      } else {                                      // z_k = M v_k, w = A z_k
        double* zk = Z + (size_t)k * nn;
        run_apply_device(F, V + (size_t)k * nn, zk, nrhs);
        timed(LRS_PROF_SPMV, spmv_flops, spmv_bytes,
              [&] { launch_spmv(n, F->d_rowptr, F->d_colind, F->d_val, zk, w, nrhs, st); });
      }
      for (int j = 0; j <= k; ++j) {
        timed(LRS_PROF_VECTOR, 2.0 * n * nrhs, 2 * vb,
              [&] { launch_dot(w, V + (size_t)j * nn, n, nrhs, sg, partial, h + (size_t)j * G, st); });
        timed(LRS_PROF_VECTOR, 2.0 * n * nrhs, 3 * vb,
              [&] { launch_axpy_col(h + (size_t)j * G, -1.0, V + (size_t)j * nn, w, n, nrhs, sg, st); });
      }
      timed(LRS_PROF_VECTOR, 2.0 * n * nrhs, vb,
            [&] { launch_dot(w, w, n, nrhs, sg, partial, h + (size_t)(k + 1) * G, st); });
      timed(LRS_PROF_VECTOR, n * nrhs, 2 * vb,
            [&] { launch_scale_col(h + (size_t)(k + 1) * G, dmask, w, V + (size_t)(k + 1) * nn, n, nrhs, sg, st); });
      cuda_check(cudaMemcpyAsync(hh.data(), h, (size_t)(k + 2) * G * sizeof(double), cudaMemcpyDeviceToHost, st),
                 "hessenberg");
      cuda_check(cudaStreamSynchronize(st), "arnoldi");
      bool mask_changed = false;
      for (int c = 0; c < G; ++c) {
        if (!running[c]) continue;
        double* col = &H[c][(size_t)k * ld];
        for (int j = 0; j <= k; ++j) col[j] = hh[(size_t)j * G + c];
        col[k + 1] = std::sqrt(std::max(hh[(size_t)(k + 1) * G + c], 0.0));
        const bool breakdown = col[k + 1] == 0.0;
        for (int j = 0; j < k; ++j) {
          const double t0 = cs[c][j] * col[j] + sn[c][j] * col[j + 1];
          col[j + 1] = -sn[c][j] * col[j] + cs[c][j] * col[j + 1];
          col[j] = t0;
        }
        const double den = std::hypot(col[k], col[k + 1]);
        const double cc = den == 0.0 ? 1.0 : col[k] / den, ss = den == 0.0 ? 0.0 : col[k + 1] / den;
        cs[c].push_back(cc);
        sn[c].push_back(ss);
        col[k] = cc * col[k] + ss * col[k + 1];
        col[k + 1] = 0.0;
        g[c][k + 1] = -ss * g[c][k];
        g[c][k] = cc * g[c][k];
        ++iters[c];
        kc[c] = k + 1;
        relres[c] = std::fabs(g[c][k + 1]) / ref[c];
        if (relres[c] <= o.tol || den == 0.0 || breakdown || iters[c] >= o.maxit) {
          running[c] = 0;
          mask_changed = true;
        }
      }
      if (mask_changed) {
        for (int c = 0; c < G; ++c) mask[c] = running[c];
        cuda_check(cudaMemcpyAsync(dmask, mask.data(), G * sizeof(int), cudaMemcpyHostToDevice, st), "mask");
      }
    }
    // x += Z y (right) or V y (left), y = H \ g per group
    std::fill(coef.begin(), coef.end(), 0.0);
    for (int c = 0; c < G; ++c) {
      const int kk = kc[c];
      std::vector<double> y(kk, 0.0);
      for (int i = kk - 1; i >= 0; --i) {
        double s = g[c][i];
        for (int j = i + 1; j < kk; ++j) s -= H[c][(size_t)j * ld + i] * y[j];
        const double d = H[c][(size_t)i * ld + i];
        y[i] = d != 0.0 ? s / d : 0.0;
      }
      for (int j = 0; j < kk; ++j) coef[(size_t)j * G + c] = y[j];
    }
    cuda_check(cudaMemcpyAsync(dcoef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, st), "coef");
    int kmax = 0;
    for (int c = 0; c < G; ++c) kmax = std::max(kmax, kc[c]);
    timed(LRS_PROF_VECTOR, 2.0 * kmax * n * nrhs, (kmax + 1) * vb,
          [&] { launch_combine(dcoef, kmax, left ? V : Z, (int64_t)nn, w, n, nrhs, sg, st); });
    const double* dx = w;
    std::vector<double> ones(G, 1.0);
    cuda_check(cudaMemcpyAsync(h, ones.data(), G * sizeof(double), cudaMemcpyHostToDevice, st), "ones");
    timed(LRS_PROF_VECTOR, 2.0 * n * nrhs, 3 * vb, [&] { launch_axpy_col(h, 1.0, dx, x, n, nrhs, sg, st); });
    timed(LRS_PROF_SPMV, spmv_flops, spmv_bytes,
          [&] { launch_spmv(n, F->d_rowptr, F->d_colind, F->d_val, x, r, nrhs, st); });
    timed(LRS_PROF_VECTOR, n * nrhs, 3 * vb, [&] { launch_residual(b, r, (int64_t)nn, st); });
    if (left) {                                     // r = M (b - A x)
      run_apply_device(F, r, z, nrhs);
      cuda_check(cudaMemcpyAsync(r, z, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "left residual");
    }
    std::vector<double> rn(G);
    col_norms(r, rn);
    for (int c = 0; c < G; ++c) {
      if (!active[c]) continue;
      beta[c] = rn[c];
      relres[c] = rn[c] / ref[c];
      if (relres[c] <= o.tol) { conv[c] = 1; active[c] = 0; }
      else if (iters[c] >= o.maxit || rn[c] == 0.0) active[c] = 0;
    }
  }
  // the residual the side did not iterate on, when it is reported
  std::vector<double> true_res(G, 0.0), prec_res(G, -1.0);
  if (left) {
    prec_res = relres;
    timed(LRS_PROF_SPMV, spmv_flops, spmv_bytes,
          [&] { launch_spmv(n, F->d_rowptr, F->d_colind, F->d_val, x, r, nrhs, st); });
    timed(LRS_PROF_VECTOR, n * nrhs, 3 * vb, [&] { launch_residual(b, r, (int64_t)nn, st); });
    std::vector<double> rn(G);
    col_norms(r, rn);
    for (int c = 0; c < G; ++c) true_res[c] = bnorm[c] > 0.0 ? rn[c] / bnorm[c] : 0.0;
  } else {
    true_res = relres;
    if (o.precond_residual) {
      // r holds b - A x of the last cycle (or b when no cycle ran)
      std::vector<double> pn(G), pb(G);
      run_apply_device(F, r, z, nrhs);
      col_norms(z, pn);
      run_apply_device(F, b, z, nrhs);
      col_norms(z, pb);
      for (int c = 0; c < G; ++c) prec_res[c] = pb[c] > 0.0 ? pn[c] / pb[c] : 0.0;
    }
  }
  info->iters = 0;
  info->rel_res = 0.0;
  info->rel_res_precond = (left || o.precond_residual) ? 0.0 : -1.0;
  info->status = LRS_OK;
  for (int c = 0; c < G; ++c) {
    info->iters = std::max(info->iters, iters[c]);
    info->rel_res = std::max(info->rel_res, true_res[c]);
    if (left || o.precond_residual) info->rel_res_precond = std::max(info->rel_res_precond, prec_res[c]);
    if (!conv[c]) info->status = LRS_ERR_NOT_CONVERGED;
  }
  F->last_iters.assign(iters.begin(), iters.end());
}

}  // namespace lrs
