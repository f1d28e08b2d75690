// Batched GMRES over many independent problems (the batched configuration:
// instances with different grids and interfaces solved together).
//
// Every instance advances its GMRES in lockstep.  One iteration of all
// instances is one CUDA graph, captured once and replayed:
//   copy V_j -> x (all instances)        one launch
//   C at irregular nodes, sparse RHS     two launches over all instances
//   mixed box solves                     persistent launches over all
//                                        instances' line pairs per pass
//   traces + BIE combination             one launch over all DOFs
//   copy y -> V_{j+1}, Arnoldi step      two launches (a CTA per instance)
// Iteration counters j live on the device, so the same graph serves every
// iteration; instances that have converged keep their state (their Arnoldi
// step is skipped).  The host reads the residual estimates of all instances
// (one small copy) once per iteration.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kfbi_internal.cuh"


struct kfbi_batch {
  std::vector<kfbi_problem*> ps;
  int n = 0, m = 0, maxnb = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  kfbi::BatchBox* bb = nullptr;
  kfbi::BatchHot* bh = nullptr;
  std::vector<double*> rhs_loop;
  kfbi::ArnDesc* darn = nullptr;
  int* jdev = nullptr;
  int* done = nullptr;
  double* res_dev = nullptr;
  double* res_host = nullptr;   // pinned
  int* done_host = nullptr;     // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long counts[KFBI_KC_COUNT] = {};
};

using namespace kfbi;

static kfbi_status batch_iteration(kfbi_batch* b, cudaStream_t st) {
  kfbi_problem* p0 = b->ps[0];
  KFBI_TRY(batch_arnoldi_copy_in(p0, b->darn, b->jdev, b->done, b->n, b->maxnb, st));
  KFBI_TRY(batch_hot_cvals_rhs(p0, b->bh, st));
  KFBI_TRY(batch_box_solve(p0, b->bb, b->done, st));
  KFBI_TRY(batch_hot_trace(p0, b->bh, st));
  return batch_arnoldi_step(p0, b->darn, b->jdev, b->done, b->res_dev, b->n, b->maxnb, b->m, st);
}

extern "C" {

kfbi_status kfbi_destroy_batch(kfbi_batch* b) {
  if (!b) return KFBI_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  batch_box_destroy(b->bb);
  batch_hot_destroy(b->bh);
  for (double* r : b->rhs_loop) cudaFree(r);
  cudaFree(b->darn);
  cudaFree(b->jdev);
  cudaFree(b->done);
  cudaFree(b->res_dev);
  if (b->res_host) cudaFreeHost(b->res_host);
  if (b->done_host) cudaFreeHost(b->done_host);
  delete b;
  return KFBI_OK;
}

kfbi_status kfbi_batch_tiles(const kfbi_batch* b, int* pass_ctas, int* row_ctas) {
  if (!b || !pass_ctas || !row_ctas) return KFBI_ERR_ARG;
  batch_box_tiles(b->bb, pass_ctas, row_ctas);
  return KFBI_OK;
}

kfbi_status kfbi_create_batch(kfbi_problem* const* problems, int count, kfbi_batch** out) {
  if (!out || !problems || count < 1) return KFBI_ERR_ARG;
  *out = nullptr;
  for (int k = 0; k < count; ++k)
    if (!problems[k]) return KFBI_ERR_ARG;
  kfbi_problem* p0 = problems[0];
  kfbi_batch* b = new kfbi_batch();
  b->ps.assign(problems, problems + count);
  b->n = count;
  b->stream = p0->stream;
  b->m = p0->gm.m;
  auto bail = [&](kfbi_status s) {
    kfbi_destroy_batch(b);
    return s;
  };
  for (kfbi_problem* p : b->ps) {
    if (p->stream != b->stream || p->g.d != p0->g.d || p->cfg.precision != KFBI_MIXED ||
        (p->cfg.kind != KFBI_DIRICHLET_INTERIOR && p->cfg.kind != KFBI_INTERFACE_MU) ||
        p->cfg.box_solver != KFBI_BOX_DST || p->gm.m != b->m || p->nb > 32768)
      return bail(fail(p0, KFBI_ERR_UNSUPPORTED,
                       "a batch needs Dirichlet or interface problems on one stream, of one dimension, "
                       "with mixed-precision DST box solves and N_b <= 32768"));
    b->maxnb = std::max(b->maxnb, p->nb);
  }
  std::vector<double*> xs, ys;
  for (kfbi_problem* p : b->ps) {
    double* r = nullptr;
    if (dalloc(&r, p->g.nodes()) != cudaSuccess)
      return bail(fail(p0, KFBI_ERR_CUDA, "out of device memory"));
    b->rhs_loop.push_back(r);
    // zero once: inside GMRES only the irregular entries are ever written
    if (cudaMemset(r, 0, sizeof(double) * p->g.nodes()) != cudaSuccess)
      return bail(fail(p0, KFBI_ERR_CUDA, "memset failed"));
    xs.push_back(p->xbuf);
    ys.push_back(p->ybuf);
  }
  kfbi_status s;
  if ((s = batch_hot_create(p0, b->ps.data(), count, xs.data(), ys.data(), b->rhs_loop.data(), &b->bh)) != KFBI_OK)
    return bail(s);
  if ((s = batch_box_create(p0, b->ps.data(), count, b->rhs_loop.data(), &b->bb)) != KFBI_OK) return bail(s);
  std::vector<ArnDesc> ad(count);
  for (int k = 0; k < count; ++k) {
    kfbi_problem* p = b->ps[k];
    Gmres& G = p->gm;
    ad[k] = ArnDesc{G.V, G.nb, G.m, G.H, G.m + 1, G.cs, G.sn, G.g, G.scal + 2, p->xbuf, p->ybuf};
  }
  if (dalloc(&b->darn, count) != cudaSuccess || dalloc(&b->jdev, count) != cudaSuccess ||
      dalloc(&b->done, count) != cudaSuccess || dalloc(&b->res_dev, count) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->res_host), sizeof(double) * count) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->done_host), sizeof(int) * count) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "out of memory"));
  if (cudaMemcpy(b->darn, ad.data(), sizeof(ArnDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "descriptor upload failed"));
  // pick the box solve's launch shapes for this batch (before the capture,
  // which records them), every instance active
  if (cudaMemset(b->done, 0, sizeof(int) * count) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "memset failed"));
  {
    // the tuning solves are set-up work: no per-launch timing events for them
    const bool prof_on = p0->prof.on;
    p0->prof.on = false;
    s = batch_box_autotune(p0, b->bb, b->ps.data(), b->rhs_loop.data(), b->done, b->stream);
    p0->prof.on = prof_on;
    if (s != KFBI_OK) return bail(s);
  }
  // capture one iteration of all instances
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "stream creation failed"));
  long long before[KFBI_KC_COUNT];
  for (int c = 0; c < KFBI_KC_COUNT; ++c) before[c] = p0->prof.launches[c];
  const bool prof = p0->prof.on;
  p0->prof.on = false;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "capture failed"));
  s = batch_iteration(b, b->cap);
  cudaError_t e = cudaStreamEndCapture(b->cap, &b->graph);
  p0->prof.on = prof;
  for (int c = 0; c < KFBI_KC_COUNT; ++c) {
    b->counts[c] = p0->prof.launches[c] - before[c];
    p0->prof.launches[c] = before[c];
  }
  if (s != KFBI_OK || e != cudaSuccess) return bail(s != KFBI_OK ? s : fail(p0, KFBI_ERR_CUDA, "capture failed"));
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "graph instantiation failed"));
  *out = b;
  return KFBI_OK;
}

kfbi_status kfbi_gmres_solve_batch(kfbi_batch* b, const kfbi_data* data, const kfbi_gmres_opts* opts,
                                   double* const* densities, kfbi_gmres_info* infos) {
  if (!b || !data || !opts || !densities) return KFBI_ERR_ARG;
  kfbi_problem* p0 = b->ps[0];
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->x0)
    return fail(p0, KFBI_ERR_ARG, "batched GMRES needs rtol > 0, max_iter >= 1 and a zero start");
  const int n = b->n;
  cudaStream_t st = b->stream;
  // Step 1 of Algorithm 1 for every instance, then the norms of the right-hand sides
  for (int k = 0; k < n; ++k) {
    kfbi_problem* p = b->ps[k];
    if (!data[k].g1 || (p->cfg.kind == KFBI_INTERFACE_MU && !data[k].g2))
      return fail(p0, KFBI_ERR_ARG, "missing boundary data for instance " + std::to_string(k));
    KFBI_TRY(bie_rhs_impl(p, &data[k], p->bvec));
    KFBI_TRY(dot_self_pub(p, p->bvec, b->res_dev + k));
  }
  KFBI_CUDA(p0, cudaMemcpyAsync(b->res_host, b->res_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaStreamSynchronize(st));
  std::vector<double> bnorm(n);
  std::vector<int> iters(n, 0);
  for (int k = 0; k < n; ++k) {
    bnorm[k] = std::sqrt(b->res_host[k]);
    if (!std::isfinite(bnorm[k])) return fail(p0, KFBI_ERR_NONFINITE, "non-finite BIE right-hand side");
    b->done_host[k] = bnorm[k] == 0.0 ? 1 : 0;
    if (!b->done_host[k]) KFBI_TRY(gmres_init_zero(b->ps[k], b->ps[k]->bvec, bnorm[k]));
  }
  KFBI_CUDA(p0, cudaMemsetAsync(b->jdev, 0, sizeof(int) * n, st));
  KFBI_CUDA(p0, cudaMemcpyAsync(b->done, b->done_host, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  const int maxit = std::min(std::min(opts->max_iter, b->m), opts->restart > 0 ? opts->restart : b->m);
  int it = 0;
  int active = 0;
  for (int k = 0; k < n; ++k) active += !b->done_host[k];
  while (active > 0 && it < maxit) {
    KFBI_CUDA(p0, cudaGraphLaunch(b->exec, st));
    for (int c = 0; c < KFBI_KC_COUNT; ++c) p0->prof.launches[c] += b->counts[c];
    ++it;
    KFBI_CUDA(p0, cudaMemcpyAsync(b->res_host, b->res_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(p0, cudaStreamSynchronize(st));
    bool changed = false;
    for (int k = 0; k < n; ++k) {
      if (b->done_host[k]) continue;
      iters[k] = it;
      if (!std::isfinite(b->res_host[k]))
        return fail(p0, KFBI_ERR_NONFINITE, "non-finite residual in instance " + std::to_string(k));
      if (b->res_host[k] <= opts->rtol * bnorm[k]) {
        b->done_host[k] = 1;
        changed = true;
        --active;
      }
    }
    if (changed)
      KFBI_CUDA(p0, cudaMemcpyAsync(b->done, b->done_host, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  }
  kfbi_status status = KFBI_OK;
  for (int k = 0; k < n; ++k) {
    KFBI_TRY(gmres_finish(b->ps[k], iters[k], densities[k]));
    const double rel = bnorm[k] > 0 ? b->res_host[k] / bnorm[k] : 0.0;
    if (infos) {
      infos[k].iters = iters[k];
      infos[k].rel_res = bnorm[k] > 0 ? rel : 0.0;
      for (double& v : infos[k].t_ms) v = 0.0;
      infos[k].x0_rejected = 0;
    }
    if (bnorm[k] > 0 && !(rel <= opts->rtol)) status = KFBI_ERR_NOT_CONVERGED;
  }
  KFBI_CUDA(p0, cudaStreamSynchronize(st));
  if (status != KFBI_OK) fail(p0, status, "some instances did not converge within max_iter");
  return status;
}

}  // extern "C"
