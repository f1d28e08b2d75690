// Batched GMRES over many independent problems (the batched configuration:
// instances with different grids and interfaces solved together).
//
// Every instance advances its GMRES in lockstep.  One iteration of all
// instances is one CUDA graph body:
//   copy V_j -> x (all instances)        one launch
//   C at irregular nodes, sparse RHS     two launches over all instances
//   mixed box solves                     persistent launches over all
//                                        instances' line pairs per pass
//   traces + BIE combination             one launch over all DOFs
//   copy y -> V_{j+1}, Arnoldi step      two launches (a CTA per instance)
//   convergence control                  one launch
// Iteration counters, thresholds and done flags live on the device, and the
// body sits inside a conditional WHILE node that the control kernel ends when
// every instance has converged or the iteration limit is reached: the whole
// Arnoldi cycle of all instances is one graph launch and one host
// synchronisation.  (If the driver refuses conditional nodes the body is
// replayed from the host, one short read of the active count per iteration.)
//
// Around the loop, the BIE right-hand sides (Algorithm 1, Step 1) and the
// final evaluations are batched the same way: each instance's corrected
// right-hand side with its data, then one batched box solve of all instances.
// Starts x0 are applied by one batched operator application and one kernel
// that takes or rejects each start with the rule of the single solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kfbi_internal.cuh"


struct kfbi_batch {
  std::vector<kfbi_problem*> ps;
  int n = 0, m = 0, maxnb = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  kfbi::BatchBox* bb = nullptr;        // box solves of the GMRES loop (sparse RHS buffers)
  kfbi::BatchBox* bb_data = nullptr;   // box solves with data (each problem's RHS buffer)
  kfbi::BatchHot* bh = nullptr;
  std::vector<double*> rhs_loop;
  kfbi::ArnDesc* darn = nullptr;
  kfbi::BatchInst* dinst = nullptr;
  kfbi::BatchInst* hinst = nullptr;    // pinned staging of the per-call pointers
  int* jdev = nullptr;
  int* done = nullptr;
  int* zeros = nullptr;                // all instances active
  int* x0_skip = nullptr;              // 1 where an instance has no start
  int* flags = nullptr;                // 0 zero start, 1 x0 taken, 2 x0 rejected
  int* ctl = nullptr;                  // [iterations, limit, active]
  double* thr = nullptr;
  double* bn = nullptr;
  double omega = 0.0;                  // inexact GMRES (the first problem's relax)
  double* tol = nullptr;               // per-instance refinement tolerance of the loop's box solves
  double* tol_base = nullptr;          // each problem's box_rtol
  double* res_dev = nullptr;
  double* res_host = nullptr;   // pinned
  int* int_host = nullptr;      // pinned: jdev, flags, done, ctl
  cudaGraph_t graph = nullptr;  // one iteration (host-driven fallback)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t loop_graph = nullptr;   // the device-driven cycle
  cudaGraphExec_t loop_exec = nullptr;
  long long counts[KFBI_KC_COUNT] = {};
};

using namespace kfbi;

static kfbi_status batch_iteration(kfbi_batch* b, cudaStream_t st, cudaGraphConditionalHandle cond, int use_cond) {
  kfbi_problem* p0 = b->ps[0];
  KFBI_TRY(batch_arnoldi_copy_in(p0, b->darn, b->jdev, b->done, b->n, b->maxnb, st));
  KFBI_TRY(batch_hot_cvals_rhs(p0, b->bh, st));
  KFBI_TRY(batch_box_solve(p0, b->bb, b->done, st));
  KFBI_TRY(batch_hot_trace(p0, b->bh, st));
  KFBI_TRY(batch_arnoldi_step(p0, b->darn, b->jdev, b->done, b->res_dev, b->n, b->maxnb, b->m, st));
  return batch_gmres_control(p0, b->res_dev, b->thr, b->done, b->n, b->ctl, cond, use_cond, b->omega,
                             b->tol_base, b->tol, st);
}

// Capture one iteration into `into` (the body of the conditional node) or
// into a new graph (*out).
static kfbi_status capture_iteration(kfbi_batch* b, cudaGraph_t into, cudaGraph_t* out,
                                     cudaGraphConditionalHandle cond, int use_cond) {
  kfbi_problem* p0 = b->ps[0];
  long long before[KFBI_KC_COUNT];
  for (int c = 0; c < KFBI_KC_COUNT; ++c) before[c] = p0->prof.launches[c];
  const bool prof = p0->prof.on;
  p0->prof.on = false;
  cudaError_t e = into ? cudaStreamBeginCaptureToGraph(b->cap, into, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal)
                       : cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  kfbi_status s = KFBI_OK;
  if (e == cudaSuccess) s = batch_iteration(b, b->cap, cond, use_cond);
  cudaGraph_t gr = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(b->cap, &gr) : e;
  p0->prof.on = prof;
  for (int c = 0; c < KFBI_KC_COUNT; ++c) {
    b->counts[c] = p0->prof.launches[c] - before[c];
    p0->prof.launches[c] = before[c];
  }
  if (e != cudaSuccess || e2 != cudaSuccess || s != KFBI_OK) {
    if (gr && !into) cudaGraphDestroy(gr);
    cudaGetLastError();
    return s != KFBI_OK ? s : fail(p0, KFBI_ERR_CUDA, "batched iteration capture failed");
  }
  if (out) *out = gr;
  return KFBI_OK;
}

// The device-driven cycle: a conditional WHILE node around one iteration.
// Returns false if the driver refuses conditional nodes.
static bool build_loop(kfbi_batch* b) {
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) ok = capture_iteration(b, np.conditional.phGraph_out[0], nullptr, h, 1) == KFBI_OK;
  if (ok) ok = cudaGraphInstantiate(&b->loop_exec, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    b->loop_exec = nullptr;
    return false;
  }
  b->loop_graph = g;
  return true;
}

// Potentials with data of every instance: per instance the correction values
// (a, b, f~ from data[k]) and the corrected right-hand side into the
// problem's RHS buffer, then one batched box solve into each problem's grid,
// then its boundary layer (the outer data g_b when use_gb).
static kfbi_status batch_potentials(kfbi_batch* b, const double* const* a, const double* const* bb,
                                    const kfbi_data* data, bool use_gb) {
  kfbi_problem* p0 = b->ps[0];
  for (int k = 0; k < b->n; ++k) {
    kfbi_problem* p = b->ps[k];
    kfbi_data dd = data[k];
    if (!use_gb) dd.g_b = nullptr;
    KFBI_TRY(launch_correction_values_data(p, a ? a[k] : nullptr, bb ? bb[k] : nullptr, &dd, p->cvals));
    KFBI_TRY(launch_rhs(p, p->cvals, &dd, p->rhs));
  }
  KFBI_TRY(batch_box_solve(p0, b->bb_data, b->zeros, b->stream));
  for (int k = 0; k < b->n; ++k)
    KFBI_TRY(launch_set_boundary(b->ps[k], b->ps[k]->ugrid, use_gb ? data[k].g_b : nullptr));
  return KFBI_OK;
}

namespace kfbi {
int batch_size(const kfbi_batch* b) { return b->n; }
kfbi_problem* batch_problem(const kfbi_batch* b, int k) { return b->ps[k]; }
}  // namespace kfbi

static bool has_data(const kfbi_problem* p, const kfbi_data& d) {
  return d.g1 && (p->cfg.kind != KFBI_INTERFACE_MU || d.g2);
}

extern "C" {

kfbi_status kfbi_destroy_batch(kfbi_batch* b) {
  if (!b) return KFBI_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
  if (b->loop_graph) cudaGraphDestroy(b->loop_graph);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  batch_box_destroy(b->bb);
  batch_box_destroy(b->bb_data);
  batch_hot_destroy(b->bh);
  for (double* r : b->rhs_loop) cudaFree(r);
  cudaFree(b->darn);
  cudaFree(b->dinst);
  cudaFree(b->jdev);
  cudaFree(b->done);
  cudaFree(b->zeros);
  cudaFree(b->x0_skip);
  cudaFree(b->flags);
  cudaFree(b->ctl);
  cudaFree(b->thr);
  cudaFree(b->bn);
  cudaFree(b->tol);
  cudaFree(b->tol_base);
  cudaFree(b->res_dev);
  if (b->res_host) cudaFreeHost(b->res_host);
  if (b->int_host) cudaFreeHost(b->int_host);
  if (b->hinst) cudaFreeHost(b->hinst);
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
        p->cfg.kind != p0->cfg.kind ||
        p->cfg.box_solver != KFBI_BOX_DST || p->gm.m != b->m || p->nb > 32768 || p->n_iface != 1)
      return bail(fail(p0, KFBI_ERR_UNSUPPORTED,
                       "a batch needs problems of one kind (Dirichlet or interface), on one stream, of "
                       "one dimension, with one interface, mixed-precision DST box solves and "
                       "N_b <= 32768"));
    b->maxnb = std::max(b->maxnb, p->nb);
  }
  std::vector<double*> xs, ys, rhs_data;
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
    rhs_data.push_back(p->rhs);
  }
  kfbi_status s;
  if ((s = batch_hot_create(p0, b->ps.data(), count, xs.data(), ys.data(), b->rhs_loop.data(), &b->bh)) != KFBI_OK)
    return bail(s);
  // per-instance refinement tolerances of the loop's box solves (each
  // problem's box_rtol, relaxed inside GMRES when relax > 0)
  b->omega = p0->cfg.relax;
  {
    std::vector<double> base(count);
    for (int k = 0; k < count; ++k) base[k] = box_tol(b->ps[k]);
    if (dalloc(&b->tol, count) != cudaSuccess || dalloc(&b->tol_base, count) != cudaSuccess ||
        cudaMemcpy(b->tol, base.data(), sizeof(double) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tol_base, base.data(), sizeof(double) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(p0, KFBI_ERR_CUDA, "out of device memory"));
  }
  if ((s = batch_box_create(p0, b->ps.data(), count, b->rhs_loop.data(), &b->bb, b->tol)) != KFBI_OK)
    return bail(s);
  if ((s = batch_box_create(p0, b->ps.data(), count, rhs_data.data(), &b->bb_data)) != KFBI_OK) return bail(s);
  std::vector<ArnDesc> ad(count);
  for (int k = 0; k < count; ++k) {
    kfbi_problem* p = b->ps[k];
    Gmres& G = p->gm;
    ad[k] = ArnDesc{G.V, G.nb, G.m, G.H, G.m + 1, G.cs, G.sn, G.g, G.scal + 2, p->xbuf, p->ybuf};
  }
  if (dalloc(&b->darn, count) != cudaSuccess || dalloc(&b->dinst, count) != cudaSuccess ||
      dalloc(&b->jdev, count) != cudaSuccess || dalloc(&b->done, count) != cudaSuccess ||
      dalloc(&b->zeros, count) != cudaSuccess || dalloc(&b->x0_skip, count) != cudaSuccess ||
      dalloc(&b->flags, count) != cudaSuccess || dalloc(&b->ctl, 4) != cudaSuccess ||
      dalloc(&b->thr, count) != cudaSuccess || dalloc(&b->bn, count) != cudaSuccess ||
      dalloc(&b->res_dev, count) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->res_host), sizeof(double) * 2 * count) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->int_host), sizeof(int) * (4 * count + 4)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->hinst), sizeof(BatchInst) * count) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "out of memory"));
  if (cudaMemcpy(b->darn, ad.data(), sizeof(ArnDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->zeros, 0, sizeof(int) * count) != cudaSuccess ||
      cudaMemset(b->done, 0, sizeof(int) * count) != cudaSuccess ||
      cudaMemset(b->ctl, 0, sizeof(int) * 4) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "descriptor upload failed"));
  // pick the box solve's launch shapes for this batch (before the capture,
  // which records them), every instance active; the data solves share them
  {
    // the tuning solves are set-up work: no per-launch timing events for them
    const bool prof_on = p0->prof.on;
    p0->prof.on = false;
    s = batch_box_autotune(p0, b->bb, b->ps.data(), b->rhs_loop.data(), b->done, b->stream);
    p0->prof.on = prof_on;
    if (s != KFBI_OK) return bail(s);
    batch_box_copy_tiles(b->bb_data, b->bb);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(p0, KFBI_ERR_CUDA, "stream creation failed"));
  if (!build_loop(b)) {
    // host-driven fallback: one iteration per replay
    if ((s = capture_iteration(b, nullptr, &b->graph, 0, 0)) != KFBI_OK) return bail(s);
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
      return bail(fail(p0, KFBI_ERR_CUDA, "graph instantiation failed"));
  }
  *out = b;
  return KFBI_OK;
}

kfbi_status kfbi_gmres_solve_batch(kfbi_batch* b, const kfbi_data* data, const kfbi_gmres_opts* opts,
                                   const double* const* x0s, double* const* densities,
                                   kfbi_gmres_info* infos) {
  if (!b || !data || !opts || !densities) return KFBI_ERR_ARG;
  kfbi_problem* p0 = b->ps[0];
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->x0)
    return fail(p0, KFBI_ERR_ARG,
                "batched GMRES needs rtol > 0, max_iter >= 1 and opts->x0 NULL (starts go in x0s)");
  const int n = b->n;
  cudaStream_t st = b->stream;
  for (int k = 0; k < n; ++k) {
    if (!has_data(b->ps[k], data[k]))
      return fail(p0, KFBI_ERR_ARG, "missing boundary data for instance " + std::to_string(k));
    if (!densities[k]) return fail(p0, KFBI_ERR_ARG, "missing density for instance " + std::to_string(k));
  }
  // Step 1 of Algorithm 1 for every instance: the potential of the data
  // (one batched box solve), then its traces into b_k
  {
    std::vector<const double*> a(n, nullptr);
    const bool mu = p0->cfg.kind == KFBI_INTERFACE_MU;
    if (mu)
      for (int k = 0; k < n; ++k) a[k] = data[k].g1;
    KFBI_TRY(batch_potentials(b, mu ? a.data() : nullptr, nullptr, data, mu));
    for (int k = 0; k < n; ++k) {
      kfbi_problem* p = b->ps[k];
      if (p->cfg.kind == KFBI_DIRICHLET_INTERIOR)
        KFBI_TRY(launch_operator_trace(p, p->ugrid, p->cvals, data[k].g1, 1.0, -1.0, p->bvec));
      else
        KFBI_TRY(launch_operator_trace(p, p->ugrid, p->cvals, data[k].g2,
                                       1.0 / (p->cfg.sigma_in + p->cfg.sigma_out), p->mu, p->bvec));
    }
  }
  // starts: y = A x0 of every instance that has one (one batched operator
  // application; instances without a start skip the box solve)
  bool any_x0 = false;
  int* skip = b->int_host;
  for (int k = 0; k < n; ++k) {
    const double* x0 = x0s ? x0s[k] : nullptr;
    b->hinst[k] = BatchInst{b->ps[k]->bvec, x0, densities[k]};
    skip[k] = x0 ? 0 : 1;
    any_x0 = any_x0 || x0;
  }
  KFBI_CUDA(p0, cudaMemcpyAsync(b->dinst, b->hinst, sizeof(BatchInst) * n, cudaMemcpyHostToDevice, st));
  // the starts' residuals at the full box-solve accuracy
  KFBI_CUDA(p0, cudaMemcpyAsync(b->tol, b->tol_base, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (any_x0) {
    KFBI_CUDA(p0, cudaMemcpyAsync(b->x0_skip, skip, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < n; ++k)
      if (x0s[k])
        KFBI_CUDA(p0, cudaMemcpyAsync(b->ps[k]->xbuf, x0s[k], sizeof(double) * b->ps[k]->nb,
                                      cudaMemcpyDeviceToDevice, st));
    KFBI_TRY(batch_hot_cvals_rhs(p0, b->bh, st));
    KFBI_TRY(batch_box_solve(p0, b->bb, b->x0_skip, st));
    KFBI_TRY(batch_hot_trace(p0, b->bh, st));
  }
  KFBI_TRY(batch_gmres_init(p0, b->darn, b->dinst, n, opts->rtol, b->thr, b->bn, b->done, b->jdev, b->flags,
                            b->res_dev, b->omega, b->tol_base, b->tol, st));
  const int maxit = std::min(std::min(opts->max_iter, b->m), opts->restart > 0 ? opts->restart : b->m);
  int* hj = b->int_host;
  int* hflags = hj + n;
  int* hdone = hj + 2 * n;
  int* hctl = hj + 3 * n;
  double* hres = b->res_host;
  double* hbn = b->res_host + n;
  KFBI_CUDA(p0, cudaMemcpyAsync(hbn, b->bn, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaMemcpyAsync(hdone, b->done, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaStreamSynchronize(st));
  int active = 0;
  for (int k = 0; k < n; ++k) {
    if (!std::isfinite(hbn[k]))
      return fail(p0, KFBI_ERR_NONFINITE, "non-finite BIE right-hand side in instance " + std::to_string(k));
    active += !hdone[k];
  }
  const int ctl0[4] = {0, maxit, active, 0};
  KFBI_CUDA(p0, cudaMemcpyAsync(b->ctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, st));
  int iterations = 0;
  if (active > 0 && maxit > 0) {
    if (b->loop_exec) {
      KFBI_CUDA(p0, cudaGraphLaunch(b->loop_exec, st));
      KFBI_CUDA(p0, cudaMemcpyAsync(hctl, b->ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
      KFBI_CUDA(p0, cudaStreamSynchronize(st));
      iterations = hctl[0];
    } else {
      while (iterations < maxit) {
        KFBI_CUDA(p0, cudaGraphLaunch(b->exec, st));
        ++iterations;
        KFBI_CUDA(p0, cudaMemcpyAsync(hctl, b->ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
        KFBI_CUDA(p0, cudaStreamSynchronize(st));
        if (hctl[2] == 0) break;
      }
    }
    for (int c = 0; c < KFBI_KC_COUNT; ++c) p0->prof.launches[c] += b->counts[c] * iterations;
  }
  KFBI_TRY(batch_gmres_finish(p0, b->darn, b->dinst, n, b->jdev, b->flags, st));
  KFBI_CUDA(p0, cudaMemcpyAsync(hj, b->jdev, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaMemcpyAsync(hflags, b->flags, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaMemcpyAsync(hres, b->res_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p0, cudaStreamSynchronize(st));
  kfbi_status status = KFBI_OK;
  for (int k = 0; k < n; ++k) {
    if (!std::isfinite(hres[k]))
      return fail(p0, KFBI_ERR_NONFINITE, "non-finite residual in instance " + std::to_string(k));
    const double rel = hbn[k] > 0 ? hres[k] / hbn[k] : 0.0;
    if (infos) {
      infos[k].iters = hj[k];
      infos[k].rel_res = rel;
      for (double& v : infos[k].t_ms) v = 0.0;
      infos[k].x0_rejected = hflags[k] == 2 ? 1 : 0;
      infos[k].refine_steps = 0;
    }
    if (hbn[k] > 0 && !(rel <= opts->rtol)) status = KFBI_ERR_NOT_CONVERGED;
  }
  if (status != KFBI_OK) fail(p0, status, "some instances did not converge within max_iter");
  return status;
}

kfbi_status kfbi_evaluate_batch(kfbi_batch* b, const kfbi_data* data, const double* const* densities,
                                double* const* u_grids) {
  if (!b || !data || !densities || !u_grids) return KFBI_ERR_ARG;
  kfbi_problem* p0 = b->ps[0];
  const int n = b->n;
  for (int k = 0; k < n; ++k) {
    if (!densities[k] || !u_grids[k]) return fail(p0, KFBI_ERR_ARG, "missing array for instance " + std::to_string(k));
    if (b->ps[k]->cfg.kind == KFBI_INTERFACE_MU && !data[k].g1)
      return fail(p0, KFBI_ERR_ARG, "interface evaluate needs data->g1 (instance " + std::to_string(k) + ")");
  }
  // Dirichlet: u = D phi + N f (a = phi); interface: [u] = g1, [d_n u] = psi,
  // f/sigma and the outer data (a = g1, b = psi)
  const bool mu = p0->cfg.kind == KFBI_INTERFACE_MU;
  std::vector<const double*> a(n), bb(n, nullptr);
  for (int k = 0; k < n; ++k) {
    a[k] = mu ? data[k].g1 : densities[k];
    if (mu) bb[k] = densities[k];
  }
  KFBI_TRY(batch_potentials(b, a.data(), mu ? bb.data() : nullptr, data, mu));
  for (int k = 0; k < n; ++k)
    KFBI_CUDA(p0, cudaMemcpyAsync(u_grids[k], b->ps[k]->ugrid, sizeof(double) * b->ps[k]->g.nodes(),
                                  cudaMemcpyDeviceToDevice, b->stream));
  return KFBI_OK;
}

}  // extern "C"
