// C ABI of the GB300 KFBI library (see include/kfbi.h): problem lifetime,
// queries, the four steps of Algorithm 1 Step 3 one at a time, the BIE
// operator, the BIE right-hand side (Algorithm 1 Step 1), GMRES (Step 4) and
// the final evaluation by superposition (Sec. 6).
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "kfbi_internal.cuh"

namespace kfbi {

kfbi_status fail(kfbi_problem* p, kfbi_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

// General interface kind: one potential per side operator with jumps
// [u] = a, [d_n u] = b and no sources, then its four one-sided traces.
static kfbi_status potential_traces(kfbi_problem* q, const double* a, const double* b, double* T) {
  const int nb = q->nb;
  KFBI_TRY(launch_correction_values(q, a, b, nullptr, q->cvals));
  KFBI_TRY(launch_rhs(q, q->cvals, nullptr, q->rhs));
  KFBI_TRY(box_solve(q, q->rhs, q->ugrid));
  return launch_traces(q, q->ugrid, q->cvals, T, T + nb, T + 2 * nb, T + 3 * nb);
}

// eq. (bie-ifp-1), left-hand side: x = [phi; psi]; w_i has [u] = phi,
// [d_n u] = psi/sigma_i under Lap - kappa_i/sigma_i;
// y = [phi - (avg w_1 - avg w_2); psi - (sigma_1 avg d_n w_1 - sigma_2 avg d_n w_2)]
static kfbi_status apply_general(kfbi_problem* p, const double* x, double* y) {
  kfbi_problem* q = p->twin;
  q->stream = p->stream;
  const int nb = p->nb;
  double* T = p->gen;
  double* s = p->gen + 8 * (size_t)nb;
  const double s1 = p->cfg.sigma_in, s2 = p->cfg.sigma_out;
  KFBI_TRY(launch_gen_scale(p, x + nb, 1.0 / s1, 1.0 / s2, s, s + nb));
  KFBI_TRY(potential_traces(p, x, s, T));
  KFBI_TRY(potential_traces(q, x, s + nb, T + 4 * (size_t)nb));
  return launch_gen_combine(p, x, 1.0, x + nb, 1.0, T, -1.0, 1.0, -s1, s2, y);
}

// One application of the discrete BIE operator: Steps 3.1-3.4 + combination.
kfbi_status apply_operator_impl(kfbi_problem* p, const double* x, double* y) {
  if (p->cfg.kind == KFBI_INTERFACE_GENERAL) return apply_general(p, x, y);
  const bool dir = p->cfg.kind == KFBI_DIRICHLET_INTERIOR;
  const bool neu = p->cfg.kind == KFBI_NEUMANN_INTERIOR;
  // Step 3.1 (fitted and evaluated at the irregular nodes)
  KFBI_TRY(launch_correction_values(p, dir ? x : nullptr, dir ? nullptr : x, nullptr, p->cvals));
  // Step 3.2
  KFBI_TRY(launch_rhs(p, p->cvals, nullptr, p->rhs));
  // Step 3.3
  KFBI_TRY(box_solve(p, p->rhs, p->ugrid));
  // Step 3.4 + BIE: Dirichlet y = x/2 + avg value; mu-form y = x/2 - mu avg d_n;
  // Neumann y = x/2 + avg d_n (= x/2 - K'x), projected when kappa~ = 0
  KFBI_TRY(launch_operator_trace(p, p->ugrid, p->cvals, x, 0.5, dir || neu ? 1.0 : -p->mu, y));
  return neu ? launch_mean_project(p, y) : KFBI_OK;
}

// One operator application through a CUDA graph captured on first use (the
// caller's stream may be the legacy stream, which cannot be captured, so the
// capture runs on a private stream and the graph is launched on p->stream).
kfbi_status apply_operator_fast(kfbi_problem* p, const double* x, double* y) {
  if (!p->use_graphs || p->prof.on) return apply_operator_impl(p, x, y);
  cudaStream_t st = p->stream;
  if (!p->op_exec) {
    if (!p->cap_stream) KFBI_CUDA(p, cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    KFBI_CUDA(p, cudaStreamSynchronize(st));
    long long before[KFBI_KC_COUNT];
    for (int k = 0; k < KFBI_KC_COUNT; ++k) before[k] = p->prof.launches[k];
    set_stream(p, p->cap_stream);
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    kfbi_status s = KFBI_OK;
    if (e == cudaSuccess) s = apply_operator_impl(p, p->xbuf, p->ybuf);
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(p->cap_stream, &gr) : e;
    set_stream(p, st);
    for (int k = 0; k < KFBI_KC_COUNT; ++k) {
      p->op_counts[k] = p->prof.launches[k] - before[k];
      p->prof.launches[k] = before[k];
    }
    if (e != cudaSuccess || e2 != cudaSuccess || s != KFBI_OK) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      p->use_graphs = false;   // fall back to direct launches (same kernels)
      return apply_operator_impl(p, x, y);
    }
    p->op_graph = gr;
    KFBI_CUDA(p, cudaGraphInstantiate(&p->op_exec, gr, 0));
  }
  KFBI_CUDA(p, cudaMemcpyAsync(p->xbuf, x, sizeof(double) * p->nx, cudaMemcpyDeviceToDevice, st));
  KFBI_CUDA(p, cudaGraphLaunch(p->op_exec, st));
  KFBI_CUDA(p, cudaMemcpyAsync(y, p->ybuf, sizeof(double) * p->nx, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < KFBI_KC_COUNT; ++k) p->prof.launches[k] += p->op_counts[k];
  return KFBI_OK;
}

static kfbi_status potential_with_data(kfbi_problem* p, const double* a, const double* b,
                                       const kfbi_data* data, bool use_gb, double* u) {
  kfbi_data dd;
  memset(&dd, 0, sizeof(dd));
  if (data) dd = *data;
  if (!use_gb) dd.g_b = nullptr;
  KFBI_TRY(launch_correction_values_data(p, a, b, &dd, p->cvals));
  KFBI_TRY(launch_rhs(p, p->cvals, &dd, p->rhs));
  KFBI_TRY(box_solve(p, p->rhs, u));
  return launch_set_boundary(p, u, use_gb ? dd.g_b : nullptr);
}

// The data of each side of the general interface problem: f_1 (Omega_1) for
// the kappa_1 operator; f_2 (Omega_2) and the outer values g_b for kappa_2.
static void side_data(const kfbi_data* data, kfbi_data* d1, kfbi_data* d2) {
  memset(d1, 0, sizeof(*d1));
  memset(d2, 0, sizeof(*d2));
  d1->f_in = data->f_in;
  d1->lapf_in = data->lapf_in;
  d1->in_per_interface = data->in_per_interface;
  d2->f_out = data->f_out;
  d2->lapf_out = data->lapf_out;
  d2->g_b = data->g_b;
}

// eq. (bie-ifp-1), right-hand side: P_1 = kappa_1 potential of [d_n u] = g2/sigma_1
// and f_1; P_2 = kappa_2 potential of [u] = g1, f_2 and g_b;
// b = [g1/2 + avg P_1 + avg P_2; -g2/2 + sigma_1 avg d_n P_1 + sigma_2 avg d_n P_2]
static kfbi_status bie_rhs_general(kfbi_problem* p, const kfbi_data* data, double* bvec) {
  kfbi_problem* q = p->twin;
  q->stream = p->stream;
  const int nb = p->nb;
  double* T = p->gen;
  double* s = p->gen + 8 * (size_t)nb;
  const double s1 = p->cfg.sigma_in, s2 = p->cfg.sigma_out;
  kfbi_data d1, d2;
  side_data(data, &d1, &d2);
  KFBI_TRY(launch_gen_scale(p, data->g2, 1.0 / s1, 0.0, s, s + nb));
  KFBI_TRY(potential_with_data(p, nullptr, s, &d1, false, p->ugrid));
  KFBI_TRY(launch_traces(p, p->ugrid, p->cvals, T, T + nb, T + 2 * nb, T + 3 * nb));
  KFBI_TRY(potential_with_data(q, data->g1, nullptr, &d2, true, q->ugrid));
  KFBI_TRY(launch_traces(q, q->ugrid, q->cvals, T + 4 * (size_t)nb, T + 5 * (size_t)nb, T + 6 * (size_t)nb,
                         T + 7 * (size_t)nb));
  return launch_gen_combine(p, data->g1, 0.5, data->g2, -0.5, T, 1.0, 1.0, s1, s2, bvec);
}

kfbi_status bie_rhs_impl(kfbi_problem* p, const kfbi_data* data, double* bvec) {
  if (p->cfg.kind == KFBI_INTERFACE_GENERAL) return bie_rhs_general(p, data, bvec);
  const bool dir = p->cfg.kind == KFBI_DIRICHLET_INTERIOR;
  if (dir) {
    // b = g_D - G f, G f = avg trace of N f (a = b = 0, F = f/sigma inside)
    KFBI_TRY(potential_with_data(p, nullptr, nullptr, data, false, p->ugrid));
    return launch_operator_trace(p, p->ugrid, p->cvals, data->g1, 1.0, -1.0, bvec);
  }
  if (p->cfg.kind == KFBI_NEUMANN_INTERIOR) {
    // b = g_N/sigma - d_n G f, d_n G f = avg d_n of N f; projected when kappa~ = 0
    KFBI_TRY(potential_with_data(p, nullptr, nullptr, data, false, p->ugrid));
    KFBI_TRY(launch_operator_trace(p, p->ugrid, p->cvals, data->g2, 1.0 / p->cfg.sigma_in, -1.0, bvec));
    return launch_mean_project(p, bvec);
  }
  // b = g2/(sigma_in + sigma_out) + mu avg d_n w, w with a = g1, F = f/sigma, g_B
  KFBI_TRY(potential_with_data(p, data->g1, nullptr, data, true, p->ugrid));
  return launch_operator_trace(p, p->ugrid, p->cvals, data->g2,
                               1.0 / (p->cfg.sigma_in + p->cfg.sigma_out), p->mu, bvec);
}

// The boundary data each kind reads: g1 (Dirichlet), g2 (Neumann), both (interface).
static bool has_boundary_data(const kfbi_problem* p, const kfbi_data* data) {
  switch (p->cfg.kind) {
    case KFBI_DIRICHLET_INTERIOR: return data->g1 != nullptr;
    case KFBI_NEUMANN_INTERIOR: return data->g2 != nullptr;
    default: return data->g1 != nullptr && data->g2 != nullptr;
  }
}

}  // namespace kfbi

using namespace kfbi;

// Message of the last failed kfbi_create_problem on this thread (the problem
// object does not survive a failed create).
static thread_local std::string g_create_error;

// Checks a level set against the problem's dimension and takes it: kind,
// parameters, interface count and, for the grid-sampled kind, a device copy
// of the node values (replacing an earlier copy).
static kfbi_status set_levelset(kfbi_problem* p, const kfbi_levelset* ls) {
  const kfbi_config* cfg = &p->cfg;
  const bool ls2d = ls->kind == KFBI_LS_ELLIPSE || ls->kind == KFBI_LS_STAR || ls->kind == KFBI_LS_DISCS;
  const bool balls = ls->kind == KFBI_LS_DISCS || ls->kind == KFBI_LS_SPHERES;
  const bool sampled = ls->kind == KFBI_LS_GRID;
  if (sampled && !ls->samples)
    return fail(p, KFBI_ERR_ARG, "a grid-sampled level set needs its node values (samples)");
  const bool uni = ls->kind == KFBI_LS_UNION;
  if (ls->n_params < 0 || ls->n_params > KFBI_LS_MAX_PARAMS || ls->kind < 1 || ls->kind > 9 ||
      (!sampled && !uni && ls2d != (cfg->dim == 2)) ||
      (balls && (ls->n_params < 2 || !(ls->p[0] > 0) || ls->p[1] < 1 ||
                 ls->p[1] > KFBI_MAX_INTERFACES ||
                 2 + cfg->dim * (int)ls->p[1] > ls->n_params)))
    return fail(p, KFBI_ERR_ARG, "level-set kind does not match the dimension");
  int n_iface = balls ? (int)ls->p[1] : 1;
  if (uni) {
    // m components, each a kind code and that kind's parameters
    bool ok = ls->n_params >= 1 && ls->p[0] >= 1 && ls->p[0] <= KFBI_MAX_INTERFACES;
    int at = 1;
    n_iface = ok ? (int)ls->p[0] : 0;
    for (int k = 0; ok && k < n_iface; ++k) {
      if (at >= ls->n_params) {
        ok = false;
        break;
      }
      const int kind = (int)ls->p[at];
      int cnt = 0;
      if (cfg->dim == 2 && (kind == KFBI_LS_ELLIPSE || kind == KFBI_LS_STAR)) cnt = 5;
      if (cfg->dim == 3 && kind == KFBI_LS_ELLIPSOID) cnt = 6;
      if (cfg->dim == 3 && kind == KFBI_LS_TORUS) cnt = 2;
      ok = cnt > 0 && at + 1 + cnt <= ls->n_params;
      at += 1 + cnt;
    }
    if (!ok)
      return fail(p, KFBI_ERR_ARG, "union level set: m in [1, 32] components of ellipse/star (2D) or "
                                   "ellipsoid/torus (3D) with their parameters");
  }
  p->n_iface = n_iface;
  p->ls.kind = ls->kind;
  p->ls.np = ls->n_params;
  memcpy(p->ls.p, ls->p, sizeof(p->ls.p));
  p->ls.grid = nullptr;
  if (sampled) {
    // the problem keeps its own copy of the node values (one buffer of the
    // grid's size, kept across updates)
    const long long nodes = p->g.nodes();
    if ((!p->ls_samples && dalloc(&p->ls_samples, nodes) != cudaSuccess) ||
        cudaMemcpy(p->ls_samples, ls->samples, sizeof(double) * nodes, cudaMemcpyDeviceToDevice) != cudaSuccess)
      return fail(p, KFBI_ERR_CUDA, "cannot copy the level-set samples");
    long long bad = 0;
    if (count_nonfinite(p->ls_samples, nodes, p->stream, &bad) != cudaSuccess)
      return fail(p, KFBI_ERR_CUDA, "cannot check the level-set samples");
    if (bad > 0) return fail(p, KFBI_ERR_ARG, "the level-set samples must be finite");
    p->ls.grid = p->ls_samples;
    p->ls.gd = p->g.d;
    p->ls.gn = p->g.n;
    p->ls.glo = p->g.lo;
    p->ls.gh = p->g.h;
  }
  return KFBI_OK;
}

namespace kfbi {

cudaError_t arena_alloc(GeoArena& A, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (A.chunks.empty() || A.used + bytes > A.cap) {
    // a new chunk of at least half of what this set-up has taken so far:
    // few chunks, and at most a third of the memory unused
    const size_t sz = std::max(bytes, std::max(A.total / 2, (size_t)16 << 20));
    char* c = nullptr;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c), sz);
    if (e != cudaSuccess) return e;
    A.chunks.push_back(c);
    A.cap = sz;
    A.used = 0;
  }
  *out = A.chunks.back() + A.used;
  A.used += bytes;
  A.total += bytes;
  return cudaSuccess;
}

void arena_reset(GeoArena& A) {
  if (A.chunks.size() > 1) {
    const size_t want = A.total + A.total / 4;
    arena_release(A);
    char* c = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&c), want) == cudaSuccess) {
      A.chunks.push_back(c);
      A.cap = want;
    }
  }
  A.used = 0;
  A.total = 0;
}

void arena_release(GeoArena& A) {
  for (char* c : A.chunks) cudaFree(c);
  A.chunks.clear();
  A.cap = A.used = A.total = 0;
}

}  // namespace kfbi

// Everything that depends on the interface: geometry, stencils, correction
// entries, trace weights, the per-DOF work vectors, the GMRES workspace and
// the captured graphs.  The box solver, the grids R and u, the stencil tables
// and the streams stay.
static void free_geometry(kfbi_problem* p, bool keep_arena = true) {
  gmres_destroy(p);
  if (p->op_exec) cudaGraphExecDestroy(p->op_exec);
  if (p->op_graph) cudaGraphDestroy(p->op_graph);
  p->op_exec = nullptr;
  p->op_graph = nullptr;
  for (int k = 0; k < KFBI_KC_COUNT; ++k) p->op_counts[k] = 0;
  // every array below lies in the geometry arena: no kernel may still read
  // them when the arena is reused (one device-wide wait, as cudaFree makes)
  cudaDeviceSynchronize();
  int32_t** i32[] = {&p->family, &p->edge, &p->axis, &p->st_axis, &p->pde_node, &p->dir_idx,
                     &p->neu_idx, &p->irr_lin, &p->dof_iface, &p->ent_lin, &p->ent_iface,
                     &p->ent_owner, &p->corr_nb, &p->corr_nb2};
  for (int32_t** b : i32) *b = nullptr;
  uint8_t** u8[] = {&p->inside, &p->irr_flag, &p->irr_inside};
  for (uint8_t** b : u8) *b = nullptr;
  double** f64[] = {&p->minv, &p->ent_w, &p->cvals, &p->tvals, &p->bvec, &p->xbuf, &p->ybuf, &p->gen};
  for (double** b : f64) *b = nullptr;
  p->d_flags = nullptr;
  for (int k = 0; k < 3; ++k) {
    p->x[k] = p->nrm[k] = nullptr;
    p->line_start[k] = nullptr;
  }
  for (int s = 0; s < 2; ++s) p->tr[s] = TraceCSR();
  // an update reuses the arena (its chunks merged into one); destroy frees it
  if (keep_arena)
    arena_reset(p->arena);
  else
    arena_release(p->arena);
  p->nb = p->nirr = p->nent = p->nx = 0;
}

// The per-DOF work vectors and the GMRES workspace of a set-up geometry (the
// grids R and u once).
static kfbi_status alloc_work(kfbi_problem* p) {
  p->nx = p->cfg.kind == KFBI_INTERFACE_GENERAL ? 2 * p->nb : p->nb;
  const long long nodes = p->g.nodes();
  if ((!p->rhs && dalloc(&p->rhs, nodes) != cudaSuccess) ||
      (!p->ugrid && dalloc(&p->ugrid, nodes) != cudaSuccess) ||
      galloc(p, &p->cvals, p->nent) != cudaSuccess || galloc(p, &p->tvals, p->nb) != cudaSuccess ||
      galloc(p, &p->bvec, p->nx) != cudaSuccess || galloc(p, &p->xbuf, p->nx) != cudaSuccess ||
      galloc(p, &p->ybuf, p->nx) != cudaSuccess ||
      (p->cfg.kind == KFBI_INTERFACE_GENERAL && galloc(p, &p->gen, 11 * (size_t)p->nb) != cudaSuccess))
    return fail(p, KFBI_ERR_CUDA, "out of device memory");
  return gmres_create(p, kMaxKrylov);
}

extern "C" {

kfbi_status kfbi_create_problem(const kfbi_config* cfg, const kfbi_levelset* ls, void* cuda_stream,
                                kfbi_problem** out) {
  if (!out) return KFBI_ERR_ARG;
  *out = nullptr;
  if (!cfg || !ls) return KFBI_ERR_ARG;
  kfbi_problem* p = new (std::nothrow) kfbi_problem();
  if (!p) return KFBI_ERR_ARG;
  p->cfg = *cfg;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  g_create_error.clear();
  auto bail = [&](kfbi_status s) {
    g_create_error = p->err;
    kfbi_destroy_problem(p);
    return s;
  };
  if (cfg->dim != 2 && cfg->dim != 3) {
    fail(p, KFBI_ERR_ARG, "dim must be 2 or 3");
    return bail(KFBI_ERR_ARG);
  }
  if (cfg->order != 2 && cfg->order != 4) {
    fail(p, KFBI_ERR_ARG, "order must be 2 or 4");
    return bail(KFBI_ERR_ARG);
  }
  if (!(cfg->hi > cfg->lo) || cfg->n < 8 || (cfg->n & (cfg->n - 1)) != 0) {
    fail(p, KFBI_ERR_ARG, "need hi > lo and N a power of two >= 8");
    return bail(KFBI_ERR_ARG);
  }
  if (cfg->kind != KFBI_DIRICHLET_INTERIOR && cfg->kind != KFBI_INTERFACE_MU &&
      cfg->kind != KFBI_NEUMANN_INTERIOR && cfg->kind != KFBI_INTERFACE_GENERAL) {
    fail(p, KFBI_ERR_ARG, "unknown problem kind");
    return bail(KFBI_ERR_ARG);
  }
  const bool two_sides = cfg->kind == KFBI_INTERFACE_MU || cfg->kind == KFBI_INTERFACE_GENERAL;
  if (!(cfg->sigma_in > 0) || (two_sides && !(cfg->sigma_out > 0)) || !(cfg->kappa >= 0) ||
      (cfg->kind == KFBI_INTERFACE_GENERAL && !(cfg->kappa_out >= 0))) {
    fail(p, KFBI_ERR_ARG, "need sigma > 0 and kappa >= 0");
    return bail(KFBI_ERR_ARG);
  }
  if (!(cfg->relax >= 0.0) || !(cfg->relax <= 1.0)) {
    fail(p, KFBI_ERR_ARG, "relax must be in [0, 1]");
    return bail(KFBI_ERR_ARG);
  }
  if (cfg->box_solver != KFBI_BOX_DST && cfg->box_solver != KFBI_BOX_MG) {
    fail(p, KFBI_ERR_ARG, "unknown box solver");
    return bail(KFBI_ERR_ARG);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    fail(p, KFBI_ERR_CUDA, "no CUDA device");
    return bail(KFBI_ERR_CUDA);
  }
  p->g.d = cfg->dim;
  p->g.n = cfg->n;
  p->g.lo = cfg->lo;
  p->g.h = (cfg->hi - cfg->lo) / cfg->n;
  {
    const kfbi_status sl = set_levelset(p, ls);
    if (sl != KFBI_OK) return bail(sl);
  }
  p->kt = cfg->kind == KFBI_INTERFACE_MU ? cfg->kappa : cfg->kappa / cfg->sigma_in;
  p->mu = cfg->kind == KFBI_INTERFACE_MU
              ? (cfg->sigma_out - cfg->sigma_in) / (cfg->sigma_out + cfg->sigma_in)
              : 0.0;
  p->cos_alpha = cfg->cos_alpha > 0 ? cfg->cos_alpha : (cfg->dim == 2 ? 0.707 : 0.4);
  const double h = p->g.h, ih2 = 1.0 / (h * h), k = p->kt;
  if (cfg->order == 2) {
    p->stencil_c[0] = -2.0 * cfg->dim * ih2 - k;
    p->stencil_c[1] = ih2;
    p->stencil_c[2] = p->stencil_c[3] = 0.0;
  } else if (cfg->dim == 2) {
    p->stencil_c[0] = -10.0 / 3.0 * ih2 - 2.0 / 3.0 * k;
    p->stencil_c[1] = 2.0 / 3.0 * ih2 - k / 12.0;
    p->stencil_c[2] = 1.0 / 6.0 * ih2;
    p->stencil_c[3] = 0.0;
  } else {
    p->stencil_c[0] = -25.0 / 6.0 * ih2 - 0.5 * k;
    p->stencil_c[1] = 5.0 / 12.0 * ih2 - k / 12.0;
    p->stencil_c[2] = 1.0 / 8.0 * ih2;
    p->stencil_c[3] = 1.0 / 48.0 * ih2;
  }
  kfbi_status s = build_geometry(p);
  if (s != KFBI_OK) return bail(s);
  if ((s = upload_neighbour_tables(p)) != KFBI_OK) return bail(s);
  if (dalloc(&p->stencil_dev, 4) != cudaSuccess ||
      cudaMemcpy(p->stencil_dev, p->stencil_c, sizeof(p->stencil_c), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    fail(p, KFBI_ERR_CUDA, "stencil upload failed");
    return bail(KFBI_ERR_CUDA);
  }
  if ((s = box_create(p)) != KFBI_OK) return bail(s);
  p->nx = cfg->kind == KFBI_INTERFACE_GENERAL ? 2 * p->nb : p->nb;
  if (cfg->kind == KFBI_INTERFACE_GENERAL) {
    // the kappa_2/sigma_2 operator: the same geometry set up once more with
    // its own collocation matrices, RHS stencil and box solver
    kfbi_config c2 = *cfg;
    c2.kind = KFBI_INTERFACE_MU;
    c2.kappa = cfg->kappa_out / cfg->sigma_out;
    if ((s = kfbi_create_problem(&c2, ls, cuda_stream, &p->twin)) != KFBI_OK) {
      fail(p, s, "kappa_2 operator: " + g_create_error);
      return bail(s);
    }
    p->twin->parent = p;
    if (p->twin->nb != p->nb || p->twin->nirr != p->nirr || p->twin->nent != p->nent) {
      fail(p, KFBI_ERR_GEOMETRY, "the two side operators set up different DOFs");
      return bail(KFBI_ERR_GEOMETRY);
    }
  }
  if ((s = alloc_work(p)) != KFBI_OK) return bail(s);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
    fail(p, KFBI_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return bail(KFBI_ERR_CUDA);
  }
  *out = p;
  return KFBI_OK;
}

kfbi_status kfbi_destroy_problem(kfbi_problem* p) {
  if (!p) return KFBI_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->twin) {
    // first, while the parent's streams exist; the twin works on the parent's stream
    p->twin->stream = p->stream;
    kfbi_destroy_problem(p->twin);
    p->twin = nullptr;
  }
  free_geometry(p, false);
  box_destroy(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->ls_samples) cudaFree(p->ls_samples);
  void* bufs[] = {p->nb_off, p->nb_coef, p->rhs, p->ugrid, p->ftilde, p->stencil_dev};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (cudaEvent_t e : p->prof.pool) cudaEventDestroy(e);
  delete p;
  return KFBI_OK;
}

kfbi_status kfbi_update_levelset(kfbi_problem* p, const kfbi_levelset* ls) {
  if (!p || !ls) return KFBI_ERR_ARG;
  if (p->parent) return fail(p, KFBI_ERR_ARG, "update the problem, not its second side operator");
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  free_geometry(p);
  KFBI_TRY(set_levelset(p, ls));
  KFBI_TRY(build_geometry(p));
  if (p->twin) {
    kfbi_problem* q = p->twin;
    q->stream = p->stream;
    KFBI_CUDA(p, cudaStreamSynchronize(q->stream));
    free_geometry(q);
    kfbi_status s = set_levelset(q, ls);
    if (s == KFBI_OK) s = build_geometry(q);
    if (s == KFBI_OK) s = alloc_work(q);
    if (s != KFBI_OK) return fail(p, s, "kappa_2 operator: " + q->err);
    if (q->nb != p->nb || q->nirr != p->nirr || q->nent != p->nent)
      return fail(p, KFBI_ERR_GEOMETRY, "the two side operators set up different DOFs");
  }
  KFBI_TRY(alloc_work(p));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  return KFBI_OK;
}

const char* kfbi_last_error(const kfbi_problem* p) {
  if (!p) return g_create_error.c_str();
  return p->err.c_str();
}

kfbi_status kfbi_sizes(const kfbi_problem* p, int* n_b, int* n_irr, int* n_coef) {
  if (!p) return KFBI_ERR_ARG;
  if (n_b) *n_b = p->nb;
  if (n_irr) *n_irr = p->nirr;
  if (n_coef) *n_coef = p->ncoef;
  return KFBI_OK;
}

kfbi_status kfbi_num_dofs(const kfbi_problem* p, int* n_b) {
  if (!p || !n_b) return KFBI_ERR_ARG;
  *n_b = p->nb;
  return KFBI_OK;
}

kfbi_status kfbi_stencil_sizes(const kfbi_problem* p, int* n_pde, int* n_dir, int* n_neu) {
  if (!p) return KFBI_ERR_ARG;
  if (n_pde) *n_pde = p->npde;
  if (n_dir) *n_dir = p->ndir;
  if (n_neu) *n_neu = p->nneu;
  return KFBI_OK;
}

kfbi_status kfbi_dof_points(const kfbi_problem* pc, double* xyz, double* normals) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p) return KFBI_ERR_ARG;
  const int d = p->g.d;
  for (int k = 0; k < d; ++k) {
    if (xyz)
      KFBI_CUDA(p, cudaMemcpy2DAsync(xyz + k, sizeof(double) * d, p->x[k], sizeof(double),
                                     sizeof(double), p->nb, cudaMemcpyDeviceToDevice, p->stream));
    if (normals)
      KFBI_CUDA(p, cudaMemcpy2DAsync(normals + k, sizeof(double) * d, p->nrm[k], sizeof(double),
                                     sizeof(double), p->nb, cudaMemcpyDeviceToDevice, p->stream));
  }
  return KFBI_OK;
}

kfbi_status kfbi_dof_info(const kfbi_problem* pc, int32_t* family, int32_t* axis,
                          int32_t* stencil_axis) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p) return KFBI_ERR_ARG;
  size_t bytes = sizeof(int32_t) * p->nb;
  if (family) KFBI_CUDA(p, cudaMemcpyAsync(family, p->family, bytes, cudaMemcpyDeviceToDevice, p->stream));
  if (axis) KFBI_CUDA(p, cudaMemcpyAsync(axis, p->axis, bytes, cudaMemcpyDeviceToDevice, p->stream));
  if (stencil_axis)
    KFBI_CUDA(p, cudaMemcpyAsync(stencil_axis, p->st_axis, bytes, cudaMemcpyDeviceToDevice, p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_collocation_stencils(const kfbi_problem* pc, int32_t* pde_nodes, int32_t* dir_dofs,
                                      int32_t* neu_dofs) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p) return KFBI_ERR_ARG;
  const size_t nb = p->nb;
  if (pde_nodes)
    KFBI_CUDA(p, cudaMemcpyAsync(pde_nodes, p->pde_node, sizeof(int32_t) * nb * p->npde,
                                 cudaMemcpyDeviceToDevice, p->stream));
  if (dir_dofs)
    KFBI_CUDA(p, cudaMemcpyAsync(dir_dofs, p->dir_idx, sizeof(int32_t) * nb * p->ndir,
                                 cudaMemcpyDeviceToDevice, p->stream));
  if (neu_dofs)
    KFBI_CUDA(p, cudaMemcpyAsync(neu_dofs, p->neu_idx, sizeof(int32_t) * nb * p->nneu,
                                 cudaMemcpyDeviceToDevice, p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_inside_mask(const kfbi_problem* pc, uint8_t* mask) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p || !mask) return KFBI_ERR_ARG;
  KFBI_CUDA(p, cudaMemcpyAsync(mask, p->inside, p->g.nodes(), cudaMemcpyDeviceToDevice, p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_irregular_nodes(const kfbi_problem* pc, int32_t* lin_index, int32_t* owner) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p) return KFBI_ERR_ARG;
  if (owner && p->n_iface > 1) return fail(p, KFBI_ERR_ARG, "several interfaces: owner must be NULL");
  size_t bytes = sizeof(int32_t) * p->nirr;
  if (lin_index) KFBI_CUDA(p, cudaMemcpyAsync(lin_index, p->irr_lin, bytes, cudaMemcpyDeviceToDevice, p->stream));
  // one interface: entry q is irregular node q
  if (owner) KFBI_CUDA(p, cudaMemcpyAsync(owner, p->ent_owner, bytes, cudaMemcpyDeviceToDevice, p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_interfaces(const kfbi_problem* p, int* n_iface, int* n_entries) {
  if (!p) return KFBI_ERR_ARG;
  if (n_iface) *n_iface = p->n_iface;
  if (n_entries) *n_entries = p->nent;
  return KFBI_OK;
}

kfbi_status kfbi_dof_iface(const kfbi_problem* pc, int32_t* iface) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p || !iface) return KFBI_ERR_ARG;
  KFBI_CUDA(p, cudaMemcpyAsync(iface, p->dof_iface, sizeof(int32_t) * p->nb, cudaMemcpyDeviceToDevice,
                               p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_correction_entries(const kfbi_problem* pc, int32_t* lin_index, int32_t* iface,
                                    int32_t* owner) {
  kfbi_problem* p = const_cast<kfbi_problem*>(pc);
  if (!p) return KFBI_ERR_ARG;
  const size_t bytes = sizeof(int32_t) * p->nent;
  if (lin_index) KFBI_CUDA(p, cudaMemcpyAsync(lin_index, p->ent_lin, bytes, cudaMemcpyDeviceToDevice, p->stream));
  if (iface) KFBI_CUDA(p, cudaMemcpyAsync(iface, p->ent_iface, bytes, cudaMemcpyDeviceToDevice, p->stream));
  if (owner) KFBI_CUDA(p, cudaMemcpyAsync(owner, p->ent_owner, bytes, cudaMemcpyDeviceToDevice, p->stream));
  return KFBI_OK;
}

kfbi_status kfbi_collocation_fit(kfbi_problem* p, const double* a, const double* b,
                                 const double* ftilde, double* coef) {
  if (!p || !coef) return KFBI_ERR_ARG;
  return launch_collocation_fit(p, a, b, ftilde, coef);
}

kfbi_status kfbi_correction_values(kfbi_problem* p, const double* a, const double* b,
                                   const double* ftilde, double* cvals) {
  if (!p || !cvals) return KFBI_ERR_ARG;
  return launch_correction_values(p, a, b, ftilde, cvals);
}

kfbi_status kfbi_corrected_rhs(kfbi_problem* p, const double* cvals, const kfbi_data* data,
                               double* rhs) {
  if (!p || !rhs) return KFBI_ERR_ARG;
  return launch_rhs(p, cvals, data, rhs);
}

kfbi_status kfbi_box_solve(kfbi_problem* p, const double* rhs, double* u) {
  if (!p || !rhs || !u) return KFBI_ERR_ARG;
  return box_solve(p, rhs, u);
}

kfbi_status kfbi_box_solve_info(kfbi_problem* p, int* steps, int* cycles, double* rel_change,
                               int* converged) {
  if (!p) return KFBI_ERR_ARG;
  int s = 0, c = 0, conv = 0;
  double rel = 0.0;
  KFBI_TRY(box_steps(p, &s, &c));
  KFBI_TRY(box_last_residual(p, &rel, &conv));
  if (steps) *steps = s;
  if (cycles) *cycles = c;
  if (rel_change) *rel_change = rel;
  if (converged) *converged = conv;
  return KFBI_OK;
}

kfbi_status kfbi_traces(kfbi_problem* p, const double* u, const double* cvals, double* val_plus,
                        double* val_minus, double* dn_plus, double* dn_minus) {
  if (!p || !u || !cvals) return KFBI_ERR_ARG;
  return launch_traces(p, u, cvals, val_plus, val_minus, dn_plus, dn_minus);
}

kfbi_status kfbi_apply_operator(kfbi_problem* p, const double* x, double* y) {
  if (!p || !x || !y) return KFBI_ERR_ARG;
  return apply_operator_fast(p, x, y);
}

kfbi_status kfbi_bie_rhs(kfbi_problem* p, const kfbi_data* data, double* b) {
  if (!p || !data || !b || !has_boundary_data(p, data)) return KFBI_ERR_ARG;
  return bie_rhs_impl(p, data, b);
}

kfbi_status kfbi_gmres_solve(kfbi_problem* p, const kfbi_data* data, const kfbi_gmres_opts* opts,
                             double* density, kfbi_gmres_info* info) {
  if (!p || !data || !opts || !density || !has_boundary_data(p, data)) return KFBI_ERR_ARG;
  if (!(opts->rtol > 0) || opts->max_iter < 1) return fail(p, KFBI_ERR_ARG, "need rtol > 0, max_iter >= 1");
  auto t0 = std::chrono::steady_clock::now();
  KFBI_TRY(bie_rhs_impl(p, data, p->bvec));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  auto t1 = std::chrono::steady_clock::now();
  int it = 0;
  double rel = 0.0;
  int rejected = 0;
  KFBI_TRY(box_steps_reset(p));
  if (p->twin) KFBI_TRY(box_steps_reset(p->twin));
  KFBI_TRY(box_tol_reset(p));
  if (p->twin) KFBI_TRY(box_tol_reset(p->twin));
  kfbi_status s = gmres_run(p, p->bvec, opts->x0, opts->rtol, opts->restart > 0 ? opts->restart : 100,
                            opts->max_iter, density, &it, &rel, &rejected);
  // every later box solve (the evaluation) at the full accuracy again
  KFBI_TRY(box_tol_reset(p));
  if (p->twin) KFBI_TRY(box_tol_reset(p->twin));
  long long steps = 0, steps2 = 0;
  KFBI_TRY(box_steps_total(p, &steps));
  if (p->twin) KFBI_TRY(box_steps_total(p->twin, &steps2));
  auto t2 = std::chrono::steady_clock::now();
  if (info) {
    info->iters = it;
    info->rel_res = rel;
    for (double& v : info->t_ms) v = 0.0;
    info->t_ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->t_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    info->t_ms[2] = std::chrono::duration<double, std::milli>(t2 - t0).count();
    info->x0_rejected = rejected;
    info->refine_steps = (int)(steps + steps2);
  }
  return s;
}

kfbi_status kfbi_evaluate(kfbi_problem* p, const kfbi_data* data, const double* density,
                          double* u_grid) {
  if (!p || !density || !u_grid) return KFBI_ERR_ARG;
  if (p->cfg.kind == KFBI_DIRICHLET_INTERIOR)
    return potential_with_data(p, density, nullptr, data, false, u_grid);
  if (p->cfg.kind == KFBI_NEUMANN_INTERIOR)
    return potential_with_data(p, nullptr, density, data, false, u_grid);
  if (p->cfg.kind == KFBI_INTERFACE_GENERAL) {
    if (!data || !data->g1 || !data->g2) return fail(p, KFBI_ERR_ARG, "interface evaluate needs g1 and g2");
    kfbi_problem* q = p->twin;
    q->stream = p->stream;
    const int nb = p->nb;
    double* s = p->gen + 8 * (size_t)nb;
    kfbi_data d1, d2;
    side_data(data, &d1, &d2);
    KFBI_TRY(launch_gen_eval_prep(p, density, density + nb, data->g1, data->g2, s, s + nb, s + 2 * (size_t)nb));
    KFBI_TRY(potential_with_data(p, density, s, &d1, false, u_grid));
    KFBI_TRY(potential_with_data(q, s + 2 * (size_t)nb, s + nb, &d2, true, q->ugrid));
    return launch_select_side(p, u_grid, q->ugrid);
  }
  if (!data || !data->g1) return fail(p, KFBI_ERR_ARG, "interface evaluate needs data->g1");
  return potential_with_data(p, data->g1, density, data, true, u_grid);
}

}  // extern "C"

namespace kfbi {

Launch::Launch(kfbi_problem* pp, int c) : p(pp->parent ? pp->parent : pp), cls(c) {
  p->prof.launches[c]++;
  if (!p->prof.on) return;
  Profiler& P = p->prof;
  if (P.used + 2 > P.pool.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      P.pool.push_back(e);
    }
  }
  rec = (int)(P.used / 2);
  P.used += 2;
  P.cls.push_back(c);
  cudaEventRecord(P.pool[2 * rec], p->stream);
}

Launch::~Launch() {
  if (rec >= 0) cudaEventRecord(p->prof.pool[2 * rec + 1], p->stream);
}

}  // namespace kfbi

extern "C" {

kfbi_status kfbi_launch_counts(kfbi_problem* p, int64_t* counts, int reset) {
  if (!p || !counts) return KFBI_ERR_ARG;
  for (int c = 0; c < KFBI_KC_COUNT; ++c) counts[c] = p->prof.launches[c];
  if (reset)
    for (int c = 0; c < KFBI_KC_COUNT; ++c) p->prof.launches[c] = 0;
  return KFBI_OK;
}

kfbi_status kfbi_profile_enable(kfbi_problem* p, int enable) {
  if (!p) return KFBI_ERR_ARG;
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  p->prof.on = enable != 0;
  p->prof.used = 0;
  p->prof.cls.clear();
  return KFBI_OK;
}

kfbi_status kfbi_profile_read(kfbi_problem* p, double* ms, int64_t* timed) {
  if (!p || !ms || !timed) return KFBI_ERR_ARG;
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int c = 0; c < KFBI_KC_COUNT; ++c) {
    ms[c] = 0.0;
    timed[c] = 0;
  }
  Profiler& P = p->prof;
  for (size_t r = 0; r < P.cls.size(); ++r) {
    float t = 0.f;
    KFBI_CUDA(p, cudaEventElapsedTime(&t, P.pool[2 * r], P.pool[2 * r + 1]));
    ms[P.cls[r]] += t;
    timed[P.cls[r]] += 1;
  }
  return KFBI_OK;
}

}  // extern "C"
