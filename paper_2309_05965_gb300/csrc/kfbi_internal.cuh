// Internal declarations of the GB300 KFBI library: the problem object, device
// buffers, small device helpers and the launch wrappers shared between the
// translation units.  Device memory layout of one problem (all in HBM):
//   grids            (N+1)^d nodes, C order (last axis fastest), FP64 (or FP32
//                    for the mixed-precision work buffers)
//   DOF arrays       structure of arrays, length N_b, DOF order of kfbi.h
//   per-DOF blocks   row-major [N_b][k] (stencils, collocation inverses)
//   per-irregular    column-major [k][n_irr] so that one thread per node reads
//                    coalesced (correction lists); per-entry the same
//                    [k][n_entries] (composite collocation rows)
//   trace weights    CSR over DOFs, one CSR per side (+, -)
// Every array that depends on the interface (DOF arrays, stencils, entries,
// trace CSRs, the per-DOF work vectors) lies in the problem's geometry arena
// (GeoArena below); the grids and the box solver's buffers are separate
// allocations kept across interface updates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kfbi.h"

namespace kfbi {

constexpr int kMaxCoef = 35;          // C(4+3, 3)
constexpr int kMaxPde = 10;
constexpr int kMaxDir = 15;
constexpr int kMaxNeu = 10;
constexpr int kMaxNeighbours = 26;    // 3^3 - 1
constexpr double kTieEps = 1e-12;     // closest-point tie tolerance (units of h^2)
constexpr double kRootTol = 1e-15;    // root iteration stop |ds| <= tol N h (the box width)
constexpr int kRootMaxIt = 64;
constexpr int kMaxKrylov = 100;     // Krylov dimension of every problem (restart length)
constexpr int kGraphArnoldi = 8192; // N_b up to which a GMRES iteration is one graph
constexpr double kTraceWeightScale = 4.0;   // exp(-|xi|^2 / 4)

// Status codes written by setup kernels into Problem::d_flags.
enum SetupFlag : int {
  kFlagGeometry = 0,      // first DOF without a complete collocation stencil (+1), 0 = none
  kFlagSingular = 1,      // first DOF with a singular collocation matrix (+1)
  kFlagTraceSingular = 2, // first DOF with a singular trace fit (+1)
  kFlagOutOfBox = 3,      // a stencil left the grid (+1)
  kFlagClosestFallback = 4,  // count of correction entries that needed the global search
  kFlagNoOwner = 5,       // first correction entry whose interface has no DOF (+1)
  kFlagCount = 8
};

struct Grid {
  int d, n;
  double lo, h;
  __host__ __device__ int np1() const { return n + 1; }
  __host__ __device__ long long nodes() const {
    long long m = n + 1;
    return d == 2 ? m * m : m * m * m;
  }
};

struct LevelSet {
  int kind;
  int np;
  double p[KFBI_LS_MAX_PARAMS];
  // KFBI_LS_GRID: the node values (device copy owned by the problem) and
  // their grid
  const double* grid;
  int gd, gn;
  double glo, gh;
};

// Trace stencil CSR for one side.
struct TraceCSR {
  int32_t* ptr = nullptr;    // N_b + 1
  int32_t* node = nullptr;   // grid linear index
  // correction entry added to the node's value, -1 if none: one interface,
  // the node's entry when it lies across Gamma (+C on the '+' side, -C on the
  // '-' side); several interfaces, C^(t) of the side's label t
  int32_t* irr = nullptr;
  int32_t* irr2 = nullptr;   // several interfaces: C^(l_q) subtracted, -1 if none
  double* wv = nullptr;      // value weights
  double* wn = nullptr;      // normal-derivative weights
  double* w = nullptr;       // weights of the operator's own trace quantity
  // 3D: wv and wn hold FP32 pairs instead (x = hi, y = lo, the weight = hi +
  // lo to ~48 bits), read through these aliases by the four-trace kernel that
  // keeps its sums off the FP64 pipe
  float2* wv2 = nullptr;
  float2* wn2 = nullptr;
  int nnz = 0;
};

struct BoxSolver;   // dst.cu
struct MgSolver;    // mg.cu

// Kernel-launch accounting: every launch is counted by class; with profiling
// enabled each launch is bracketed by CUDA events on the problem's stream.
struct Profiler {
  bool on = false;
  long long launches[KFBI_KC_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> cls;              // class of record r (events 2r, 2r+1)
};

struct Gmres {
  int nb = 0, m = 0;
  double* V = nullptr;       // (m+1) x N_b
  double* H = nullptr;       // column j at H + j*(m+1)
  double* cs = nullptr;
  double* sn = nullptr;
  double* g = nullptr;       // m+1
  double* y = nullptr;       // m
  double* part = nullptr;    // partial sums
  double* scal = nullptr;    // device scalars: [0] beta, [1] bnorm, [2] res, [3] tmp
  double* hcol = nullptr;    // (m+1) coefficient scratch
  double* host_res = nullptr;  // pinned
  int nchunk = 0;
  // one GMRES iteration (operator + Arnoldi step) as a CUDA graph with the
  // step index on the device, for N_b <= kGraphArnoldi
  int* jdev = nullptr;          // [0] j, [1] done flag (always 0 here), [2] iteration limit
  double* h1 = nullptr;         // (m+1)
  double* h2 = nullptr;         // (m+1)
  double* npart = nullptr;      // partial norms (one per CTA of the update)
  void* desc = nullptr;         // ArnDesc of this problem (device)
  cudaGraphExec_t it_exec = nullptr;
  cudaGraph_t it_graph = nullptr;
  // the whole Arnoldi cycle as a conditional WHILE node around that iteration
  cudaGraphExec_t loop_exec = nullptr;
  cudaGraph_t loop_graph = nullptr;
  bool loop_failed = false;
  long long it_counts[KFBI_KC_COUNT] = {};
};

// Device memory of one geometry: every array that the set-up and the per-DOF
// work allocation make, temporaries included, bump-allocated (256-byte
// aligned) from chunks of cudaMalloc.  A new interface on the same grid
// resets it instead of freeing and allocating each array; after a set-up
// that needed several chunks the reset replaces them by one that holds them
// all, so the next set-up of a similar interface makes no allocation.
struct GeoArena {
  std::vector<char*> chunks;
  size_t cap = 0;     // bytes of the last chunk
  size_t used = 0;    // bytes handed out from the last chunk
  size_t total = 0;   // bytes handed out since the last reset
};
cudaError_t arena_alloc(GeoArena& A, size_t bytes, void** out);
// number of non-finite values of a device array (synchronises the stream)
cudaError_t count_nonfinite(const double* a, long long n, cudaStream_t st, long long* out);
void arena_reset(GeoArena& A);
void arena_release(GeoArena& A);

}  // namespace kfbi

struct kfbi_problem {
  kfbi_config cfg;
  kfbi::Grid g;
  kfbi::LevelSet ls;
  double* ls_samples = nullptr;   // device copy of a grid-sampled level set
  cudaStream_t stream = nullptr;
  std::string err;
  double kt = 0.0;           // kappa~ of the box operator
  double mu = 0.0;           // (sigma_out - sigma_in)/(sigma_out + sigma_in)
  double cos_alpha = 0.0;
  double stencil_c[4] = {0, 0, 0, 0};   // coefficients by number of nonzero offsets
  double* stencil_dev = nullptr;         // the same four on the device

  // geometry
  uint8_t* inside = nullptr;
  uint8_t* irr_flag = nullptr;
  int nb = 0;
  double* x[3] = {nullptr, nullptr, nullptr};
  double* nrm[3] = {nullptr, nullptr, nullptr};
  int n_iface = 1;               // interfaces (side labels 1..n_iface)
  int32_t* dof_iface = nullptr;  // [N_b] interface of each DOF
  int32_t* family = nullptr;
  int32_t* edge = nullptr;
  int32_t* axis = nullptr;
  int32_t* st_axis = nullptr;
  int32_t* line_start[3] = {nullptr, nullptr, nullptr};
  int nlines = 0;

  // collocation
  int npde = 0, ndir = 0, nneu = 0, ncoef = 0;
  int32_t* pde_node = nullptr;   // [N_b][npde] linear node index
  int32_t* dir_idx = nullptr;    // [N_b][ndir]
  int32_t* neu_idx = nullptr;    // [N_b][nneu]
  double* minv = nullptr;        // [N_b][ncoef][ncoef], row-major M^{-1}

  // irregular nodes (the rows of the correction terms)
  int nirr = 0;
  int32_t* irr_lin = nullptr;    // [n_irr]
  uint8_t* irr_inside = nullptr; // [n_irr] side label
  // correction entries (node, interface k) holding C^(k); one interface: one
  // per irregular node, entry q = irregular node q
  int nent = 0;
  int32_t* ent_lin = nullptr;    // [n_ent]
  int32_t* ent_iface = nullptr;  // [n_ent]
  int32_t* ent_owner = nullptr;  // [n_ent] closest primary point on interface k
  double* ent_w = nullptr;       // [ncoef][n_ent] composite rows phi(xi)^T M^{-1}
  // [n_nb][n_irr] one interface: entry of an other-side neighbour or -1
  // (C_P = -+ sum c C); several interfaces: entry of C^(l_Q)(Q) (+c)
  int32_t* corr_nb = nullptr;
  int32_t* corr_nb2 = nullptr;   // several interfaces: entry of C^(l_P)(Q) (-c), or -1
  int n_nb = 0;
  int8_t* nb_off = nullptr;      // [n_nb][3] neighbour offsets (setup enumeration order)
  double* nb_coef = nullptr;     // [n_nb] stencil coefficient c of each neighbour

  // traces
  kfbi::TraceCSR tr[2];

  // box solver + work
  kfbi::BoxSolver* box = nullptr;
  double* cvals = nullptr;       // [n_ent]
  double* rhs = nullptr;         // grid
  double* ugrid = nullptr;       // grid
  double* tvals = nullptr;       // [N_b]
  double* ftilde = nullptr;      // grid scratch
  double* bvec = nullptr;        // [N_b]
  int* d_flags = nullptr;        // kFlagCount ints
  kfbi::Gmres gm;
  kfbi::Profiler prof;
  kfbi::MgSolver* mg = nullptr;
  // CUDA graph of one operator application on fixed buffers (xbuf -> ybuf)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t op_graph = nullptr;
  cudaGraphExec_t op_exec = nullptr;
  long long op_counts[KFBI_KC_COUNT] = {};
  double* xbuf = nullptr;
  double* ybuf = nullptr;
  bool use_graphs = true;
  int nx = 0;                    // unknowns of the BIE: N_b, or 2 N_b for the general interface kind
  kfbi_problem* twin = nullptr;  // general interface kind: the kappa_2/sigma_2 operator (owned)
  kfbi_problem* parent = nullptr;  // set on a twin: its launches are counted and timed there
  double* gen = nullptr;         // general interface kind: 8 N_b traces + 3 N_b scaled data
  kfbi::GeoArena arena;          // the geometry's arrays and the set-up's temporaries
};

namespace kfbi {

// ---- error handling ------------------------------------------------------
kfbi_status fail(kfbi_problem* p, kfbi_status s, const std::string& msg);
#define KFBI_CUDA(p, call)                                                       \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return ::kfbi::fail((p), KFBI_ERR_CUDA,                                     \
                          std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)
#define KFBI_TRY(expr)                                                           \
  do {                                                                            \
    kfbi_status s_ = (expr);                                                      \
    if (s_ != KFBI_OK) return s_;                                                 \
  } while (0)

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T) + 16);
}

// the same from the problem's geometry arena (released with the geometry)
template <typename T>
cudaError_t galloc(kfbi_problem* p, T** ptr, size_t count) {
  return arena_alloc(p->arena, count * sizeof(T) + 16, reinterpret_cast<void**>(ptr));
}

inline int div_up(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// Interior BVPs (Dirichlet, Neumann) take f on Omega only, in unit-sigma form
// with sigma_in, and no outer boundary data.
inline bool interior_bvp(const kfbi_problem* p) { return p->cfg.kind != KFBI_INTERFACE_MU; }

// The stream a problem launches on, and its twin with it (graph captures
// switch both to the capture stream and back).
inline void set_stream(kfbi_problem* p, cudaStream_t s) {
  p->stream = s;
  if (p->twin) p->twin->stream = s;
}

// ---- device helpers -------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Totals of four per-lane values over the warp, by a reduce-scatter
// butterfly (6 adds per lane instead of 4 x 5): lane 8 q returns the total of
// s[q], as do the other lanes of its group of 8.
__device__ __forceinline__ double warp_sum4(const double* s) {
  const int lane = threadIdx.x & 31;
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
  double k0 = h4 ? s[2] : s[0], k1 = h4 ? s[3] : s[1];
  const double o0 = h4 ? s[0] : s[2], o1 = h4 ? s[1] : s[3];
  k0 += __shfl_xor_sync(0xffffffffu, o0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, o1, 16);
  double k = h3 ? k1 : k0;
  const double o = h3 ? k0 : k1;
  k += __shfl_xor_sync(0xffffffffu, o, 8);
#pragma unroll
  for (int m = 4; m > 0; m >>= 1) k += __shfl_xor_sync(0xffffffffu, k, m);
  return k;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Graded-lexicographic exponents (total degree ascending, then the exponent of
// x descending, then y descending), the monomial basis of Sec. 5.3.1.
struct Exponents {
  int n;
  int8_t e[kMaxCoef][3];
};
void make_exponents(int d, int p, Exponents* out);

// Scope object bracketing one kernel launch (see Profiler).
struct Launch {
  kfbi_problem* p;
  int cls;
  int rec = -1;
  Launch(kfbi_problem* pp, int c);
  ~Launch();
};

#define KFBI_LAUNCH(p, cls, ...)        \
  do {                                   \
    ::kfbi::Launch launch_((p), (cls));  \
    __VA_ARGS__;                         \
  } while (0)

// ---- launch wrappers implemented in the .cu files ---------------------------
// setup.cu
kfbi_status build_geometry(kfbi_problem* p);
// hotpath.cu
kfbi_status launch_correction_values(kfbi_problem* p, const double* a, const double* b,
                                     const double* ftilde, double* cvals);
kfbi_status launch_collocation_fit(kfbi_problem* p, const double* a, const double* b,
                                   const double* ftilde, double* coef);
kfbi_status launch_rhs(kfbi_problem* p, const double* cvals, const kfbi_data* data,
                       double* rhs);
kfbi_status launch_correction_values_data(kfbi_problem* p, const double* a, const double* b,
                                          const kfbi_data* data, double* cvals);
kfbi_status upload_neighbour_tables(kfbi_problem* p);
kfbi_status launch_traces(kfbi_problem* p, const double* u, const double* cvals,
                          double* vp, double* vm, double* dp, double* dm);
kfbi_status launch_operator_trace(kfbi_problem* p, const double* u, const double* cvals,
                                  const double* x, double alpha_x, double beta_t,
                                  double* y);
kfbi_status launch_set_boundary(kfbi_problem* p, double* u, const double* g_b);
// Neumann BVP with kappa~ = 0 (Sec. 7.2.1): y -= mean(y) over the N_b DOFs;
// a no-op for every other problem.
kfbi_status launch_mean_project(kfbi_problem* p, double* y);
// General interface kind (eq. (bie-ifp-1)): out1 = s1 v, out2 = s2 v
// (N_b values); the combination y[i] = c1 x1[i] + a1 avgV_1 + a2 avgV_2,
// y[N_b + i] = c2 x2[i] + b1 avgDn_1 + b2 avgDn_2 of the two trace sets
// T = [vp1, vm1, dp1, dm1, vp2, vm2, dp2, dm2]; the evaluation data
// s1 = (psi + g2)/sigma_1, s2 = -psi/sigma_2, a = g1 - phi; and the side
// selection u = inside ? u : u2.
kfbi_status launch_gen_scale(kfbi_problem* p, const double* v, double s1, double s2, double* out1,
                             double* out2);
kfbi_status launch_gen_combine(kfbi_problem* p, const double* x1, double c1, const double* x2, double c2,
                               const double* T, double a1, double a2, double b1, double b2, double* y);
kfbi_status launch_gen_eval_prep(kfbi_problem* p, const double* phi, const double* psi, const double* g1,
                                 const double* g2, double* s1, double* s2, double* a);
kfbi_status launch_select_side(kfbi_problem* p, double* u, const double* u2);
// dst.cu / mg.cu
kfbi_status box_create(kfbi_problem* p);
void box_destroy(kfbi_problem* p);
kfbi_status box_solve(kfbi_problem* p, const double* rhs, double* u);
kfbi_status box_last_residual(kfbi_problem* p, double* rel, int* converged);
kfbi_status box_steps(kfbi_problem* p, int* steps, int* cycles);
double* box_tol_dev(kfbi_problem* p);
double box_tol(const kfbi_problem* p);
kfbi_status box_tol_reset(kfbi_problem* p);
kfbi_status box_steps_reset(kfbi_problem* p);
kfbi_status box_steps_total(kfbi_problem* p, long long* out);
// exact fixed-point refinement state (dst.cu), used by the mixed multigrid
struct FixState;
kfbi_status fix_create(kfbi_problem* p, FixState** out);
void fix_destroy(FixState* F);
kfbi_status fix_init(kfbi_problem* p, FixState* F, const float* u0, const double* R, cudaStream_t st);
kfbi_status fix_residual(kfbi_problem* p, FixState* F, float* r32, const int* skip, cudaStream_t st);
kfbi_status fix_add(kfbi_problem* p, FixState* F, const float* e, unsigned long long* corr, const int* skip,
                    cudaStream_t st);
kfbi_status fix_out(kfbi_problem* p, FixState* F, double* u, cudaStream_t st);
// gmres.cu
kfbi_status gmres_create(kfbi_problem* p, int m);
void gmres_destroy(kfbi_problem* p);
kfbi_status apply_operator_fast(kfbi_problem* p, const double* x, double* y);
kfbi_status gmres_run(kfbi_problem* p, const double* b, const double* x0, double rtol,
                      int restart, int max_iter, double* x, int* iters, double* rel,
                      int* x0_rejected = nullptr);
kfbi_status dot_self_pub(kfbi_problem* p, const double* v, double* out);
kfbi_status gmres_init_zero(kfbi_problem* p, const double* b, double bnorm);
kfbi_status gmres_finish(kfbi_problem* p, int k, double* x);
// capi.cu
kfbi_status bie_rhs_impl(kfbi_problem* p, const kfbi_data* data, double* bvec);

// ---- batched pieces (many independent problems in lockstep) -------------------
// One GMRES instance as seen by the batched Arnoldi kernels.
struct ArnDesc {
  double* V;
  int nb, m;
  double* H;
  int ld;
  double* cs;
  double* sn;
  double* g;
  double* res;
  double* x;   // operator input buffer
  double* y;   // operator output buffer
};
// Per-call pointers of one batched instance: its BIE right-hand side, its
// start (NULL = zero) and where its density goes.
struct BatchInst {
  const double* b;
  const double* x0;
  double* out;
};
struct BatchBox;
struct BatchHot;
// dst.cu
kfbi_status batch_box_create(kfbi_problem* p0, kfbi_problem* const* ps, int ninst,
                             double* const* rhs, BatchBox** out, const double* tol_dev = nullptr);
void batch_box_destroy(BatchBox* bb);
kfbi_status batch_box_autotune(kfbi_problem* p0, BatchBox* bb, kfbi_problem* const* ps, double* const* rhs,
                               const int* done, cudaStream_t st);
void batch_box_tiles(const BatchBox* bb, int* pass_ctas, int* row_ctas);
kfbi_status batch_box_solve(kfbi_problem* p0, BatchBox* bb, const int* done, cudaStream_t st);
// hotpath.cu
kfbi_status batch_hot_create(kfbi_problem* p0, kfbi_problem* const* ps, int ninst, double* const* x,
                             double* const* y, double* const* rhs, BatchHot** out);
void batch_hot_destroy(BatchHot* bh);
kfbi_status batch_hot_cvals_rhs(kfbi_problem* p0, BatchHot* bh, cudaStream_t st);
kfbi_status batch_hot_trace(kfbi_problem* p0, BatchHot* bh, cudaStream_t st);
// gmres.cu
kfbi_status batch_arnoldi_copy_in(kfbi_problem* p0, const ArnDesc* d, const int* jdev, const int* done,
                                  int ninst, int maxnb, cudaStream_t st);
kfbi_status batch_arnoldi_step(kfbi_problem* p0, const ArnDesc* d, int* jdev, const int* done,
                               double* res_out, int ninst, int maxnb, int m, cudaStream_t st);
kfbi_status batch_gmres_init(kfbi_problem* p0, const ArnDesc* d, const BatchInst* inst, int n, double rtol,
                             double* thr, double* bn, int* done, int* jdev, int* flags, double* res_out,
                             double omega, const double* base_tol, double* tol, cudaStream_t st);
kfbi_status batch_gmres_control(kfbi_problem* p0, const double* res, const double* thr, int* done, int n, int* ctl,
                                cudaGraphConditionalHandle cond, int use_cond, double omega,
                                const double* base_tol, double* tol, cudaStream_t st);
kfbi_status batch_gmres_finish(kfbi_problem* p0, const ArnDesc* d, const BatchInst* inst, int n, const int* jdev,
                               const int* flags, cudaStream_t st);
void batch_box_copy_tiles(BatchBox* dst, const BatchBox* src);
// batch.cu: the instances of a batch
int batch_size(const kfbi_batch* b);
kfbi_problem* batch_problem(const kfbi_batch* b, int k);

}  // namespace kfbi
