// Matrix-free GMRES on the device (Algorithm 1, Step 4): Arnoldi with
// classical Gram-Schmidt applied twice (CGS2: two block-parallel projections
// instead of j sequential ones), Givens rotations of the Hessenberg column on
// the device, restarts after `restart` steps.  Reductions are two-level and in
// a fixed order, so results are reproducible run to run.  The only host
// transfer per iteration is the residual estimate |g_{j+1}| (8 bytes).
#include <cmath>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

kfbi_status apply_operator_impl(kfbi_problem* p, const double* x, double* y);

namespace {

constexpr int kDotThreads = 256;

// part[i * nchunk + c] = partial dot of V_i and w over chunk c
__global__ void k_dots(const double* __restrict__ V, int nb, int count,
                       const double* __restrict__ w, int nchunk, double* __restrict__ part) {
  const int i = blockIdx.y;
  const int c = blockIdx.x;
  const int per = (nb + nchunk - 1) / nchunk;
  const int b = c * per, e = min(nb, b + per);
  const double* v = V + (size_t)i * nb;
  double s = 0.0;
  for (int k = b + threadIdx.x; k < e; k += blockDim.x) s += v[k] * w[k];
  s = warp_sum(s);
  __shared__ double ws[kDotThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kDotThreads / 32 ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[(size_t)i * nchunk + c] = t;
  }
}

// out[i] = (accumulate ? out[i] : 0) + sum_c part[i * nchunk + c], one block per i
__global__ void k_reduce(const double* __restrict__ part, int nchunk, double* __restrict__ out,
                         int accumulate) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) s += part[(size_t)i * nchunk + c];
  s = warp_sum(s);
  __shared__ double ws[kDotThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kDotThreads / 32 ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[i] = accumulate ? out[i] + t : t;
  }
}

// w -= sum_{i<count} h[i] V_i
__global__ void k_project(const double* __restrict__ V, int nb, int count,
                          const double* __restrict__ h, double* __restrict__ w) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    double s = w[k];
    for (int i = 0; i < count; ++i) s -= h[i] * V[(size_t)i * nb + k];
    w[k] = s;
  }
}

__global__ void k_scale(double* __restrict__ w, int nb, const double* __restrict__ s, int invert) {
  double f = invert ? 1.0 / s[0] : s[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
    w[k] = w[k] * f;
}

__global__ void k_sub(const double* __restrict__ b, double* __restrict__ w, int nb) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
    w[k] = b[k] - w[k];
}

__global__ void k_sqrt(double* s) { s[0] = sqrt(s[0]); }

__global__ void k_add(double* __restrict__ a, const double* __restrict__ b, int k) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) a[i] += b[i];
}

// Hessenberg column j: H[0..j] = h1 + h2, H[j+1] = sqrt(nn); Givens update; res = |g[j+1]|
__global__ void k_givens(double* __restrict__ H, int ld, int j, const double* __restrict__ h1,
                         const double* __restrict__ hn2, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res,
                         double* __restrict__ hnorm) {
  double* col = H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = h1[i];
  double hn = sqrt(hn2[0]);
  col[j + 1] = hn;
  hnorm[0] = hn;
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double rr = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / rr;
  sn[j] = col[j + 1] / rr;
  col[j] = rr;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  res[0] = fabs(g[j + 1]);
}

__global__ void k_init_g(double* g, int m, const double* beta) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta[0] : 0.0;
}

// upper-triangular solve H y = g (k x k)
__global__ void k_solve_y(const double* __restrict__ H, int ld, int k, const double* __restrict__ g,
                          double* __restrict__ y) {
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < k; ++j) s -= H[(size_t)j * ld + i] * y[j];
    y[i] = s / H[(size_t)i * ld + i];
  }
}

// x += sum_{i<k} y[i] V_i
__global__ void k_update_x(const double* __restrict__ V, int nb, int k, const double* __restrict__ y,
                           double* __restrict__ x) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += gridDim.x * blockDim.x) {
    double s = x[e];
    for (int i = 0; i < k; ++i) s += y[i] * V[(size_t)i * nb + e];
    x[e] = s;
  }
}

// One Arnoldi step in one CTA (N_b moderate): w = V_{j+1} holds A v_j on entry.
// CGS2 projections, norm, normalisation and the Givens update of column j.
constexpr int kArnThreads = 1024;

// One Arnoldi step by one CTA (N_b moderate): w = V_{j+1} holds A v_j on entry.
// CGS2 projections (each warp owns whole dot products), norm, normalisation
// and the Givens update of column j; res = |g_{j+1}|.
__device__ void arnoldi_step(double* __restrict__ V, int nb, int j, double* __restrict__ H, int ld,
                             double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                             double* __restrict__ res, double* sm) {
  const int nw = kArnThreads / 32;
  double* part = sm;                       // (j+2) x nw
  double* h = part + (size_t)(j + 2) * nw; // j+2
  double* hacc = h + (j + 2);              // j+2
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* w = V + (size_t)(j + 1) * nb;
  for (int i = tid; i <= j + 1; i += kArnThreads) hacc[i] = 0.0;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = warp; i <= j; i += nw) {
      const double* v = V + (size_t)i * nb;
      double s = 0.0;
      for (int k = lane; k < nb; k += 32) s += v[k] * w[k];
      s = warp_sum(s);
      if (lane == 0) {
        h[i] = s;
        hacc[i] += s;
      }
    }
    __syncthreads();
    for (int k = tid; k < nb; k += kArnThreads) {
      double s = w[k];
      for (int i = 0; i <= j; ++i) s -= h[i] * V[(size_t)i * nb + k];
      w[k] = s;
    }
    __syncthreads();
  }
  double s = 0.0;
  for (int k = tid; k < nb; k += kArnThreads) s += w[k] * w[k];
  s = warp_sum(s);
  if (lane == 0) part[warp] = s;
  __syncthreads();
  if (tid == 0) {
    double nn = 0.0;
    for (int q = 0; q < nw; ++q) nn += part[q];
    double hn = sqrt(nn);
    double* col = H + (size_t)j * ld;
    for (int i = 0; i <= j; ++i) col[i] = hacc[i];
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      double t = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t;
    }
    double rr = hypot(col[j], col[j + 1]);
    cs[j] = col[j] / rr;
    sn[j] = col[j + 1] / rr;
    col[j] = rr;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    res[0] = fabs(g[j + 1]);
    h[0] = hn;
  }
  __syncthreads();
  const double inv = 1.0 / h[0];
  for (int k = tid; k < nb; k += kArnThreads) w[k] *= inv;
}

__global__ void __launch_bounds__(kArnThreads) k_arnoldi_small(
    double* __restrict__ V, int nb, int j, double* __restrict__ H, int ld,
    double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
    double* __restrict__ res) {
  extern __shared__ double sm[];
  arnoldi_step(V, nb, j, H, ld, cs, sn, g, res, sm);
}

}  // namespace

// ---- batched Arnoldi over instances (iteration counters on the device) -------


namespace {

__global__ void k_copy_in_batched(const ArnDesc* __restrict__ D, const int* __restrict__ jdev,
                                  const int* __restrict__ done) {
  const int k = blockIdx.y;
  if (done[k]) return;
  const ArnDesc& a = D[k];
  const double* v = a.V + (size_t)jdev[k] * a.nb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.nb; e += gridDim.x * blockDim.x) a.x[e] = v[e];
}

__global__ void k_copy_out_batched(const ArnDesc* __restrict__ D, const int* __restrict__ jdev,
                                   const int* __restrict__ done) {
  const int k = blockIdx.y;
  if (done[k]) return;
  const ArnDesc& a = D[k];
  if (jdev[k] + 1 > a.m) return;
  double* v = a.V + (size_t)(jdev[k] + 1) * a.nb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.nb; e += gridDim.x * blockDim.x) v[e] = a.y[e];
}

__global__ void __launch_bounds__(kArnThreads) k_arnoldi_batched(const ArnDesc* __restrict__ D,
                                                                 int* __restrict__ jdev,
                                                                 const int* __restrict__ done,
                                                                 double* __restrict__ res_out) {
  extern __shared__ double sm[];
  const int k = blockIdx.x;
  const ArnDesc& a = D[k];
  const int j = jdev[k];
  if (done[k] || j + 1 > a.m) {
    if (threadIdx.x == 0) res_out[k] = a.res[0];
    return;
  }
  arnoldi_step(a.V, a.nb, j, a.H, a.ld, a.cs, a.sn, a.g, a.res, sm);
  if (threadIdx.x == 0) {
    jdev[k] = j + 1;
    res_out[k] = a.res[0];
  }
}

}  // namespace

namespace {

// ---- one GMRES iteration as a graph (moderate N_b) ----------------------------
// CGS2 across many CTAs with the step index j on the device: the Arnoldi step
// of one CTA is bound by that SM's FP64 rate (2 FMA/clk), so the projections
// run on every SM and the Givens update on one CTA.
constexpr int kCgsThreads = 256;

// h[i] = V_i . V_{j+1} for i <= j (CTA i; CTAs beyond j exit)
__global__ void __launch_bounds__(kCgsThreads) k_cgs_dots(const double* __restrict__ V, int nb,
                                                          const int* __restrict__ jdev, double* __restrict__ h) {
  const int j = jdev[0];
  const int i = blockIdx.x;
  if (i > j) return;
  const double* v = V + (size_t)i * nb;
  const double* w = V + (size_t)(j + 1) * nb;
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += kCgsThreads) s += v[k] * w[k];
  s = warp_sum(s);
  __shared__ double ws[kCgsThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kCgsThreads / 32; ++q) t += ws[q];
    h[i] = t;
  }
}

// V_{j+1} -= sum_{i <= j} h[i] V_i; with part: the CTA's sum of squares of the result
__global__ void __launch_bounds__(kCgsThreads) k_cgs_update(double* __restrict__ V, int nb,
                                                            const int* __restrict__ jdev,
                                                            const double* __restrict__ h,
                                                            double* __restrict__ part) {
  const int j = jdev[0];
  __shared__ double hs[kMaxKrylov + 1];
  for (int i = threadIdx.x; i <= j; i += kCgsThreads) hs[i] = h[i];
  __syncthreads();
  double* w = V + (size_t)(j + 1) * nb;
  double acc = 0.0;
  for (int k = blockIdx.x * kCgsThreads + threadIdx.x; k < nb; k += gridDim.x * kCgsThreads) {
    double s = w[k];
    for (int i = 0; i <= j; ++i) s -= hs[i] * V[(size_t)i * nb + k];
    w[k] = s;
    acc += s * s;
  }
  if (!part) return;
  acc = warp_sum(acc);
  __shared__ double ws[kCgsThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kCgsThreads / 32; ++q) t += ws[q];
    part[blockIdx.x] = t;
  }
}

// Hessenberg column j = h1 + h2, h_{j+1,j} = |V_{j+1}| (from the partials, in a
// fixed order), Givens update, res = |g_{j+1}|, scal = 1/h_{j+1,j}, j <- j + 1
// With use_cond (the body of the device-driven loop): the loop continues while
// res > thr and j + 1 < jdev[2], so it ends after at most jdev[2] iterations
// whatever the residual (NaN included).
__global__ void k_cgs_finish(double* __restrict__ H, int ld, double* __restrict__ cs, double* __restrict__ sn,
                             double* __restrict__ g, double* __restrict__ res, const double* __restrict__ h1,
                             const double* __restrict__ h2, const double* __restrict__ part, int npart,
                             int* __restrict__ jdev, double* __restrict__ scal, cudaGraphConditionalHandle cond,
                             int use_cond, const double* __restrict__ thr) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int c = threadIdx.x; c < npart; c += blockDim.x) s += part[c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double nn = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) nn += ws[q];
  const int j = jdev[0];
  double* col = H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  const double hn = sqrt(nn);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rr = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / rr;
  sn[j] = col[j + 1] / rr;
  col[j] = rr;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  res[0] = fabs(g[j + 1]);
  scal[0] = 1.0 / hn;
  jdev[0] = j + 1;
  if (use_cond) cudaGraphSetConditional(cond, (res[0] > thr[0] && j + 1 < jdev[2]) ? 1u : 0u);
}

// Inexact GMRES (relaxation of the operator's accuracy as the residual
// falls, after Simoncini & Szyld 2003 and Bouras & Fraysse 2005): before
// operator application j the refinement tolerance of the mixed box solves
// becomes max(base, omega rtol ||b|| / ||r_j||), with thr = rtol ||b|| and
// res = ||r_j|| the current estimate.  While GMRES runs, res > thr, so the
// tolerance stays below omega.
__global__ void k_relax_tol(const double* __restrict__ thr, const double* __restrict__ res, double omega,
                            double base, double* __restrict__ t1, double* __restrict__ t2) {
  double t = omega * thr[0] / res[0];
  if (!(t > base)) t = base;
  if (t1) *t1 = t;
  if (t2) *t2 = t;
}

// V_j *= scal (j already advanced)
__global__ void k_cgs_normalize(double* __restrict__ V, int nb, const int* __restrict__ jdev,
                                const double* __restrict__ scal) {
  const int j = jdev[0];
  const double f = scal[0];
  double* w = V + (size_t)j * nb;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) w[k] *= f;
}

}  // namespace

// The relaxed refinement tolerance before an operator application inside
// GMRES (k_relax_tol), for the problem and its twin; nothing when relax = 0.
kfbi_status relax_box_tol(kfbi_problem* p) {
  if (!(p->cfg.relax > 0)) return KFBI_OK;
  Gmres& G = p->gm;
  double* t1 = box_tol_dev(p);
  double* t2 = p->twin ? box_tol_dev(p->twin) : nullptr;
  if (t1 || t2)
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_relax_tol<<<1, 1, 0, p->stream>>>(G.scal + 5, G.scal + 2, p->cfg.relax,
                                                                       box_tol(p), t1, t2));
  return KFBI_OK;
}

namespace {

constexpr int kBatchThreads = 256;

// fixed-order sum of one value per thread over a CTA of kBatchThreads
__device__ double cta_sum(double v, double* ws) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < kBatchThreads / 32; ++q) t += ws[q];
  __syncthreads();
  return t;
}

// Start of every instance's GMRES (a CTA per instance): ||b||; with a start x0
// (y = A x0 already in the instance's operator output) r0 = b - y is taken
// when ||r0|| < ||b|| (finite), else the zero start (the single solve's rule);
// V_0 = r/||r||, g = (||r||, 0, ...), threshold rtol ||b||; an instance whose
// start already meets it (or is not finite) is marked done.
// The refinement tolerance of instance k's box solves before its next
// iteration: relaxed as in the single solve (k_relax_tol), base when omega = 0.
__device__ __forceinline__ double relaxed_tol(double omega, double base, double thr, double res) {
  double t = omega * thr / res;
  return omega > 0.0 && t > base ? t : base;
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_init(const ArnDesc* __restrict__ D,
                                                             const BatchInst* __restrict__ I, double rtol,
                                                             double* __restrict__ thr, double* __restrict__ bn,
                                                             int* __restrict__ done, int* __restrict__ jdev,
                                                             int* __restrict__ flags, double* __restrict__ res_out,
                                                             double omega, const double* __restrict__ base_tol,
                                                             double* __restrict__ tol) {
  __shared__ double ws[kBatchThreads / 32];
  __shared__ double sc[2];
  const int k = blockIdx.x;
  const ArnDesc& a = D[k];
  const BatchInst& in = I[k];
  const bool has_x0 = in.x0 != nullptr;
  double sb = 0.0, sr = 0.0;
  for (int e = threadIdx.x; e < a.nb; e += kBatchThreads) {
    const double bv = in.b[e];
    sb += bv * bv;
    if (has_x0) {
      const double r = bv - a.y[e];
      sr += r * r;
    }
  }
  const double bnorm = sqrt(cta_sum(sb, ws));
  const double rnorm = has_x0 ? sqrt(cta_sum(sr, ws)) : 0.0;
  const bool use = has_x0 && rnorm < bnorm;   // false for a NaN residual
  const double beta = use ? rnorm : bnorm;
  if (threadIdx.x == 0) {
    sc[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    sc[1] = beta;
  }
  __syncthreads();
  const double f = sc[0];
  for (int e = threadIdx.x; e < a.nb; e += kBatchThreads)
    a.V[e] = (use ? in.b[e] - a.y[e] : in.b[e]) * f;
  for (int i = threadIdx.x; i <= a.m; i += kBatchThreads) a.g[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    const double t = rtol * bnorm;
    thr[k] = t;
    bn[k] = bnorm;
    flags[k] = has_x0 ? (use ? 1 : 2) : 0;
    done[k] = (beta > t) ? 0 : 1;
    jdev[k] = 0;
    a.res[0] = beta;
    res_out[k] = beta;
    if (tol) tol[k] = relaxed_tol(omega, base_tol[k], t, beta);
  }
}

// After each batched iteration: instances whose residual estimate reached
// their threshold (or is not finite) are marked done; ctl[0] counts the
// iterations, ctl[2] the instances still active; with use_cond the loop
// continues while some instance is active and ctl[0] < ctl[1].
__global__ void __launch_bounds__(kBatchThreads) k_batch_control(const double* __restrict__ res,
                                                                const double* __restrict__ thr,
                                                                int* __restrict__ done, int n,
                                                                int* __restrict__ ctl,
                                                                cudaGraphConditionalHandle cond, int use_cond,
                                                                double omega, const double* __restrict__ base_tol,
                                                                double* __restrict__ tol) {
  __shared__ int wa[kBatchThreads / 32];
  int active = 0;
  for (int k = threadIdx.x; k < n; k += kBatchThreads) {
    if (done[k]) continue;
    if (res[k] > thr[k]) {
      ++active;
      if (tol) tol[k] = relaxed_tol(omega, base_tol[k], thr[k], res[k]);
    } else {
      done[k] = 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) active += __shfl_xor_sync(0xffffffffu, active, o);
  if ((threadIdx.x & 31) == 0) wa[threadIdx.x >> 5] = active;
  __syncthreads();
  if (threadIdx.x != 0) return;
  int tot = 0;
  for (int q = 0; q < kBatchThreads / 32; ++q) tot += wa[q];
  ctl[0] += 1;
  ctl[2] = tot;
  if (use_cond) cudaGraphSetConditional(cond, (tot > 0 && ctl[0] < ctl[1]) ? 1u : 0u);
}

// x = (x0 if taken) + sum_{i < k} y_i V_i with H y = g (k x k upper
// triangular, k = the instance's iterations), a CTA per instance
__global__ void __launch_bounds__(kBatchThreads) k_batch_finish(const ArnDesc* __restrict__ D,
                                                               const BatchInst* __restrict__ I,
                                                               const int* __restrict__ jdev,
                                                               const int* __restrict__ flags) {
  __shared__ double y[kMaxKrylov];
  const int k = blockIdx.x;
  const ArnDesc& a = D[k];
  const BatchInst& in = I[k];
  const int kk = min(jdev[k], a.m);
  if (threadIdx.x == 0) {
    for (int i = kk - 1; i >= 0; --i) {
      double s = a.g[i];
      for (int j = i + 1; j < kk; ++j) s -= a.H[(size_t)j * a.ld + i] * y[j];
      y[i] = s / a.H[(size_t)i * a.ld + i];
    }
  }
  __syncthreads();
  const bool base = flags[k] == 1;
  for (int e = threadIdx.x; e < a.nb; e += kBatchThreads) {
    double s = base ? in.x0[e] : 0.0;
    for (int i = 0; i < kk; ++i) s += y[i] * a.V[(size_t)i * a.nb + e];
    in.out[e] = s;
  }
}

}  // namespace

kfbi_status batch_gmres_init(kfbi_problem* p0, const ArnDesc* d, const BatchInst* inst, int n, double rtol,
                             double* thr, double* bn, int* done, int* jdev, int* flags, double* res_out,
                             double omega, const double* base_tol, double* tol, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_batch_init<<<n, kBatchThreads, 0, st>>>(d, inst, rtol, thr, bn, done, jdev,
                                                                            flags, res_out, omega, base_tol, tol));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status batch_gmres_control(kfbi_problem* p0, const double* res, const double* thr, int* done, int n, int* ctl,
                                cudaGraphConditionalHandle cond, int use_cond, double omega,
                                const double* base_tol, double* tol, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_batch_control<<<1, kBatchThreads, 0, st>>>(res, thr, done, n, ctl, cond,
                                                                               use_cond, omega, base_tol, tol));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status batch_gmres_finish(kfbi_problem* p0, const ArnDesc* d, const BatchInst* inst, int n, const int* jdev,
                               const int* flags, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_batch_finish<<<n, kBatchThreads, 0, st>>>(d, inst, jdev, flags));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status batch_arnoldi_copy_in(kfbi_problem* p0, const ArnDesc* d, const int* jdev, const int* done,
                                  int ninst, int maxnb, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_copy_in_batched<<<dim3(div_up(maxnb, 256), ninst), 256, 0, st>>>(d, jdev, done));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status batch_arnoldi_step(kfbi_problem* p0, const ArnDesc* d, int* jdev, const int* done,
                               double* res_out, int ninst, int maxnb, int m, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_copy_out_batched<<<dim3(div_up(maxnb, 256), ninst), 256, 0, st>>>(d, jdev, done));
  size_t smem = sizeof(double) * ((size_t)(m + 2) * (kArnThreads / 32) + 2 * (size_t)(m + 2));
  KFBI_LAUNCH(p0, KFBI_KC_GMRES, k_arnoldi_batched<<<ninst, kArnThreads, smem, st>>>(d, jdev, done, res_out));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

// Initialise GMRES of instance p with zero start: V_0 = b/|b|, g = (|b|, 0, ...).
kfbi_status gmres_init_zero(kfbi_problem* p, const double* b, double bnorm) {
  Gmres& G = p->gm;
  cudaStream_t st = p->stream;
  const int eb = std::min(div_up(G.nb, 256), 152 * 4);
  KFBI_CUDA(p, cudaMemcpyAsync(G.scal, &bnorm, sizeof(double), cudaMemcpyHostToDevice, st));
  KFBI_CUDA(p, cudaMemcpyAsync(G.V, b, sizeof(double) * G.nb, cudaMemcpyDeviceToDevice, st));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_scale<<<eb, 256, 0, st>>>(G.V, G.nb, G.scal, 1));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_init_g<<<1, 128, 0, st>>>(G.g, G.m, G.scal));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status gmres_norm2(kfbi_problem* p, const double* v, double* out_dev) { return dot_self_pub(p, v, out_dev); }

// x = sum_{i < k} y_i V_i after solving H y = g (k x k)
kfbi_status gmres_finish(kfbi_problem* p, int k, double* x) {
  Gmres& G = p->gm;
  cudaStream_t st = p->stream;
  const int eb = std::min(div_up(G.nb, 256), 152 * 4);
  KFBI_CUDA(p, cudaMemsetAsync(x, 0, sizeof(double) * G.nb, st));
  if (k <= 0) return KFBI_OK;
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_solve_y<<<1, 1, 0, st>>>(G.H, G.m + 1, k, G.g, G.y));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_update_x<<<eb, 256, 0, st>>>(G.V, G.nb, k, G.y, x));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

constexpr int kSmallArnoldi = 32768;   // N_b up to which one CTA runs the Arnoldi step

kfbi_status gmres_create(kfbi_problem* p, int m) {
  Gmres& G = p->gm;
  G.nb = p->nx;   // the BIE's unknowns (2 N_b for the general interface kind)
  G.m = m;
  G.nchunk = std::max(1, std::min(1024, div_up(G.nb, 2048)));
  KFBI_CUDA(p, dalloc(&G.V, (size_t)(m + 1) * G.nb));
  KFBI_CUDA(p, dalloc(&G.H, (size_t)(m + 1) * m));
  KFBI_CUDA(p, dalloc(&G.cs, m));
  KFBI_CUDA(p, dalloc(&G.sn, m));
  KFBI_CUDA(p, dalloc(&G.g, m + 1));
  KFBI_CUDA(p, dalloc(&G.y, m));
  KFBI_CUDA(p, dalloc(&G.part, (size_t)(m + 1) * G.nchunk));
  KFBI_CUDA(p, dalloc(&G.scal, 8));
  KFBI_CUDA(p, dalloc(&G.hcol, 2 * (m + 1)));
  KFBI_CUDA(p, cudaMallocHost(reinterpret_cast<void**>(&G.host_res), 4 * sizeof(double)));
  KFBI_CUDA(p, dalloc(&G.jdev, 4));
  KFBI_CUDA(p, cudaMemset(G.jdev, 0, 4 * sizeof(int)));
  KFBI_CUDA(p, dalloc(&G.h1, m + 1));
  KFBI_CUDA(p, dalloc(&G.h2, m + 1));
  KFBI_CUDA(p, dalloc(&G.npart, 152 * 4));
  return KFBI_OK;
}

void gmres_destroy(kfbi_problem* p) {
  Gmres& G = p->gm;
  cudaFree(G.V);
  cudaFree(G.H);
  cudaFree(G.cs);
  cudaFree(G.sn);
  cudaFree(G.g);
  cudaFree(G.y);
  cudaFree(G.part);
  cudaFree(G.scal);
  cudaFree(G.hcol);
  if (G.host_res) cudaFreeHost(G.host_res);
  if (G.it_exec) cudaGraphExecDestroy(G.it_exec);
  if (G.it_graph) cudaGraphDestroy(G.it_graph);
  if (G.loop_exec) cudaGraphExecDestroy(G.loop_exec);
  if (G.loop_graph) cudaGraphDestroy(G.loop_graph);
  cudaFree(G.jdev);
  cudaFree(G.h1);
  cudaFree(G.h2);
  cudaFree(G.npart);
  cudaFree(G.desc);
  G = Gmres();
}

// ||v||^2 into out[0] (device)
static kfbi_status dot_self(kfbi_problem* p, const double* v, double* out) { return dot_self_pub(p, v, out); }
kfbi_status dot_self_pub(kfbi_problem* p, const double* v, double* out) {
  Gmres& G = p->gm;
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_dots<<<dim3(G.nchunk, 1), kDotThreads, 0, p->stream>>>(v, G.nb, 1, v, G.nchunk, G.part));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_reduce<<<1, kDotThreads, 0, p->stream>>>(G.part, G.nchunk, out, 0));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status read_scalar(kfbi_problem* p, const double* dev, double* host) {
  KFBI_CUDA(p, cudaMemcpyAsync(p->gm.host_res, dev, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  *host = p->gm.host_res[0];
  return KFBI_OK;
}

// The kernels of one GMRES iteration of problem p on its stream: x = V_j;
// y = A x (the operator's kernels); V_{j+1} = y; CGS2 over all SMs; Givens;
// normalise; j <- j + 1.  With use_cond the finish kernel also sets the
// condition of the enclosing device-driven loop.
static kfbi_status iteration_body(kfbi_problem* p, cudaGraphConditionalHandle cond, int use_cond) {
  Gmres& G = p->gm;
  const int nb = G.nb;
  const int eb = std::min(div_up(nb, kCgsThreads), 152 * 4);
  const ArnDesc* d = static_cast<const ArnDesc*>(G.desc);
  const int* done = G.jdev + 1;
  KFBI_TRY(batch_arnoldi_copy_in(p, d, G.jdev, done, 1, nb, p->stream));
  KFBI_TRY(relax_box_tol(p));
  KFBI_TRY(apply_operator_impl(p, p->xbuf, p->ybuf));
  cudaStream_t cs = p->stream;
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_copy_out_batched<<<dim3(div_up(nb, 256), 1), 256, 0, cs>>>(d, G.jdev, done));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_dots<<<G.m + 1, kCgsThreads, 0, cs>>>(G.V, nb, G.jdev, G.h1));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_update<<<eb, kCgsThreads, 0, cs>>>(G.V, nb, G.jdev, G.h1, nullptr));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_dots<<<G.m + 1, kCgsThreads, 0, cs>>>(G.V, nb, G.jdev, G.h2));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_update<<<eb, kCgsThreads, 0, cs>>>(G.V, nb, G.jdev, G.h2, G.npart));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_finish<<<1, 256, 0, cs>>>(G.H, G.m + 1, G.cs, G.sn, G.g, G.scal + 2, G.h1,
                                                                 G.h2, G.npart, eb, G.jdev, G.scal + 3, cond,
                                                                 use_cond, G.scal + 5));
  KFBI_LAUNCH(p, KFBI_KC_GMRES, k_cgs_normalize<<<eb, 256, 0, cs>>>(G.V, nb, G.jdev, G.scal + 3));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status ensure_desc(kfbi_problem* p) {
  Gmres& G = p->gm;
  if (!p->cap_stream) KFBI_CUDA(p, cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  if (!G.desc) {
    ArnDesc d{G.V, G.nb, G.m, G.H, G.m + 1, G.cs, G.sn, G.g, G.scal + 2, p->xbuf, p->ybuf};
    ArnDesc* dd = nullptr;
    KFBI_CUDA(p, dalloc(&dd, 1));
    KFBI_CUDA(p, cudaMemcpy(dd, &d, sizeof(d), cudaMemcpyHostToDevice));
    G.desc = dd;
  }
  return KFBI_OK;
}

// Capture iteration_body on the private stream, into `into` when given
// (cudaStreamBeginCaptureToGraph), else into a new graph returned in *out.
static kfbi_status capture_body(kfbi_problem* p, cudaGraph_t into, cudaGraph_t* out,
                                cudaGraphConditionalHandle cond, int use_cond) {
  Gmres& G = p->gm;
  cudaStream_t st = p->stream;
  KFBI_CUDA(p, cudaStreamSynchronize(st));
  long long before[KFBI_KC_COUNT];
  for (int k = 0; k < KFBI_KC_COUNT; ++k) before[k] = p->prof.launches[k];
  const bool prof = p->prof.on;
  p->prof.on = false;
  set_stream(p, p->cap_stream);
  kfbi_status s = KFBI_OK;
  cudaError_t e = into ? cudaStreamBeginCaptureToGraph(p->cap_stream, into, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal)
                       : cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) s = iteration_body(p, cond, use_cond);
  cudaGraph_t gr = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(p->cap_stream, &gr) : e;
  set_stream(p, st);
  p->prof.on = prof;
  for (int k = 0; k < KFBI_KC_COUNT; ++k) {
    G.it_counts[k] = p->prof.launches[k] - before[k];
    p->prof.launches[k] = before[k];
  }
  if (e != cudaSuccess || e2 != cudaSuccess || s != KFBI_OK) {
    if (gr && !into) cudaGraphDestroy(gr);
    cudaGetLastError();
    return s != KFBI_OK ? s : fail(p, KFBI_ERR_CUDA, "GMRES iteration capture failed");
  }
  *out = gr;
  return KFBI_OK;
}

// One GMRES iteration of problem p as a graph, replayed once per iteration.
static kfbi_status iteration_graph(kfbi_problem* p) {
  Gmres& G = p->gm;
  if (G.it_exec) return KFBI_OK;
  KFBI_TRY(ensure_desc(p));
  cudaGraph_t gr = nullptr;
  KFBI_TRY(capture_body(p, nullptr, &gr, 0, 0));
  G.it_graph = gr;
  KFBI_CUDA(p, cudaGraphInstantiate(&G.it_exec, gr, 0));
  return KFBI_OK;
}

// The whole Arnoldi cycle on the device: a conditional WHILE node whose body is
// one iteration; the finish kernel ends the loop when the residual estimate
// reaches the threshold or after the iteration limit jdev[2], so the host
// synchronises once per cycle instead of once per iteration.  Returns false
// (the caller then replays the single-iteration graph) if the driver refuses
// conditional nodes.
static bool loop_graph(kfbi_problem* p) {
  Gmres& G = p->gm;
  if (G.loop_exec) return true;
  if (G.loop_failed) return false;
  G.loop_failed = true;
  if (ensure_desc(p) != KFBI_OK) return false;
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
  cudaGraph_t body = ok ? np.conditional.phGraph_out[0] : nullptr;
  cudaGraph_t captured = nullptr;
  if (ok) ok = capture_body(p, body, &captured, h, 1) == KFBI_OK;
  if (ok) ok = cudaGraphInstantiate(&G.loop_exec, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    G.loop_exec = nullptr;
    return false;
  }
  G.loop_graph = g;
  G.loop_failed = false;
  return true;
}

kfbi_status gmres_run(kfbi_problem* p, const double* b, const double* x0, double rtol, int restart,
                      int max_iter, double* x, int* iters, double* rel, int* x0_rejected) {
  Gmres& G = p->gm;
  const int nb = G.nb;
  const int m = std::max(1, std::min(restart, G.m));
  const int ld = G.m + 1;
  cudaStream_t st = p->stream;
  const int eb = std::min(div_up(nb, 256), 152 * 4);
  double* beta = G.scal + 0;
  double* bn2 = G.scal + 1;
  double* res = G.scal + 2;
  double* hn2 = G.scal + 3;
  double* hnorm = G.scal + 4;
  double* h1 = G.hcol;
  double* h2 = G.hcol + (G.m + 1);
  KFBI_TRY(dot_self(p, b, bn2));
  double bnorm2;
  KFBI_TRY(read_scalar(p, bn2, &bnorm2));
  const double bnorm = std::sqrt(bnorm2);
  *iters = 0;
  *rel = 0.0;
  if (x0_rejected) *x0_rejected = 0;
  if (!std::isfinite(bnorm)) return fail(p, KFBI_ERR_NONFINITE, "non-finite BIE right-hand side");
  if (bnorm == 0.0) {
    KFBI_CUDA(p, cudaMemsetAsync(x, 0, sizeof(double) * nb, st));
    return KFBI_OK;
  }
  if (x0) {
    if (x0 != x) KFBI_CUDA(p, cudaMemcpyAsync(x, x0, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
  } else {
    KFBI_CUDA(p, cudaMemsetAsync(x, 0, sizeof(double) * nb, st));
  }
  bool nonzero_x = x0 != nullptr;
  int total = 0;
  for (;;) {
    double* V0 = G.V;
    if (nonzero_x) {
      // the residual of a start or a restart at the full box-solve accuracy
      KFBI_TRY(box_tol_reset(p));
      if (p->twin) KFBI_TRY(box_tol_reset(p->twin));
      KFBI_TRY(apply_operator_fast(p, x, V0));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_sub<<<eb, 256, 0, st>>>(b, V0, nb));
    } else {
      KFBI_CUDA(p, cudaMemcpyAsync(V0, b, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
    }
    KFBI_TRY(dot_self(p, V0, beta));
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_sqrt<<<1, 1, 0, st>>>(beta));
    double hbeta;
    KFBI_TRY(read_scalar(p, beta, &hbeta));
    if (!std::isfinite(hbeta) && !(total == 0 && x0)) return fail(p, KFBI_ERR_NONFINITE, "non-finite GMRES residual");
    if (total == 0 && nonzero_x && x0 && !(hbeta < bnorm)) {
      // the initial guess is no better than zero: start from zero instead
      if (x0_rejected) *x0_rejected = 1;
      KFBI_CUDA(p, cudaMemsetAsync(x, 0, sizeof(double) * nb, st));
      nonzero_x = false;
      continue;
    }
    if (hbeta <= rtol * bnorm) {
      *iters = total;
      *rel = hbeta / bnorm;
      return KFBI_OK;
    }
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_scale<<<eb, 256, 0, st>>>(V0, nb, beta, 1));
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_init_g<<<1, 128, 0, st>>>(G.g, G.m, beta));
    // the residual estimate starts at beta and the threshold is rtol ||b||
    // (both read on the device by the loop and by the relaxation)
    {
      const double thr0 = rtol * bnorm;
      KFBI_CUDA(p, cudaMemcpyAsync(res, beta, sizeof(double), cudaMemcpyDeviceToDevice, st));
      KFBI_CUDA(p, cudaMemcpyAsync(G.scal + 5, &thr0, sizeof(double), cudaMemcpyHostToDevice, st));
    }
    int jend = 0;
    double hres = hbeta;
    const bool graph_it = nb <= kGraphArnoldi && p->use_graphs && !p->prof.on;
    if (graph_it && loop_graph(p)) {
      // one launch runs the cycle: at most min(m, max_iter - total) iterations
      const int jmax = std::min(m, max_iter - total);
      const int head[3] = {0, 0, jmax};
      const double thr = rtol * bnorm;
      KFBI_CUDA(p, cudaMemcpyAsync(G.jdev, head, sizeof(head), cudaMemcpyHostToDevice, st));
      KFBI_CUDA(p, cudaMemcpyAsync(G.scal + 5, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
      KFBI_CUDA(p, cudaGraphLaunch(G.loop_exec, st));
      int jdone = 0;
      KFBI_CUDA(p, cudaMemcpyAsync(G.host_res, res, sizeof(double), cudaMemcpyDeviceToHost, st));
      KFBI_CUDA(p, cudaMemcpyAsync(&jdone, G.jdev, sizeof(int), cudaMemcpyDeviceToHost, st));
      KFBI_CUDA(p, cudaStreamSynchronize(st));
      hres = G.host_res[0];
      if (jdone < 1 || jdone > jmax) return fail(p, KFBI_ERR_CUDA, "device-driven GMRES loop lost its step count");
      for (int k = 0; k < KFBI_KC_COUNT; ++k) p->prof.launches[k] += G.it_counts[k] * jdone;
      total += jdone;
      jend = jdone;
      if (!std::isfinite(hres)) return fail(p, KFBI_ERR_NONFINITE, "non-finite GMRES residual");
    } else if (graph_it) {
      KFBI_TRY(iteration_graph(p));
      KFBI_CUDA(p, cudaMemsetAsync(G.jdev, 0, 3 * sizeof(int), st));
    }
    const bool stepwise = !(graph_it && G.loop_exec);
    for (int j = 0; stepwise && j < m; ++j) {
      double* Vj = G.V + (size_t)j * nb;
      double* w = G.V + (size_t)(j + 1) * nb;
      if (graph_it) {
        KFBI_CUDA(p, cudaGraphLaunch(G.it_exec, st));
        for (int k = 0; k < KFBI_KC_COUNT; ++k) p->prof.launches[k] += G.it_counts[k];
        ++total;
        KFBI_TRY(read_scalar(p, res, &hres));
        jend = j + 1;
        if (!std::isfinite(hres)) return fail(p, KFBI_ERR_NONFINITE, "non-finite GMRES residual");
        if (hres <= rtol * bnorm || total >= max_iter) break;
        continue;
      }
      KFBI_TRY(relax_box_tol(p));
      KFBI_TRY(apply_operator_fast(p, Vj, w));
      ++total;
      if (nb <= kSmallArnoldi) {
        size_t smem = sizeof(double) * ((size_t)(j + 2) * (kArnThreads / 32) + 2 * (size_t)(j + 2));
        KFBI_LAUNCH(p, KFBI_KC_GMRES, k_arnoldi_small<<<1, kArnThreads, smem, st>>>(
            G.V, nb, j, G.H, ld, G.cs, G.sn, G.g, res));
        KFBI_CUDA(p, cudaGetLastError());
        KFBI_TRY(read_scalar(p, res, &hres));
        jend = j + 1;
        if (!std::isfinite(hres)) return fail(p, KFBI_ERR_NONFINITE, "non-finite GMRES residual");
        if (hres <= rtol * bnorm || total >= max_iter) break;
        continue;
      }
      // CGS2: h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_dots<<<dim3(G.nchunk, j + 1), kDotThreads, 0, st>>>(G.V, nb, j + 1, w, G.nchunk, G.part));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_reduce<<<j + 1, kDotThreads, 0, st>>>(G.part, G.nchunk, h1, 0));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_project<<<eb, 256, 0, st>>>(G.V, nb, j + 1, h1, w));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_dots<<<dim3(G.nchunk, j + 1), kDotThreads, 0, st>>>(G.V, nb, j + 1, w, G.nchunk, G.part));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_reduce<<<j + 1, kDotThreads, 0, st>>>(G.part, G.nchunk, h2, 0));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_project<<<eb, 256, 0, st>>>(G.V, nb, j + 1, h2, w));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_add<<<1, 128, 0, st>>>(h1, h2, j + 1));
      KFBI_TRY(dot_self(p, w, hn2));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_givens<<<1, 1, 0, st>>>(G.H, ld, j, h1, hn2, G.cs, G.sn, G.g, res, hnorm));
      KFBI_LAUNCH(p, KFBI_KC_GMRES, k_scale<<<eb, 256, 0, st>>>(w, nb, hnorm, 1));
      KFBI_CUDA(p, cudaGetLastError());
      KFBI_TRY(read_scalar(p, res, &hres));
      jend = j + 1;
      if (!std::isfinite(hres)) return fail(p, KFBI_ERR_NONFINITE, "non-finite GMRES residual");
      if (hres <= rtol * bnorm || total >= max_iter) break;
    }
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_solve_y<<<1, 1, 0, st>>>(G.H, ld, jend, G.g, G.y));
    KFBI_LAUNCH(p, KFBI_KC_GMRES, k_update_x<<<eb, 256, 0, st>>>(G.V, nb, jend, G.y, x));
    KFBI_CUDA(p, cudaGetLastError());
    nonzero_x = true;
    *iters = total;
    *rel = hres / bnorm;
    if (hres <= rtol * bnorm) {
      KFBI_CUDA(p, cudaStreamSynchronize(st));
      return KFBI_OK;
    }
    if (total >= max_iter)
      return fail(p, KFBI_ERR_NOT_CONVERGED,
                  "GMRES reached max_iter = " + std::to_string(max_iter) +
                      " (relative residual " + std::to_string(hres / bnorm) + ")");
  }
}

}  // namespace kfbi
