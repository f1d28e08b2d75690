// Hot-path kernels of one operator application (Algorithm 1, Step 3):
//   3.1+  correction function C at every irregular node from the collocation
//         data of its closest primary point (composite rows phi(xi)^T M^{-1},
//         so the local polynomial of Sec. 5.3.1 is fitted and evaluated in one
//         pass);
//   3.2   corrected right-hand side of eq. (corrected-FDS) with the correction
//         terms of eq. (crc-formula);
//   3.4   corrected interpolation of the traces (Sec. 5.5), fused with the BIE
//         combination y = alpha x + beta t.
// All arithmetic is FP64.
#include "kfbi_internal.cuh"

namespace kfbi {

namespace {

// C(q) = sum_j W[j][q] Q_j, Q = [h^2 f~(PDE nodes); a(Dirichlet DOFs); h b(Neumann DOFs)]
// of the owner's collocation system (eq. (cau-ls)), one thread per correction
// entry.  f~ = fa/sa - fb/sb at the PDE nodes (either pointer may be null);
// fa holds one grid per interface when fstride > 0 (the entry's interface's).
__global__ void k_cvals(int nirr, int npde, int ndir, int nneu, double h,
                        const int32_t* __restrict__ owner, const double* __restrict__ W,
                        const int32_t* __restrict__ pde_node, const int32_t* __restrict__ dir_idx,
                        const int32_t* __restrict__ neu_idx, const double* __restrict__ a,
                        const double* __restrict__ b, const double* __restrict__ fa, double sa,
                        const double* __restrict__ fb, double sb, double* __restrict__ out,
                        const int32_t* __restrict__ eiface, long long fstride) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  int i = owner[q];
  if (fa && fstride) fa += eiface[q] * fstride;
  double acc = 0.0;
  int j = 0;
  if (fa != nullptr || fb != nullptr) {
    double h2 = h * h;
    for (int s = 0; s < npde; ++s, ++j) {
      int node = pde_node[i * npde + s];
      double ft = 0.0;
      if (fa) ft = fa[node] / sa;
      if (fb) ft = ft - fb[node] / sb;
      acc += W[(size_t)j * nirr + q] * (h2 * ft);
    }
  } else {
    j = npde;
  }
  if (a != nullptr) {
    for (int s = 0; s < ndir; ++s, ++j) acc += W[(size_t)j * nirr + q] * a[dir_idx[i * ndir + s]];
  } else {
    j += ndir;
  }
  if (b != nullptr) {
    for (int s = 0; s < nneu; ++s, ++j)
      acc += W[(size_t)j * nirr + q] * (h * b[neu_idx[i * nneu + s]]);
  }
  out[q] = acc;
}

// d_i = M_i^{-1} Q_i, one warp per primary point (stage output).
__global__ void k_coef(int nb, int nc, int npde, int ndir, int nneu, double h,
                       const double* __restrict__ minv, const int32_t* __restrict__ pde_node,
                       const int32_t* __restrict__ dir_idx, const int32_t* __restrict__ neu_idx,
                       const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ ft, double* __restrict__ coef) {
  int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= nb) return;
  __shared__ double Qs[8][kMaxCoef];
  double* Q = Qs[threadIdx.x / 32];
  for (int j = lane; j < nc; j += 32) {
    double v;
    if (j < npde) {
      v = ft ? (h * h) * ft[pde_node[i * npde + j]] : 0.0;
    } else if (j < npde + ndir) {
      v = a ? a[dir_idx[i * ndir + (j - npde)]] : 0.0;
    } else {
      v = b ? h * b[neu_idx[i * nneu + (j - npde - ndir)]] : 0.0;
    }
    Q[j] = v;
  }
  __syncwarp();
  const double* M = minv + (size_t)i * nc * nc;
  for (int k = lane; k < nc; k += 32) {
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s += M[k * nc + j] * Q[j];
    coef[(size_t)i * nc + k] = s;
  }
}

// R = F + h^2/12 Lap F (order 4) from each node's own side, minus the lift of
// the outer boundary data, at interior nodes; 0 on the boundary layer.  The
// coefficient divisions are reciprocals from the host and the node indices
// are 32-bit (grids of up to 1025^3 nodes): FP64 divides and 64-bit integer
// divides run as long FP64-pipe sequences on GB300.
__global__ void k_rhs_source(Grid g, int order, const uint8_t* __restrict__ inside,
                             const double* __restrict__ fi, const double* __restrict__ fo,
                             const double* __restrict__ li, const double* __restrict__ lo_,
                             double rsi, double rso, double h2_12, const double* __restrict__ gb,
                             const double* __restrict__ nbc, const int8_t* __restrict__ nboff,
                             int nnb, double* __restrict__ R, long long fstride) {
  const int tot = (int)g.nodes();
  const int n1 = g.n + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    int idx[3];
    if (g.d == 2) {
      idx[1] = t % n1;
      idx[0] = t / n1;
      idx[2] = 1;
    } else {
      const int r = t / n1;
      idx[2] = t - r * n1;
      idx[1] = r % n1;
      idx[0] = r / n1;
    }
    bool interior = idx[0] >= 1 && idx[0] < g.n && idx[1] >= 1 && idx[1] < g.n &&
                    (g.d == 2 || (idx[2] >= 1 && idx[2] < g.n));
    if (!interior) {
      R[t] = 0.0;
      continue;
    }
    double v = 0.0;
    const int lab = inside[t];
    const bool in = lab != 0;
    // f of the node's own side (of its interface's component with fstride > 0)
    const long long off = in ? (long long)(lab - 1) * fstride : 0;
    const double* F = in ? (fi ? fi + off : nullptr) : fo;
    const double* Lp = in ? (li ? li + off : nullptr) : lo_;
    const double rs = in ? rsi : rso;
    if (F) v = F[t] * rs;
    if (order == 4 && Lp) v = v + h2_12 * (Lp[t] * rs);
    if (gb) {
      bool near = idx[0] == 1 || idx[0] == g.n - 1 || idx[1] == 1 || idx[1] == g.n - 1 ||
                  (g.d == 3 && (idx[2] == 1 || idx[2] == g.n - 1));
      if (near) {
        double lift = 0.0;
        for (int k = 0; k < nnb; ++k) {
          int q0 = idx[0] + nboff[3 * k], q1 = idx[1] + nboff[3 * k + 1];
          int q2 = g.d == 3 ? idx[2] + nboff[3 * k + 2] : 0;
          bool bnd = q0 == 0 || q0 == g.n || q1 == 0 || q1 == g.n ||
                     (g.d == 3 && (q2 == 0 || q2 == g.n));
          if (!bnd) continue;
          const int qi = g.d == 2 ? q0 * n1 + q1 : (q0 * n1 + q1) * n1 + q2;
          lift += nbc[k] * gb[qi];
        }
        v = v - lift;
      }
    }
    R[t] = v;
  }
}

// R[P] += C_P (eq. (crc-formula)): -sum c C(Q) over outside Q if P is inside,
// +sum c C(Q) over inside Q if P is outside.
__global__ void k_rhs_correct(int nirr, int nnb, const int32_t* __restrict__ lin,
                              const uint8_t* __restrict__ irr_inside,
                              const int32_t* __restrict__ corr_nb, const double* __restrict__ nbc,
                              const double* __restrict__ cv, double* __restrict__ R, int add) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  double acc = 0.0;
  for (int s = 0; s < nnb; ++s) {
    int j = corr_nb[(size_t)s * nirr + q];
    if (j >= 0) acc += nbc[s] * cv[j];
  }
  double c = irr_inside[q] ? -acc : acc;
  long long t = lin[q];
  R[t] = add ? R[t] + c : c;
}

// Several interfaces: R[P] += -sum_{l_Q != l_P} c (C^(l_P)(Q) - C^(l_Q)(Q)),
// i.e. + c C^(l_Q)(Q) - c C^(l_P)(Q) with C^(0) = 0 (entries -1).
__global__ void k_rhs_correct_multi(int nirr, int nnb, const int32_t* __restrict__ lin,
                                    const int32_t* __restrict__ corr_a,
                                    const int32_t* __restrict__ corr_b,
                                    const double* __restrict__ nbc, const double* __restrict__ cv,
                                    double* __restrict__ R) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  double acc = 0.0;
  for (int s = 0; s < nnb; ++s) {
    const int ja = corr_a[(size_t)s * nirr + q];
    const int jb = corr_b[(size_t)s * nirr + q];
    if (ja >= 0 || jb >= 0) acc += nbc[s] * ((ja >= 0 ? cv[ja] : 0.0) - (jb >= 0 ? cv[jb] : 0.0));
  }
  R[lin[q]] += acc;
}

// The corrected datum of trace stencil entry e: one interface, u + C across
// Gamma on the '+' side, u - C on the '-' side (MINUS); several interfaces
// u + (C^(t) - C^(l_q)) across, C^(0) = 0.
template <bool MULTI, bool MINUS>
__device__ __forceinline__ double trace_datum(const TraceCSR& T, int e,
                                              const double* __restrict__ u,
                                              const double* __restrict__ cv) {
  double w = u[T.node[e]];
  const int j = T.irr[e];
  if (!MULTI) {
    if (j >= 0) w = MINUS ? w - cv[j] : w + cv[j];
  } else {
    const int j2 = T.irr2[e];
    if (j >= 0 || j2 >= 0) w += (j >= 0 ? cv[j] : 0.0) - (j2 >= 0 ? cv[j2] : 0.0);
  }
  return w;
}

// Four one-sided traces (stage output), one warp per DOF.
template <bool MULTI>
__global__ void k_traces4(int nb, TraceCSR tp, TraceCSR tm, const double* __restrict__ u,
                          const double* __restrict__ cv, double* vp, double* vm, double* dp,
                          double* dm) {
  int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= nb) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = tp.ptr[i] + lane; e < tp.ptr[i + 1]; e += 32) {
    const double w = trace_datum<MULTI, false>(tp, e, u, cv);
    s[0] += tp.wv[e] * w;
    s[1] += tp.wn[e] * w;
  }
  for (int e = tm.ptr[i] + lane; e < tm.ptr[i + 1]; e += 32) {
    const double w = trace_datum<MULTI, true>(tm, e, u, cv);
    s[2] += tm.wv[e] * w;
    s[3] += tm.wn[e] * w;
  }
  // lane 8 q holds sum q: value+, d_n+, value-, d_n-
  const double t = warp_sum4(s);
  double* out = (lane >> 3) == 0 ? vp : (lane >> 3) == 1 ? dp : (lane >> 3) == 2 ? vm : dm;
  if ((lane & 7) == 0 && out) out[i] = t;
}

// ---- the 3D trace sums in FP32 pairs ------------------------------------------
// GB300 issues FP64 at 2 lanes per clock per SM against 128 for FP32, and the
// 3D trace kernels spend their time there (two FMAs per stencil entry).  Their
// sums run here in "double-float" arithmetic on the FP32 pipe instead: a value
// is an unevaluated pair hi + lo of floats (~48 bits), products use the exact
// FMA residual, sums the error-free two-sum (Dekker 1971; Knuth, TAOCP vol. 2,
// 4.2.2); every step is written with the _rn intrinsics so that no product
// and sum are contracted into an FMA.
struct DFlt {
  float hi, lo;
};

// An FP64 value as hi + lo: hi its leading 24 bits, lo the next 23, both
// assembled from the bit pattern with integer operations (the FP64-to-FP32
// conversion would issue to the FP64 pipe).  |x| < 2^-126 gives 0 (far below
// any term of a trace sum), non-finite values stay non-finite in hi.
__device__ __forceinline__ float2 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7ffu);
  if (e == 0x7ff)
    return make_float2(__uint_as_float(sign | 0x7f800000u | (((h32 & 0xfffffu) | l32) ? 0x400000u : 0u)), 0.f);
  const int fe = e - 896;                          // FP32 exponent field of x
  if (fe <= 0) return make_float2(0.f, 0.f);
  if (fe >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29));
  // the remaining 29 mantissa bits are r 2^(e - 1075); their top 23 bits,
  // (r >> 6) 2^(e - 1069), are exact in FP32
  const unsigned r = (l32 & 0x1fffffffu) >> 6;
  const float rf = __fsub_rn(__uint_as_float(0x4b000000u | r), 8388608.f);
  const int le = e - 942;                          // FP32 exponent field of 2^(e - 1069)
  float lo = le > 0 ? __fmul_rn(rf, __uint_as_float((unsigned)le << 23)) : 0.f;
  return make_float2(hi, sign ? -lo : lo);
}

// acc += w u (w, u as pairs; the lo x lo product is dropped)
__device__ __forceinline__ void df_fma(DFlt& acc, float2 w, float2 u) {
  const float p = __fmul_rn(w.x, u.x);
  float e = __fmaf_rn(w.x, u.x, -p);
  e = __fmaf_rn(w.x, u.y, e);
  e = __fmaf_rn(w.y, u.x, e);
  const float t = __fadd_rn(acc.hi, p);
  const float z = __fsub_rn(t, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
  acc.hi = t;
}

__device__ __forceinline__ DFlt df_add(DFlt a, DFlt b) {
  const float t = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(t, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(b.hi, z));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  // renormalise (fast two-sum: |t| >= |lo|)
  const float s = __fadd_rn(t, lo);
  return DFlt{s, __fsub_rn(lo, __fsub_rn(s, t))};
}

__device__ __forceinline__ DFlt df_shfl_xor(DFlt a, int m) {
  return DFlt{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

__device__ __forceinline__ double df_value(DFlt a) { return (double)a.hi + (double)a.lo; }

// One stencil entry into the pair sums of the value and normal-derivative
// weights: w (u + corrections), the corrections C as in trace_datum, each its
// own product.
template <bool MULTI, bool MINUS>
__device__ __forceinline__ void trace_entry2_df(const TraceCSR& T, int e, const double* __restrict__ u,
                                                const double* __restrict__ cv, DFlt& av, DFlt& an) {
  const float2 wv = T.wv2[e], wn = T.wn2[e];
  const float2 uu = split_f64(u[T.node[e]]);
  df_fma(av, wv, uu);
  df_fma(an, wn, uu);
  const int j = T.irr[e];
  if (!MULTI) {
    if (j >= 0) {
      float2 c = split_f64(cv[j]);
      if (MINUS) c = make_float2(-c.x, -c.y);
      df_fma(av, wv, c);
      df_fma(an, wn, c);
    }
  } else {
    const int j2 = T.irr2[e];
    if (j >= 0) {
      const float2 c = split_f64(cv[j]);
      df_fma(av, wv, c);
      df_fma(an, wn, c);
    }
    if (j2 >= 0) {
      float2 c = split_f64(cv[j2]);
      c = make_float2(-c.x, -c.y);
      df_fma(av, wv, c);
      df_fma(an, wn, c);
    }
  }
}

// k_traces4 in pair arithmetic (3D), the four sums reduced by the same
// reduce-scatter butterfly as warp_sum4
template <bool MULTI>
__global__ void k_traces4_df(int nb, TraceCSR tp, TraceCSR tm, const double* __restrict__ u,
                             const double* __restrict__ cv, double* vp, double* vm, double* dp,
                             double* dm) {
  int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= nb) return;
  DFlt s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int e = tp.ptr[i] + lane; e < tp.ptr[i + 1]; e += 32)
    trace_entry2_df<MULTI, false>(tp, e, u, cv, s[0], s[1]);
  for (int e = tm.ptr[i] + lane; e < tm.ptr[i + 1]; e += 32)
    trace_entry2_df<MULTI, true>(tm, e, u, cv, s[2], s[3]);
  for (int q = 0; q < 4; ++q) s[q] = df_add(s[q], DFlt{0.f, 0.f});
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
  DFlt k0 = h4 ? s[2] : s[0], k1 = h4 ? s[3] : s[1];
  const DFlt o0 = h4 ? s[0] : s[2], o1 = h4 ? s[1] : s[3];
  k0 = df_add(k0, df_shfl_xor(o0, 16));
  k1 = df_add(k1, df_shfl_xor(o1, 16));
  DFlt k = h3 ? k1 : k0;
  const DFlt o = h3 ? k0 : k1;
  k = df_add(k, df_shfl_xor(o, 8));
#pragma unroll
  for (int m = 4; m > 0; m >>= 1) k = df_add(k, df_shfl_xor(k, m));
  double* out = (lane >> 3) == 0 ? vp : (lane >> 3) == 1 ? dp : (lane >> 3) == 2 ? vm : dm;
  if ((lane & 7) == 0 && out) out[i] = df_value(k);
}

// The operator's trace quantity t (average value for the Dirichlet form,
// average normal derivative for the mu-form; weights carry the 1/2) fused with
// the BIE combination y = alpha x + beta t.
template <bool MULTI>
__global__ void k_trace_op(int nb, TraceCSR tp, TraceCSR tm, const double* __restrict__ u,
                           const double* __restrict__ cv, const double* __restrict__ x,
                           double alpha, double beta, double* __restrict__ y) {
  int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= nb) return;
  double acc = 0.0;
  for (int e = tp.ptr[i] + lane; e < tp.ptr[i + 1]; e += 32)
    acc += tp.w[e] * trace_datum<MULTI, false>(tp, e, u, cv);
  for (int e = tm.ptr[i] + lane; e < tm.ptr[i + 1]; e += 32)
    acc += tm.w[e] * trace_datum<MULTI, true>(tm, e, u, cv);
  acc = warp_sum(acc);
  if (lane == 0) y[i] = (x ? alpha * x[i] : 0.0) + beta * acc;
}

// y -= mean(y): one CTA, each thread a strided partial sum, then a fixed
// warp/CTA tree, so the result does not depend on timing.
__global__ void __launch_bounds__(1024) k_mean_project(int n, double* __restrict__ y) {
  __shared__ double part[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[0] = t;
  }
  __syncthreads();
  const double m = part[0] / n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] -= m;
}

// ---- general interface problem, eq. (bie-ifp-1) ----------------------------
__global__ void k_gen_scale(int nb, const double* __restrict__ v, double s1, double s2,
                            double* __restrict__ o1, double* __restrict__ o2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const double x = v[i];
  o1[i] = x * s1;
  o2[i] = x * s2;
}

__global__ void k_gen_combine(int nb, const double* __restrict__ x1, double c1,
                              const double* __restrict__ x2, double c2, const double* __restrict__ T,
                              double a1, double a2, double b1, double b2, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const double v1 = 0.5 * (T[i] + T[nb + i]), d1 = 0.5 * (T[2 * nb + i] + T[3 * nb + i]);
  const double v2 = 0.5 * (T[4 * nb + i] + T[5 * nb + i]), d2 = 0.5 * (T[6 * nb + i] + T[7 * nb + i]);
  y[i] = c1 * x1[i] + a1 * v1 + a2 * v2;
  y[nb + i] = c2 * x2[i] + b1 * d1 + b2 * d2;
}

__global__ void k_gen_eval_prep(int nb, const double* __restrict__ phi, const double* __restrict__ psi,
                                const double* __restrict__ g1, const double* __restrict__ g2, double r1,
                                double r2, double* __restrict__ s1, double* __restrict__ s2,
                                double* __restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  s1[i] = (psi[i] + g2[i]) * r1;
  s2[i] = -psi[i] * r2;
  a[i] = g1[i] - phi[i];
}

__global__ void k_select_side(int tot, const uint8_t* __restrict__ inside, double* __restrict__ u,
                              const double* __restrict__ u2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x)
    if (!inside[t]) u[t] = u2[t];
}

__global__ void k_set_boundary(Grid g, const double* __restrict__ gb, double* __restrict__ u) {
  const int tot = (int)g.nodes();
  const int n1 = g.n + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    int i2 = 1, i1, i0;
    if (g.d == 2) {
      i1 = t % n1;
      i0 = t / n1;
    } else {
      const int r = t / n1;
      i2 = t - r * n1;
      i1 = r % n1;
      i0 = r / n1;
    }
    bool bnd = i0 == 0 || i0 == g.n || i1 == 0 || i1 == g.n ||
               (g.d == 3 && (i2 == 0 || i2 == g.n));
    if (bnd) u[t] = gb ? gb[t] : 0.0;
  }
}

}  // namespace

// Grid stride between the per-interface f_in grids of the data (0: one grid).
static long long in_stride(const kfbi_problem* p, const kfbi_data* data) {
  return data && data->in_per_interface && p->n_iface > 1 ? p->g.nodes() : 0;
}

kfbi_status launch_correction_values(kfbi_problem* p, const double* a, const double* b,
                                     const double* ftilde, double* cvals) {
  KFBI_LAUNCH(p, KFBI_KC_CORRECTION, k_cvals<<<div_up(p->nent, 128), 128, 0, p->stream>>>(
      p->nent, p->npde, p->ndir, p->nneu, p->g.h, p->ent_owner, p->ent_w, p->pde_node,
      p->dir_idx, p->neu_idx, a, b, ftilde, 1.0, nullptr, 1.0, cvals, p->ent_iface, 0));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

// C values from the physical data (f~ = f_in/sigma_in - f_out/sigma_out).
kfbi_status launch_correction_values_data(kfbi_problem* p, const double* a, const double* b,
                                          const kfbi_data* data, double* cvals) {
  const double* fi = data ? data->f_in : nullptr;
  const double* fo = data ? data->f_out : nullptr;
  double so = interior_bvp(p) ? 1.0 : p->cfg.sigma_out;
  if (interior_bvp(p)) fo = nullptr;
  KFBI_LAUNCH(p, KFBI_KC_CORRECTION, k_cvals<<<div_up(p->nent, 128), 128, 0, p->stream>>>(
      p->nent, p->npde, p->ndir, p->nneu, p->g.h, p->ent_owner, p->ent_w, p->pde_node,
      p->dir_idx, p->neu_idx, a, b, fi, p->cfg.sigma_in, fo, so, cvals, p->ent_iface,
      in_stride(p, data)));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_collocation_fit(kfbi_problem* p, const double* a, const double* b,
                                   const double* ftilde, double* coef) {
  KFBI_LAUNCH(p, KFBI_KC_CORRECTION, k_coef<<<div_up(p->nb, 8), 256, 0, p->stream>>>(p->nb, p->ncoef, p->npde, p->ndir, p->nneu,
                                                   p->g.h, p->minv, p->pde_node, p->dir_idx,
                                                   p->neu_idx, a, b, ftilde, coef));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

// Neighbour coefficients in the enumeration order of the setup (a, b[, c] in
// {-1,0,1}, last fastest, centre skipped; star only for order 2).
static void neighbour_table(kfbi_problem* p, std::vector<double>* coef, std::vector<int8_t>* off) {
  const int d = p->g.d;
  coef->clear();
  off->clear();
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int e = (d == 3 ? -1 : 0); e <= (d == 3 ? 1 : 0); ++e) {
        int nz = (a != 0) + (b != 0) + (e != 0);
        if (nz == 0) continue;
        if (p->cfg.order == 2 && nz > 1) continue;
        coef->push_back(p->stencil_c[nz]);
        off->push_back((int8_t)a);
        off->push_back((int8_t)b);
        off->push_back((int8_t)e);
      }
}

kfbi_status launch_rhs(kfbi_problem* p, const double* cvals, const kfbi_data* data,
                       double* rhs) {
  const Grid g = p->g;
  const double* d_nbc = p->nb_coef;
  const int8_t* d_off = p->nb_off;
  const bool src = data && (data->f_in || data->f_out || data->lapf_in || data->lapf_out);
  const bool gb = data && data->g_b;
  if (src || gb) {
    const double* fi = data->f_in;
    const double* fo = interior_bvp(p) ? nullptr : data->f_out;
    const double* li = data->lapf_in;
    const double* lo_ = interior_bvp(p) ? nullptr : data->lapf_out;
    double so = interior_bvp(p) ? 1.0 : p->cfg.sigma_out;
    KFBI_LAUNCH(p, KFBI_KC_RHS, k_rhs_source<<<std::min(div_up(g.nodes(), 256), 152 * 32), 256, 0, p->stream>>>(
        g, p->cfg.order, p->inside, fi, fo, li, lo_, 1.0 / p->cfg.sigma_in, 1.0 / so, g.h * g.h / 12.0,
        interior_bvp(p) ? nullptr : data->g_b, d_nbc, d_off, p->n_nb, rhs, in_stride(p, data)));
    KFBI_CUDA(p, cudaGetLastError());
  } else {
    KFBI_CUDA(p, cudaMemsetAsync(rhs, 0, sizeof(double) * g.nodes(), p->stream));
  }
  if (cvals && p->n_iface > 1) {
    KFBI_LAUNCH(p, KFBI_KC_RHS, k_rhs_correct_multi<<<div_up(p->nirr, 128), 128, 0, p->stream>>>(
        p->nirr, p->n_nb, p->irr_lin, p->corr_nb, p->corr_nb2, d_nbc, cvals, rhs));
    KFBI_CUDA(p, cudaGetLastError());
  } else if (cvals) {
    KFBI_LAUNCH(p, KFBI_KC_RHS, k_rhs_correct<<<div_up(p->nirr, 128), 128, 0, p->stream>>>(
        p->nirr, p->n_nb, p->irr_lin, p->irr_inside, p->corr_nb, d_nbc, cvals, rhs, 1));
    KFBI_CUDA(p, cudaGetLastError());
  }
  return KFBI_OK;
}

kfbi_status launch_traces(kfbi_problem* p, const double* u, const double* cvals, double* vp,
                          double* vm, double* dp, double* dm) {
  // 3D: the pair-arithmetic kernels (FP64 pipe bound otherwise)
  const bool df = p->tr[0].wv2 != nullptr;
  if (p->n_iface > 1 && df)
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_traces4_df<true><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, vp, vm, dp, dm));
  else if (df)
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_traces4_df<false><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, vp, vm, dp, dm));
  else if (p->n_iface > 1)
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_traces4<true><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, vp, vm, dp, dm));
  else
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_traces4<false><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, vp, vm, dp, dm));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_operator_trace(kfbi_problem* p, const double* u, const double* cvals,
                                  const double* x, double alpha_x, double beta_t, double* y) {
  if (p->n_iface > 1)
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_trace_op<true><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, x, alpha_x, beta_t, y));
  else
    KFBI_LAUNCH(p, KFBI_KC_TRACE, k_trace_op<false><<<div_up(p->nb, 8), 256, 0, p->stream>>>(
        p->nb, p->tr[0], p->tr[1], u, cvals, x, alpha_x, beta_t, y));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_mean_project(kfbi_problem* p, double* y) {
  if (p->cfg.kind != KFBI_NEUMANN_INTERIOR || p->kt != 0.0) return KFBI_OK;
  KFBI_LAUNCH(p, KFBI_KC_TRACE, k_mean_project<<<1, 1024, 0, p->stream>>>(p->nb, y));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_gen_scale(kfbi_problem* p, const double* v, double s1, double s2, double* out1,
                             double* out2) {
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_gen_scale<<<div_up(p->nb, 256), 256, 0, p->stream>>>(p->nb, v, s1, s2, out1, out2));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_gen_combine(kfbi_problem* p, const double* x1, double c1, const double* x2, double c2,
                               const double* T, double a1, double a2, double b1, double b2, double* y) {
  KFBI_LAUNCH(p, KFBI_KC_TRACE, k_gen_combine<<<div_up(p->nb, 256), 256, 0, p->stream>>>(
      p->nb, x1, c1, x2, c2, T, a1, a2, b1, b2, y));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_gen_eval_prep(kfbi_problem* p, const double* phi, const double* psi, const double* g1,
                                 const double* g2, double* s1, double* s2, double* a) {
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_gen_eval_prep<<<div_up(p->nb, 256), 256, 0, p->stream>>>(
      p->nb, phi, psi, g1, g2, 1.0 / p->cfg.sigma_in, 1.0 / p->cfg.sigma_out, s1, s2, a));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_select_side(kfbi_problem* p, double* u, const double* u2) {
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_select_side<<<std::min(div_up(p->g.nodes(), 256), 152 * 32), 256, 0, p->stream>>>(
      (int)p->g.nodes(), p->inside, u, u2));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status launch_set_boundary(kfbi_problem* p, double* u, const double* g_b) {
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_set_boundary<<<std::min(div_up(p->g.nodes(), 256), 152 * 32), 256, 0, p->stream>>>(p->g, g_b, u));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status upload_neighbour_tables(kfbi_problem* p) {
  std::vector<double> c;
  std::vector<int8_t> o;
  neighbour_table(p, &c, &o);
  KFBI_CUDA(p, dalloc(&p->nb_coef, c.size()));
  KFBI_CUDA(p, dalloc(&p->nb_off, o.size()));
  KFBI_CUDA(p, cudaMemcpyAsync(p->nb_coef, c.data(), sizeof(double) * c.size(),
                               cudaMemcpyHostToDevice, p->stream));
  KFBI_CUDA(p, cudaMemcpyAsync(p->nb_off, o.data(), o.size(), cudaMemcpyHostToDevice, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  return KFBI_OK;
}

}  // namespace kfbi

// ---------------------------------------------------------------------------
// Batched variants over many instances (flattened work, instance found by a
// binary search in a prefix array).  Used by the batched GMRES of batch.cu.
// ---------------------------------------------------------------------------
namespace kfbi {

struct BatchHot {
  int ninst = 0;
  void* dcv = nullptr;     // CvDesc[ninst]
  void* dcorr = nullptr;   // CorrDesc[ninst]
  void* dtr = nullptr;     // TrDesc[ninst]
  int* dirr_start = nullptr;
  int* ddof_start = nullptr;
  int tot_irr = 0, tot_dof = 0;
};

namespace {

struct CvDesc {
  int nirr, npde, ndir, nneu;
  double h;
  const int32_t* owner;
  const double* W;
  const int32_t* dir_idx;
  const int32_t* neu_idx;
  const double* a;     // Dirichlet data (density of the Dirichlet form) or null
  const double* b;     // Neumann data (density of the mu-form) or null
  double* out;
};

struct CorrDesc {
  int nirr, nnb;
  const int32_t* lin;
  const uint8_t* irr_inside;
  const int32_t* corr_nb;
  const double* nbc;
  const double* cv;
  double* R;
};

struct TrDesc {
  int nb;
  TraceCSR tp, tm;
  const double* u;
  const double* cv;
  const double* x;
  double alpha, beta;
  double* y;
};

__device__ __forceinline__ int inst_of(const int* start, int ninst, int item) {
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_cvals_batched(const CvDesc* __restrict__ D, const int* __restrict__ start, int ninst) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= start[ninst]) return;
  const int k = inst_of(start, ninst, item);
  const CvDesc& c = D[k];
  const int q = item - start[k];
  const int i = c.owner[q];
  double acc = 0.0;
  int j = c.npde;
  if (c.a) {
    for (int s = 0; s < c.ndir; ++s, ++j) acc += c.W[(size_t)j * c.nirr + q] * c.a[c.dir_idx[i * c.ndir + s]];
  } else {
    j += c.ndir;
  }
  if (c.b) {
    for (int s = 0; s < c.nneu; ++s, ++j)
      acc += c.W[(size_t)j * c.nirr + q] * (c.h * c.b[c.neu_idx[i * c.nneu + s]]);
  }
  c.out[q] = acc;
}

// R[P] = C_P (the loop right-hand side is zero away from the irregular nodes)
__global__ void k_rhs_correct_batched(const CorrDesc* __restrict__ D, const int* __restrict__ start,
                                      int ninst) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= start[ninst]) return;
  const int k = inst_of(start, ninst, item);
  const CorrDesc& c = D[k];
  const int q = item - start[k];
  double acc = 0.0;
  for (int s = 0; s < c.nnb; ++s) {
    const int j = c.corr_nb[(size_t)s * c.nirr + q];
    if (j >= 0) acc += c.nbc[s] * c.cv[j];
  }
  c.R[c.lin[q]] = c.irr_inside[q] ? -acc : acc;
}

__global__ void k_trace_op_batched(const TrDesc* __restrict__ D, const int* __restrict__ start,
                                   int ninst) {
  const int item = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (item >= start[ninst]) return;
  const int k = inst_of(start, ninst, item);
  const TrDesc& t = D[k];
  const int i = item - start[k];
  double acc = 0.0;
  for (int e = t.tp.ptr[i] + lane; e < t.tp.ptr[i + 1]; e += 32) {
    double w = t.u[t.tp.node[e]];
    const int j = t.tp.irr[e];
    if (j >= 0) w += t.cv[j];
    acc += t.tp.w[e] * w;
  }
  for (int e = t.tm.ptr[i] + lane; e < t.tm.ptr[i + 1]; e += 32) {
    double w = t.u[t.tm.node[e]];
    const int j = t.tm.irr[e];
    if (j >= 0) w -= t.cv[j];
    acc += t.tm.w[e] * w;
  }
  acc = warp_sum(acc);
  if (lane == 0) t.y[i] = t.alpha * t.x[i] + t.beta * acc;
}

}  // namespace

kfbi_status batch_hot_create(kfbi_problem* p0, kfbi_problem* const* ps, int ninst, double* const* x,
                             double* const* y, double* const* rhs, BatchHot** out) {
  BatchHot* bh = new BatchHot();
  *out = bh;
  bh->ninst = ninst;
  std::vector<CvDesc> cv(ninst);
  std::vector<CorrDesc> co(ninst);
  std::vector<TrDesc> tr(ninst);
  std::vector<int> is(ninst + 1, 0), ds(ninst + 1, 0);
  for (int k = 0; k < ninst; ++k) {
    kfbi_problem* p = ps[k];
    const bool dir = p->cfg.kind == KFBI_DIRICHLET_INTERIOR;
    // one interface per instance (checked at batch creation): entry q is
    // irregular node q, so one prefix array serves both item kinds
    cv[k] = CvDesc{p->nent, p->npde, p->ndir, p->nneu, p->g.h, p->ent_owner, p->ent_w,
                   p->dir_idx, p->neu_idx, dir ? x[k] : nullptr, dir ? nullptr : x[k], p->cvals};
    co[k] = CorrDesc{p->nirr, p->n_nb, p->irr_lin, p->irr_inside, p->corr_nb, p->nb_coef, p->cvals, rhs[k]};
    tr[k] = TrDesc{p->nb, p->tr[0], p->tr[1], p->ugrid, p->cvals, x[k], 0.5, dir ? 1.0 : -p->mu, y[k]};
    is[k + 1] = is[k] + p->nirr;
    ds[k + 1] = ds[k] + p->nb;
  }
  bh->tot_irr = is[ninst];
  bh->tot_dof = ds[ninst];
  CvDesc* a = nullptr;
  CorrDesc* b = nullptr;
  TrDesc* c = nullptr;
  KFBI_CUDA(p0, dalloc(&a, ninst));
  KFBI_CUDA(p0, dalloc(&b, ninst));
  KFBI_CUDA(p0, dalloc(&c, ninst));
  KFBI_CUDA(p0, dalloc(&bh->dirr_start, ninst + 1));
  KFBI_CUDA(p0, dalloc(&bh->ddof_start, ninst + 1));
  bh->dcv = a;
  bh->dcorr = b;
  bh->dtr = c;
  KFBI_CUDA(p0, cudaMemcpy(a, cv.data(), sizeof(CvDesc) * ninst, cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(b, co.data(), sizeof(CorrDesc) * ninst, cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(c, tr.data(), sizeof(TrDesc) * ninst, cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bh->dirr_start, is.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bh->ddof_start, ds.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  return KFBI_OK;
}

void batch_hot_destroy(BatchHot* bh) {
  if (!bh) return;
  cudaFree(bh->dcv);
  cudaFree(bh->dcorr);
  cudaFree(bh->dtr);
  cudaFree(bh->dirr_start);
  cudaFree(bh->ddof_start);
  delete bh;
}

kfbi_status batch_hot_cvals_rhs(kfbi_problem* p0, BatchHot* bh, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_CORRECTION, k_cvals_batched<<<div_up(bh->tot_irr, 128), 128, 0, st>>>(
      static_cast<const CvDesc*>(bh->dcv), bh->dirr_start, bh->ninst));
  KFBI_LAUNCH(p0, KFBI_KC_RHS, k_rhs_correct_batched<<<div_up(bh->tot_irr, 128), 128, 0, st>>>(
      static_cast<const CorrDesc*>(bh->dcorr), bh->dirr_start, bh->ninst));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status batch_hot_trace(kfbi_problem* p0, BatchHot* bh, cudaStream_t st) {
  KFBI_LAUNCH(p0, KFBI_KC_TRACE, k_trace_op_batched<<<div_up(bh->tot_dof, 8), 256, 0, st>>>(
      static_cast<const TrDesc*>(bh->dtr), bh->ddof_start, bh->ninst));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
