// Geometry set-up of one problem on the GPU (Sec. 5.1, 5.2, 5.4, 5.5):
// node classes, grid-line intersections (DOFs), reference axes, collocation
// stencils, inverses of the collocation matrices (eq. (cau-ls)), irregular
// nodes, closest primary points, correction neighbour lists (eq.
// (crc-formula)) and the least-squares trace weights.
//
// This translation unit is compiled with -fmad=false: every product and sum is
// rounded on its own, so the integer decisions (classification, root
// brackets, stencil lines, closest points, stencil radii) follow the written
// rules operation by operation.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "kfbi_internal.cuh"
#include "levelset.cuh"

namespace kfbi {

namespace {

constexpr int kFlagSentinel = INT_MAX;

__device__ __forceinline__ double coord(const Grid& g, int i) { return g.lo + (double)i * g.h; }

__device__ __forceinline__ long long node_index(const Grid& g, const int* idx) {
  long long n1 = g.n + 1;
  if (g.d == 2) return (long long)idx[0] * n1 + idx[1];
  return ((long long)idx[0] * n1 + idx[1]) * n1 + idx[2];
}

__device__ __forceinline__ void node_multi(const Grid& g, long long t, int* idx) {
  int n1 = g.n + 1;
  if (g.d == 2) {
    idx[1] = (int)(t % n1);
    idx[0] = (int)(t / n1);
    idx[2] = 0;
  } else {
    idx[2] = (int)(t % n1);
    t /= n1;
    idx[1] = (int)(t % n1);
    idx[0] = (int)(t / n1);
  }
}

__device__ __forceinline__ void flag_min(int* flags, int which, int value) {
  atomicMin(&flags[which], value);
}

// ---------------------------------------------------------------------------
// Scan (single block): out[i] = base + sum_{j<i} in[j], out[n] = total.
// ---------------------------------------------------------------------------
__global__ void k_exclusive_scan(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                 int n, int32_t base) {
  __shared__ int32_t part[1024];
  int t = threadIdx.x;
  int chunk = (n + 1023) / 1024;
  int b = t * chunk;
  int e = min(n, b + chunk);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = base + (t ? part[t - 1] : 0);
  for (int i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == 1023) out[n] = base + part[1023];
}

// Multi-block exclusive scan for long arrays: per chunk of kScanChunk elements
// its sum, a single-block scan of the sums, then each chunk's scan from its
// offset (integer sums: the result does not depend on the decomposition).
constexpr int kScanChunk = 4096;   // 1024 threads x 4 elements

__device__ __forceinline__ int32_t warp_scan_incl_i(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive prefix of v over the 1024 threads of the block, and the total
__device__ __forceinline__ int32_t block_scan_excl(int32_t v, int32_t* total) {
  __shared__ int32_t wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t incl = warp_scan_incl_i(v);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int32_t x = wsum[lane];
    wsum[lane] = warp_scan_incl_i(x) - x;
  }
  __syncthreads();
  const int32_t r = wsum[w] + incl - v;
  if (total) *total = wsum[31] + __shfl_sync(0xffffffffu, incl, 31);
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_sums(const int32_t* __restrict__ in, int n,
                                                    int32_t* __restrict__ bsum) {
  const long long i0 = (long long)blockIdx.x * kScanChunk + 4 * threadIdx.x;
  int32_t s = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (i0 + e < n) s += in[i0 + e];
  int32_t tot = 0;
  block_scan_excl(s, &tot);
  if (threadIdx.x == 1023) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int32_t* __restrict__ in, int n,
                                                     const int32_t* __restrict__ boff, int nblk,
                                                     int32_t* __restrict__ out) {
  const long long i0 = (long long)blockIdx.x * kScanChunk + 4 * threadIdx.x;
  int32_t v[4];
  int32_t s = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[e] = i0 + e < n ? in[i0 + e] : 0;
    s += v[e];
  }
  int32_t run = boff[blockIdx.x] + block_scan_excl(s, nullptr);
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (i0 + e < n) {
      out[i0 + e] = run;
      run += v[e];
    }
  if (blockIdx.x == nblk - 1 && threadIdx.x == 0) out[n] = boff[nblk];
}

// ---------------------------------------------------------------------------
// Classification (Sec. 5.2): inside iff H(node) < 0, stored as the node's side
// label (0 outside, 1 + k in Omega^(k); 1 inside for one interface).
// ---------------------------------------------------------------------------
// A grid-sampled H is its sample at a node (the interpolant's weights there
// are 1 and +-0, and every sample is finite), so its labels are read directly.
__global__ void k_classify(Grid g, LevelSet L, uint8_t* __restrict__ inside) {
  long long tot = g.nodes();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    if (L.kind == KFBI_LS_GRID) {
      inside[t] = L.grid[t] < 0.0 ? 1 : 0;
      continue;
    }
    int idx[3];
    node_multi(g, t, idx);
    double X[3] = {coord(g, idx[0]), coord(g, idx[1]), g.d == 3 ? coord(g, idx[2]) : 0.0};
    inside[t] = (uint8_t)ls_label(L, X);
  }
}

__global__ void k_count_nonfinite(const double* __restrict__ a, long long n,
                                  unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    c += isfinite(a[t]) ? 0ull : 1ull;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// Grid-line intersections (Sec. 5.1).
// ---------------------------------------------------------------------------
struct LineDesc {
  int r;          // family (direction of the lines)
  int oa, ob;     // other axes (ascending); ob = -1 in 2D
  long long sr, sa, sb;   // node strides of r, oa, ob
};

__device__ __forceinline__ void line_other(const Grid& g, const LineDesc& D, int li, int* ia, int* ib) {
  if (g.d == 2) {
    *ia = li;
    *ib = 0;
  } else {
    *ia = li / (g.n + 1);
    *ib = li % (g.n + 1);
  }
}

// Root of H_k (interface k) on the edge [x0, x0 + h e_r]: start at the
// linear interpolant, Newton step, bisection whenever Newton leaves the
// bracket or df = 0, stop at |ds| <= 1e-15 N h or after 64 steps.  1e-15 of
// the box width is about the FP64 spacing of a coordinate in the box; the
// rounding noise of H makes the Newton steps near the root ~1e-16 / |grad H|
// long, so a tolerance of 1e-15 h (1e-18 at N = 1024) is met only by chance
// (8-11 steps on average and up to the step limit, where about 3 suffice),
// and a warp waits for its slowest lane.
__device__ double edge_root(const Grid& g, const LevelSet& L, int k, const double* x0, int r,
                            int j) {
  double xa[3] = {x0[0], x0[1], x0[2]};
  double xb[3] = {x0[0], x0[1], x0[2]};
  xa[r] = coord(g, j);
  xb[r] = coord(g, j + 1);
  double ha = ls_H_iface(L, k, xa), hb = ls_H_iface(L, k, xb);
  bool neg_a = ha < 0.0;
  double h = g.h;
  double s = h * ha / (ha - hb);
  double lo_s = 0.0, hi_s = h;
  for (int it = 0; it < kRootMaxIt; ++it) {
    double X[3] = {xa[0], xa[1], xa[2]};
    X[r] = xa[r] + s;
    double f = ls_H_iface(L, k, X);
    double gr[3];
    ls_grad_iface(L, k, X, gr);
    double df = gr[r];
    bool done_zero = f == 0.0;
    bool same = (f < 0.0) == neg_a;
    if (same) lo_s = s; else hi_s = s;
    double s_new = s - f / df;
    bool bad = !((s_new > lo_s) && (s_new < hi_s)) || (df == 0.0);
    if (bad) s_new = 0.5 * (lo_s + hi_s);
    if (done_zero) s_new = s;
    bool conv = done_zero || (fabs(s_new - s) <= kRootTol * (g.n * h));
    s = s_new;
    if (conv) break;
  }
  return s;
}

__device__ bool crossing_point(const Grid& g, const LevelSet& L, int k, const LineDesc& D, int ia,
                               int ib, int j, double cos_alpha, double* X, double* nv) {
  double x0[3] = {0.0, 0.0, 0.0};
  x0[D.oa] = coord(g, ia);
  if (g.d == 3) x0[D.ob] = coord(g, ib);
  x0[D.r] = coord(g, j);
  double s = edge_root(g, L, k, x0, D.r, j);
  X[0] = x0[0];
  X[1] = x0[1];
  X[2] = x0[2];
  X[D.r] = x0[D.r] + s;
  double gr[3];
  ls_grad_iface(L, k, X, gr);
  double nn = g.d == 2 ? gr[0] * gr[0] + gr[1] * gr[1] : gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
  double inv = sqrt(nn);
  nv[0] = gr[0] / inv;
  nv[1] = gr[1] / inv;
  nv[2] = g.d == 3 ? gr[2] / inv : 0.0;
  return fabs(nv[D.r]) > cos_alpha;
}

// The interfaces crossed on edge j of a line whose end nodes carry labels
// la != lb: slot 0 on interface la - 1 (if la > 0), slot 1 on lb - 1 (if
// lb > 0), with several interfaces only where that H_k changes sign along
// the edge (with one interface the labels decide: exactly one slot).
__device__ __forceinline__ int edge_slots(const Grid& g, const LevelSet& L, const LineDesc& D, int ia,
                                          int ib, int j, int la, int lb, bool multi, int* ks) {
  int c = 0;
  const int cand[2] = {la - 1, lb - 1};
  for (int slot = 0; slot < 2; ++slot) {
    const int k = cand[slot];
    if (k < 0) continue;
    if (multi) {
      double xa[3] = {0.0, 0.0, 0.0};
      xa[D.oa] = coord(g, ia);
      if (g.d == 3) xa[D.ob] = coord(g, ib);
      double xb[3] = {xa[0], xa[1], xa[2]};
      xa[D.r] = coord(g, j);
      xb[D.r] = coord(g, j + 1);
      if ((ls_H_iface(L, k, xa) < 0.0) == (ls_H_iface(L, k, xb) < 0.0)) continue;
    }
    ks[c++] = k;
  }
  return c;
}

// inclusive warp prefix sum
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Candidate points (edge, interface) of the grid lines of one family, a warp
// per line: the lanes test 32 consecutive edges at a time for a change of
// node label.  Count pass, then the fill pass writes each line's candidates
// in edge order (slot order within an edge) after those of the lower lanes.
constexpr int kLineWarps = 4;
__global__ void __launch_bounds__(32 * kLineWarps) k_cand_count(Grid g, LevelSet L, LineDesc D,
                                                                const uint8_t* __restrict__ inside,
                                                                bool multi, int nlines,
                                                                int32_t* __restrict__ count) {
  const int li = blockIdx.x * kLineWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (li >= nlines) return;
  int ia, ib;
  line_other(g, D, li, &ia, &ib);
  const long long base = ia * D.sa + (g.d == 3 ? ib * D.sb : 0);
  int c = 0;
  for (int j0 = 0; j0 < g.n; j0 += 32) {
    const int j = j0 + lane;
    int hits = 0;
    if (j < g.n) {
      const int la = inside[base + j * D.sr], lb = inside[base + (j + 1) * D.sr];
      int ks[2];
      if (la != lb) hits = edge_slots(g, L, D, ia, ib, j, la, lb, multi, ks);
    }
    c += __shfl_sync(0xffffffffu, warp_incl_scan(hits), 31);
  }
  if (lane == 0) count[li] = c;
}

__global__ void __launch_bounds__(32 * kLineWarps) k_cand_fill(Grid g, LevelSet L, LineDesc D,
                                                               const uint8_t* __restrict__ inside,
                                                               bool multi, int nlines,
                                                               const int32_t* __restrict__ start,
                                                               int32_t* __restrict__ cline,
                                                               int32_t* __restrict__ cedge,
                                                               int32_t* __restrict__ ciface) {
  const int li = blockIdx.x * kLineWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (li >= nlines) return;
  int ia, ib;
  line_other(g, D, li, &ia, &ib);
  const long long base = ia * D.sa + (g.d == 3 ? ib * D.sb : 0);
  int pos0 = start[li];
  for (int j0 = 0; j0 < g.n; j0 += 32) {
    const int j = j0 + lane;
    int hits = 0, ks[2];
    if (j < g.n) {
      const int la = inside[base + j * D.sr], lb = inside[base + (j + 1) * D.sr];
      if (la != lb) hits = edge_slots(g, L, D, ia, ib, j, la, lb, multi, ks);
    }
    const int incl = warp_incl_scan(hits);
    for (int c = 0; c < hits; ++c) {
      const int pos = pos0 + incl - hits + c;
      cline[pos] = li;
      cedge[pos] = j;
      ciface[pos] = ks[c];
    }
    pos0 += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// One thread per candidate: the root of H_k on its edge (Sec. 5.1), the unit
// normal, and whether the point is a DOF of this family (|n_r| > cos alpha).
__global__ void k_cand_roots(Grid g, LevelSet L, LineDesc D, int ncand, double cos_alpha,
                             const int32_t* __restrict__ cline, const int32_t* __restrict__ cedge,
                             const int32_t* __restrict__ ciface, double* __restrict__ cx,
                             double* __restrict__ cn, int32_t* __restrict__ keep) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  int ia, ib;
  line_other(g, D, cline[c], &ia, &ib);
  double X[3], nv[3];
  const bool k = crossing_point(g, L, ciface[c], D, ia, ib, cedge[c], cos_alpha, X, nv);
  for (int e = 0; e < 3; ++e) {
    cx[(size_t)e * ncand + c] = X[e];
    cn[(size_t)e * ncand + c] = nv[e];
  }
  keep[c] = k ? 1 : 0;
}

// The kept candidates in candidate order are the family's DOFs in DOF order:
// DOF base + kpos[c].
__global__ void k_cand_scatter(Grid g, LineDesc D, int ncand, int base, const int32_t* __restrict__ kpos,
                               const int32_t* __restrict__ keep, const int32_t* __restrict__ cedge,
                               const int32_t* __restrict__ ciface, const double* __restrict__ cx,
                               const double* __restrict__ cn, double* x0, double* x1, double* x2,
                               double* n0, double* n1, double* n2, int32_t* family, int32_t* edge,
                               int32_t* axis, int32_t* iface) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand || !keep[c]) return;
  const int pos = base + kpos[c];
  double nv[3];
  for (int e = 0; e < 3; ++e) nv[e] = cn[(size_t)e * ncand + c];
  x0[pos] = cx[c];
  x1[pos] = cx[(size_t)ncand + c];
  n0[pos] = nv[0];
  n1[pos] = nv[1];
  if (g.d == 3) {
    x2[pos] = cx[2 * (size_t)ncand + c];
    n2[pos] = nv[2];
  }
  family[pos] = D.r;
  edge[pos] = cedge[c];
  iface[pos] = ciface[c];
  int m = 0;
  double best = fabs(nv[0]);
  for (int k = 1; k < g.d; ++k)
    if (fabs(nv[k]) > best) {
      best = fabs(nv[k]);
      m = k;
    }
  axis[pos] = m;
}

// line_start[li] = DOF base + kept candidates before the line's first
__global__ void k_cand_line_start(int nlines, int base, const int32_t* __restrict__ cstart,
                                  const int32_t* __restrict__ kpos, int32_t* __restrict__ line_start) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li > nlines) return;
  line_start[li] = base + kpos[cstart[li]];
}

// ---------------------------------------------------------------------------
// Collocation stencils (Sec. 5.4).
// ---------------------------------------------------------------------------
struct StencilTables {
  int npde, ndir, nneu;
  int pde_off[kMaxPde][3];
  int ntries;                 // 3D lattice variants (shifted / unshifted)
  int dset[2][kMaxDir][2];
  int nset_pos[2][kMaxNeu];   // positions of the Neumann points inside dset
};
__constant__ StencilTables c_st;

struct DofView {
  const double* x[3];
  const double* n[3];
  const int32_t* line_start[3];
  const int32_t* iface;
};


// Family-`fam` DOF of interface `ifc` on the line through other-axis node
// indices (j, k), nearest to s_pred along e_fam within 2h; ties to the lower
// index; -1 if none.
__device__ int nearest_on_line(const Grid& g, const DofView& V, int fam, int j, int k,
                               double s_pred, int ifc) {
  if (j < 0 || j > g.n) return -1;
  int li = j;
  if (g.d == 3) {
    if (k < 0 || k > g.n) return -1;
    li = j * (g.n + 1) + k;
  }
  const int32_t* st = V.line_start[fam];
  int best = -1;
  double bestd = INFINITY;
  double win = 2.0 * g.h;
  for (int q = st[li]; q < st[li + 1]; ++q) {
    if (V.iface[q] != ifc) continue;
    double dist = fabs(V.x[fam][q] - s_pred);
    if (dist <= win && dist < bestd) {
      best = q;
      bestd = dist;
    }
  }
  return best;
}

__global__ void k_stencils(Grid g, int order, double cos_alpha, DofView V, int nb,
                           const int32_t* __restrict__ axis, int32_t* __restrict__ pde_node,
                           int32_t* __restrict__ dir_idx, int32_t* __restrict__ neu_idx,
                           int32_t* __restrict__ st_axis, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const int d = g.d;
  double p[3] = {V.x[0][i], V.x[1][i], d == 3 ? V.x[2][i] : 0.0};
  double nv[3] = {V.n[0][i], V.n[1][i], d == 3 ? V.n[2][i] : 0.0};
  int n0[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) n0[k] = (int)floor((p[k] - g.lo) / g.h + 0.5);
  for (int s = 0; s < c_st.npde; ++s) {
    int idx[3] = {n0[0] + c_st.pde_off[s][0], n0[1] + c_st.pde_off[s][1],
                  n0[2] + c_st.pde_off[s][2]};
    bool ok = true;
    for (int k = 0; k < d; ++k) ok = ok && idx[k] >= 0 && idx[k] <= g.n;
    if (!ok) {
      flag_min(flags, kFlagOutOfBox, i + 1);
      return;
    }
    pde_node[i * c_st.npde + s] = (int32_t)node_index(g, idx);
  }
  // reference axes to try: m first, then the others by decreasing |n_k| with |n_k| > cos(alpha)
  int m0 = axis[i];
  int axes[3];
  int na = 0;
  axes[na++] = m0;
  {
    int rest[2], nr = 0;
    for (int k = 0; k < d; ++k)
      if (k != m0 && fabs(nv[k]) > cos_alpha) rest[nr++] = k;
    if (nr == 2 && (fabs(nv[rest[1]]) > fabs(nv[rest[0]]))) {
      int t = rest[0];
      rest[0] = rest[1];
      rest[1] = t;
    }
    for (int q = 0; q < nr; ++q) axes[na++] = rest[q];
  }
  for (int ai = 0; ai < na; ++ai) {
    int m = axes[ai];
    if (d == 2) {
      int t = 1 - m;
      double kap = (p[t] - g.lo) / g.h;
      int j0 = (int)floor(kap + 0.5);
      int cand[9];
      double key[9];
      for (int c = 0; c < 9; ++c) {
        cand[c] = j0 - 4 + c;
        key[c] = fabs((double)cand[c] - kap);
      }
      for (int a = 1; a < 9; ++a) {   // insertion sort by (key, index)
        int cv = cand[a];
        double kv = key[a];
        int b = a - 1;
        while (b >= 0 && (key[b] > kv || (key[b] == kv && cand[b] > cv))) {
          cand[b + 1] = cand[b];
          key[b + 1] = key[b];
          --b;
        }
        cand[b + 1] = cv;
        key[b + 1] = kv;
      }
      int found[kMaxDir];
      int nf = 0;
      for (int c = 0; c < 9 && nf < c_st.ndir; ++c) {
        double xt = g.lo + (double)cand[c] * g.h;
        double s_pred = p[m] - nv[t] * (xt - p[t]) / nv[m];
        int q = nearest_on_line(g, V, m, cand[c], 0, s_pred, V.iface[i]);
        if (q >= 0) found[nf++] = q;
      }
      if (nf == c_st.ndir) {
        for (int s = 0; s < c_st.ndir; ++s) dir_idx[i * c_st.ndir + s] = found[s];
        for (int s = 0; s < c_st.nneu; ++s) neu_idx[i * c_st.nneu + s] = found[s];
        st_axis[i] = m;
        return;
      }
    } else {
      int t1 = m == 0 ? 1 : 0;
      int t2 = m == 2 ? 1 : 2;
      double k1 = (p[t1] - g.lo) / g.h;
      double k2 = (p[t2] - g.lo) / g.h;
      int j0 = (int)floor(k1 + 0.5);
      int l0 = (int)floor(k2 + 0.5);
      int s1 = k1 >= (double)j0 ? 1 : -1;
      int s2 = k2 >= (double)l0 ? 1 : -1;
      const int ori[4][2] = {{s1, s2}, {-s1, s2}, {s1, -s2}, {-s1, -s2}};
      for (int tv = 0; tv < c_st.ntries; ++tv) {
        for (int o = 0; o < 4; ++o) {
          int found[kMaxDir];
          bool ok = true;
          for (int s = 0; s < c_st.ndir; ++s) {
            int j = j0 + ori[o][0] * c_st.dset[tv][s][0];
            int k = l0 + ori[o][1] * c_st.dset[tv][s][1];
            double x1 = g.lo + (double)j * g.h;
            double x2 = g.lo + (double)k * g.h;
            double s_pred = p[m] - (nv[t1] * (x1 - p[t1]) + nv[t2] * (x2 - p[t2])) / nv[m];
            int q = nearest_on_line(g, V, m, j, k, s_pred, V.iface[i]);
            if (q < 0) {
              ok = false;
              break;
            }
            found[s] = q;
          }
          if (ok) {
            for (int s = 0; s < c_st.ndir; ++s) dir_idx[i * c_st.ndir + s] = found[s];
            for (int s = 0; s < c_st.nneu; ++s)
              neu_idx[i * c_st.nneu + s] = found[c_st.nset_pos[tv][s]];
            st_axis[i] = m;
            return;
          }
        }
      }
    }
  }
  flag_min(flags, kFlagGeometry, i + 1);
  st_axis[i] = -1;
}

// ---------------------------------------------------------------------------
// Monomials in scaled coordinates (graded-lexicographic order).
// ---------------------------------------------------------------------------
__constant__ Exponents c_exp;

__device__ __forceinline__ void powers(const double* xi, int d, double pw[3][5]) {
  for (int k = 0; k < 3; ++k) {
    double v = k < d ? xi[k] : 0.0;
    pw[k][0] = 1.0;
    pw[k][1] = v;
    pw[k][2] = v * v;
    pw[k][3] = pw[k][2] * v;
    pw[k][4] = pw[k][3] * v;
  }
}

__device__ __forceinline__ double mono(const double pw[3][5], int e) {
  return pw[0][c_exp.e[e][0]] * pw[1][c_exp.e[e][1]] * pw[2][c_exp.e[e][2]];
}

__device__ __forceinline__ double mono_d(const double pw[3][5], int e, int k) {
  int ek = c_exp.e[e][k];
  if (ek == 0) return 0.0;
  double v = (double)ek * pw[k][ek - 1];
  for (int j = 0; j < 3; ++j)
    if (j != k) v = v * pw[j][c_exp.e[e][j]];
  return v;
}

__device__ __forceinline__ double mono_lap(const double pw[3][5], int e, int d) {
  double tot = 0.0;
  for (int k = 0; k < d; ++k) {
    int ek = c_exp.e[e][k];
    if (ek < 2) continue;
    double v = (double)(ek * (ek - 1)) * pw[k][ek - 2];
    for (int j = 0; j < 3; ++j)
      if (j != k) v = v * pw[j][c_exp.e[e][j]];
    tot = tot + v;
  }
  return tot;
}

// ---------------------------------------------------------------------------
// Warp Householder QR of a column-major m x n matrix in shared memory.
// R: upper triangle of A plus rdiag; reflector v_k in A[k.., k];
// vn2[k] = 2 / |v_k|^2 (0 for a zero column), so that applying H_k costs a
// multiply: an FP64 divide is a long sequence on GB300's FP64 pipe (2 lanes
// per clock per SM), and one per column pair made the fits FP64-bound.
// ---------------------------------------------------------------------------
__device__ bool warp_householder(double* A, int lda, int m, int n, double* rdiag, double* vn2) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    double* ak = A + (size_t)k * lda;
    double s = 0.0;
    for (int i = k + lane; i < m; i += 32) s += ak[i] * ak[i];
    s = warp_sum(s);
    double akk = ak[k];
    double nrm = sqrt(s);
    double alpha = akk >= 0.0 ? -nrm : nrm;
    double vk = akk - alpha;
    double vnorm2 = s - akk * akk + vk * vk;
    const bool good = nrm > 0.0 && vnorm2 > 0.0;
    const double rv = good ? 2.0 / vnorm2 : 0.0;
    __syncwarp();
    if (lane == 0) {
      ak[k] = vk;
      rdiag[k] = alpha;
      vn2[k] = rv;
    }
    __syncwarp();
    if (!good) {
      ok = false;
      continue;
    }
    for (int j = k + 1; j < n; ++j) {
      double* aj = A + (size_t)j * lda;
      double t = 0.0;
      for (int i = k + lane; i < m; i += 32) t += ak[i] * aj[i];
      t = warp_sum(t);
      double f = t * rv;
      for (int i = k + lane; i < m; i += 32) aj[i] -= f * ak[i];
      __syncwarp();
    }
  }
  return ok;
}

// y <- H_k y for k = n-1..0 (y = Q y) or k = 0..n-1 (y = Q^T y).
__device__ void warp_apply_q(const double* A, int lda, int m, int n, const double* vn2, double* y,
                             bool transpose) {
  const int lane = threadIdx.x & 31;
  for (int kk = 0; kk < n; ++kk) {
    int k = transpose ? kk : n - 1 - kk;
    if (!(vn2[k] > 0.0)) continue;
    const double* ak = A + (size_t)k * lda;
    double t = 0.0;
    for (int i = k + lane; i < m; i += 32) t += ak[i] * y[i];
    t = warp_sum(t);
    double f = t * vn2[k];
    __syncwarp();
    for (int i = k + lane; i < m; i += 32) y[i] -= f * ak[i];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Collocation matrices M (eq. (cau-appro), rows scaled to O(1)) and M^{-1}.
// One warp per primary point; M^{-1} by Gauss-Jordan elimination with partial
// pivoting on [M | I], one lane per column (a pivot search is the only warp
// reduction of a step), the columns at an odd stride in shared memory so
// that the lanes' column walks fall in different banks.
// ---------------------------------------------------------------------------
__global__ void k_collocation_factor(Grid g, double kt, DofView V, int nb,
                                     const int32_t* __restrict__ pde_node,
                                     const int32_t* __restrict__ dir_idx,
                                     const int32_t* __restrict__ neu_idx,
                                     double* __restrict__ minv, int* flags) {
  extern __shared__ double sm[];
  const int n = c_exp.n;
  const int lda = n | 1;                // odd column stride (>= n)
  double* A = sm;                       // [M | I]: 2n columns of n rows, column-major, lda
  double* fcol = A + (size_t)lda * 2 * n;   // the pivot column of a step
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  if (i >= nb) return;
  const int d = g.d;
  double p[3] = {V.x[0][i], V.x[1][i], d == 3 ? V.x[2][i] : 0.0};
  const int npde = c_st.npde, ndir = c_st.ndir;
  for (int r = lane; r < n; r += 32) {
    double xi[3] = {0.0, 0.0, 0.0};
    double nq[3] = {0.0, 0.0, 0.0};
    int kind;
    if (r < npde) {
      long long t = pde_node[i * npde + r];
      int idx[3];
      node_multi(g, t, idx);
      for (int k = 0; k < d; ++k) xi[k] = (coord(g, idx[k]) - p[k]) / g.h;
      kind = 0;
    } else if (r < npde + ndir) {
      int q = dir_idx[i * ndir + (r - npde)];
      for (int k = 0; k < d; ++k) xi[k] = (V.x[k][q] - p[k]) / g.h;
      kind = 1;
    } else {
      int q = neu_idx[i * c_st.nneu + (r - npde - ndir)];
      for (int k = 0; k < d; ++k) {
        xi[k] = (V.x[k][q] - p[k]) / g.h;
        nq[k] = V.n[k][q];
      }
      kind = 2;
    }
    double pw[3][5];
    powers(xi, d, pw);
    for (int e = 0; e < n; ++e) {
      double v;
      if (kind == 0) {
        v = mono_lap(pw, e, d) - kt * g.h * g.h * mono(pw, e);
      } else if (kind == 1) {
        v = mono(pw, e);
      } else {
        v = nq[0] * mono_d(pw, e, 0) + nq[1] * mono_d(pw, e, 1);
        if (d == 3) v = v + nq[2] * mono_d(pw, e, 2);
      }
      A[(size_t)e * lda + r] = v;
    }
  }
  __syncwarp();
  // ||M||_1
  double colmax = 0.0;
  for (int e = lane; e < n; e += 32) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += fabs(A[(size_t)e * lda + r]);
    colmax = fmax(colmax, s);
  }
  for (int o = 16; o > 0; o >>= 1) colmax = fmax(colmax, __shfl_xor_sync(0xffffffffu, colmax, o));
  for (int c = n + lane; c < 2 * n; c += 32)
    for (int r = 0; r < n; ++r) A[(size_t)c * lda + r] = (r == c - n) ? 1.0 : 0.0;
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    const double* ak = A + (size_t)k * lda;
    // pivot: the first row of the largest |a_ik|, i >= k
    double best = -1.0;
    int prow = n;
    for (int r = k + lane; r < n; r += 32) {
      const double v = fabs(ak[r]);
      if (v > best) {
        best = v;
        prow = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orow = __shfl_xor_sync(0xffffffffu, prow, o);
      if (ob > best || (ob == best && orow < prow)) {
        best = ob;
        prow = orow;
      }
    }
    if (!(best > 0.0)) {
      ok = false;
      break;
    }
    // the multipliers: column k after the row swap, copied before any lane
    // changes that column
    for (int r = lane; r < n; r += 32) fcol[r] = ak[r == k ? prow : (r == prow ? k : r)];
    __syncwarp();
    const double piv = fcol[k];
    for (int c = lane; c < 2 * n; c += 32) {
      double* col = A + (size_t)c * lda;
      const double t = col[prow];
      col[prow] = col[k];
      const double rk = t / piv;
      col[k] = rk;
      for (int r = 0; r < n; ++r)
        if (r != k) col[r] = col[r] - fcol[r] * rk;
    }
    __syncwarp();
  }
  // ||M^{-1}||_1 and output (row-major M^{-1}[k][j] = X[k][j], X column j =
  // augmented column n + j)
  double invmax = 0.0;
  for (int c = n + lane; c < 2 * n; c += 32) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += fabs(A[(size_t)c * lda + r]);
    invmax = fmax(invmax, s);
  }
  for (int o = 16; o > 0; o >>= 1) invmax = fmax(invmax, __shfl_xor_sync(0xffffffffu, invmax, o));
  double* out = minv + (size_t)i * n * n;
  for (int t = lane; t < n * n; t += 32) {
    int k = t / n, j = t % n;
    out[t] = A[(size_t)(n + j) * lda + k];
  }
  double cond = colmax * invmax;
  if (lane == 0 && (!ok || !(cond < 1e10))) flag_min(flags, kFlagSingular, i + 1);
}

// ---------------------------------------------------------------------------
// Irregular nodes (Sec. 5.2).
// ---------------------------------------------------------------------------
struct NbTable {
  int count;
  int off[kMaxNeighbours][3];
};
__constant__ NbTable c_nb;

__global__ void k_irregular_flags(Grid g, const uint8_t* __restrict__ inside,
                                  uint8_t* __restrict__ flag) {
  long long tot = g.nodes();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_multi(g, t, idx);
    bool interior = true;
    for (int k = 0; k < g.d; ++k) interior = interior && idx[k] >= 1 && idx[k] <= g.n - 1;
    uint8_t f = 0;
    if (interior) {
      uint8_t c0 = inside[t];
      for (int s = 0; s < c_nb.count; ++s) {
        int q[3] = {idx[0] + c_nb.off[s][0], idx[1] + c_nb.off[s][1], idx[2] + c_nb.off[s][2]};
        if (inside[node_index(g, q)] != c0) {
          f = 1;
          break;
        }
      }
    }
    flag[t] = f;
  }
}

// rows along the last axis
__global__ void k_row_count(Grid g, const uint8_t* __restrict__ flag, int nrows,
                            int32_t* __restrict__ count) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const uint8_t* f = flag + (long long)r * (g.n + 1);
  int c = 0;
  for (int j = 0; j <= g.n; ++j) c += f[j];
  count[r] = c;
}

__global__ void k_row_fill(Grid g, const uint8_t* __restrict__ flag,
                           const uint8_t* __restrict__ inside, int nrows,
                           const int32_t* __restrict__ start, int32_t* __restrict__ lin,
                           uint8_t* __restrict__ irr_inside, int32_t* __restrict__ map) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  long long base = (long long)r * (g.n + 1);
  int pos = start[r];
  for (int j = 0; j <= g.n; ++j) {
    if (flag[base + j]) {
      lin[pos] = (int32_t)(base + j);
      irr_inside[pos] = inside[base + j];
      map[base + j] = pos;
      ++pos;
    }
  }
}

// ---------------------------------------------------------------------------
// Closest primary points (Sec. 5.3, closest-point partition of unity).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_of(const Grid& g, double x) {
  int c = (int)floor((x - g.lo) / g.h);
  return min(max(c, 0), g.n - 1);
}

__device__ __forceinline__ long long cell_index(const Grid& g, const int* c) {
  long long n = g.n;
  if (g.d == 2) return (long long)c[0] * n + c[1];
  return ((long long)c[0] * n + c[1]) * n + c[2];
}

__global__ void k_cell_count(Grid g, DofView V, int nb, int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int c[3] = {cell_of(g, V.x[0][i]), cell_of(g, V.x[1][i]), g.d == 3 ? cell_of(g, V.x[2][i]) : 0};
  atomicAdd(&cnt[cell_index(g, c)], 1);
}

__global__ void k_cell_fill(Grid g, DofView V, int nb, const int32_t* __restrict__ start,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ items) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int c[3] = {cell_of(g, V.x[0][i]), cell_of(g, V.x[1][i]), g.d == 3 ? cell_of(g, V.x[2][i]) : 0};
  long long ci = cell_index(g, c);
  int pos = atomicAdd(&cursor[ci], 1);
  items[start[ci] + pos] = i;
}

__device__ __forceinline__ double dist2(const DofView& V, int d, int q, const double* X) {
  double dx = X[0] - V.x[0][q];
  double s = dx * dx;
  double dy = X[1] - V.x[1][q];
  s = s + dy * dy;
  if (d == 3) {
    double dz = X[2] - V.x[2][q];
    s = s + dz * dz;
  }
  return s;
}

// Per correction entry (node, interface k): the closest primary point among
// the DOFs of interface k.
__global__ void k_closest(Grid g, DofView V, int nb, int nent, const int32_t* __restrict__ lin,
                          const int32_t* __restrict__ ent_iface,
                          const int32_t* __restrict__ cstart, const int32_t* __restrict__ items,
                          int32_t* __restrict__ owner, int* flags) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nent) return;
  const int ifc = ent_iface[q];
  const int K = 3;
  int idx[3];
  node_multi(g, lin[q], idx);
  double X[3] = {coord(g, idx[0]), coord(g, idx[1]), g.d == 3 ? coord(g, idx[2]) : 0.0};
  int c0[3] = {min(idx[0], g.n - 1), min(idx[1], g.n - 1), g.d == 3 ? min(idx[2], g.n - 1) : 0};
  double eps = kTieEps * g.h * g.h;
  double dmin = INFINITY;
  int lo3 = g.d == 3 ? -K : 0, hi3 = g.d == 3 ? K : 0;
  for (int pass = 0; pass < 2; ++pass) {
    int best = INT_MAX;
    for (int a = -K; a <= K; ++a)
      for (int b = -K; b <= K; ++b)
        for (int c = lo3; c <= hi3; ++c) {
          int cc[3] = {c0[0] + a, c0[1] + b, c0[2] + c};
          if (cc[0] < 0 || cc[0] >= g.n || cc[1] < 0 || cc[1] >= g.n) continue;
          if (g.d == 3 && (cc[2] < 0 || cc[2] >= g.n)) continue;
          long long ci = cell_index(g, cc);
          for (int t = cstart[ci]; t < cstart[ci + 1]; ++t) {
            int i = items[t];
            if (V.iface[i] != ifc) continue;
            double d2 = dist2(V, g.d, i, X);
            if (pass == 0) dmin = fmin(dmin, d2);
            else if (d2 <= dmin + eps && i < best) best = i;
          }
        }
    if (pass == 0 && !(dmin < (double)(K * K) * g.h * g.h)) {
      // nothing certain within K h: global search
      atomicAdd(&flags[kFlagClosestFallback], 1);
      dmin = INFINITY;
      for (int i = 0; i < nb; ++i)
        if (V.iface[i] == ifc) dmin = fmin(dmin, dist2(V, g.d, i, X));
      int b2 = INT_MAX;
      for (int i = 0; i < nb; ++i)
        if (V.iface[i] == ifc && dist2(V, g.d, i, X) <= dmin + eps) {
          b2 = i;
          break;
        }
      if (b2 == INT_MAX) {
        // no DOF on this interface at all: reported, and an in-range owner
        flag_min(flags, kFlagNoOwner, q + 1);
        b2 = 0;
      }
      owner[q] = b2;
      return;
    }
    if (pass == 1) owner[q] = best;
  }
}

// Composite rows W[j][q] = sum_k phi_k(xi_q) (M^{-1})[k][j], so that C(q) =
// sum_j W[j][q] Q_j of the owner's collocation data.
__global__ void k_composite(Grid g, DofView V, int nent, const int32_t* __restrict__ lin,
                            const int32_t* __restrict__ owner, const double* __restrict__ minv,
                            double* __restrict__ W) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nent) return;
  const int n = c_exp.n;
  int idx[3];
  node_multi(g, lin[q], idx);
  int i = owner[q];
  double xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g.d; ++k) xi[k] = (coord(g, idx[k]) - V.x[k][i]) / g.h;
  double pw[3][5];
  powers(xi, g.d, pw);
  double ph[kMaxCoef];
  for (int e = 0; e < n; ++e) ph[e] = mono(pw, e);
  const double* Mi = minv + (size_t)i * n * n;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += ph[k] * Mi[k * n + j];
    W[(size_t)j * nent + q] = s;
  }
}

__global__ void k_corr_lists(Grid g, int nirr, const int32_t* __restrict__ lin,
                             const uint8_t* __restrict__ inside, const int32_t* __restrict__ map,
                             int32_t* __restrict__ corr_nb) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  int idx[3];
  node_multi(g, lin[q], idx);
  uint8_t c0 = inside[lin[q]];
  for (int s = 0; s < c_nb.count; ++s) {
    int nq[3] = {idx[0] + c_nb.off[s][0], idx[1] + c_nb.off[s][1], idx[2] + c_nb.off[s][2]};
    long long t = node_index(g, nq);
    corr_nb[(size_t)s * nirr + q] = (inside[t] != c0) ? map[t] : -1;
  }
}

// ---- several interfaces: correction entries (node, k) as a bit mask per
// node (bit k = C^(k+1) held there), then numbered in node order, then k.
__device__ __forceinline__ uint32_t label_bit(int lab) { return lab > 0 ? (1u << (lab - 1)) : 0u; }

// entries of the correction terms: every irregular node, for each label >= 1
// of its stencil (itself included)
__global__ void k_need_rhs(Grid g, int nirr, const int32_t* __restrict__ lin,
                           const uint8_t* __restrict__ inside, uint32_t* __restrict__ need) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  int idx[3];
  node_multi(g, lin[q], idx);
  uint32_t m = label_bit(inside[lin[q]]);
  for (int s = 0; s < c_nb.count; ++s) {
    int nq[3] = {idx[0] + c_nb.off[s][0], idx[1] + c_nb.off[s][1], idx[2] + c_nb.off[s][2]};
    m |= label_bit(inside[node_index(g, nq)]);
  }
  need[lin[q]] = m;
}

// entries per grid row (last axis), then numbered: emap[node] = the node's
// first entry, ent_lin / ent_iface per entry
__global__ void k_ent_row_count(Grid g, const uint32_t* __restrict__ need, int nrows,
                                int32_t* __restrict__ count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const uint32_t* f = need + (long long)r * (g.n + 1);
  int c = 0;
  for (int j = 0; j <= g.n; ++j) c += __popc(f[j]);
  count[r] = c;
}

__global__ void k_ent_row_fill(Grid g, const uint32_t* __restrict__ need, int nrows,
                               const int32_t* __restrict__ start, int32_t* __restrict__ emap,
                               int32_t* __restrict__ ent_lin, int32_t* __restrict__ ent_iface) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const long long base = (long long)r * (g.n + 1);
  int pos = start[r];
  for (int j = 0; j <= g.n; ++j) {
    uint32_t m = need[base + j];
    if (!m) continue;
    emap[base + j] = pos;
    for (int k = 0; k < KFBI_MAX_INTERFACES; ++k)
      if ((m >> k) & 1u) {
        ent_lin[pos] = (int32_t)(base + j);
        ent_iface[pos] = k;
        ++pos;
      }
  }
}

// the entry holding C^(k+1) at a node (the bit must be set)
__device__ __forceinline__ int entry_of(const uint32_t* need, const int32_t* emap, long long node,
                                        int k) {
  return emap[node] + __popc(need[node] & ((1u << k) - 1u));
}

// C_P = -sum_{l_Q != l_P} c (C^(l_P)(Q) - C^(l_Q)(Q)): per neighbour the entry
// of C^(l_Q)(Q) (added with +c) and of C^(l_P)(Q) (with -c), -1 for label 0
__global__ void k_corr_lists_multi(Grid g, int nirr, const int32_t* __restrict__ lin,
                                   const uint8_t* __restrict__ inside,
                                   const uint32_t* __restrict__ need,
                                   const int32_t* __restrict__ emap, int32_t* __restrict__ corr_a,
                                   int32_t* __restrict__ corr_b) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  int idx[3];
  node_multi(g, lin[q], idx);
  const int lp = inside[lin[q]];
  for (int s = 0; s < c_nb.count; ++s) {
    int nq[3] = {idx[0] + c_nb.off[s][0], idx[1] + c_nb.off[s][1], idx[2] + c_nb.off[s][2]};
    const long long t = node_index(g, nq);
    const int lq = inside[t];
    int a = -1, b = -1;
    if (lq != lp) {
      if (lq > 0) a = entry_of(need, emap, t, lq - 1);
      if (lp > 0) b = entry_of(need, emap, t, lp - 1);
    }
    corr_a[(size_t)s * nirr + q] = a;
    corr_b[(size_t)s * nirr + q] = b;
  }
}

// FP64 weights replaced in place by FP32 pairs (same 8 bytes): hi = the FP32
// rounding, lo = that of the rest.
__global__ void k_split_weights(int n, double* a, double* b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double* arr[2] = {a, b};
  for (int k = 0; k < 2; ++k) {
    const double v = arr[k][e];
    const float h = (float)v;
    reinterpret_cast<float2*>(arr[k])[e] = make_float2(h, (float)(v - (double)h));
  }
}

// ---------------------------------------------------------------------------
// Trace stencils and weighted least-squares weights (Sec. 5.5).
// ---------------------------------------------------------------------------
struct TraceParams {
  double rs2, ro2;     // squared radii in units of h
  int win;             // window half-width (ceil(R_s) + 1)
  int wside;           // 2 win + 1
  int wtotal;          // wside^d
};

// Window offset o of a trace stencil for side label t: nodes of label t
// within R_s, and nodes of another label within R_o that are irregular and
// hold C^(t) (need == nullptr: one interface, where they always do) or, where
// another interface is close (`close`), every node of another label within R_o.
__device__ __forceinline__ bool trace_select(const Grid& g, const TraceParams& T, const double* p,
                                             const int* n0, int o, int tlab, bool close,
                                             const uint8_t* inside, const uint8_t* irr,
                                             const uint32_t* need,
                                             long long* node_out, double* xi_out, double* r2_out,
                                             bool* across) {
  int off[3] = {0, 0, 0};
  int rem = o;
  for (int k = g.d - 1; k >= 0; --k) {
    off[k] = rem % T.wside - T.win;
    rem /= T.wside;
  }
  int idx[3] = {n0[0] + off[0], n0[1] + off[1], n0[2] + off[2]};
  for (int k = 0; k < g.d; ++k)
    if (idx[k] < 0 || idx[k] > g.n) return false;
  double xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g.d; ++k) xi[k] = (coord(g, idx[k]) - p[k]) / g.h;
  double r2 = xi[0] * xi[0];
  r2 = r2 + xi[1] * xi[1];
  if (g.d == 3) r2 = r2 + xi[2] * xi[2];
  long long t = node_index(g, idx);
  bool same = inside[t] == tlab;
  bool holds = close || tlab == 0 || need == nullptr || ((need[t] >> (tlab - 1)) & 1u);
  bool keep = (same && r2 <= T.rs2) || (!same && (close || irr[t]) && holds && r2 <= T.ro2);
  if (!keep) return false;
  *node_out = t;
  xi_out[0] = xi[0];
  xi_out[1] = xi[1];
  xi_out[2] = xi[2];
  *r2_out = r2;
  *across = !same;
  return true;
}

__device__ __forceinline__ void trace_centre(const Grid& g, const DofView& V, int i, double* p,
                                             int* n0) {
  p[0] = V.x[0][i];
  p[1] = V.x[1][i];
  p[2] = g.d == 3 ? V.x[2][i] : 0.0;
  n0[0] = n0[1] = n0[2] = 0;
  for (int k = 0; k < g.d; ++k) n0[k] = (int)floor((p[k] - g.lo) / g.h + 0.5);
}

// Several interfaces: a DOF of interface k is close to another interface if a
// node of a third label (not 0, not 1 + k) lies within R_s of it.
__global__ void k_trace_close(Grid g, TraceParams T, DofView V, int nb,
                              const uint8_t* __restrict__ inside, uint8_t* __restrict__ close) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double p[3];
  int n0[3];
  trace_centre(g, V, i, p, n0);
  const int own = V.iface[i] + 1;
  uint8_t c = 0;
  for (int o = 0; o < T.wtotal && !c; ++o) {
    int rem = o, idx[3] = {0, 0, 0};
    bool ok = true;
    double r2 = 0.0;
    for (int k = g.d - 1; k >= 0; --k) {
      idx[k] = n0[k] + rem % T.wside - T.win;
      rem /= T.wside;
      ok = ok && idx[k] >= 0 && idx[k] <= g.n;
    }
    if (!ok) continue;
    double xi[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < g.d; ++k) xi[k] = (coord(g, idx[k]) - p[k]) / g.h;
    r2 = xi[0] * xi[0];
    r2 = r2 + xi[1] * xi[1];
    if (g.d == 3) r2 = r2 + xi[2] * xi[2];
    const int lab = inside[node_index(g, idx)];
    if (lab != 0 && lab != own && r2 <= T.rs2) c = 1;
  }
  close[i] = c;
}

__global__ void k_trace_count(Grid g, TraceParams T, DofView V, int nb,
                              const uint8_t* __restrict__ inside, const uint8_t* __restrict__ irr,
                              const uint8_t* __restrict__ close, const uint32_t* __restrict__ need,
                              int32_t* __restrict__ count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nb) return;
  int side = t / nb, i = t % nb;
  double p[3];
  int n0[3];
  trace_centre(g, V, i, p, n0);
  const int tlab = side == 0 ? V.iface[i] + 1 : 0;
  const bool cl = close && close[i];
  int c = 0;
  for (int o = 0; o < T.wtotal; ++o) {
    long long node;
    double xi[3], r2;
    bool across;
    if (trace_select(g, T, p, n0, o, tlab, cl, inside, irr, need, &node, xi, &r2, &across)) ++c;
  }
  count[t] = c;
}

// Several interfaces: the entries the trace stencils of close DOFs need,
// C^(t) and C^(l_q) at each selected node q of another label, or-ed into need2.
__global__ void k_need_trace(Grid g, TraceParams T, DofView V, int nb,
                             const uint8_t* __restrict__ inside, const uint8_t* __restrict__ irr,
                             const uint8_t* __restrict__ close, uint32_t* __restrict__ need2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nb) return;
  int side = t / nb, i = t % nb;
  if (!close[i]) return;
  double p[3];
  int n0[3];
  trace_centre(g, V, i, p, n0);
  const int tlab = side == 0 ? V.iface[i] + 1 : 0;
  for (int o = 0; o < T.wtotal; ++o) {
    long long node;
    double xi[3], r2;
    bool across;
    if (trace_select(g, T, p, n0, o, tlab, true, inside, irr, nullptr, &node, xi, &r2, &across) &&
        across)
      atomicOr(&need2[node], label_bit(tlab) | label_bit(inside[node]));
  }
}

// One warp per (DOF, side).  A = diag(wt) V (m x n, column-major), QR, then
// the rows e_0^T pinv(A) diag(wt) (value) and c_n^T pinv(A) diag(wt) with
// c_n = (0, n/h, 0...) (normal derivative).
__global__ void k_trace_fill(Grid g, TraceParams T, DofView V, int nb,
                             const uint8_t* __restrict__ inside, const uint8_t* __restrict__ irr,
                             const int32_t* __restrict__ map, const int32_t* __restrict__ ptr_all,
                             const uint8_t* __restrict__ close, const uint32_t* __restrict__ need,
                             const uint32_t* __restrict__ need2, const int32_t* __restrict__ emap,
                             int mmax, double alpha, double beta, int32_t* __restrict__ node_out,
                             int32_t* __restrict__ irr_out, int32_t* __restrict__ irr2_out,
                             double* __restrict__ wv_out,
                             double* __restrict__ wn_out, double* __restrict__ w_out, int* flags) {
  extern __shared__ double sm[];
  const int n = c_exp.n;
  const int lda = mmax + 1;
  double* A = sm;                            // lda x n
  double* y0 = A + (size_t)lda * n;          // lda
  double* y1 = y0 + lda;                     // lda
  double* wt = y1 + lda;                     // lda
  double* rdiag = wt + lda;                  // n
  double* vn2 = rdiag + n;                   // n
  double* z = vn2 + n;                       // 2n
  int* nodes = (int*)(z + 2 * n);            // lda ints
  int* acr = nodes + lda;                    // lda ints
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x;
  if (t >= 2 * nb) return;
  const int side = t / nb, i = t % nb;
  const int d = g.d;
  double p[3] = {V.x[0][i], V.x[1][i], d == 3 ? V.x[2][i] : 0.0};
  double nv[3] = {V.n[0][i], V.n[1][i], d == 3 ? V.n[2][i] : 0.0};
  int n0[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) n0[k] = (int)floor((p[k] - g.lo) / g.h + 0.5);
  const int tlab = side == 0 ? V.iface[i] + 1 : 0;
  const bool cl = close && close[i];
  // ordered compaction of the selected window offsets
  int m = 0;
  for (int base = 0; base < T.wtotal; base += 32) {
    int o = base + lane;
    long long node = 0;
    double xi[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    bool across = false;
    bool sel = o < T.wtotal && trace_select(g, T, p, n0, o, tlab, cl, inside, irr, need, &node,
                                            xi, &r2, &across);
    unsigned ball = __ballot_sync(0xffffffffu, sel);
    if (sel) {
      int pos = m + __popc(ball & ((1u << lane) - 1u));
      if (pos < mmax) {
        nodes[pos] = (int)node;
        acr[pos] = across ? 1 : 0;
        double w = exp(-r2 / kTraceWeightScale);
        wt[pos] = w;
        double pw[3][5];
        powers(xi, d, pw);
        for (int e = 0; e < n; ++e) A[(size_t)e * lda + pos] = w * mono(pw, e);
      }
    }
    m += __popc(ball);
  }
  __syncwarp();
  m = min(m, mmax);
  bool ok = m >= n && warp_householder(A, lda, m, n, rdiag, vn2);
  // z0 = R^{-T} e_0, z1 = R^{-T} c_n  (forward substitution, lane 0)
  if (lane == 0) {
    for (int k = 0; k < n; ++k) {
      double c0 = (k == 0) ? 1.0 : 0.0;
      double c1 = 0.0;
      if (k >= 1 && k <= d) c1 = nv[k - 1] / g.h;
      double a0 = c0, a1 = c1;
      for (int j = 0; j < k; ++j) {
        double rjk = A[(size_t)k * lda + j];
        a0 -= rjk * z[j];
        a1 -= rjk * z[n + j];
      }
      const double ir = 1.0 / rdiag[k];
      z[k] = a0 * ir;
      z[n + k] = a1 * ir;
    }
  }
  __syncwarp();
  for (int r = lane; r < m; r += 32) {
    y0[r] = r < n ? z[r] : 0.0;
    y1[r] = r < n ? z[n + r] : 0.0;
  }
  __syncwarp();
  warp_apply_q(A, lda, m, n, vn2, y0, false);
  warp_apply_q(A, lda, m, n, vn2, y1, false);
  int off = ptr_all[t];
  for (int r = lane; r < m; r += 32) {
    double a = y0[r] * wt[r], b = y1[r] * wt[r];
    int node = nodes[r];
    node_out[off + r] = node;
    if (need2) {
      // several interfaces: u + C^(t) - C^(l_q) across, with C^(0) = 0
      const int lq = inside[node];
      irr_out[off + r] = acr[r] && tlab > 0 ? entry_of(need2, emap, node, tlab - 1) : -1;
      irr2_out[off + r] = acr[r] && lq > 0 ? entry_of(need2, emap, node, lq - 1) : -1;
    } else {
      irr_out[off + r] = acr[r] ? map[node] : -1;
    }
    wv_out[off + r] = a;
    wn_out[off + r] = b;
    w_out[off + r] = alpha * a + beta * b;
  }
  double rmax = 0.0, rmin = INFINITY;
  for (int k = 0; k < n; ++k) {
    rmax = fmax(rmax, fabs(rdiag[k]));
    rmin = fmin(rmin, fabs(rdiag[k]));
  }
  if (lane == 0 && (!ok || !(rmin > 1e-10 * rmax))) flag_min(flags, kFlagTraceSingular, i + 1);
}

}  // namespace

cudaError_t count_nonfinite(const double* a, long long n, cudaStream_t st, long long* out) {
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(*d), st);
  if (e != cudaSuccess) return e;
  unsigned long long h = 0;
  cudaMemsetAsync(d, 0, sizeof(*d), st);
  k_count_nonfinite<<<(int)std::min<long long>(div_up(n, 256), 152 * 8), 256, 0, st>>>(a, n, d);
  cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  *out = (long long)h;
  return e;
}

// ---------------------------------------------------------------------------
// Host orchestration.
// ---------------------------------------------------------------------------
void make_exponents(int d, int p, Exponents* out) {
  int c = 0;
  for (int t = 0; t <= p; ++t) {
    if (d == 2) {
      for (int l = t; l >= 0; --l) {
        out->e[c][0] = (int8_t)l;
        out->e[c][1] = (int8_t)(t - l);
        out->e[c][2] = 0;
        ++c;
      }
    } else {
      for (int l = t; l >= 0; --l)
        for (int m = t - l; m >= 0; --m) {
          out->e[c][0] = (int8_t)l;
          out->e[c][1] = (int8_t)m;
          out->e[c][2] = (int8_t)(t - l - m);
          ++c;
        }
    }
  }
  out->n = c;
}

static void lattice(int order, bool shifted, std::vector<std::pair<int, int>>* dset,
                    std::vector<int>* npos) {
  int low = (order == 4 && shifted) ? -1 : 0;
  int top_d = order + 2 * low;
  int top_n = order - 1 + 2 * low;
  dset->clear();
  npos->clear();
  for (int a = low; a <= order; ++a)
    for (int b = low; b <= order; ++b)
      if (a + b <= top_d) dset->push_back({a, b});
  for (size_t k = 0; k < dset->size(); ++k)
    if ((*dset)[k].first + (*dset)[k].second <= top_n) npos->push_back((int)k);
}

static kfbi_status check_flags(kfbi_problem* p, const char* stage) {
  int h[kFlagCount];
  KFBI_CUDA(p, cudaMemcpyAsync(h, p->d_flags, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  if (h[kFlagNoOwner] != kFlagSentinel)
    return fail(p, KFBI_ERR_GEOMETRY, std::string(stage) + ": interface of correction entry " +
                                          std::to_string(h[kFlagNoOwner] - 1) + " has no DOF");
  if (h[kFlagOutOfBox] != kFlagSentinel)
    return fail(p, KFBI_ERR_GEOMETRY, std::string(stage) + ": stencil of DOF " +
                                          std::to_string(h[kFlagOutOfBox] - 1) + " leaves the box");
  if (h[kFlagGeometry] != kFlagSentinel)
    return fail(p, KFBI_ERR_GEOMETRY, std::string(stage) + ": no complete collocation stencil at DOF " +
                                          std::to_string(h[kFlagGeometry] - 1));
  if (h[kFlagSingular] != kFlagSentinel)
    return fail(p, KFBI_ERR_SINGULAR, std::string(stage) + ": singular collocation matrix at DOF " +
                                          std::to_string(h[kFlagSingular] - 1));
  if (h[kFlagTraceSingular] != kFlagSentinel)
    return fail(p, KFBI_ERR_SINGULAR, std::string(stage) + ": singular trace fit at DOF " +
                                          std::to_string(h[kFlagTraceSingular] - 1));
  return KFBI_OK;
}

// out[i] = base + sum_{j<i} in[j] and out[n] = base + total, on stream st:
// one block for short arrays, the multi-block scan otherwise.
static kfbi_status scan_exclusive(kfbi_problem* p, const int32_t* in, int32_t* out, int n,
                                  int32_t base, cudaStream_t st) {
  if (n <= (1 << 16)) {
    k_exclusive_scan<<<1, 1024, 0, st>>>(in, out, n, base);
    KFBI_CUDA(p, cudaGetLastError());
    return KFBI_OK;
  }
  const int nblk = div_up(n, kScanChunk);
  int32_t *bsum = nullptr, *boff = nullptr;
  KFBI_CUDA(p, galloc(p, &bsum, nblk));
  KFBI_CUDA(p, galloc(p, &boff, nblk + 1));
  k_scan_sums<<<nblk, 1024, 0, st>>>(in, n, bsum);
  k_exclusive_scan<<<1, 1024, 0, st>>>(bsum, boff, nblk, base);
  k_scan_apply<<<nblk, 1024, 0, st>>>(in, n, boff, nblk, out);
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status build_geometry(kfbi_problem* p) {
  const Grid g = p->g;
  const int d = g.d, n = g.n, n1 = n + 1;
  const long long nodes = g.nodes();
  cudaStream_t st = p->stream;
  LevelSet L = p->ls;

  {
    int h[kFlagCount];
    for (int k = 0; k < kFlagCount; ++k) h[k] = kFlagSentinel;
    h[kFlagClosestFallback] = 0;
    KFBI_CUDA(p, galloc(p, &p->d_flags, kFlagCount));
    KFBI_CUDA(p, cudaMemcpyAsync(p->d_flags, h, sizeof(h), cudaMemcpyHostToDevice, st));
  }
  KFBI_CUDA(p, galloc(p, &p->inside, nodes));
  k_classify<<<div_up(nodes, 256), 256, 0, st>>>(g, L, p->inside);
  KFBI_CUDA(p, cudaGetLastError());

  // ---- DOFs, per family: candidate points per line (a warp per line),
  // their roots (a thread per candidate), then the kept ones in DOF order
  const int nlines = d == 2 ? n1 : n1 * n1;
  p->nlines = nlines;
  const bool multi = p->n_iface > 1;
  LineDesc D[3];
  long long strides[3] = {d == 2 ? n1 : (long long)n1 * n1, d == 2 ? 1 : n1, 1};
  struct Cand {
    int n = 0, kept = 0;
    int32_t *start = nullptr, *line = nullptr, *edge = nullptr, *iface = nullptr, *keep = nullptr,
            *kpos = nullptr;
    double *x = nullptr, *nv = nullptr;
  } C[3];
  // (the candidate arrays are arena temporaries: nothing to free)
  auto free_cand = [&]() {
    for (int r = 0; r < 3; ++r) C[r] = Cand();
  };
  int32_t* ccnt = nullptr;
  KFBI_CUDA(p, galloc(p, &ccnt, nlines));
  int32_t base = 0;
  for (int r = 0; r < d; ++r) {
    D[r].r = r;
    int o[2], no = 0;
    for (int k = 0; k < d; ++k)
      if (k != r) o[no++] = k;
    D[r].oa = o[0];
    D[r].ob = d == 3 ? o[1] : -1;
    D[r].sr = strides[r];
    D[r].sa = strides[o[0]];
    D[r].sb = d == 3 ? strides[o[1]] : 0;
    Cand& c = C[r];
    k_cand_count<<<div_up(nlines, kLineWarps), 32 * kLineWarps, 0, st>>>(g, L, D[r], p->inside, multi,
                                                                        nlines, ccnt);
    KFBI_CUDA(p, cudaGetLastError());
    KFBI_CUDA(p, galloc(p, &c.start, nlines + 1));
    KFBI_TRY(scan_exclusive(p, ccnt, c.start, nlines, 0, st));
    KFBI_CUDA(p, cudaMemcpyAsync(&c.n, c.start + nlines, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(p, cudaStreamSynchronize(st));
    KFBI_CUDA(p, galloc(p, &c.kpos, c.n + 1));
    if (c.n > 0) {
      KFBI_CUDA(p, galloc(p, &c.line, c.n));
      KFBI_CUDA(p, galloc(p, &c.edge, c.n));
      KFBI_CUDA(p, galloc(p, &c.iface, c.n));
      KFBI_CUDA(p, galloc(p, &c.keep, c.n));
      KFBI_CUDA(p, galloc(p, &c.x, 3 * (size_t)c.n));
      KFBI_CUDA(p, galloc(p, &c.nv, 3 * (size_t)c.n));
      k_cand_fill<<<div_up(nlines, kLineWarps), 32 * kLineWarps, 0, st>>>(g, L, D[r], p->inside, multi,
                                                                         nlines, c.start, c.line, c.edge,
                                                                         c.iface);
      // one warp per block: the FP64-bound root iterations spread over all SMs
      k_cand_roots<<<div_up(c.n, 32), 32, 0, st>>>(g, L, D[r], c.n, p->cos_alpha, c.line, c.edge, c.iface,
                                                   c.x, c.nv, c.keep);
      KFBI_CUDA(p, cudaGetLastError());
      KFBI_TRY(scan_exclusive(p, c.keep, c.kpos, c.n, 0, st));
      KFBI_CUDA(p, cudaMemcpyAsync(&c.kept, c.kpos + c.n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      KFBI_CUDA(p, cudaStreamSynchronize(st));
    } else {
      KFBI_CUDA(p, cudaMemsetAsync(c.kpos, 0, sizeof(int32_t), st));
    }
    KFBI_CUDA(p, galloc(p, &p->line_start[r], nlines + 1));
    k_cand_line_start<<<div_up(nlines + 1, 256), 256, 0, st>>>(nlines, base, c.start, c.kpos,
                                                               p->line_start[r]);
    KFBI_CUDA(p, cudaGetLastError());
    base += c.kept;
  }
  p->nb = base;
  if (p->nb == 0) {
    free_cand();
    return fail(p, KFBI_ERR_GEOMETRY, "the interface does not cross the grid");
  }
  const int nb = p->nb;
  for (int k = 0; k < d; ++k) {
    KFBI_CUDA(p, galloc(p, &p->x[k], nb));
    KFBI_CUDA(p, galloc(p, &p->nrm[k], nb));
  }
  KFBI_CUDA(p, galloc(p, &p->family, nb));
  KFBI_CUDA(p, galloc(p, &p->dof_iface, nb));
  KFBI_CUDA(p, galloc(p, &p->edge, nb));
  KFBI_CUDA(p, galloc(p, &p->axis, nb));
  KFBI_CUDA(p, galloc(p, &p->st_axis, nb));
  {
    int32_t fbase = 0;
    for (int r = 0; r < d; ++r) {
      const Cand& c = C[r];
      if (c.n > 0)
        k_cand_scatter<<<div_up(c.n, 128), 128, 0, st>>>(
            g, D[r], c.n, fbase, c.kpos, c.keep, c.edge, c.iface, c.x, c.nv, p->x[0], p->x[1],
            d == 3 ? p->x[2] : p->x[0], p->nrm[0], p->nrm[1], d == 3 ? p->nrm[2] : p->nrm[0], p->family,
            p->edge, p->axis, p->dof_iface);
      KFBI_CUDA(p, cudaGetLastError());
      fbase += c.kept;
    }
  }
  free_cand();

  DofView V;
  for (int k = 0; k < 3; ++k) {
    V.x[k] = k < d ? p->x[k] : nullptr;
    V.n[k] = k < d ? p->nrm[k] : nullptr;
    V.line_start[k] = k < d ? p->line_start[k] : nullptr;
  }
  V.iface = p->dof_iface;

  // ---- stencil tables
  StencilTables T;
  memset(&T, 0, sizeof(T));
  const int order = p->cfg.order;
  if (order == 2) {
    T.npde = 1;
  } else if (d == 2) {
    const int off[6][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}};
    T.npde = 6;
    for (int s = 0; s < 6; ++s) {
      T.pde_off[s][0] = off[s][0];
      T.pde_off[s][1] = off[s][1];
    }
  } else {
    const int off[10][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                            {0, 0, 1}, {0, 0, -1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    T.npde = 10;
    for (int s = 0; s < 10; ++s)
      for (int k = 0; k < 3; ++k) T.pde_off[s][k] = off[s][k];
  }
  if (d == 2) {
    T.ndir = order + 1;
    T.nneu = order;
    T.ntries = 1;
  } else {
    T.ntries = order == 4 ? 2 : 1;
    for (int tv = 0; tv < T.ntries; ++tv) {
      std::vector<std::pair<int, int>> ds;
      std::vector<int> np;
      lattice(order, tv == 0, &ds, &np);
      T.ndir = (int)ds.size();
      T.nneu = (int)np.size();
      for (size_t s = 0; s < ds.size(); ++s) {
        T.dset[tv][s][0] = ds[s].first;
        T.dset[tv][s][1] = ds[s].second;
      }
      for (size_t s = 0; s < np.size(); ++s) T.nset_pos[tv][s] = np[s];
    }
  }
  p->npde = T.npde;
  p->ndir = T.ndir;
  p->nneu = T.nneu;
  KFBI_CUDA(p, cudaMemcpyToSymbolAsync(c_st, &T, sizeof(T), 0, cudaMemcpyHostToDevice, st));
  Exponents E;
  make_exponents(d, order, &E);
  p->ncoef = E.n;
  if (p->npde + p->ndir + p->nneu != p->ncoef)
    return fail(p, KFBI_ERR_UNSUPPORTED, "collocation system is not square");
  KFBI_CUDA(p, cudaMemcpyToSymbolAsync(c_exp, &E, sizeof(E), 0, cudaMemcpyHostToDevice, st));

  KFBI_CUDA(p, galloc(p, &p->pde_node, (size_t)nb * p->npde));
  KFBI_CUDA(p, galloc(p, &p->dir_idx, (size_t)nb * p->ndir));
  KFBI_CUDA(p, galloc(p, &p->neu_idx, (size_t)nb * p->nneu));
  k_stencils<<<div_up(nb, 128), 128, 0, st>>>(g, order, p->cos_alpha, V, nb, p->axis,
                                               p->pde_node, p->dir_idx, p->neu_idx, p->st_axis,
                                               p->d_flags);
  KFBI_CUDA(p, cudaGetLastError());
  KFBI_TRY(check_flags(p, "collocation stencils"));

  const int nc = p->ncoef;
  KFBI_CUDA(p, galloc(p, &p->minv, (size_t)nb * nc * nc));
  {
    size_t smem = sizeof(double) * ((size_t)(nc + 1) * nc * 2 + 2 * nc);
    // per-kernel process-wide attribute: raise it to the device maximum once
    int dev = 0, optin = 0;
    KFBI_CUDA(p, cudaGetDevice(&dev));
    KFBI_CUDA(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KFBI_CUDA(p, cudaFuncSetAttribute(k_collocation_factor,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KFBI_CUDA(p, cudaFuncSetAttribute(k_trace_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin));
    k_collocation_factor<<<nb, 32, smem, st>>>(g, p->kt, V, nb, p->pde_node, p->dir_idx,
                                               p->neu_idx, p->minv, p->d_flags);
    KFBI_CUDA(p, cudaGetLastError());
  }
  KFBI_TRY(check_flags(p, "collocation factor"));

  // ---- irregular nodes
  NbTable NT;
  memset(&NT, 0, sizeof(NT));
  {
    int c = 0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        for (int e = (d == 3 ? -1 : 0); e <= (d == 3 ? 1 : 0); ++e) {
          int nz = (a != 0) + (b != 0) + (e != 0);
          if (nz == 0) continue;
          if (order == 2 && nz > 1) continue;
          NT.off[c][0] = a;
          NT.off[c][1] = b;
          NT.off[c][2] = e;
          ++c;
        }
    NT.count = c;
  }
  p->n_nb = NT.count;
  KFBI_CUDA(p, cudaMemcpyToSymbolAsync(c_nb, &NT, sizeof(NT), 0, cudaMemcpyHostToDevice, st));
  KFBI_CUDA(p, galloc(p, &p->irr_flag, nodes));
  k_irregular_flags<<<div_up(nodes, 256), 256, 0, st>>>(g, p->inside, p->irr_flag);
  KFBI_CUDA(p, cudaGetLastError());
  const int nrows = (int)(nodes / n1);
  int32_t *rcnt = nullptr, *rstart = nullptr, *map = nullptr;
  KFBI_CUDA(p, galloc(p, &rcnt, nrows));
  KFBI_CUDA(p, galloc(p, &rstart, nrows + 1));
  KFBI_CUDA(p, galloc(p, &map, nodes));
  KFBI_CUDA(p, cudaMemsetAsync(map, 0xff, sizeof(int32_t) * nodes, st));
  k_row_count<<<div_up(nrows, 128), 128, 0, st>>>(g, p->irr_flag, nrows, rcnt);
  KFBI_TRY(scan_exclusive(p, rcnt, rstart, nrows, 0, st));
  int32_t nirr = 0;
  KFBI_CUDA(p, cudaMemcpyAsync(&nirr, rstart + nrows, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p, cudaStreamSynchronize(st));
  p->nirr = nirr;
  if (nirr == 0) return fail(p, KFBI_ERR_GEOMETRY, "no irregular nodes");
  KFBI_CUDA(p, galloc(p, &p->irr_lin, nirr));
  KFBI_CUDA(p, galloc(p, &p->irr_inside, nirr));
  k_row_fill<<<div_up(nrows, 128), 128, 0, st>>>(g, p->irr_flag, p->inside, nrows, rstart,
                                                  p->irr_lin, p->irr_inside, map);
  KFBI_CUDA(p, cudaGetLastError());

  // ---- trace stencil parameters (Sec. 5.5)
  TraceParams TP;
  double rs = order == 4 ? 4.0 : 3.0, ro = order == 4 ? 2.5 : 1.5;
  TP.rs2 = rs * rs;
  TP.ro2 = ro * ro;
  TP.win = (int)std::ceil(rs) + 1;
  TP.wside = 2 * TP.win + 1;
  TP.wtotal = d == 2 ? TP.wside * TP.wside : TP.wside * TP.wside * TP.wside;

  // ---- correction entries (node, interface k)
  uint32_t *need = nullptr, *need2 = nullptr;
  uint8_t* close = nullptr;
  int32_t* emap = nullptr;
  if (!multi) {
    // one per irregular node, in its order
    p->nent = nirr;
    KFBI_CUDA(p, galloc(p, &p->ent_lin, nirr));
    KFBI_CUDA(p, galloc(p, &p->ent_iface, nirr));
    KFBI_CUDA(p, cudaMemcpyAsync(p->ent_lin, p->irr_lin, sizeof(int32_t) * nirr,
                                 cudaMemcpyDeviceToDevice, st));
    KFBI_CUDA(p, cudaMemsetAsync(p->ent_iface, 0, sizeof(int32_t) * nirr, st));
  } else {
    KFBI_CUDA(p, galloc(p, &need, nodes));
    KFBI_CUDA(p, galloc(p, &need2, nodes));
    KFBI_CUDA(p, galloc(p, &close, nb));
    KFBI_CUDA(p, galloc(p, &emap, nodes));
    KFBI_CUDA(p, cudaMemsetAsync(need, 0, sizeof(uint32_t) * nodes, st));
    KFBI_CUDA(p, cudaMemsetAsync(emap, 0xff, sizeof(int32_t) * nodes, st));
    k_need_rhs<<<div_up(nirr, 128), 128, 0, st>>>(g, nirr, p->irr_lin, p->inside, need);
    KFBI_CUDA(p, cudaMemcpyAsync(need2, need, sizeof(uint32_t) * nodes, cudaMemcpyDeviceToDevice, st));
    k_trace_close<<<div_up(nb, 128), 128, 0, st>>>(g, TP, V, nb, p->inside, close);
    k_need_trace<<<div_up(2 * nb, 128), 128, 0, st>>>(g, TP, V, nb, p->inside, p->irr_flag, close,
                                                      need2);
    KFBI_CUDA(p, cudaGetLastError());
    int32_t *ecnt = nullptr, *estart = nullptr;
    KFBI_CUDA(p, galloc(p, &ecnt, nrows));
    KFBI_CUDA(p, galloc(p, &estart, nrows + 1));
    k_ent_row_count<<<div_up(nrows, 128), 128, 0, st>>>(g, need2, nrows, ecnt);
    KFBI_TRY(scan_exclusive(p, ecnt, estart, nrows, 0, st));
    int32_t nent = 0;
    KFBI_CUDA(p, cudaMemcpyAsync(&nent, estart + nrows, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(p, cudaStreamSynchronize(st));
    p->nent = nent;
    KFBI_CUDA(p, galloc(p, &p->ent_lin, nent));
    KFBI_CUDA(p, galloc(p, &p->ent_iface, nent));
    k_ent_row_fill<<<div_up(nrows, 128), 128, 0, st>>>(g, need2, nrows, estart, emap, p->ent_lin,
                                                        p->ent_iface);
    KFBI_CUDA(p, cudaGetLastError());
  }
  const int nent = p->nent;
  KFBI_CUDA(p, galloc(p, &p->ent_owner, nent));

  // ---- closest primary points via a cell list
  {
    long long ncell = d == 2 ? (long long)n * n : (long long)n * n * n;
    int32_t *ccnt = nullptr, *cstart = nullptr, *cur = nullptr, *items = nullptr;
    KFBI_CUDA(p, galloc(p, &ccnt, ncell));
    KFBI_CUDA(p, galloc(p, &cstart, ncell + 1));
    KFBI_CUDA(p, galloc(p, &cur, ncell));
    KFBI_CUDA(p, galloc(p, &items, nb));
    KFBI_CUDA(p, cudaMemsetAsync(ccnt, 0, sizeof(int32_t) * ncell, st));
    KFBI_CUDA(p, cudaMemsetAsync(cur, 0, sizeof(int32_t) * ncell, st));
    k_cell_count<<<div_up(nb, 256), 256, 0, st>>>(g, V, nb, ccnt);
    KFBI_TRY(scan_exclusive(p, ccnt, cstart, (int)ncell, 0, st));
    k_cell_fill<<<div_up(nb, 256), 256, 0, st>>>(g, V, nb, cstart, cur, items);
    k_closest<<<div_up(nent, 128), 128, 0, st>>>(g, V, nb, nent, p->ent_lin, p->ent_iface, cstart,
                                                 items, p->ent_owner, p->d_flags);
    KFBI_CUDA(p, cudaGetLastError());
  }
  KFBI_TRY(check_flags(p, "closest primary points"));
  KFBI_CUDA(p, galloc(p, &p->ent_w, (size_t)nc * nent));
  k_composite<<<div_up(nent, 128), 128, 0, st>>>(g, V, nent, p->ent_lin, p->ent_owner, p->minv,
                                                  p->ent_w);
  KFBI_CUDA(p, cudaGetLastError());
  KFBI_CUDA(p, galloc(p, &p->corr_nb, (size_t)p->n_nb * nirr));
  if (!multi) {
    k_corr_lists<<<div_up(nirr, 128), 128, 0, st>>>(g, nirr, p->irr_lin, p->inside, map, p->corr_nb);
  } else {
    KFBI_CUDA(p, galloc(p, &p->corr_nb2, (size_t)p->n_nb * nirr));
    k_corr_lists_multi<<<div_up(nirr, 128), 128, 0, st>>>(g, nirr, p->irr_lin, p->inside, need2,
                                                          emap, p->corr_nb, p->corr_nb2);
  }
  KFBI_CUDA(p, cudaGetLastError());

  // ---- trace stencils
  int32_t *tcnt = nullptr, *tptr = nullptr;
  KFBI_CUDA(p, galloc(p, &tcnt, 2 * nb));
  KFBI_CUDA(p, galloc(p, &tptr, 2 * nb + 1));
  k_trace_count<<<div_up(2 * nb, 128), 128, 0, st>>>(g, TP, V, nb, p->inside, p->irr_flag, close,
                                                       need, tcnt);
  KFBI_TRY(scan_exclusive(p, tcnt, tptr, 2 * nb, 0, st));
  KFBI_CUDA(p, cudaGetLastError());
  std::vector<int32_t> hptr(2 * nb + 1), hcnt(2 * nb);
  KFBI_CUDA(p, cudaMemcpyAsync(hptr.data(), tptr, sizeof(int32_t) * (2 * nb + 1),
                               cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p, cudaMemcpyAsync(hcnt.data(), tcnt, sizeof(int32_t) * 2 * nb, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(p, cudaStreamSynchronize(st));
  int mmax = 0;
  for (int k = 0; k < 2 * nb; ++k) mmax = std::max(mmax, hcnt[k]);
  const int nnz_all = hptr[2 * nb];
  int32_t *tnode = nullptr, *tirr = nullptr, *tirr2 = nullptr;
  double *twv = nullptr, *twn = nullptr, *tw = nullptr;
  KFBI_CUDA(p, galloc(p, &tnode, nnz_all));
  KFBI_CUDA(p, galloc(p, &tirr, nnz_all));
  if (multi) KFBI_CUDA(p, galloc(p, &tirr2, nnz_all));
  KFBI_CUDA(p, galloc(p, &twv, nnz_all));
  KFBI_CUDA(p, galloc(p, &twn, nnz_all));
  KFBI_CUDA(p, galloc(p, &tw, nnz_all));
  {
    double alpha = p->cfg.kind == KFBI_DIRICHLET_INTERIOR ? 0.5 : 0.0;
    double beta = p->cfg.kind == KFBI_DIRICHLET_INTERIOR ? 0.0 : 0.5;
    const int lda = mmax + 1;
    size_t smem = sizeof(double) * ((size_t)lda * nc + 3 * (size_t)lda + 4 * nc) +
                  sizeof(int) * 2 * (size_t)lda;
    int dev = 0, optin = 0;
    KFBI_CUDA(p, cudaGetDevice(&dev));
    KFBI_CUDA(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin)
      return fail(p, KFBI_ERR_UNSUPPORTED, "trace stencil too large for shared memory");
    k_trace_fill<<<2 * nb, 32, smem, st>>>(g, TP, V, nb, p->inside, p->irr_flag, map, tptr, close,
                                           need, need2, emap, mmax, alpha, beta, tnode, tirr,
                                           tirr2, twv, twn, tw, p->d_flags);
    KFBI_CUDA(p, cudaGetLastError());
  }
  KFBI_TRY(check_flags(p, "trace weights"));
  // split the all-sides CSR into the two per-side CSRs (pointers into one allocation)
  for (int s = 0; s < 2; ++s) {
    TraceCSR& c = p->tr[s];
    KFBI_CUDA(p, galloc(p, &c.ptr, nb + 1));
    std::vector<int32_t> sp(nb + 1);
    int32_t b0 = hptr[(size_t)s * nb];
    for (int k = 0; k <= nb; ++k) sp[k] = hptr[(size_t)s * nb + k] - b0;
    KFBI_CUDA(p, cudaMemcpyAsync(c.ptr, sp.data(), sizeof(int32_t) * (nb + 1),
                                 cudaMemcpyHostToDevice, st));
    c.nnz = sp[nb];
    c.node = tnode + b0;
    c.irr = tirr + b0;
    c.irr2 = multi ? tirr2 + b0 : nullptr;
    c.wv = twv + b0;
    c.wn = twn + b0;
    c.w = tw + b0;
  }
  if (d == 3 && nnz_all > 0) {
    // the 3D four-trace kernel reads value and normal-derivative weights as
    // FP32 pairs (the operator's own trace keeps FP64: it is memory-bound)
    k_split_weights<<<div_up(nnz_all, 256), 256, 0, st>>>(nnz_all, twv, twn);
    KFBI_CUDA(p, cudaGetLastError());
    for (int s = 0; s < 2; ++s) {
      TraceCSR& c = p->tr[s];
      c.wv2 = reinterpret_cast<float2*>(c.wv);
      c.wn2 = reinterpret_cast<float2*>(c.wn);
    }
  }
  KFBI_CUDA(p, cudaStreamSynchronize(st));
  return KFBI_OK;
}

}  // namespace kfbi
