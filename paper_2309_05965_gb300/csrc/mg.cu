// Geometric multigrid box solve (Algorithm 1, Step 3.3; the paper names
// geometric multigrid as the alternative fast solver but gives no design).
//
// Design (this library's):
//   * levels N, N/2, ..., 4 with the compact operator rediscretised at h_l =
//     2^l h (same kappa~);
//   * smoother: weighted Jacobi, omega = 0.909 (2D) / 1.136 (3D), the values that
//     minimise the high-frequency amplification of the 9/27-point compact
//     operators (smoothing factor 0.45 in both); 4/5 and 6/7 for the 2nd-order
//     5/7-point operators (smoothing factors 0.6 and 5/7);
//   * full-weighting restriction, (bi/tri)linear prolongation, V(2,2) cycles;
//   * coarsest level (3^d unknowns) solved exactly with a dense inverse;
//   * levels with N <= kCoarseN run the rest of the V-cycle inside one CTA
//     (grids of at most 31^2 / 15^3 unknowns), removing per-level launches;
//   * FP64 mode: V-cycles until max|R - A u| <= tol max|R|;
//   * mixed mode: FP32 V-cycles on A e = r with the FP64 residual r = R - A u
//     recomputed after each group of cycles (iterative refinement);
//   * convergence is tracked on the device; cycles after convergence exit at
//     their first instruction (graph-capturable, no host synchronisation).
#include <cmath>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

namespace {

constexpr int kCoarseN2 = 32;   // 2D: levels with N <= 32 run in one CTA
constexpr int kCoarseN3 = 16;   // 3D
constexpr int kNu = 2;          // pre- and post-smoothing sweeps (the kernels ping-pong u -> t -> u)
static_assert(kNu == 2, "the sweeps alternate between u and t");

template <typename T>
struct Lvl {
  int n;
  T c[4];        // stencil coefficients by number of nonzero offsets
  T dinv_w;      // omega / c0
  T* u;
  T* f;
  T* t;          // Jacobi ping-pong / residual
};

template <typename T>
struct LvlArgs {
  int d, order, nlev;
  Lvl<T> L[16];
  const T* cinv;   // coarsest dense inverse, m x m, m = 3^d
};

__device__ __forceinline__ long long lin(int d, int n1, int i0, int i1, int i2) {
  return d == 2 ? (long long)i1 * n1 + i2 : ((long long)i0 * n1 + i1) * n1 + i2;
}

// A u at interior node t (grid of n1 nodes per axis)
template <typename T>
__device__ __forceinline__ T apply_at(int d, int order, int n1, const T* c, const T* up) {
  if (d == 2) {
    T s1 = (up[-1] + up[1]) + (up[-n1] + up[n1]);
    T a = c[0] * up[0] + c[1] * s1;
    if (order == 4) a += c[2] * ((up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]));
    return a;
  }
  const long long s = (long long)n1 * n1;
  T f = (up[-1] + up[1]) + (up[-n1] + up[n1]) + (up[-s] + up[s]);
  T a = c[0] * up[0] + c[1] * f;
  if (order == 4) {
    T e = (up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]) + (up[-s - 1] + up[-s + 1]) +
          (up[s - 1] + up[s + 1]) + (up[-s - n1] + up[-s + n1]) + (up[s - n1] + up[s + n1]);
    T k = (up[-s - n1 - 1] + up[-s - n1 + 1]) + (up[-s + n1 - 1] + up[-s + n1 + 1]) +
          (up[s - n1 - 1] + up[s - n1 + 1]) + (up[s + n1 - 1] + up[s + n1 + 1]);
    a += c[2] * e + c[3] * k;
  }
  return a;
}

// ---- marching stencil sweeps ------------------------------------------------
// A thread owns one line along the slowest axis (a column (i1, j) in 3D, a
// column j in 2D) and marches along it, keeping three consecutive slices of
// the per-slice sums in registers:
//   3D slice k: centre C, in-plane edge sum S1 (4), in-plane corner sum S2 (4);
//     A u = c0 C(k) + c1 (S1(k) + C(k-1) + C(k+1)) + c2 (S2(k) + S1(k-1) + S1(k+1))
//           + c3 (S2(k-1) + S2(k+1));
//   2D row k: centre C, horizontal pair H;
//     A u = c0 C(k) + c1 (H(k) + C(k-1) + C(k+1)) + c2 (H(k-1) + H(k+1)).
// Each new slice costs 9 (3D) / 3 (2D) loads instead of 27 / 9 per point.
// mode 0: Jacobi uout = uin + w D^-1 (f - A uin) (zero_guess: uout = w D^-1 f);
// mode 1: residual r = f - A u.  Only interior nodes are written (boundary
// nodes of every level buffer are zero from allocation and never written).
constexpr int kMarchX = 128;
constexpr int kMarchZ = 16;   // slices per thread

template <typename T>
struct Slice {
  T C, S1, S2;
};

template <typename T>
__device__ __forceinline__ Slice<T> slice3(const T* __restrict__ u, int t, int n1) {
  const T* p = u + t;
  Slice<T> s;
  s.C = p[0];
  s.S1 = (p[-1] + p[1]) + (p[-n1] + p[n1]);
  s.S2 = (p[-n1 - 1] + p[-n1 + 1]) + (p[n1 - 1] + p[n1 + 1]);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kMarchX) k_march(int d, Lvl<T> L, const T* __restrict__ uin, T* __restrict__ out,
                                                   int mode, int zero_guess, const int* skip) {
  if (skip && *skip) return;
  const int n = L.n, n1 = n + 1;
  const int j = 1 + blockIdx.x * kMarchX + threadIdx.x;
  if (j >= n) return;
  const T c0 = L.c[0], c1 = L.c[1], c2 = L.c[2], c3 = L.c[3];
  if (d == 2) {
    const int k0 = 1 + blockIdx.y * kMarchZ, k1 = min(n, k0 + kMarchZ);
    if (zero_guess) {
      for (int k = k0; k < k1; ++k) out[k * n1 + j] = L.dinv_w * L.f[k * n1 + j];
      return;
    }
    int t = (k0 - 1) * n1 + j;
    T Cm = uin[t], Hm = uin[t - 1] + uin[t + 1];
    t += n1;
    T C0 = uin[t], H0 = uin[t - 1] + uin[t + 1];
    for (int k = k0; k < k1; ++k, t += n1) {
      const T Cp = uin[t + n1], Hp = uin[t + n1 - 1] + uin[t + n1 + 1];
      const T au = c0 * C0 + c1 * (H0 + Cm + Cp) + c2 * (Hm + Hp);
      const T f = L.f[t];
      out[t] = mode == 0 ? C0 + L.dinv_w * (f - au) : f - au;
      Cm = C0; Hm = H0;
      C0 = Cp; H0 = Hp;
    }
    return;
  }
  const int i1 = 1 + blockIdx.y;
  const int k0 = 1 + blockIdx.z * kMarchZ, k1 = min(n, k0 + kMarchZ);
  const int plane = n1 * n1;
  if (zero_guess) {
    for (int k = k0; k < k1; ++k) {
      const int t = (k * n1 + i1) * n1 + j;
      out[t] = L.dinv_w * L.f[t];
    }
    return;
  }
  int t = ((k0 - 1) * n1 + i1) * n1 + j;
  Slice<T> m = slice3(uin, t, n1);
  t += plane;
  Slice<T> c = slice3(uin, t, n1);
  for (int k = k0; k < k1; ++k, t += plane) {
    const Slice<T> q = slice3(uin, t + plane, n1);
    const T au = c0 * c.C + c1 * (c.S1 + m.C + q.C) + c2 * (c.S2 + m.S1 + q.S1) + c3 * (m.S2 + q.S2);
    const T f = L.f[t];
    out[t] = mode == 0 ? c.C + L.dinv_w * (f - au) : f - au;
    m = c;
    c = q;
  }
}

template <typename T>
dim3 march_grid(int d, int n) {
  const unsigned gx = (unsigned)div_up(n - 1, kMarchX);
  const unsigned gz = (unsigned)div_up(n - 1, kMarchZ);
  return d == 2 ? dim3(gx, gz, 1) : dim3(gx, (unsigned)(n - 1), gz);
}

// ---- 3D sweeps ----------------------------------------------------------------
// First pre-smoothing sweep from a zero iterate: out = omega D^-1 f at the
// interior nodes (a thread per (y, x) column over kz slices).
template <typename T>
__global__ void k_jacobi0_3(Lvl<T> L, T* __restrict__ out, int kz, const int* skip) {
  if (skip && *skip) return;
  const int n = L.n, n1 = n + 1, plane = n1 * n1;
  const int x = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int y = 1 + blockIdx.y;
  if (x >= n) return;
  const int z0 = 1 + blockIdx.z * kz, z1 = min(n, z0 + kz);
  const T dw = L.dinv_w;
  for (int z = z0; z < z1; ++z) {
    const int t = z * plane + y * n1 + x;
    out[t] = dw * L.f[t];
  }
}

// ---- register-blocked 3D sweep ---------------------------------------------
// A thread owns one x-column and kRB consecutive y-rows and marches along z;
// no shared memory and no barriers.  Per slice it loads the (kRB + 2) x 3
// in-plane neighbourhood (rows y-1 .. y+kRB, columns x-1 .. x+1; a warp's
// load of one row and offset is 32 consecutive words), forms the horizontal
// pair sums once per row and the slice sums of its kRB rows from them (the
// grouping of k_march), and keeps the slice sums of three slices in
// registers.  The next slice's u and f loads are issued before the current
// slice is computed and stored; f goes through a restrict pointer so that its
// loads are not held behind the stores to out (with f read through the level
// struct, each row's f load waited for the previous row's store: 72 against
// 56 us per 256^3 sweep); u through the read-only path and 8-slice z-chunks
// (51 us, 3.9 TB/s).  Measured alternatives, all slower at 256^3: a
// shared-memory tiled sweep (halo tile staged per slice, one barrier per
// slice; ~110 instructions per point, issue-bound), the same with cp.async
// staging six slices deep, L2 prefetches ahead of the loads, two-slice-deep
// register prefetch, 1, 2 or 8 rows per thread and persistent CTAs.
constexpr int kRB = 4;           // rows per thread
constexpr int kRX = 32;          // x-columns per CTA
constexpr int kRY = 4;           // row groups per CTA (CTA = 32 x 16 columns)
constexpr int kRThreads = kRX * kRY;

template <typename T>
__global__ void __launch_bounds__(kRThreads, sizeof(T) == 4 ? 6 : 3) k_sweep3r(Lvl<T> L, const T* __restrict__ uin, T* __restrict__ out,
                                                         int mode, int kz, const int* skip) {
  if (skip && *skip) return;
  const int n = L.n, n1 = n + 1, plane = n1 * n1;
  const int x = 1 + blockIdx.x * kRX + (threadIdx.x % kRX);
  const int yb = 1 + blockIdx.y * (kRY * kRB) + (threadIdx.x / kRX) * kRB;
  if (x >= n || yb >= n) return;
  const int z0 = 1 + blockIdx.z * kz, z1 = min(n, z0 + kz);
  const T c0 = L.c[0], c1 = L.c[1], c2 = L.c[2], c3 = L.c[3], dw = L.dinv_w;
  // rows yb - 1 .. yb + kRB (those beyond the grid read as 0)
  int roff[kRB + 2];
  bool rok[kRB + 2];
#pragma unroll
  for (int r = 0; r < kRB + 2; ++r) {
    rok[r] = yb - 1 + r <= n;
    roff[r] = (yb - 1 + r) * n1 + x;
  }
  T raw[kRB + 2][3];
  auto load = [&](int z) {
    const T* s = uin + z * plane;
#pragma unroll
    for (int r = 0; r < kRB + 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) raw[r][c] = rok[r] ? __ldg(s + roff[r] + c - 1) : (T)0;
  };
  T mC[kRB], mS1[kRB], mS2[kRB], cC[kRB], cS1[kRB], cS2[kRB];
  auto sums = [&](T* C, T* S1, T* S2) {
    T H[kRB + 2];
#pragma unroll
    for (int r = 0; r < kRB + 2; ++r) H[r] = raw[r][0] + raw[r][2];
#pragma unroll
    for (int r = 0; r < kRB; ++r) {
      C[r] = raw[r + 1][1];
      S1[r] = H[r + 1] + (raw[r][1] + raw[r + 2][1]);
      S2[r] = H[r] + H[r + 2];
    }
  };
  const T* __restrict__ fp = L.f;
  T fcur[kRB], fnext[kRB];
  auto loadf = [&](int z, T* dst) {
    const int tb = z * plane + yb * n1 + x;
#pragma unroll
    for (int r = 0; r < kRB; ++r) dst[r] = (yb + r < n) ? fp[tb + r * n1] : (T)0;
  };
  loadf(z0, fcur);
  load(z0 - 1);
  sums(mC, mS1, mS2);
  load(z0);
  sums(cC, cS1, cS2);
  load(z0 + 1);
  for (int z = z0; z < z1; ++z) {
    T qC[kRB], qS1[kRB], qS2[kRB];
    sums(qC, qS1, qS2);
    if (z + 1 < z1) {
      load(z + 2);
      loadf(z + 1, fnext);
    }
    const int t = z * plane + yb * n1 + x;
#pragma unroll
    for (int r = 0; r < kRB; ++r) {
      if (yb + r < n) {
        const T f = fcur[r];
        const T au = c0 * cC[r] + c1 * (cS1[r] + mC[r] + qC[r]) + c2 * (cS2[r] + mS1[r] + qS1[r]) +
                     c3 * (mS2[r] + qS2[r]);
        out[t + r * n1] = mode == 0 ? cC[r] + dw * (f - au) : f - au;
      }
      mC[r] = cC[r];
      mS1[r] = cS1[r];
      mS2[r] = cS2[r];
      cC[r] = qC[r];
      cS1[r] = qS1[r];
      cS2[r] = qS2[r];
      fcur[r] = fnext[r];
    }
  }
}

// slices per thread of the column kernels (k_jacobi0_3, k_prolong3): 16, or
// fewer where a level has too few columns to fill the GPU
inline int column_kz(int n) {
  const long long cols = (long long)div_up(n - 1, 128) * (n - 1);
  int kz = 16;
  while (kz > 1 && cols * div_up(n - 1, kz) < 1000) kz >>= 1;
  return kz;
}

inline int sweep_r_kz(int n) {
  const int cols = div_up(n - 1, kRX) * div_up(n - 1, kRY * kRB);
  int kz = 1;
  while (kz < 8 && kz < n - 1 && (long long)cols * div_up(n - 1, kz) > 2 * 152 * 6) kz <<= 1;
  return kz;
}

// uf += P uc in 3D, a thread per fine (y, x) column marching along z: the
// in-plane (bi)linear value of coarse slice k serves fine slices 2k - 1, 2k
// and 2k + 1 (fine slice 2k takes it, 2k + 1 the mean of slices k and k + 1)
template <typename T>
__global__ void k_prolong3(int nf, const T* __restrict__ uc, T* __restrict__ uf, int kz, const int* skip) {
  if (skip && *skip) return;
  const int nf1 = nf + 1, nc1 = nf / 2 + 1, cplane = nc1 * nc1, plane = nf1 * nf1;
  const int x = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int y = 1 + blockIdx.y;
  if (x >= nf) return;
  const int z0 = 1 + blockIdx.z * kz, z1 = min(nf, z0 + kz);
  const int ox = x & 1, oy = y & 1;
  const int cb = (y >> 1) * nc1 + (x >> 1);
  const T w = (oy ? (T)0.5 : (T)1) * (ox ? (T)0.5 : (T)1);
  auto inplane = [&](int k) -> T {
    const T* c = uc + k * cplane + cb;
    T s = __ldg(c);
    if (ox) s += __ldg(c + 1);
    if (oy) s += ox ? __ldg(c + nc1) + __ldg(c + nc1 + 1) : __ldg(c + nc1);
    return w * s;
  };
  int k = z0 >> 1;
  T vlo = inplane(k), vhi = inplane(k + 1);
  T* __restrict__ p = uf + z0 * plane + y * nf1 + x;
  T cur = p[0];
  for (int z = z0; z < z1; ++z, p += plane) {
    const T nxt = z + 1 < z1 ? p[plane] : (T)0;   // issued before this slice's store
    if ((z >> 1) != k) {
      k = z >> 1;
      vlo = vhi;
      vhi = inplane(k + 1);
    }
    const T v = (z & 1) ? (T)0.5 * (vlo + vhi) : vlo;
    p[0] = cur + v;
    cur = nxt;
  }
}

// ---- per-level transfer kernels: x over the last axis, y (z) over the others ----

// full weighting: weight prod_k w(o_k), w(0) = 1/2, w(+-1) = 1/4 (32-bit
// indices: grids of up to 1025^3 nodes).  Threads run over the nodes of one
// coarse slice (x fastest), blockIdx.y over the slices (3D).
template <typename T>
__global__ void k_restrict(int d, int nc, const T* __restrict__ rf, T* __restrict__ fc,
                           const int* skip) {
  if (skip && *skip) return;
  const int nf1 = 2 * nc + 1, nc1 = nc + 1;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nc1 * nc1) return;
  const int i1 = q / nc1, j = q - i1 * nc1, i0 = blockIdx.y;
  const int tc = d == 2 ? q : i0 * nc1 * nc1 + q;
  const bool interior = j >= 1 && j < nc && i1 >= 1 && i1 < nc && (d == 2 || (i0 >= 1 && i0 < nc));
  if (!interior) {
    fc[tc] = (T)0;
    return;
  }
  T acc = (T)0;
  const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
  if (d == 2) {
    const int base = (2 * i1) * nf1 + 2 * j;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) acc += w[a + 1] * w[b + 1] * __ldg(rf + base + a * nf1 + b);
  } else {
    const int base = ((2 * i0) * nf1 + 2 * i1) * nf1 + 2 * j;
    const int pl = nf1 * nf1;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int c = -1; c <= 1; ++c)
          acc += w[a + 1] * w[b + 1] * w[c + 1] * __ldg(rf + base + a * pl + b * nf1 + c);
  }
  fc[tc] = acc;
}

// uf += P uc ((bi/tri)linear interpolation): the coarse neighbours of a fine
// node are lo = i >> 1 and lo + 1 along each axis with an odd index, weight
// 1/2 per odd axis; 32-bit indices, the combination loop unrolled
template <typename T>
__global__ void k_prolong_add(int d, int nf, const T* __restrict__ uc, T* __restrict__ uf,
                              const int* skip) {
  if (skip && *skip) return;
  const int nf1 = nf + 1, nc1 = nf / 2 + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y, i0 = blockIdx.z;
  if (j > nf) return;
  const bool interior = j >= 1 && j < nf && i1 >= 1 && i1 < nf && (d == 2 || (i0 >= 1 && i0 < nf));
  if (!interior) return;
  const int o0 = d == 3 ? (i0 & 1) : 0, o1 = i1 & 1, o2 = j & 1;
  T wgt = (T)1;
  if (o0) wgt *= (T)0.5;
  if (o1) wgt *= (T)0.5;
  if (o2) wgt *= (T)0.5;
  const int base = d == 2 ? (i1 >> 1) * nc1 + (j >> 1) : ((i0 >> 1) * nc1 + (i1 >> 1)) * nc1 + (j >> 1);
  const int s0 = nc1 * nc1;
  T acc = (T)0;
  if (d == 2) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b1 = m & 1, b2 = (m >> 1) & 1;
      if ((b1 && !o1) || (b2 && !o2)) continue;
      acc += wgt * uc[base + b1 * nc1 + b2];
    }
    uf[i1 * nf1 + j] += acc;
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int b0 = m & 1, b1 = (m >> 1) & 1, b2 = (m >> 2) & 1;
      if ((b0 && !o0) || (b1 && !o1) || (b2 && !o2)) continue;
      acc += wgt * uc[base + b0 * s0 + b1 * nc1 + b2];
    }
    uf[(i0 * nf1 + i1) * nf1 + j] += acc;
  }
}

// ---- the coarse part of the V-cycle in one CTA ------------------------------

template <typename T>
__device__ void blk_jacobi(int d, int order, const Lvl<T>& L, const T* uin, T* uout, bool zero) {
  const int n = L.n, n1 = n + 1;
  const int m = n - 1;
  const int tot = d == 2 ? m * m : m * m * m;
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    int j = q % m + 1, r = q / m;
    int i1 = r % m + 1, i0 = d == 3 ? r / m + 1 : 0;
    long long t = lin(d, n1, i0, i1, j);
    uout[t] = zero ? L.dinv_w * L.f[t]
                   : uin[t] + L.dinv_w * (L.f[t] - apply_at<T>(d, order, n1, L.c, uin + t));
  }
  __syncthreads();
}

// The V-cycle from level lstart down to the coarsest and back, in one CTA.
// start_zero: the iterate at lstart starts from zero (a coarse correction, or
// the first cycle on a grid that is coarse from the start).
template <typename T>
__global__ void k_coarse_cycle(LvlArgs<T> A, int lstart, int start_zero, const int* skip) {
  if (skip && *skip) return;
  const int d = A.d;
  for (int l = lstart; l < A.nlev; ++l) {
    const int n1 = A.L[l].n + 1;
    const int tot = d == 2 ? n1 * n1 : n1 * n1 * n1;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      A.L[l].t[q] = (T)0;
      if (l > lstart || start_zero) A.L[l].u[q] = (T)0;
    }
  }
  __syncthreads();
  // descend
  for (int l = lstart; l < A.nlev - 1; ++l) {
    const Lvl<T>& L = A.L[l];
    bool zero = l > lstart || start_zero;   // corrections start from zero
    // two sweeps, u -> t -> u (kNu = 2)
    blk_jacobi<T>(d, A.order, L, L.u, L.t, zero);
    blk_jacobi<T>(d, A.order, L, L.t, L.u, false);
    // residual into t, restrict to the next f
    {
      const int n = L.n, n1 = n + 1, m = n - 1;
      const int tot = d == 2 ? m * m : m * m * m;
      for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        int j = q % m + 1, r = q / m;
        int i1 = r % m + 1, i0 = d == 3 ? r / m + 1 : 0;
        long long t = lin(d, n1, i0, i1, j);
        L.t[t] = L.f[t] - apply_at<T>(d, A.order, n1, L.c, L.u + t);
      }
      __syncthreads();
      const Lvl<T>& C = A.L[l + 1];
      const int nc = C.n, nc1 = nc + 1, mc = nc - 1;
      const int totc = d == 2 ? mc * mc : mc * mc * mc;
      const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
      for (int q = threadIdx.x; q < totc; q += blockDim.x) {
        int j = q % mc + 1, r = q / mc;
        int i1 = r % mc + 1, i0 = d == 3 ? r / mc + 1 : 0;
        T acc = (T)0;
        if (d == 2) {
          for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b) acc += w[a + 1] * w[b + 1] * L.t[lin(2, n1, 0, 2 * i1 + a, 2 * j + b)];
        } else {
          for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
              for (int c = -1; c <= 1; ++c)
                acc += w[a + 1] * w[b + 1] * w[c + 1] *
                       L.t[lin(3, n1, 2 * i0 + a, 2 * i1 + b, 2 * j + c)];
        }
        C.f[lin(d, nc1, i0, i1, j)] = acc;
      }
      __syncthreads();
    }
  }
  // coarsest: u = C^{-1} f on its 3^d interior unknowns
  {
    const Lvl<T>& C = A.L[A.nlev - 1];
    const int n1 = C.n + 1, m = C.n - 1;
    const int tot = d == 2 ? m * m : m * m * m;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      T acc = (T)0;
      for (int k = 0; k < tot; ++k) {
        int j = k % m + 1, r = k / m;
        int i1 = r % m + 1, i0 = d == 3 ? r / m + 1 : 0;
        acc += A.cinv[q * tot + k] * C.f[lin(d, n1, i0, i1, j)];
      }
      int j = q % m + 1, r = q / m;
      int i1 = r % m + 1, i0 = d == 3 ? r / m + 1 : 0;
      C.t[lin(d, n1, i0, i1, j)] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (d == 2 ? n1 * n1 : n1 * n1 * n1); q += blockDim.x) C.u[q] = C.t[q];
    __syncthreads();
  }
  // ascend
  for (int l = A.nlev - 2; l >= lstart; --l) {
    const Lvl<T>& L = A.L[l];
    const Lvl<T>& C = A.L[l + 1];
    const int nf = L.n, nf1 = nf + 1, m = nf - 1, nc1 = C.n + 1;
    const int tot = d == 2 ? m * m : m * m * m;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      int j = q % m + 1, r = q / m;
      int i1 = r % m + 1, i0 = d == 3 ? r / m + 1 : 0;
      const int idx[3] = {i0, i1, j};
      int lo[3], hi[3];
      for (int k = 0; k < 3; ++k) {
        lo[k] = idx[k] >> 1;
        hi[k] = (idx[k] + 1) >> 1;
      }
      T acc = (T)0;
      const int k0 = d == 2 ? 1 : 0;
      for (int mm = 0; mm < (1 << (3 - k0)); ++mm) {
        int ci[3] = {lo[0], lo[1], lo[2]};
        T wgt = (T)1;
        bool dup = false;
        for (int k = k0; k < 3; ++k) {
          int bit = (mm >> (k - k0)) & 1;
          bool odd = (idx[k] & 1) != 0;
          if (!odd && bit) dup = true;
          ci[k] = bit ? hi[k] : lo[k];
          if (odd) wgt *= (T)0.5;
        }
        if (dup) continue;
        acc += wgt * C.u[lin(d, nc1, ci[0], ci[1], ci[2])];
      }
      L.u[lin(d, nf1, i0, i1, j)] += acc;
    }
    __syncthreads();
    blk_jacobi<T>(d, A.order, L, L.u, L.t, false);   // two sweeps, u -> t -> u (kNu = 2)
    blk_jacobi<T>(d, A.order, L, L.t, L.u, false);
  }
}

// ---- refinement helpers ------------------------------------------------------

__global__ void k_to_float(long long tot, const double* __restrict__ a, float* __restrict__ b,
                           const int* skip) {
  if (skip && *skip) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

// mixed: conv = (max|e_k| <= tol max|u|), the FP32 cycles contract the error by
// orders of magnitude per outer step, so the last correction bounds the error
__global__ void k_mg_check_corr(unsigned long long* nrm, const double* tolp, int* conv) {
  const double tol = tolp[0];
  if (*conv) return;
  double em = __longlong_as_double((long long)nrm[6]);
  double um = __longlong_as_double((long long)nrm[7]);
  nrm[8] = nrm[6];
  nrm[9] = nrm[7];
  if (em <= tol * um) *conv = 1;
  nrm[10] += 1ull;   // the outer step just checked ran
  nrm[6] = 0ull;
  nrm[7] = 0ull;
}

__global__ void k_mg_residual64(Grid g, int order, const double* __restrict__ c,
                                const double* __restrict__ R, const double* __restrict__ u,
                                double* __restrict__ r, unsigned long long* __restrict__ nrm,
                                const int* skip) {
  if (skip && *skip) return;
  const int n1 = g.n + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y, i0 = blockIdx.z;
  double mx = 0.0, ux = 0.0;
  if (j <= g.n) {
    const long long t = lin(g.d, n1, i0, i1, j);
    const bool interior = j >= 1 && j < g.n && i1 >= 1 && i1 < g.n && (g.d == 2 || (i0 >= 1 && i0 < g.n));
    double v = interior ? R[t] - apply_at<double>(g.d, order, n1, c, u + t) : 0.0;
    if (r) r[t] = v;
    mx = fabs(v);
    ux = fabs(u[t]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    ux = fmax(ux, __shfl_xor_sync(0xffffffffu, ux, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx > 0.0) atomicMax(nrm, (unsigned long long)__double_as_longlong(mx));
    if (ux > 0.0) atomicMax(nrm + 2, (unsigned long long)__double_as_longlong(ux));
  }
}

__global__ void k_absmax_mg(long long tot, const double* __restrict__ R, unsigned long long* nrm) {
  double mx = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(R[t]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(nrm, (unsigned long long)__double_as_longlong(mx));
}

// FP64 V-cycles: stop at the normwise backward error max|r| <= tol (max|R| +
// ||A||_inf max|u|) or when the residual stagnates (r_k > 0.7 r_{k-1}) at the
// rounding floor eps ||A|| ||u|| of the FP64 residual.
__global__ void k_mg_check(unsigned long long* nrm, double tol, double anorm, int* conv) {
  if (*conv) return;
  double R = __longlong_as_double((long long)nrm[0]);
  double r = __longlong_as_double((long long)nrm[1]);
  double um = __longlong_as_double((long long)nrm[2]);
  double rp = __longlong_as_double((long long)nrm[4]);
  nrm[4] = nrm[1];
  nrm[5] = nrm[2];
  if (r <= tol * (R + anorm * um) || (rp > 0.0 && r > 0.7 * rp)) *conv = 1;
  nrm[10] += 1ull;   // the V-cycle just checked ran
  nrm[1] = 0ull;
  nrm[2] = 0ull;
}

__global__ void k_mg_reset(unsigned long long* nrm, int* conv) {
  for (int k = 0; k < 11; ++k) nrm[k] = 0ull;
  *conv = 0;
}

}  // namespace

struct MgSolver {
  int nlev = 0, lcoarse = 0;
  int precision = KFBI_FP64;
  LvlArgs<double> A64;
  LvlArgs<float> A32;
  double* cinv64 = nullptr;
  float* cinv32 = nullptr;
  std::vector<void*> bufs;
  double* u64 = nullptr;       // mixed: FP64 accumulated solution lives in the caller's u
  FixState* fix = nullptr;     // mixed: exact fixed-point residual between FP32 solves
  unsigned long long* nrm = nullptr;
  int* conv = nullptr;
  int max_cycles = 60;
  int inner_cycles = 4;
  int outer_max = 6;
  double tol = 1e-13;
  double* tol_dev = nullptr;   // mixed: the outer-step tolerance the check reads (relaxed in GMRES)
  double anorm = 0.0;          // ||A_h||_inf = sum of |stencil coefficients|
};

namespace {

void stencil_for(int d, int order, double h, double k, double* c) {
  const double ih2 = 1.0 / (h * h);
  if (order == 2) {
    c[0] = -2.0 * d * ih2 - k;
    c[1] = ih2;
    c[2] = c[3] = 0.0;
  } else if (d == 2) {
    c[0] = -10.0 / 3.0 * ih2 - 2.0 / 3.0 * k;
    c[1] = 2.0 / 3.0 * ih2 - k / 12.0;
    c[2] = 1.0 / 6.0 * ih2;
    c[3] = 0.0;
  } else {
    c[0] = -25.0 / 6.0 * ih2 - 0.5 * k;
    c[1] = 5.0 / 12.0 * ih2 - k / 12.0;
    c[2] = 1.0 / 8.0 * ih2;
    c[3] = 1.0 / 48.0 * ih2;
  }
}

// dense inverse of the coarsest operator (3^d interior unknowns) by Gauss-Jordan
std::vector<double> coarse_inverse(int d, int order, double h, double kt) {
  double c[4];
  stencil_for(d, order, h, kt, c);
  const int m = 3;
  const int tot = d == 2 ? m * m : m * m * m;
  std::vector<double> A(tot * tot, 0.0), I(tot * tot, 0.0);
  for (int q = 0; q < tot; ++q) {
    int qi[3] = {0, 0, 0};
    int r = q;
    for (int k = d - 1; k >= 0; --k) {
      qi[k] = r % m;
      r /= m;
    }
    for (int p = 0; p < tot; ++p) {
      int pi[3] = {0, 0, 0};
      int rr = p;
      for (int k = d - 1; k >= 0; --k) {
        pi[k] = rr % m;
        rr /= m;
      }
      int nz = 0, far = 0;
      for (int k = 0; k < d; ++k) {
        int dd = std::abs(pi[k] - qi[k]);
        if (dd > 1) far = 1;
        nz += dd;
      }
      if (far) continue;
      int cnt = 0;
      for (int k = 0; k < d; ++k) cnt += pi[k] != qi[k];
      if (order == 2 && cnt > 1) continue;
      A[q * tot + p] = c[cnt];
    }
    I[q * tot + q] = 1.0;
  }
  for (int col = 0; col < tot; ++col) {
    int piv = col;
    for (int r = col + 1; r < tot; ++r)
      if (std::fabs(A[r * tot + col]) > std::fabs(A[piv * tot + col])) piv = r;
    if (piv != col)
      for (int k = 0; k < tot; ++k) {
        std::swap(A[col * tot + k], A[piv * tot + k]);
        std::swap(I[col * tot + k], I[piv * tot + k]);
      }
    double dv = A[col * tot + col];
    for (int k = 0; k < tot; ++k) {
      A[col * tot + k] /= dv;
      I[col * tot + k] /= dv;
    }
    for (int r = 0; r < tot; ++r) {
      if (r == col) continue;
      double f = A[r * tot + col];
      if (f == 0.0) continue;
      for (int k = 0; k < tot; ++k) {
        A[r * tot + k] -= f * A[col * tot + k];
        I[r * tot + k] -= f * I[col * tot + k];
      }
    }
  }
  return I;
}

template <typename T>
dim3 lvl_grid(int d, int n) {
  return dim3((unsigned)div_up(n + 1, 128), (unsigned)(n + 1), d == 3 ? (unsigned)(n + 1) : 1u);
}

// One smoothing (mode 0) or residual (mode 1) sweep on level L: the tiled
// kernel in 3D, the marching kernel in 2D (2D levels are L2-resident).
template <typename T>
kfbi_status sweep(kfbi_problem* p, int d, const Lvl<T>& L, const T* uin, T* out, int mode, bool zero,
                  const int* skip, const T* uc = nullptr) {
  cudaStream_t st = p->stream;
  if (d == 3) {
    if (zero) {
      const int jz = column_kz(L.n);
      const dim3 jg((unsigned)div_up(L.n - 1, 128), (unsigned)(L.n - 1), (unsigned)div_up(L.n - 1, jz));
      KFBI_LAUNCH(p, KFBI_KC_MG, k_jacobi0_3<T><<<jg, 128, 0, st>>>(L, out, jz, skip));
      return KFBI_OK;
    }
    if (uc) {   // u += P uc first (the corrected u is then read by the sweep)
      const int pz = column_kz(L.n);
      const dim3 pg((unsigned)div_up(L.n - 1, 128), (unsigned)(L.n - 1), (unsigned)div_up(L.n - 1, pz));
      KFBI_LAUNCH(p, KFBI_KC_MG, k_prolong3<T><<<pg, 128, 0, st>>>(L.n, uc, const_cast<T*>(uin), pz, skip));
    }
    const int rz = sweep_r_kz(L.n);
    const dim3 rg((unsigned)div_up(L.n - 1, kRX), (unsigned)div_up(L.n - 1, kRY * kRB),
                  (unsigned)div_up(L.n - 1, rz));
    KFBI_LAUNCH(p, KFBI_KC_MG, k_sweep3r<T><<<rg, kRThreads, 0, st>>>(L, uin, out, mode, rz, skip));
  } else {
    KFBI_LAUNCH(p, KFBI_KC_MG, k_march<T><<<march_grid<T>(d, L.n), kMarchX, 0, st>>>(d, L, uin, out, mode,
                                                                                       zero ? 1 : 0, skip));
  }
  return KFBI_OK;
}

// One V-cycle starting at level 0 of A (u_0 holds the current iterate).
template <typename T>
kfbi_status vcycle(kfbi_problem* p, LvlArgs<T>& A, int lcoarse, bool zero_guess, const int* skip) {
  const int d = A.d, order = A.order;
  cudaStream_t st = p->stream;
  for (int l = 0; l < lcoarse; ++l) {
    Lvl<T>& L = A.L[l];
    const bool zero = (l > 0) || zero_guess;
    // two sweeps u -> t -> u, then the residual into t
    KFBI_TRY(sweep<T>(p, d, L, L.u, L.t, 0, zero, skip));
    KFBI_TRY(sweep<T>(p, d, L, L.t, L.u, 0, false, skip));
    KFBI_TRY(sweep<T>(p, d, L, L.u, L.t, 1, false, skip));
    const int nc1 = A.L[l + 1].n + 1;
    const dim3 rg((unsigned)div_up((long long)nc1 * nc1, 128), d == 3 ? (unsigned)nc1 : 1u);
    KFBI_LAUNCH(p, KFBI_KC_MG, k_restrict<T><<<rg, 128, 0, st>>>(
        d, A.L[l + 1].n, L.t, A.L[l + 1].f, skip));
  }
  KFBI_LAUNCH(p, KFBI_KC_MG, k_coarse_cycle<T><<<1, 1024, 0, st>>>(
      A, lcoarse, (lcoarse > 0 || zero_guess) ? 1 : 0, skip));
  for (int l = lcoarse - 1; l >= 0; --l) {
    Lvl<T>& L = A.L[l];
    if (d == 3) {   // prolongation folded into the first post-smoothing sweep
      KFBI_TRY(sweep<T>(p, d, L, L.u, L.t, 0, false, skip, A.L[l + 1].u));
    } else {
      KFBI_LAUNCH(p, KFBI_KC_MG, k_prolong_add<T><<<lvl_grid<T>(d, L.n), 128, 0, st>>>(d, L.n, A.L[l + 1].u, L.u,
                                                                                       skip));
      KFBI_TRY(sweep<T>(p, d, L, L.u, L.t, 0, false, skip));
    }
    KFBI_TRY(sweep<T>(p, d, L, L.t, L.u, 0, false, skip));
  }
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
kfbi_status build_levels(kfbi_problem* p, MgSolver* M, LvlArgs<T>& A, T** cinv, bool level0_owned) {
  const Grid g = p->g;
  const int d = g.d;
  A.d = d;
  A.order = p->cfg.order;
  int n = g.n, l = 0;
  // weighted Jacobi: 0.909 / 1.136 for the compact 9-/27-point operators,
  // 4/5 / 6/7 for the 5-/7-point ones (at the 27-point value the 7-point
  // sweep amplifies the highest mode by |1 - 2 omega| > 1)
  const double omega = A.order == 2 ? (d == 2 ? 0.8 : 6.0 / 7.0) : (d == 2 ? 0.909 : 1.136);
  while (true) {
    if (l >= 16) return fail(p, KFBI_ERR_UNSUPPORTED, "too many multigrid levels");
    Lvl<T>& L = A.L[l];
    L.n = n;
    double c[4];
    stencil_for(d, A.order, g.h * (double)(g.n / n), p->kt, c);
    for (int k = 0; k < 4; ++k) L.c[k] = (T)c[k];
    L.dinv_w = (T)(omega / c[0]);
    const long long nodes = d == 2 ? (long long)(n + 1) * (n + 1) : (long long)(n + 1) * (n + 1) * (n + 1);
    if (l > 0 || level0_owned) {
      KFBI_CUDA(p, dalloc(&L.u, nodes));
      KFBI_CUDA(p, dalloc(&L.f, nodes));
      KFBI_CUDA(p, cudaMemset(L.u, 0, sizeof(T) * nodes));
      KFBI_CUDA(p, cudaMemset(L.f, 0, sizeof(T) * nodes));
      M->bufs.push_back(L.u);
      M->bufs.push_back(L.f);
    }
    KFBI_CUDA(p, dalloc(&L.t, nodes));
    KFBI_CUDA(p, cudaMemset(L.t, 0, sizeof(T) * nodes));
    M->bufs.push_back(L.t);
    ++l;
    if (n == 4) break;
    n /= 2;
  }
  A.nlev = l;
  const int cn = d == 2 ? kCoarseN2 : kCoarseN3;
  int lc = 0;
  while (lc < A.nlev - 1 && A.L[lc].n > cn) ++lc;
  M->lcoarse = lc;
  std::vector<double> ci = coarse_inverse(d, A.order, g.h * (double)(g.n / 4), p->kt);
  std::vector<T> cit(ci.begin(), ci.end());
  KFBI_CUDA(p, dalloc(cinv, cit.size()));
  KFBI_CUDA(p, cudaMemcpy(*cinv, cit.data(), sizeof(T) * cit.size(), cudaMemcpyHostToDevice));
  M->bufs.push_back(*cinv);
  A.cinv = *cinv;
  return KFBI_OK;
}

}  // namespace

kfbi_status mg_create(kfbi_problem* p) {
  const Grid g = p->g;
  if (g.n < 8 || (g.n & (g.n - 1)) != 0) return fail(p, KFBI_ERR_UNSUPPORTED, "MG needs N a power of two >= 8");
  MgSolver* M = new MgSolver();
  p->mg = M;
  M->precision = p->cfg.precision;
  M->tol = p->cfg.box_rtol > 0 ? p->cfg.box_rtol : 1e-13;
  M->outer_max = p->cfg.box_max_iters > 0 ? std::min(p->cfg.box_max_iters, 12) : 8;
  M->max_cycles = p->cfg.box_max_iters > 0 ? p->cfg.box_max_iters : 40;
  const long long nodes = g.nodes();
  if (M->precision == KFBI_MIXED) {
    KFBI_TRY(build_levels<float>(p, M, M->A32, &M->cinv32, true));
    KFBI_TRY(fix_create(p, &M->fix));
  } else {
    KFBI_TRY(build_levels<double>(p, M, M->A64, &M->cinv64, false));
  }
  {
    const double* c = p->stencil_c;
    const int d = g.d;
    double a = std::fabs(c[0]);
    if (p->cfg.order == 2) a += 2 * d * std::fabs(c[1]);
    else if (d == 2) a += 4 * std::fabs(c[1]) + 4 * std::fabs(c[2]);
    else a += 6 * std::fabs(c[1]) + 12 * std::fabs(c[2]) + 8 * std::fabs(c[3]);
    M->anorm = a;
  }
  KFBI_CUDA(p, dalloc(&M->nrm, 11));
  KFBI_CUDA(p, dalloc(&M->conv, 1));
  KFBI_CUDA(p, dalloc(&M->tol_dev, 1));
  KFBI_CUDA(p, cudaMemcpy(M->tol_dev, &M->tol, sizeof(double), cudaMemcpyHostToDevice));
  M->bufs.push_back(M->nrm);
  M->bufs.push_back(M->conv);
  M->bufs.push_back(M->tol_dev);
  return KFBI_OK;
}

// the mixed multigrid's outer-step tolerance (device) and its base value
double* mg_tol_dev(kfbi_problem* p) {
  return (p->mg && p->mg->precision == KFBI_MIXED) ? p->mg->tol_dev : nullptr;
}
double mg_tol(const kfbi_problem* p) { return p->mg ? p->mg->tol : 0.0; }

void mg_destroy(kfbi_problem* p) {
  MgSolver* M = p->mg;
  if (!M) return;
  for (void* b : M->bufs) cudaFree(b);
  fix_destroy(M->fix);
  delete M;
  p->mg = nullptr;
}

kfbi_status mg_solve(kfbi_problem* p, const double* rhs, double* u) {
  MgSolver* M = p->mg;
  const Grid g = p->g;
  cudaStream_t st = p->stream;
  const long long nodes = g.nodes();
  const dim3 gr = lvl_grid<double>(g.d, g.n);
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_mg_reset<<<1, 1, 0, st>>>(M->nrm, M->conv));
  if (M->precision != KFBI_MIXED) {
    KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_absmax_mg<<<std::min(div_up(nodes, 256), 152 * 8), 256, 0, st>>>(
        nodes, rhs, M->nrm));
    KFBI_CUDA(p, cudaMemsetAsync(u, 0, sizeof(double) * nodes, st));
    LvlArgs<double>& A = M->A64;
    A.L[0].u = u;
    A.L[0].f = const_cast<double*>(rhs);
    for (int c = 0; c < M->max_cycles; ++c) {
      KFBI_TRY(vcycle<double>(p, A, M->lcoarse, c == 0, M->conv));
      KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_mg_residual64<<<gr, 128, 0, st>>>(
          g, p->cfg.order, p->stencil_dev, rhs, u, nullptr, M->nrm + 1, M->conv));
      KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_mg_check<<<1, 1, 0, st>>>(M->nrm, M->tol, M->anorm, M->conv));
    }
    KFBI_CUDA(p, cudaGetLastError());
    return KFBI_OK;
  }
  // mixed: u0 = FP32 MG(R); then u is kept in fixed point and each outer step
  // solves A e = r with r = R - A_h u exact (integer stencil), e by FP32 V-cycles
  LvlArgs<float>& A = M->A32;
  KFBI_LAUNCH(p, KFBI_KC_MG, k_to_float<<<std::min(div_up(nodes, 256), 152 * 8), 256, 0, st>>>(
      nodes, rhs, A.L[0].f, nullptr));
  for (int c = 0; c < M->inner_cycles; ++c) KFBI_TRY(vcycle<float>(p, A, M->lcoarse, c == 0, nullptr));
  KFBI_TRY(fix_init(p, M->fix, A.L[0].u, rhs, st));
  for (int o = 1; o < M->outer_max; ++o) {
    KFBI_TRY(fix_residual(p, M->fix, A.L[0].f, M->conv, st));
    for (int c = 0; c < M->inner_cycles; ++c) KFBI_TRY(vcycle<float>(p, A, M->lcoarse, c == 0, M->conv));
    KFBI_TRY(fix_add(p, M->fix, A.L[0].u, M->nrm + 6, M->conv, st));
    KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_mg_check_corr<<<1, 1, 0, st>>>(M->nrm, M->tol_dev, M->conv));
  }
  KFBI_TRY(fix_out(p, M->fix, u, st));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

// Outer steps and V-cycles of the last multigrid box solve (mixed: the first
// FP32 cycles plus every outer step that ran, inner_cycles V-cycles each;
// FP64: the V-cycles that ran, one step).
kfbi_status mg_steps(kfbi_problem* p, int* steps, int* cycles) {
  MgSolver* M = p->mg;
  unsigned long long c = 0;
  KFBI_CUDA(p, cudaMemcpyAsync(&c, M->nrm + 10, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  if (M->precision == KFBI_MIXED) {
    *steps = 1 + (int)c;
    *cycles = M->inner_cycles * *steps;
  } else {
    *steps = 1;
    *cycles = (int)c;
  }
  return KFBI_OK;
}

kfbi_status mg_last_residual(kfbi_problem* p, double* rel, int* converged) {
  MgSolver* M = p->mg;
  unsigned long long h[10];
  int c = 0;
  KFBI_CUDA(p, cudaMemcpyAsync(h, M->nrm, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaMemcpyAsync(&c, M->conv, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  double R, r, um;
  if (M->precision == KFBI_MIXED) {
    memcpy(&r, &h[8], 8);
    memcpy(&um, &h[9], 8);
    *rel = um > 0 ? r / um : 0.0;
  } else {
    memcpy(&R, &h[0], 8);
    memcpy(&r, &h[4], 8);
    memcpy(&um, &h[5], 8);
    *rel = (R + M->anorm * um) > 0 ? r / (R + M->anorm * um) : 0.0;
  }
  *converged = c;
  return KFBI_OK;
}

}  // namespace kfbi
