// Box solve by the discrete sine transform (Algorithm 1, Step 3.3): the
// compact 9/27-point (or 5/7-point) operators with homogeneous Dirichlet data
// are diagonal in the basis prod_k sin(p_k pi i_k / N), with eigenvalues
//   9-pt:  h^-2 [-10/3 + 4/3 (c_p + c_q) + 2/3 c_p c_q] - k [2/3 + (c_p + c_q)/6]
//   27-pt: h^-2 [-25/6 + 5/6 S1 + 1/2 S2 + 1/6 S3] - k [1/2 + S1/6]
//   5/7-pt: h^-2 sum_k (2 c_k - 2) - k
// (c = cos(p pi / N), S1/S2/S3 the elementary symmetric sums), derived from the
// stencils of eqs. (9p-cds)/(27p-cds).
//
// GB300 design.  A DST-I of length N-1 is a complex FFT of length L = 2N of the
// odd extension; two real lines are packed as the real and imaginary parts of
// one complex sequence (Z_k = -2i (A_k + i B_k)).  Each CTA transforms P such
// pairs in shared memory with a radix-2 FFT:
//   * edge passes: decimation in frequency (natural in, bit-reversed out);
//   * the middle pass along the slowest axis: DIF, then the spectral division
//     by the eigenvalue applied in place in bit-reversed order (the odd
//     symmetry Z_{L-k} = -Z_k makes the rescaled sequence exactly the odd
//     extension of the next input), then decimation in time (bit-reversed in,
//     natural out) — no reordering pass.
// 2D: 3 passes (axis 1, axis 0 fused, axis 1); 3D: 5 passes.  Each pass reads
// and writes the grid once.  T = double (FP64 path) or float (mixed path:
// FP32 transforms, FP64 residual r = R - A_h u and iterative refinement, with a
// device-side convergence flag so that no host synchronisation is needed).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

template <typename T>
struct Cx {
  T x, y;
};

struct BoxSolver {
  int L = 0, logL = 0;
  double* tw64 = nullptr;     // L/2 twiddles exp(-2 pi i t / L)
  float* tw32 = nullptr;
  double* cosv = nullptr;     // cos(k pi / N), k = 0..N
  double* s64 = nullptr;      // sin^2(k pi / 2N), k = 0..N
  float* s32 = nullptr;
  double* scale64 = nullptr;  // FP64 path: (2/N)^d / lambda on the mode grid (N-1)^d
  double* work64 = nullptr;   // grid of doubles
  float* work32 = nullptr;    // grid of floats
  double* res = nullptr;      // FP64 residual grid
  unsigned long long* nrm = nullptr;   // [0] max|R| [1] max|r| [2] last max|delta| [3] max|delta| [4] max|u| [5] last max|u|
  int* conv = nullptr;        // device flag
  int refine_steps = 4;
  double tol = 1e-13;
};

namespace {

struct PassArgs {
  const void* src;
  void* dst;
  int src64, dst64, accumulate;
  long long sa, sb, es;     // line strides: line(a, b) at a*sa + b*sb, element j at +j*es
  int n;                    // N
  int logL;
  const void* tw;
  // spectral scaling (fused pass only)
  const double* cosv;
  const float* s32;           // sin^2(k pi/2N) for the FP32 path
  const double* scale64;      // precomputed scale for the FP64 path (mode grid, C order)
  double ih2, kt, gscale;   // gscale = (2/N)^d
  int d, order;
  int fused;
  int amode;                // 1 if the a index is a mode index of the scaling (3D)
  const int* skip;          // convergence flag (skip when *skip != 0), may be null
  unsigned long long* corr_max;   // accumulate pass: max |correction|, max |u + correction|
  float* delta_out;               // accumulate pass: also keep the FP32 correction (in place)
};

template <typename T>
__device__ __forceinline__ T ld(const void* p, int is64, long long i) {
  return is64 ? (T)static_cast<const double*>(p)[i] : (T)static_cast<const float*>(p)[i];
}

// lambda h^2 with s_k = sin^2(k pi / 2N) (c_k = 1 - 2 s_k), free of the
// cancellation of the cosine form for low modes:
//   9-pt:  -4 (s_p + s_q) + 8/3 s_p s_q          - kappa h^2 (1 - (s_p + s_q)/3)
//   27-pt: -4 S1 + 8/3 S2 - 4/3 S3                - kappa h^2 (1 - S1/3)
//   5/7-pt: -4 S1                                  - kappa h^2
template <typename R>
__device__ __forceinline__ R lam_h2(int d, int order, R kh2, R sp, R sq, R sr) {
  if (order == 2) return (R)-4 * (d == 2 ? sp + sq : sp + sq + sr) - kh2;
  if (d == 2) return (R)-4 * (sp + sq) + (R)(8.0 / 3.0) * sp * sq - kh2 * ((R)1 - (sp + sq) / (R)3);
  R s1 = sp + sq + sr;
  R s2 = sp * sq + sq * sr + sr * sp;
  R s3 = sp * sq * sr;
  return (R)-4 * s1 + (R)(8.0 / 3.0) * s2 - (R)(4.0 / 3.0) * s3 - kh2 * ((R)1 - s1 / (R)3);
}

__global__ void k_scale_table(int d, int order, int n, double kh2, double gh2,
                              const double* __restrict__ sv, double* __restrict__ out) {
  const long long m = n - 1;
  const long long tot = d == 2 ? m * m : m * m * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int q = (int)(t % m) + 1;
    long long r = t / m;
    int p = (int)(r % m) + 1;
    int pr = d == 3 ? (int)(r / m) + 1 : 0;
    // index order (slowest..fastest) = (transform mode j, a, b) of the fused pass
    double v = d == 2 ? lam_h2<double>(2, order, kh2, sv[p], sv[q], 0.0)
                      : lam_h2<double>(3, order, kh2, sv[pr], sv[p], sv[q]);
    out[t] = gh2 / v;
  }
}

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Self-sorting (Stockham) FFT of length L = 2^k on P sequences in shared
// memory, natural order in and out, radix-4 stages and one radix-2 stage when
// k is odd.  x and y are ping-pong buffers; returns the buffer holding the
// result.  tw[t] = exp(-2 pi i t / L), t in [0, L).
template <typename T, int P>
__device__ Cx<T>* fft_stockham(Cx<T>* x, Cx<T>* y, int L, const Cx<T>* __restrict__ tw) {
  int n = L, s = 1, ls = 0;
  const int lq4 = __ffs(L) - 3;     // log2(L / 4)
  while (n >= 4) {
    const int m = n >> 2;
    const int q4 = L >> 2;          // butterflies per sequence per stage (m * s)
    const int tstep = L / n;        // twiddle index scale
    for (int t = threadIdx.x; t < q4 * P; t += blockDim.x) {
      const int pr = t >> lq4;
      const int b = t & (q4 - 1);
      const int q = b & (s - 1);
      const int p = b >> ls;
      const Cx<T>* xx = x + pr * L;
      Cx<T>* yy = y + pr * L;
      const Cx<T> a = xx[q + s * p];
      const Cx<T> bb = xx[q + s * (p + m)];
      const Cx<T> c = xx[q + s * (p + 2 * m)];
      const Cx<T> d = xx[q + s * (p + 3 * m)];
      const Cx<T> apc = {a.x + c.x, a.y + c.y}, amc = {a.x - c.x, a.y - c.y};
      const Cx<T> bpd = {bb.x + d.x, bb.y + d.y};
      const Cx<T> jbmd = {bb.y - d.y, d.x - bb.x};   // -i (b - d)
      const int o = q + s * 4 * p;
      yy[o] = {apc.x + bpd.x, apc.y + bpd.y};
      yy[o + s] = cmul(Cx<T>{amc.x + jbmd.x, amc.y + jbmd.y}, tw[p * tstep]);
      yy[o + 2 * s] = cmul(Cx<T>{apc.x - bpd.x, apc.y - bpd.y}, tw[2 * p * tstep]);
      yy[o + 3 * s] = cmul(Cx<T>{amc.x - jbmd.x, amc.y - jbmd.y}, tw[3 * p * tstep]);
    }
    __syncthreads();
    Cx<T>* tmp = x;
    x = y;
    y = tmp;
    n = m;
    s <<= 2;
    ls += 2;
  }
  if (n == 2) {
    const int q2 = L >> 1;
    for (int t = threadIdx.x; t < q2 * P; t += blockDim.x) {
      const int pr = t >> (lq4 + 1);
      const int q = t & (q2 - 1);    // p = 0, m = 1: no twiddle
      const Cx<T>* xx = x + pr * L;
      Cx<T>* yy = y + pr * L;
      const Cx<T> a = xx[q], b = xx[q + s];
      yy[q] = {a.x + b.x, a.y + b.y};
      yy[q + s] = {a.x - b.x, a.y - b.y};
    }
    __syncthreads();
    x = y;
  }
  return x;
}

// One DST-I pass over P line pairs (see file comment): line pairs starting at
// b0 = 1 + 2 P bx of the line family a = by + 1.
template <typename T, int P>
__device__ __forceinline__ void dst_pass_device(const PassArgs& A, int bx, int by,
                                                unsigned char* smraw) {
  Cx<T>* z = reinterpret_cast<Cx<T>*>(smraw);
  Cx<T>* zb = z + (size_t)P * 2 * A.n;      // ping-pong buffer
  const Cx<T>* tw = static_cast<const Cx<T>*>(A.tw);
  const int n = A.n;
  const int L = 2 * n;
  const int nm1 = n - 1;
  const int a = by + 1;
  const int b0 = 1 + 2 * P * bx;
  const long long abase = (long long)a * A.sa;
  const bool contig = A.es == 1;
  const int nval = nm1 * 2 * P;
  // load the odd extensions
  for (int t = threadIdx.x; t < nval; t += blockDim.x) {
    int j, q;
    if (contig) {
      j = 1 + t % nm1;
      q = t / nm1;
    } else {
      q = t % (2 * P);
      j = 1 + t / (2 * P);
    }
    const int b = b0 + q;
    T v = (T)0;
    if (b <= nm1) v = ld<T>(A.src, A.src64, abase + (long long)b * A.sb + (long long)j * A.es);
    Cx<T>* zz = z + (q >> 1) * L;
    if (q & 1) {
      zz[j].y = v;
      zz[L - j].y = -v;
    } else {
      zz[j].x = v;
      zz[L - j].x = -v;
    }
  }
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    z[t * L] = {(T)0, (T)0};
    z[t * L + n] = {(T)0, (T)0};
  }
  __syncthreads();
  z = fft_stockham<T, P>(z, zb, L, tw);
  zb = (z == reinterpret_cast<Cx<T>*>(smraw)) ? z + (size_t)P * L : reinterpret_cast<Cx<T>*>(smraw);
  if (A.fused) {
    // spectral division in place (natural order; Z_{L-k} = -Z_k makes the
    // rescaled sequence the odd extension of the next input), then the same FFT
    for (int t = threadIdx.x; t < L * P; t += blockDim.x) {
      const int pr = t >> A.logL;
      const int pos = t & (L - 1);
      const int k = pos;
      Cx<T>* zz = z + pr * L;
      if (k == 0 || k == n) {
        zz[pos] = {(T)0, (T)0};
        continue;
      }
      const int km = k < n ? k : L - k;     // the mode of k and of L - k
      const int bA = b0 + 2 * pr, bB = min(bA + 1, nm1);
      T scA, scB;
      if (sizeof(T) == 8) {
        // FP64: precomputed (2/N)^d h^2 / (lambda h^2), table index (km, a, b)
        const long long m1 = nm1;
        long long base = (A.d == 2) ? (long long)(km - 1) * m1
                                    : ((long long)(km - 1) * m1 + (a - 1)) * m1;
        scA = (T)A.scale64[base + bA - 1];
        scB = (T)A.scale64[base + bB - 1];
      } else {
        const float kh2 = (float)A.kt;   // kappa h^2 (precomputed on the host)
        const float g = (float)A.gscale;
        const float sk = A.s32[km];
        const float sa = A.d == 3 ? A.s32[a] : 0.f;
        if (A.d == 2) {
          scA = (T)(g / lam_h2<float>(2, A.order, kh2, sk, A.s32[bA], 0.f));
          scB = (T)(g / lam_h2<float>(2, A.order, kh2, sk, A.s32[bB], 0.f));
        } else {
          scA = (T)(g / lam_h2<float>(3, A.order, kh2, sk, sa, A.s32[bA]));
          scB = (T)(g / lam_h2<float>(3, A.order, kh2, sk, sa, A.s32[bB]));
        }
      }
      Cx<T> Z = zz[pos];
      // A_k = -Im(Z)/2 (line bA), B_k = Re(Z)/2 (line bB); repack x = sA A + i sB B
      zz[pos] = {scA * ((T)-0.5 * Z.y), scB * ((T)0.5 * Z.x)};
    }
    __syncthreads();
    z = fft_stockham<T, P>(z, zb, L, tw);
  }
  // extract S_k = -Im(Z_k)/2 (first line) and Re(Z_k)/2 (second line) and store
  float dmx = 0.f, umx = 0.f;
  for (int t = threadIdx.x; t < nval; t += blockDim.x) {
    int j, q;
    if (contig) {
      j = 1 + t % nm1;
      q = t / nm1;
    } else {
      q = t % (2 * P);
      j = 1 + t / (2 * P);
    }
    const int b = b0 + q;
    if (b > nm1) continue;
    const Cx<T>* zz = z + (q >> 1) * L;
    Cx<T> Z = zz[j];
    T v = (q & 1) ? (T)0.5 * Z.x : (T)-0.5 * Z.y;
    long long off = abase + (long long)b * A.sb + (long long)j * A.es;
    if (A.dst64) {
      double* o = static_cast<double*>(A.dst);
      double nv = A.accumulate ? o[off] + (double)v : (double)v;
      o[off] = nv;
      if (A.delta_out) A.delta_out[off] = (float)v;
      if (A.corr_max) {
        dmx = fmaxf(dmx, fabsf((float)v));
        umx = fmaxf(umx, fabsf((float)nv));
      }
    } else {
      static_cast<float*>(A.dst)[off] = (float)v;
    }
  }
  if (A.corr_max) {
    for (int o = 16; o > 0; o >>= 1) {
      dmx = fmaxf(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
      umx = fmaxf(umx, __shfl_xor_sync(0xffffffffu, umx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      // non-negative doubles order like their bit patterns
      if (dmx > 0.f) atomicMax(A.corr_max, (unsigned long long)__double_as_longlong((double)dmx));
      if (umx > 0.f) atomicMax(A.corr_max + 1, (unsigned long long)__double_as_longlong((double)umx));
    }
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_dst_pass(PassArgs A) {
  if (A.skip && *A.skip) return;
  extern __shared__ unsigned char smraw[];
  dst_pass_device<T, P>(A, blockIdx.x, blockIdx.y, smraw);
}

// Persistent batched pass over many independent grids (one pair per work
// item): item -> instance by binary search in the prefix `start`, each
// instance with its own PassArgs (its own N, pointers and convergence flag).
template <typename T>
__global__ void __launch_bounds__(256) k_dst_pass_batched(const PassArgs* __restrict__ args,
                                                         const int* __restrict__ start, int ninst) {
  extern __shared__ unsigned char smraw[];
  const int total = start[ninst];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = ninst;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (start[mid] <= item) lo = mid; else hi = mid;
    }
    const PassArgs& A = args[lo];
    if (A.skip && *A.skip) continue;
    const int local = item - start[lo];
    const int npx = A.n / 2;
    dst_pass_device<T, 1>(A, local % npx, local / npx, smraw);
    __syncthreads();
  }
}

// r = R - A_h u at interior nodes (u zero on the boundary layer), and max|r|.
// Launch: x over the last (contiguous) axis, y (and z) over the others.
__global__ void k_residual(Grid g, int order, const double* __restrict__ c, const double* __restrict__ R,
                           const double* __restrict__ u, double* __restrict__ r,
                           unsigned long long* __restrict__ nrm, const int* skip) {
  if (skip && *skip) return;
  const int n1 = g.n + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = blockIdx.y;
  const int i0 = blockIdx.z;
  double mx = 0.0;
  if (j <= g.n) {
    const long long t = g.d == 2 ? (long long)i1 * n1 + j : ((long long)i0 * n1 + i1) * n1 + j;
    const bool interior = j >= 1 && j < g.n && i1 >= 1 && i1 < g.n && (g.d == 2 || (i0 >= 1 && i0 < g.n));
    if (!interior) {
      r[t] = 0.0;
    } else {
      const double* up = u + t;
      double acc;
      if (g.d == 2) {
        double s1 = (up[-1] + up[1]) + (up[-n1] + up[n1]);
        acc = c[0] * up[0] + c[1] * s1;
        if (order == 4) acc += c[2] * ((up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]));
      } else {
        const long long s = (long long)n1 * n1;
        double f = (up[-1] + up[1]) + (up[-n1] + up[n1]) + (up[-s] + up[s]);
        acc = c[0] * up[0] + c[1] * f;
        if (order == 4) {
          double e = (up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]) + (up[-s - 1] + up[-s + 1]) +
                     (up[s - 1] + up[s + 1]) + (up[-s - n1] + up[-s + n1]) + (up[s - n1] + up[s + n1]);
          double k = (up[-s - n1 - 1] + up[-s - n1 + 1]) + (up[-s + n1 - 1] + up[-s + n1 + 1]) +
                     (up[s - n1 - 1] + up[s - n1 + 1]) + (up[s + n1 - 1] + up[s + n1 + 1]);
          acc += c[2] * e + c[3] * k;
        }
      }
      double v = R[t] - acc;
      r[t] = v;
      mx = fabs(v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(nrm, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_absmax(long long tot, const double* __restrict__ R, unsigned long long* nrm) {
  double mx = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(R[t]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(nrm, (unsigned long long)__double_as_longlong(mx));
}

// Refinement stop: conv = (max|delta_k| <= tol max|u_{k+1}|), the size of the
// last FP32 correction against the solution (a residual test would sit on the
// rounding floor eps cond(A_h) of the FP64 residual itself at large N).
// Keeps the last ratio's terms in nrm[2..] and resets the accumulation slots.
__global__ void k_check(unsigned long long* nrm, double tol, int* conv) {
  if (*conv) return;
  double dm = __longlong_as_double((long long)nrm[3]);
  double um = __longlong_as_double((long long)nrm[4]);
  nrm[2] = nrm[3];
  nrm[5] = nrm[4];
  if (dm <= tol * um) *conv = 1;
  nrm[3] = 0ull;
  nrm[4] = 0ull;
}

__global__ void k_zero_flags(unsigned long long* nrm, int* conv) {
  for (int k = 0; k < 6; ++k) nrm[k] = 0ull;
  *conv = 0;
}

template <typename T, int P>
void launch_pass_p(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st) {
  dim3 grid((unsigned)((npairs_b + P - 1) / P), (unsigned)na);
  size_t smem = sizeof(Cx<T>) * (size_t)(2 * A.n) * P * 2;
  KFBI_LAUNCH(p, KFBI_KC_DST, k_dst_pass<T, P><<<grid, 256, smem, st>>>(A));
}

// pairs per CTA: enough butterflies for 256 threads (P L / 4 >= 256), at least
// `pmin` (strided passes read 2 P adjacent lines per row)
template <typename T>
void launch_pass(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st, int pmin) {
  const int L = 2 * A.n;
  int P = std::max(pmin, 1024 / L);
  if (sizeof(T) == 8 && L >= 2048) P = std::min(P, 1);
  if (P >= 8) launch_pass_p<T, 8>(p, A, npairs_b, na, st);
  else if (P >= 4) launch_pass_p<T, 4>(p, A, npairs_b, na, st);
  else if (P >= 2) launch_pass_p<T, 2>(p, A, npairs_b, na, st);
  else launch_pass_p<T, 1>(p, A, npairs_b, na, st);
}

// The dynamic shared-memory limit is a per-kernel, process-wide attribute:
// raise it once to the device maximum (problems of different N share it).
template <typename T, int P>
cudaError_t set_smem(int max_optin) {
  return cudaFuncSetAttribute(k_dst_pass<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_optin);
}

// The passes of one DST solve of `src` (grid, FP64 or FP32) into `dst` (grid,
// FP64), overwriting or accumulating, with a work buffer of type T: the
// argument block of each pass, the pairs-per-CTA floor (strided passes read
// 2 P adjacent lines) and the number of line families.
struct PassPlan {
  PassArgs args[5];
  int pmin[5];
  int npass = 0, npairs = 0, na = 1;
};

template <typename T>
PassPlan plan_passes(kfbi_problem* p, const void* src, int src64, double* dst, int accumulate,
                     const int* skip, unsigned long long* corr_max) {
  BoxSolver* B = p->box;
  const Grid g = p->g;
  const int n = g.n, n1 = n + 1;
  T* work = std::is_same<T, double>::value ? reinterpret_cast<T*>(B->work64)
                                            : reinterpret_cast<T*>(B->work32);
  const void* tw = std::is_same<T, double>::value ? (const void*)B->tw64 : (const void*)B->tw32;
  PassArgs A;
  memset(&A, 0, sizeof(A));
  A.n = n;
  A.logL = B->logL;
  A.tw = tw;
  A.cosv = B->cosv;
  A.s32 = B->s32;
  A.scale64 = B->scale64;
  A.ih2 = 1.0 / (g.h * g.h);
  A.kt = p->kt * g.h * g.h;   // kappa h^2
  A.d = g.d;
  A.order = p->cfg.order;
  A.skip = skip;
  A.gscale = (g.d == 2 ? (2.0 / n) * (2.0 / n) : (2.0 / n) * (2.0 / n) * (2.0 / n)) * g.h * g.h;
  const int is64 = std::is_same<T, double>::value ? 1 : 0;
  PassPlan P;
  P.npairs = n / 2;   // ceil((N-1)/2) for even N
  P.na = g.d == 2 ? 1 : n - 1;
  auto add = [&](const void* s, int s64, void* d, int d64, int acc, long long sa, long long sb,
                 long long es, int fused, int pmin) {
    PassArgs& Q = P.args[P.npass];
    Q = A;
    Q.src = s;
    Q.src64 = s64;
    Q.dst = d;
    Q.dst64 = d64;
    Q.accumulate = acc;
    Q.corr_max = (d64 && acc) ? corr_max : nullptr;
    Q.sa = sa;
    Q.sb = sb;
    Q.es = es;
    Q.fused = fused;
    P.pmin[P.npass] = pmin;
    ++P.npass;
  };
  if (g.d == 2) {
    add(src, src64, work, is64, 0, 0, n1, 1, 0, 1);          // axis 1, lines b = i0
    add(work, is64, work, is64, 0, 0, 1, n1, 1, 2);          // axis 0 fused, lines b = i1
    add(work, is64, dst, 1, accumulate, 0, n1, 1, 0, 1);     // axis 1
  } else {
    const long long s0 = (long long)n1 * n1;
    add(src, src64, work, is64, 0, s0, n1, 1, 0, 1);         // axis 2, lines (i0, i1)
    add(work, is64, work, is64, 0, s0, 1, n1, 0, 2);         // axis 1, lines (i0, i2)
    add(work, is64, work, is64, 0, n1, 1, s0, 1, 2);         // axis 0 fused, lines (i1, i2)
    add(work, is64, work, is64, 0, s0, 1, n1, 0, 2);         // axis 1
    add(work, is64, dst, 1, accumulate, s0, n1, 1, 0, 1);    // axis 2
  }
  return P;
}

template <typename T>
kfbi_status dst_solve_t(kfbi_problem* p, const void* src, int src64, double* dst, int accumulate,
                        const int* skip, unsigned long long* corr_max = nullptr) {
  PassPlan P = plan_passes<T>(p, src, src64, dst, accumulate, skip, corr_max);
  for (int k = 0; k < P.npass; ++k)
    launch_pass<T>(p, P.args[k], P.npairs, P.na, p->stream, P.pmin[k]);
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

}  // namespace

kfbi_status mg_create(kfbi_problem* p);
void mg_destroy(kfbi_problem* p);
kfbi_status mg_solve(kfbi_problem* p, const double* rhs, double* u);
kfbi_status mg_last_residual(kfbi_problem* p, double* rel, int* converged);

kfbi_status box_create(kfbi_problem* p) {
  if (p->cfg.box_solver == KFBI_BOX_MG) return mg_create(p);
  const Grid g = p->g;
  const int n = g.n;
  if (n < 8 || (n & (n - 1)) != 0) return fail(p, KFBI_ERR_UNSUPPORTED, "N must be a power of two >= 8");
  if ((g.d == 2 && n > 4096) || (g.d == 3 && n > 1024))
    return fail(p, KFBI_ERR_UNSUPPORTED, "N too large for the shared-memory DST");
  BoxSolver* B = new BoxSolver();
  p->box = B;
  B->L = 2 * n;
  B->logL = 0;
  while ((1 << B->logL) < B->L) ++B->logL;
  std::vector<double> tw(2 * B->L);    // interleaved re, im over the full circle
  std::vector<float> tw32(2 * B->L);
  for (int t = 0; t < B->L; ++t) {
    double ang = -2.0 * M_PI * (double)t / (double)B->L;
    tw[2 * t] = std::cos(ang);
    tw[2 * t + 1] = std::sin(ang);
    tw32[2 * t] = (float)tw[2 * t];
    tw32[2 * t + 1] = (float)tw[2 * t + 1];
  }
  std::vector<double> cs(n + 1);
  for (int k = 0; k <= n; ++k) cs[k] = std::cos((double)k * M_PI / (double)n);
  std::vector<double> sv(n + 1);
  std::vector<float> sv32(n + 1);
  for (int k = 0; k <= n; ++k) {
    double t = std::sin((double)k * M_PI / (2.0 * n));
    sv[k] = t * t;
    sv32[k] = (float)sv[k];
  }
  KFBI_CUDA(p, dalloc(&B->s64, n + 1));
  KFBI_CUDA(p, dalloc(&B->s32, n + 1));
  KFBI_CUDA(p, cudaMemcpy(B->s64, sv.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice));
  KFBI_CUDA(p, cudaMemcpy(B->s32, sv32.data(), sizeof(float) * (n + 1), cudaMemcpyHostToDevice));
  KFBI_CUDA(p, dalloc(&B->tw64, 2 * B->L));
  KFBI_CUDA(p, dalloc(&B->tw32, 2 * B->L));
  KFBI_CUDA(p, dalloc(&B->cosv, n + 1));
  KFBI_CUDA(p, cudaMemcpy(B->tw64, tw.data(), sizeof(double) * 2 * B->L, cudaMemcpyHostToDevice));
  KFBI_CUDA(p, cudaMemcpy(B->tw32, tw32.data(), sizeof(float) * 2 * B->L, cudaMemcpyHostToDevice));
  KFBI_CUDA(p, cudaMemcpy(B->cosv, cs.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice));
  const long long nodes = g.nodes();
  if (p->cfg.precision == KFBI_MIXED) {
    KFBI_CUDA(p, dalloc(&B->work32, nodes));
    KFBI_CUDA(p, cudaMemset(B->work32, 0, sizeof(float) * nodes));
    KFBI_CUDA(p, dalloc(&B->res, nodes));
    KFBI_CUDA(p, cudaMemset(B->res, 0, sizeof(double) * nodes));

  } else {
    KFBI_CUDA(p, dalloc(&B->work64, nodes));
    const long long m = n - 1;
    const long long nm = g.d == 2 ? m * m : m * m * m;
    KFBI_CUDA(p, dalloc(&B->scale64, nm));
    const double gh2 = (g.d == 2 ? (2.0 / n) * (2.0 / n) : (2.0 / n) * (2.0 / n) * (2.0 / n)) * g.h * g.h;
    k_scale_table<<<std::min(div_up(nm, 256), 152 * 16), 256>>>(g.d, p->cfg.order, n, p->kt * g.h * g.h,
                                                                gh2, B->s64, B->scale64);
    KFBI_CUDA(p, cudaGetLastError());
    KFBI_CUDA(p, cudaDeviceSynchronize());
  }
  KFBI_CUDA(p, dalloc(&B->nrm, 6));
  KFBI_CUDA(p, dalloc(&B->conv, 1));
  B->tol = p->cfg.box_rtol > 0 ? p->cfg.box_rtol : 1e-13;
  B->refine_steps = p->cfg.box_max_iters > 0 ? std::min(p->cfg.box_max_iters, 8) : 5;
  int dev = 0, optin = 0;
  KFBI_CUDA(p, cudaGetDevice(&dev));
  KFBI_CUDA(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if ((size_t)optin < sizeof(Cx<double>) * (size_t)(2 * n) * 2 * std::max(1, 1024 / (2 * n)) ||
      (size_t)optin < sizeof(Cx<float>) * (size_t)(2 * n) * 2 * std::max(2, 1024 / (2 * n)))
    return fail(p, KFBI_ERR_UNSUPPORTED, "N too large for the shared-memory DST on this device");
  KFBI_CUDA(p, (set_smem<double, 1>(optin)));
  KFBI_CUDA(p, (set_smem<double, 2>(optin)));
  KFBI_CUDA(p, (set_smem<double, 4>(optin)));
  KFBI_CUDA(p, (set_smem<double, 8>(optin)));
  KFBI_CUDA(p, (set_smem<float, 1>(optin)));
  KFBI_CUDA(p, (set_smem<float, 2>(optin)));
  KFBI_CUDA(p, (set_smem<float, 4>(optin)));
  KFBI_CUDA(p, (set_smem<float, 8>(optin)));
  return KFBI_OK;
}

void box_destroy(kfbi_problem* p) {
  mg_destroy(p);
  BoxSolver* B = p->box;
  if (!B) return;
  cudaFree(B->tw64);
  cudaFree(B->tw32);
  cudaFree(B->cosv);
  cudaFree(B->s64);
  cudaFree(B->s32);
  cudaFree(B->scale64);
  cudaFree(B->work64);
  cudaFree(B->work32);
  cudaFree(B->res);
  cudaFree(B->nrm);
  cudaFree(B->conv);
  delete B;
  p->box = nullptr;
}

kfbi_status box_solve(kfbi_problem* p, const double* rhs, double* u) {
  if (p->mg) {
    KFBI_TRY(mg_solve(p, rhs, u));
    return launch_set_boundary(p, u, nullptr);
  }
  BoxSolver* B = p->box;
  const Grid g = p->g;
  if (p->cfg.precision != KFBI_MIXED) {
    KFBI_TRY(dst_solve_t<double>(p, rhs, 1, u, 0, nullptr));
    return launch_set_boundary(p, u, nullptr);
  }
  // mixed: u = 0; repeat { u += DST32^{-1}(r); r = R - A_h u } until max|r| <= tol max|R|
  cudaStream_t st = p->stream;
  const long long nodes = g.nodes();
  KFBI_CUDA(p, cudaMemsetAsync(u, 0, sizeof(double) * nodes, st));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_zero_flags<<<1, 1, 0, st>>>(B->nrm, B->conv));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_absmax<<<std::min(div_up(nodes, 256), 152 * 8), 256, 0, st>>>(nodes, rhs, B->nrm));
  KFBI_CUDA(p, cudaGetLastError());
  // u += delta_k = DST32(r_k); r_{k+1} = R - A_h u in FP64 every step.  (An
  // update r_k - A_h delta_k with A_h delta_k in FP32 is not enough: delta_k is
  // smooth, A_h delta_k cancels by ~cond(A_h), and its FP32 rounding is then as
  // large as the residual itself.)
  const dim3 rgrid((unsigned)div_up(g.n + 1, 128), (unsigned)(g.n + 1), g.d == 3 ? (unsigned)(g.n + 1) : 1u);
  for (int it = 0; it < B->refine_steps; ++it) {
    KFBI_TRY(dst_solve_t<float>(p, it == 0 ? (const void*)rhs : (const void*)B->res, 1, u, 1, B->conv,
                                B->nrm + 3));
    KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_check<<<1, 1, 0, st>>>(B->nrm, B->tol, B->conv));
    if (it + 1 < B->refine_steps) {
      KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_residual<<<rgrid, 128, 0, st>>>(
          g, p->cfg.order, p->stencil_dev, rhs, u, B->res, B->nrm + 1, B->conv));
    }
    KFBI_CUDA(p, cudaGetLastError());
  }
  return KFBI_OK;
}

// Host-visible diagnostics of the last mixed solve: max|R - A_h u| / max|R|.
kfbi_status box_last_residual(kfbi_problem* p, double* rel, int* converged) {
  if (p->mg) return mg_last_residual(p, rel, converged);
  BoxSolver* B = p->box;
  unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
  int c = 1;
  if (p->cfg.precision == KFBI_MIXED) {
    KFBI_CUDA(p, cudaMemcpyAsync(h, B->nrm, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    KFBI_CUDA(p, cudaMemcpyAsync(&c, B->conv, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  }
  double dm, um;
  memcpy(&dm, &h[2], 8);
  memcpy(&um, &h[5], 8);
  *rel = um > 0 ? dm / um : 0.0;
  *converged = c;
  return KFBI_OK;
}

}  // namespace kfbi

// ---------------------------------------------------------------------------
// Box solve that allocates nothing (kfbi_box_solve_noalloc).
//
// For callers that cannot call cudaMalloc — code running where the allocator
// is unavailable or forbidden, e.g. inside another library's memory pool
// discipline, a plugin host that owns all device memory, or a context where an
// allocation could synchronise or fail mid-pipeline.  The caller passes the
// right-hand side and the output grid; everything else the FP64 sine-transform
// solve needs (work grid, spectral scale table, twiddles, sin^2 table) lives in
// one file-scope __device__ array of fixed size.  Every GPU that loads this
// library holds that array (about 4.4 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace kfbi {
namespace {

constexpr int kNoAllocMaxN2 = 512;                // 2D: N <= 512
constexpr int kNoAllocMaxN3 = 64;                 // 3D: N <= 64
constexpr long long kNoAllocGrid = 65LL * 65 * 65;   // >= max (N+1)^d = 274625
constexpr long long kNoAllocTw = 4 * 1024;        // full-circle twiddles, L <= 1024
constexpr long long kNoAllocS = 1024;             // sin^2 table, N + 1 <= 513
constexpr long long kNoAllocTotal = 2 * kNoAllocGrid + kNoAllocTw + kNoAllocS;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocTotal];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

__global__ void k_noalloc_tables(int n, double* __restrict__ tw, double* __restrict__ sv) {
  const int L = 2 * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)L, &s, &c);
    tw[2 * t] = c;
    tw[2 * t + 1] = s;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
    double s = sinpi((double)k / (2.0 * n));
    sv[k] = s * s;
  }
}

template <int P>
void noalloc_pass(const PassArgs& A, int npairs, int na, cudaStream_t st) {
  dim3 grid((unsigned)((npairs + P - 1) / P), (unsigned)na);
  size_t smem = sizeof(Cx<double>) * (size_t)(2 * A.n) * P * 2;
  k_dst_pass<double, P><<<grid, 256, smem, st>>>(A);
}

void noalloc_launch(const PassArgs& A, int npairs, int na, cudaStream_t st, int pmin) {
  const int P = std::max(pmin, 1024 / (2 * A.n));
  if (P >= 8) noalloc_pass<8>(A, npairs, na, st);
  else if (P >= 4) noalloc_pass<4>(A, npairs, na, st);
  else if (P >= 2) noalloc_pass<2>(A, npairs, na, st);
  else noalloc_pass<1>(A, npairs, na, st);
}

}  // namespace

}  // namespace kfbi

extern "C" kfbi_status kfbi_box_solve_noalloc(int dim, int n, double lo, double hi, int order,
                                              double kappa, const double* rhs, double* u,
                                              void* cuda_stream) {
  using namespace kfbi;
  if ((dim != 2 && dim != 3) || (order != 2 && order != 4) || !(hi > lo) || !(kappa >= 0.0) ||
      !rhs || !u || n < 8 || (n & (n - 1)) != 0)
    return KFBI_ERR_ARG;
  if ((dim == 2 && n > kNoAllocMaxN2) || (dim == 3 && n > kNoAllocMaxN3))
    return KFBI_ERR_ARG;   // beyond the fixed scratch: 2D N <= 512, 3D N <= 64
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return KFBI_ERR_CUDA;
  double* base = nullptr;
  {
    // one-time set-up per device: the array's device address (a host-side
    // reference to it is only a stand-in) and the shared-memory limits
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      double* ptr = nullptr;
      if (cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_scratch) != cudaSuccess ||
          !ptr)
        return KFBI_ERR_CUDA;
      int optin = 0;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return KFBI_ERR_CUDA;
      if (cudaFuncSetAttribute(k_dst_pass<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
          cudaFuncSetAttribute(k_dst_pass<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
          cudaFuncSetAttribute(k_dst_pass<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
          cudaFuncSetAttribute(k_dst_pass<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess)
        return KFBI_ERR_CUDA;
      g_noalloc_ptr[dev] = ptr;
    }
    base = g_noalloc_ptr[dev];
  }
  double* work = base;
  double* scale = base + kNoAllocGrid;
  double* tw = base + 2 * kNoAllocGrid;
  double* sv = tw + kNoAllocTw;
  const double h = (hi - lo) / n;
  const double kt = kappa;
  const double gh2 = (dim == 2 ? (2.0 / n) * (2.0 / n) : (2.0 / n) * (2.0 / n) * (2.0 / n)) * h * h;
  const long long m = n - 1;
  const long long nm = dim == 2 ? m * m : m * m * m;
  const long long nodes = dim == 2 ? (long long)(n + 1) * (n + 1) : (long long)(n + 1) * (n + 1) * (n + 1);
  // the tables depend on N and kappa, so every call rebuilds them
  k_noalloc_tables<<<4, 256, 0, st>>>(n, tw, sv);
  k_scale_table<<<std::min(div_up(nm, 256), 152 * 16), 256, 0, st>>>(dim, order, n, kt * h * h, gh2, sv, scale);
  if (cudaMemsetAsync(u, 0, sizeof(double) * nodes, st) != cudaSuccess) return KFBI_ERR_CUDA;
  PassArgs A;
  memset(&A, 0, sizeof(A));
  A.n = n;
  int logL = 0;
  while ((1 << logL) < 2 * n) ++logL;
  A.logL = logL;
  A.tw = tw;
  A.scale64 = scale;
  A.d = dim;
  A.order = order;
  const int npairs = n / 2;
  const int n1 = n + 1;
  auto io = [&](const void* s, void* d, int d64) {
    A.src = s;
    A.src64 = 1;
    A.dst = d;
    A.dst64 = d64;
    A.accumulate = 0;
  };
  if (dim == 2) {
    io(rhs, work, 1);
    A.sa = 0; A.sb = n1; A.es = 1; A.fused = 0;
    noalloc_launch(A, npairs, 1, st, 1);
    io(work, work, 1);
    A.sa = 0; A.sb = 1; A.es = n1; A.fused = 1;
    noalloc_launch(A, npairs, 1, st, 2);
    io(work, u, 1);
    A.sa = 0; A.sb = n1; A.es = 1; A.fused = 0;
    noalloc_launch(A, npairs, 1, st, 1);
  } else {
    const long long s0 = (long long)n1 * n1;
    io(rhs, work, 1);
    A.sa = s0; A.sb = n1; A.es = 1; A.fused = 0;
    noalloc_launch(A, npairs, n - 1, st, 1);
    io(work, work, 1);
    A.sa = s0; A.sb = 1; A.es = n1;
    noalloc_launch(A, npairs, n - 1, st, 2);
    A.sa = n1; A.sb = 1; A.es = s0; A.fused = 1;
    noalloc_launch(A, npairs, n - 1, st, 2);
    A.fused = 0;
    A.sa = s0; A.sb = 1; A.es = n1;
    noalloc_launch(A, npairs, n - 1, st, 2);
    io(work, u, 1);
    A.sa = s0; A.sb = n1; A.es = 1;
    noalloc_launch(A, npairs, n - 1, st, 1);
  }
  return cudaGetLastError() == cudaSuccess ? KFBI_OK : KFBI_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Batched mixed-precision box solve: many independent grids (different N) in
// one launch per pass (persistent CTAs over all instances' line pairs) and one
// launch per residual / check, with per-instance convergence flags.
// ---------------------------------------------------------------------------
namespace kfbi {
namespace {

struct ResDesc {
  Grid g;
  int order;
  const double* c;
  const double* R;
  double* u;
  double* r;
  unsigned long long* nrm;
  int* conv;
  double tol;
};

__device__ __forceinline__ int find_inst(const int* start, int ninst, int item) {
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// one grid row (last axis) per work item
__global__ void k_residual_batched(const ResDesc* __restrict__ rd, const int* __restrict__ rstart, int ninst) {
  const int total = rstart[ninst];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int inst = find_inst(rstart, ninst, item);
    const ResDesc& D = rd[inst];
    if (*D.conv) continue;
    const Grid g = D.g;
    const int n1 = g.n + 1;
    const int row = item - rstart[inst];
    const int i1 = row % n1, i0 = row / n1;   // 2D: i0 = 0
    double mx = 0.0;
    for (int j = threadIdx.x; j <= g.n; j += blockDim.x) {
      const long long t = g.d == 2 ? (long long)i1 * n1 + j : ((long long)i0 * n1 + i1) * n1 + j;
      const bool interior = j >= 1 && j < g.n && i1 >= 1 && i1 < g.n && (g.d == 2 || (i0 >= 1 && i0 < g.n));
      if (!interior) {
        D.r[t] = 0.0;
        continue;
      }
      const double* up = D.u + t;
      const double* c = D.c;
      double acc;
      if (g.d == 2) {
        double s1 = (up[-1] + up[1]) + (up[-n1] + up[n1]);
        acc = c[0] * up[0] + c[1] * s1;
        if (D.order == 4) acc += c[2] * ((up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]));
      } else {
        const long long s = (long long)n1 * n1;
        double f = (up[-1] + up[1]) + (up[-n1] + up[n1]) + (up[-s] + up[s]);
        acc = c[0] * up[0] + c[1] * f;
        if (D.order == 4) {
          double e = (up[-n1 - 1] + up[-n1 + 1]) + (up[n1 - 1] + up[n1 + 1]) + (up[-s - 1] + up[-s + 1]) +
                     (up[s - 1] + up[s + 1]) + (up[-s - n1] + up[-s + n1]) + (up[s - n1] + up[s + n1]);
          double k = (up[-s - n1 - 1] + up[-s - n1 + 1]) + (up[-s + n1 - 1] + up[-s + n1 + 1]) +
                     (up[s - n1 - 1] + up[s - n1 + 1]) + (up[s + n1 - 1] + up[s + n1 + 1]);
          acc += c[2] * e + c[3] * k;
        }
      }
      const double v = D.R[t] - acc;
      D.r[t] = v;
      mx = fmax(mx, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0)
      atomicMax(D.nrm + 1, (unsigned long long)__double_as_longlong(mx));
  }
}

__global__ void k_check_batched(const ResDesc* __restrict__ rd, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  const ResDesc& D = rd[i];
  unsigned long long* nrm = D.nrm;
  if (*D.conv) return;
  double dm = __longlong_as_double((long long)nrm[3]);
  double um = __longlong_as_double((long long)nrm[4]);
  nrm[2] = nrm[3];
  nrm[5] = nrm[4];
  if (dm <= D.tol * um) *D.conv = 1;
  nrm[3] = 0ull;
  nrm[4] = 0ull;
}

// Reset the refinement state; instances flagged in `done` (outer iteration
// finished) start as converged, so every pass and residual skips them.
__global__ void k_zero_batched(const ResDesc* __restrict__ rd, int ninst, const int* __restrict__ done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  for (int k = 0; k < 6; ++k) rd[i].nrm[k] = 0ull;
  *rd[i].conv = done ? done[i] : 0;
}

}  // namespace

struct BatchBox {
  int ninst = 0, npass = 0, steps = 4;
  PassArgs* dargs = nullptr;   // [npass + 1][ninst]: pass 0 from R, pass 0 from r, passes 1..
  int* dstart = nullptr;       // [ninst + 1] line-pair work items
  ResDesc* dres = nullptr;     // [ninst]
  int* drstart = nullptr;      // [ninst + 1] residual rows
  std::vector<double*> u, rhs;
  std::vector<size_t> ubytes;
  size_t smem = 0;
  int grid = 0;
};

kfbi_status batch_box_create(kfbi_problem* p0, kfbi_problem* const* ps, int ninst,
                             double* const* rhs, BatchBox** out) {
  BatchBox* bb = new BatchBox();
  *out = bb;
  bb->ninst = ninst;
  const int d = ps[0]->g.d;
  std::vector<PassArgs> args;
  std::vector<int> start(ninst + 1, 0), rstart(ninst + 1, 0);
  std::vector<ResDesc> res(ninst);
  std::vector<PassPlan> plans(ninst), plans_r(ninst);
  int maxn = 0;
  for (int i = 0; i < ninst; ++i) {
    kfbi_problem* p = ps[i];
    if (p->g.d != d || p->cfg.precision != KFBI_MIXED || p->box == nullptr || p->mg != nullptr)
      return fail(p0, KFBI_ERR_UNSUPPORTED,
                  "batched solves need mixed-precision DST problems of one dimension");
    BoxSolver* B = p->box;
    plans[i] = plan_passes<float>(p, rhs[i], 1, p->ugrid, 1, B->conv, B->nrm + 3);
    plans_r[i] = plan_passes<float>(p, B->res, 1, p->ugrid, 1, B->conv, B->nrm + 3);
    start[i + 1] = start[i] + plans[i].npairs * plans[i].na;
    const int n1 = p->g.n + 1;
    rstart[i + 1] = rstart[i] + (d == 2 ? n1 : n1 * n1);
    res[i] = ResDesc{p->g, p->cfg.order, p->stencil_dev, rhs[i], p->ugrid, B->res, B->nrm, B->conv, B->tol};
    maxn = std::max(maxn, p->g.n);
    bb->steps = std::max(bb->steps, B->refine_steps);
    bb->u.push_back(p->ugrid);
    bb->rhs.push_back(rhs[i]);
    bb->ubytes.push_back(sizeof(double) * (size_t)p->g.nodes());
  }
  bb->npass = plans[0].npass;
  for (int v = 0; v <= bb->npass; ++v)
    for (int i = 0; i < ninst; ++i)
      args.push_back(v == 0 ? plans[i].args[0] : v == 1 ? plans_r[i].args[0] : plans[i].args[v - 1]);
  KFBI_CUDA(p0, dalloc(&bb->dargs, args.size()));
  KFBI_CUDA(p0, dalloc(&bb->dstart, ninst + 1));
  KFBI_CUDA(p0, dalloc(&bb->dres, ninst));
  KFBI_CUDA(p0, dalloc(&bb->drstart, ninst + 1));
  KFBI_CUDA(p0, cudaMemcpy(bb->dargs, args.data(), sizeof(PassArgs) * args.size(), cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->dstart, start.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->dres, res.data(), sizeof(ResDesc) * ninst, cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->drstart, rstart.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  bb->smem = sizeof(Cx<float>) * (size_t)(2 * maxn) * 2;
  int dev = 0, optin = 0, sms = 0;
  KFBI_CUDA(p0, cudaGetDevice(&dev));
  KFBI_CUDA(p0, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  KFBI_CUDA(p0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  KFBI_CUDA(p0, cudaFuncSetAttribute(k_dst_pass_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  int per_sm = 0;
  KFBI_CUDA(p0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dst_pass_batched<float>, 256, bb->smem));
  bb->grid = sms * std::max(1, per_sm);
  return KFBI_OK;
}

void batch_box_destroy(BatchBox* bb) {
  if (!bb) return;
  cudaFree(bb->dargs);
  cudaFree(bb->dstart);
  cudaFree(bb->dres);
  cudaFree(bb->drstart);
  delete bb;
}

// All instances not flagged in `done` (may be null): u_i = A_i^{-1} rhs_i by
// FP32 transforms with FP64 refinement.
kfbi_status batch_box_solve(kfbi_problem* p0, BatchBox* bb, const int* done, cudaStream_t st) {
  const int ni = bb->ninst;
  for (int i = 0; i < ni; ++i)   // grid sizes differ: one memset per instance
    KFBI_CUDA(p0, cudaMemsetAsync(bb->u[i], 0, bb->ubytes[i], st));
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_zero_batched<<<div_up(ni, 128), 128, 0, st>>>(bb->dres, ni, done));
  for (int it = 0; it < bb->steps; ++it) {
    for (int v = 0; v < bb->npass; ++v) {
      const PassArgs* a = bb->dargs + (size_t)(v == 0 ? (it == 0 ? 0 : 1) : v + 1) * ni;
      KFBI_LAUNCH(p0, KFBI_KC_DST, k_dst_pass_batched<float><<<bb->grid, 256, bb->smem, st>>>(a, bb->dstart, ni));
    }
    KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_check_batched<<<div_up(ni, 128), 128, 0, st>>>(bb->dres, ni));
    if (it + 1 < bb->steps)
      KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_residual_batched<<<bb->grid, 128, 0, st>>>(bb->dres, bb->drstart, ni));
  }
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
