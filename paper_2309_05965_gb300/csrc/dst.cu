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
// one complex sequence (Z_k = -2i (A_k + i B_k)).  A pass transforms every line
// of one axis, each CTA P line pairs in shared memory, natural order in and
// out (self-sorting Stockham FFTs):
//   * FP64 path (k_dst_pass<double>): radix-4 stages (and one radix-2 stage)
//     over the shared buffer, FP64-ALU bound on GB300;
//   * FP32 path (k_dst32<LOGL, P>): a thread owns 16 points per stage,
//     radix-16 register DFTs, per-stage twiddle tables, a padded buffer.
// The pass along the slowest axis applies the spectral division in place
// between the forward and the inverse transform (Z_{L-k} = -Z_k keeps the
// rescaled sequence the odd extension of the next input), so 2D takes 3
// passes (axis 1, axis 0 fused, axis 1) and 3D 5; each pass reads and writes
// the grid once.  The mixed path (FP32 transforms) refines with an exact
// fixed-point residual r = R - A_h u and a device-side convergence flag, so
// no host synchronisation is needed.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

// max(a, b) that returns NaN when either operand is NaN (fmaxf returns the
// other operand): the norms of the mixed path must see a non-finite solve
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}

template <typename T>
struct Cx {
  T x, y;
};

struct BoxSolver {
  int L = 0, logL = 0;
  double* tw64 = nullptr;     // L/2 twiddles exp(-2 pi i t / L)
  float* tw32 = nullptr;
  float* twst = nullptr;      // FP32 stage twiddle tables (stage_twiddles)
  double* cosv = nullptr;     // cos(k pi / N), k = 0..N
  double* s64 = nullptr;      // sin^2(k pi / 2N), k = 0..N
  float* s32 = nullptr;
  double* scale64 = nullptr;  // FP64 path: (2/N)^d / lambda on the mode grid (N-1)^d
  double* work64 = nullptr;   // grid of doubles
  float* work32 = nullptr;    // grid of floats
  double* res = nullptr;      // FP64 residual grid
  unsigned long long* nrm = nullptr;   // [0] max|R| [1] max|r| [2] last max|delta| [3] max|delta| [4] max|u| [5] last max|u|
                                       // [6] correction steps of the last solve, [7] of all solves since reset,
                                       // [8] relative size of the last first correction (FP32 error estimate)
  double* tol_dev = nullptr;  // the refinement tolerance the checks read (relaxed inside GMRES)
  int* conv = nullptr;        // device flag
  int refine_steps = 4;
  double tol = 1e-13;
  // exact residual of the mixed path in fixed point: mult h^2 A_h = S - kappa h^2 K
  // with S integer weights w[c] by the number c of nonzero offsets and
  // K u = kscale (kA u_P + kB sum of edge neighbours)
  long long* ufix = nullptr;  // u 2^F
  long long* rfix = nullptr;  // mult h^2 R 2^F
  double* fixd = nullptr;     // [0] mult h^2 2^F, [1] 2^-F, [2] kscale kappa h^2
  float* fixf = nullptr;      // 2^Fa, 2^Fb, 2^-Fa, 2^-Fb, 2^-Fb / (mult h^2) (Fa + Fb = F)
  int w[4] = {0, 0, 0, 0};
  int kA = 0, kB = 0;
  double multh2 = 0.0, kc = 0.0;
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
  unsigned long long* corr_max;   // last pass: max |correction|, max |u + correction|
  float* delta_out;               // accumulate pass: also keep the FP32 correction (in place)
  long long* dstfix;              // last pass of a refinement step: u_fix += round(delta 2^F)
  const void* twst;               // FP32 path: stage twiddle tables (stage_twiddles)
  const float* fixf;              // [0..1] 2^Fa, 2^Fb; [2..3] 2^-Fa, 2^-Fb (k_fix_scale)
  const double* fixd;             // [1] mult h^2 2^-F (with uout)
  double* uout;                   // with dstfix: also u = u_fix mult h^2 2^-F in FP64
  unsigned long long* zero_nrm;   // first pass of a mixed solve: CTA 0 clears nrm[0..6] and
  int* zero_conv;                 // the convergence flag before anything reads them
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

// lambda h^2 = alpha + beta s_k along a line of the fused pass, the other
// indices' s fixed (sq = s of the slow mode index in 3D, sr = s of the line):
// the expansions of lam_h2 in s_p = s_k.  alpha < 0 (in 3D -4 (sq + sr)
// outweighs 8/3 sq sr), and beta > 0 only where beta <= kappa h^2 / 3 <= |alpha|,
// so alpha + beta s_k does not cancel.
__device__ __forceinline__ void lam_affine(int d, int order, float kh2, float sq, float sr, float& alpha,
                                           float& beta) {
  const float q = d == 2 ? sr : sq + sr;
  if (order == 2) {
    alpha = -4.f * q - kh2;
    beta = -4.f;
  } else if (d == 2) {
    alpha = -4.f * sr - kh2 * (1.f - sr / 3.f);
    beta = -4.f + (8.f / 3.f) * sr + kh2 / 3.f;
  } else {
    const float p = sq * sr;
    alpha = -4.f * q + (8.f / 3.f) * p - kh2 * (1.f - q / 3.f);
    beta = -4.f + (8.f / 3.f) * q - (4.f / 3.f) * p + kh2 / 3.f;
  }
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
        dmx = fmax_nan(dmx, fabsf((float)v));
        umx = fmax_nan(umx, fabsf((float)nv));
      }
    } else {
      static_cast<float*>(A.dst)[off] = (float)v;
    }
  }
  if (A.corr_max) {
    for (int o = 16; o > 0; o >>= 1) {
      dmx = fmax_nan(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
      umx = fmax_nan(umx, __shfl_xor_sync(0xffffffffu, umx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      // non-negative doubles order like their bit patterns
      if (!(dmx <= 0.f)) atomicMax(A.corr_max, (unsigned long long)__double_as_longlong((double)dmx));
      if (!(umx <= 0.f)) atomicMax(A.corr_max + 1, (unsigned long long)__double_as_longlong((double)umx));
    }
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_dst_pass(PassArgs A) {
  if (A.skip && *A.skip) return;
  extern __shared__ unsigned char smraw[];
  dst_pass_device<T, P>(A, blockIdx.x, blockIdx.y, smraw);
}

// ---------------------------------------------------------------------------
// FP32 passes of the mixed-precision path with register DFTs.
//
// Each CTA transforms P line pairs (sequences of length L = 2^LOGL); a thread
// owns 16 points of one sequence per stage.  Stockham autosort stages of
// radix 16 (and one of radix 2^(LOGL mod 4)): a thread reads its R inputs at
// stride L/R, multiplies by the stage twiddles, runs the R-point DFT in
// registers and writes the R outputs at stride NS (the product of the earlier
// radices), natural order in and out.  The shared buffer is padded by one
// element per 16 so that the stride-R writes of the first stage and the
// stride-L/R reads are free of bank conflicts.  Compared with the radix-4
// shared-memory kernel above this takes 2-3 exchanges instead of 5-6 and all
// index arithmetic is compile-time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// v * exp(-2 pi i j / 16), j known at compile time after unrolling
__device__ __forceinline__ Cx<float> mulw16(Cx<float> v, int j) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  float c, s;   // exp(-2 pi i j/16) = c + i s
  switch (j & 15) {
    case 0: return v;
    case 1: c = c1; s = -s1; break;
    case 2: c = r2; s = -r2; break;
    case 3: c = s1; s = -c1; break;
    case 4: return {v.y, -v.x};
    case 5: c = -s1; s = -c1; break;
    case 6: c = -r2; s = -r2; break;
    case 7: c = -c1; s = -s1; break;
    case 8: return {-v.x, -v.y};
    case 9: c = -c1; s = s1; break;
    case 10: c = -r2; s = r2; break;
    case 11: c = -s1; s = c1; break;
    case 12: return {-v.y, v.x};
    case 13: c = s1; s = c1; break;
    case 14: c = r2; s = r2; break;
    default: c = c1; s = s1; break;
  }
  return {v.x * c - v.y * s, v.x * s + v.y * c};
}

__device__ __forceinline__ void dft4(Cx<float>& a0, Cx<float>& a1, Cx<float>& a2, Cx<float>& a3) {
  const Cx<float> t0 = {a0.x + a2.x, a0.y + a2.y}, t1 = {a0.x - a2.x, a0.y - a2.y};
  const Cx<float> t2 = {a1.x + a3.x, a1.y + a3.y}, t3 = {a1.x - a3.x, a1.y - a3.y};
  a0 = {t0.x + t2.x, t0.y + t2.y};
  a2 = {t0.x - t2.x, t0.y - t2.y};
  a1 = {t1.x + t3.y, t1.y - t3.x};   // t1 - i t3
  a3 = {t1.x - t3.y, t1.y + t3.x};   // t1 + i t3
}

// out = DFT_R(in), R in {2, 4, 8, 16}: four-step splits r = (R/4) a + b.
template <int R>
__device__ __forceinline__ void dftr(Cx<float>* v, Cx<float>* out) {
  if constexpr (R == 2) {
    out[0] = {v[0].x + v[1].x, v[0].y + v[1].y};
    out[1] = {v[0].x - v[1].x, v[0].y - v[1].y};
  } else if constexpr (R == 4) {
    dft4(v[0], v[1], v[2], v[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = v[k];
  } else if constexpr (R == 8) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      dft4(v[b], v[2 + b], v[4 + b], v[6 + b]);   // Y[b][k1] in v[2 k1 + b]
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) v[2 * k1 + b] = mulw16(v[2 * k1 + b], 2 * b * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      const Cx<float> y0 = v[2 * k1], y1 = v[2 * k1 + 1];
      out[k1] = {y0.x + y1.x, y0.y + y1.y};
      out[k1 + 4] = {y0.x - y1.x, y0.y - y1.y};
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      dft4(v[b], v[4 + b], v[8 + b], v[12 + b]);   // Y[b][k1] in v[4 k1 + b]
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) v[4 * k1 + b] = mulw16(v[4 * k1 + b], b * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) out[k1 + 4 * k2] = v[4 * k1 + k2];
    }
  }
}

// One radix-R Stockham stage in place on the padded buffer s (one sequence).
// tw is this stage's twiddle table T[r NS + k] = exp(-2 pi i r k / (NS R)):
// the lanes of a warp have consecutive k, so each load is coalesced.
template <int L, int R, int NS>
__device__ __forceinline__ void reg_stage(Cx<float>* s, int tid, const Cx<float>* __restrict__ tw) {
  constexpr int G = L / R;    // R-point DFTs per stage
  constexpr int T = L / 16;   // threads per sequence
  constexpr int Q = 16 / R;   // DFTs per thread
  Cx<float> v[16];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = tid + q * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = s[padi(j + r * G)];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = tid + q * T;
    const int k = j & (NS - 1);
    Cx<float>* x = v + q * R;
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = __ldg(reinterpret_cast<const float2*>(tw) + r * NS + k);
        x[r] = cmul(x[r], Cx<float>{w.x, w.y});
      }
    }
    Cx<float> y[R];
    dftr<R>(x, y);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[padi(base + r * NS)] = y[r];
  }
  __syncthreads();
}

// Stage plan of length 2^LOGL: radix-16 stages, then one of radix 2^(LOGL mod 4).
// The twiddle tables of the stages after the first lie back to back.
template <int LOGL>
__device__ __forceinline__ void reg_fft(Cx<float>* s, int tid, const Cx<float>* __restrict__ tw) {
  constexpr int L = 1 << LOGL;
  constexpr int N16 = LOGL / 4, REM = LOGL % 4;
  constexpr int NSF = 1 << (4 * N16);
  constexpr int OFF3 = 16 * 16, OFFR = (N16 >= 2 ? 256 : 0) + (N16 >= 3 ? 16 * 256 : 0);
  if constexpr (N16 >= 1) reg_stage<L, 16, 1>(s, tid, tw);
  if constexpr (N16 >= 2) reg_stage<L, 16, 16>(s, tid, tw);
  if constexpr (N16 >= 3) reg_stage<L, 16, 256>(s, tid, tw + OFF3);
  if constexpr (REM == 1) reg_stage<L, 2, NSF>(s, tid, tw + OFFR);
  if constexpr (REM == 2) reg_stage<L, 4, NSF>(s, tid, tw + OFFR);
  if constexpr (REM == 3) reg_stage<L, 8, NSF>(s, tid, tw + OFFR);
}

// Host copy of the same plan: the stage twiddle tables for length 2^logL.
std::vector<float> stage_twiddles(int logL) {
  const int L = 1 << logL;
  std::vector<int> radix;
  for (int k = 0; k < logL / 4; ++k) radix.push_back(16);
  if (logL % 4) radix.push_back(1 << (logL % 4));
  std::vector<float> out;
  int ns = 1;
  for (int R : radix) {
    if (ns > 1)
      for (int r = 0; r < R; ++r)
        for (int k = 0; k < ns; ++k) {
          const double ang = -2.0 * M_PI * (double)(r * k) / (double)(ns * R);
          out.push_back((float)std::cos(ang));
          out.push_back((float)std::sin(ang));
        }
    ns *= R;
  }
  (void)L;
  if (out.empty()) out.assign(2, 0.f);
  return out;
}

// ---- 64-bit fixed-point arithmetic on 32-bit pieces ---------------------------
// On GB300 integer-to-float conversions (and FP64 divides and 64-bit integer
// divides) issue to the FP64 pipe, 2 per clock per SM; these helpers keep the
// fixed-point steps on the 32-bit integer and FP32 pipes: adds with an
// explicit carry, shifts as funnel shifts, conversions through 16- and 32-bit
// pieces.
__device__ __forceinline__ void split64(long long v, unsigned& lo, unsigned& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v));
}
__device__ __forceinline__ long long join64(unsigned lo, unsigned hi) {
  long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}
__device__ __forceinline__ long long add64(long long a, long long b) {
  unsigned al, ah, bl, bh, rl, rh;
  split64(a, al, ah);
  split64(b, bl, bh);
  asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;" : "=r"(rl), "=r"(rh) : "r"(al), "r"(ah), "r"(bl), "r"(bh));
  return join64(rl, rh);
}
__device__ __forceinline__ long long sub64(long long a, long long b) {
  unsigned al, ah, bl, bh, rl, rh;
  split64(a, al, ah);
  split64(b, bl, bh);
  asm("sub.cc.u32 %0, %2, %4;\n\tsubc.u32 %1, %3, %5;" : "=r"(rl), "=r"(rh) : "r"(al), "r"(ah), "r"(bl), "r"(bh));
  return join64(rl, rh);
}
template <int K>
__device__ __forceinline__ long long shl64(long long a) {
  unsigned l, h;
  split64(a, l, h);
  return join64(l << K, __funnelshift_l(l, h, K));
}
__device__ __forceinline__ void neg32pair(unsigned& l, unsigned& h) {
  asm("sub.cc.u32 %0, 0, %2;\n\tsubc.u32 %1, 0, %3;" : "=r"(l), "=r"(h) : "r"(l), "r"(h));
}

// round(x) as int64 for |x| < 2^62
__device__ __forceinline__ long long f2ll(float x) {
  const float ax = fabsf(x);
  const float hi = floorf(ax * 2.3283064365386963e-10f);   // ax / 2^32
  const float lo = fmaf(hi, -4294967296.f, ax);            // ax - hi 2^32, exact, in [0, 2^32)
  unsigned l = __float2uint_rn(lo), h = __float2uint_rz(hi);
  if (x < 0.f) neg32pair(l, h);
  return join64(l, h);
}

// x in [0, 2^16) -> FP32 exactly without a conversion instruction: 2^23 + x
// has x as its low mantissa bits.  The bits go through an inline-asm move so
// that the compiler cannot fold the subtraction back into an integer-to-float
// conversion instruction, which issues to the FP64 pipe on GB300.
__device__ __forceinline__ float u16f(unsigned x) {
  float f;
  asm("mov.b32 %0, %1;" : "=f"(f) : "r"(0x4B000000u | x));
  return f - 8388608.f;
}

// int64 -> FP32 (within 2 ulp) from four 16-bit pieces of |v|
__device__ __forceinline__ float ll2f(long long v) {
  unsigned l, h;
  split64(v, l, h);
  const bool neg = (int)h < 0;
  if (neg) neg32pair(l, h);
  float m = fmaf(u16f(h >> 16), 65536.f, u16f(h & 0xffffu));
  m = fmaf(m, 65536.f, u16f(l >> 16));
  m = fmaf(m, 65536.f, u16f(l & 0xffffu));
  return neg ? -m : m;
}

// int64 -> FP64 (round half up) by assembling the bits
__device__ __forceinline__ double ll2d(long long v) {
  unsigned l, h;
  split64(v, l, h);
  const unsigned sign = h & 0x80000000u;
  if (sign) neg32pair(l, h);
  if ((h | l) == 0u) return 0.0;
  const int lz = h ? __clz(h) : 32 + __clz(l);
  if (lz >= 32) {                      // normalise: bit 63 set
    h = l << (lz - 32);
    l = 0u;
  } else if (lz > 0) {
    h = __funnelshift_l(l, h, lz);
    l <<= lz;
  }
  int E = 1086 - lz;                   // the value is (h:l) 2^-lz, top bit worth 2^(63 - lz)
  unsigned cy;
  asm("add.cc.u32 %0, %0, 1024;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, 0, 0;" : "+r"(l), "+r"(h), "=r"(cy));
  if (cy) {                            // rounded up to 2^64
    h = 0x80000000u;
    l = 0u;
    E += 1;
  }
  const unsigned mh = (h >> 11) & 0xfffffu;
  const unsigned ml = (h << 21) | (l >> 11);
  return __hiloint2double((int)(sign | ((unsigned)E << 20) | mh), (int)ml);
}

// round(x 2^F) as int64 for |x 2^F| < 2^62, from the bits of x (no FP64 arithmetic)
__device__ __forceinline__ long long d2ll_pow2(double x, int F) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0) return 0;                       // zero (subnormals are far below the scale)
  unsigned ml = lo, mh = (hi & 0xfffffu) | 0x100000u;   // 53-bit significand m, x = m 2^(e - 1075)
  const int sft = e - 1075 + F;
  unsigned rl, rh;
  if (sft >= 0) {
    const int k = min(sft, 31);
    rh = __funnelshift_l(ml, mh, k);
    rl = ml << k;
  } else {
    const int k = -sft;
    if (k > 54) return 0;
    // add 2^(k-1), then shift right by k: round half up
    const unsigned al = k - 1 < 32 ? (1u << (k - 1)) : 0u;
    const unsigned ah = k - 1 < 32 ? 0u : (1u << (k - 1 - 32));
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(ml), "+r"(mh) : "r"(al), "r"(ah));
    if (k < 32) {
      rl = __funnelshift_r(ml, mh, k);
      rh = mh >> k;
    } else {
      rl = mh >> (k - 32);
      rh = 0u;
    }
  }
  if (hi >> 31) neg32pair(rl, rh);
  return join64(rl, rh);
}

template <int LOGL, int P>
struct Reg {
  static constexpr int L = 1 << LOGL;
  static constexpr int T = L / 16;          // threads per sequence
  static constexpr int THREADS = P * T;
  static constexpr int LP = L + L / 16;     // padded sequence length
  static constexpr size_t SMEM = sizeof(Cx<float>) * (size_t)P * LP;
};

// Default pairs per CTA: 128 threads per CTA up to L = 2048.
__host__ __device__ constexpr int reg_pairs(int logL) { return logL >= 11 ? 1 : (1 << (11 - logL)); }

// One FP32 pass over the 2P lines b0 = 1 + 2 P bx ... of line family a = by + 1.
// Offsets are 32-bit (grids up to 1025^3 nodes); each load/store item is one
// complex pair (the same element of lines 2q and 2q+1).
template <int LOGL, int P>
__device__ __forceinline__ void dst32_body(const PassArgs& A, int bx, int by, Cx<float>* sm) {
  using F = Reg<LOGL, P>;
  constexpr int L = F::L, LP = F::LP;
  constexpr int n = L / 2, nm1 = n - 1;
  if (A.zero_nrm && bx == 0 && by == 0 && threadIdx.x == 0) {
    for (int k = 0; k < 7; ++k) A.zero_nrm[k] = 0ull;
    *A.zero_conv = 0;
  }
  const Cx<float>* tw = static_cast<const Cx<float>*>(A.twst);
  const int a = by + 1;
  const int b0 = 1 + 2 * P * bx;
  const int sa = (int)A.sa, sb = (int)A.sb, es = (int)A.es;
  const int abase = a * sa;
  const bool contig = es == 1;
  constexpr int nitem = nm1 * P;                      // (element, pair) items
  constexpr int NIT = (nitem + F::THREADS - 1) / F::THREADS;
  // contiguous lines: element fastest (coalesced along each line); strided
  // lines: pair fastest (the 2P adjacent lines of a row together)
  auto coords = [&](int t, int& j, int& q) {
    if (contig) {
      j = 1 + t % nm1;
      q = t / nm1;
    } else {
      q = t % P;
      j = 1 + t / P;
    }
  };
  {
    float2 vals[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int t = threadIdx.x + it * F::THREADS;
      int j, q;
      coords(t < nitem ? t : 0, j, q);
      const int bA = b0 + 2 * q;
      const int off = abase + bA * sb + j * es;
      float2 v = {0.f, 0.f};
      if (t < nitem && bA <= nm1) {
        if (A.src64) {
          const double* src = static_cast<const double*>(A.src);
          v.x = (float)__ldg(src + off);
          if (bA + 1 <= nm1) v.y = (float)__ldg(src + off + sb);
        } else {
          const float* src = static_cast<const float*>(A.src);
          v.x = __ldg(src + off);
          if (bA + 1 <= nm1) v.y = __ldg(src + off + sb);
        }
      }
      vals[it] = v;
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int t = threadIdx.x + it * F::THREADS;
      if (t < nitem) {
        int j, q;
        coords(t, j, q);
        Cx<float>* zz = sm + q * LP;
        zz[padi(j)] = {vals[it].x, vals[it].y};
        zz[padi(L - j)] = {-vals[it].x, -vals[it].y};
      }
    }
  }
  for (int t = threadIdx.x; t < P; t += F::THREADS) {
    sm[t * LP + padi(0)] = {0.f, 0.f};
    sm[t * LP + padi(n)] = {0.f, 0.f};
  }
  __syncthreads();
  const int pr = threadIdx.x / F::T, tid = threadIdx.x % F::T;
  Cx<float>* s = sm + pr * LP;
  reg_fft<LOGL>(s, tid, tw);
  if (A.fused) {
    // spectral division in place, then the same FFT gives the inverse
    // transform.  lambda h^2 is affine in s_k along the line: alpha + beta s_k
    // with alpha, beta fixed by the line's other mode indices.  Only k < n is
    // divided; Z_{L-k} = -Z_k is written from it, so the rescaled sequence is
    // exactly the odd extension of the next input.
    const float kh2 = (float)A.kt, g = (float)A.gscale;
    const int bA = b0 + 2 * pr, bB = min(bA + 1, nm1);
    const float sa3 = A.d == 3 ? A.s32[a] : 0.f;
    float alA, beA, alB, beB;
    lam_affine(A.d, A.order, kh2, sa3, A.s32[min(bA, nm1)], alA, beA);
    lam_affine(A.d, A.order, kh2, sa3, A.s32[bB], alB, beB);
    const float gA = -0.5f * g, gB = 0.5f * g;
#pragma unroll
    for (int i = 0; i < n / F::T; ++i) {
      const int k = tid + i * F::T;
      if (k == 0) {
        s[padi(0)] = {0.f, 0.f};
        s[padi(n)] = {0.f, 0.f};
        continue;
      }
      const float sk = A.s32[k];
      const Cx<float> Z = s[padi(k)];
      const Cx<float> V = {__fdividef(gA, fmaf(beA, sk, alA)) * Z.y, __fdividef(gB, fmaf(beB, sk, alB)) * Z.x};
      s[padi(k)] = V;
      s[padi(L - k)] = {-V.x, -V.y};
    }
    __syncthreads();
    reg_fft<LOGL>(s, tid, tw);
  }
  // S_k = -Im(Z_k)/2 (line 2q), Re(Z_k)/2 (line 2q+1); in the accumulating
  // modes all old values are loaded before the first store
  float dmx = 0.f, umx = 0.f;
  {
    float2 vals[NIT];
    int offs[NIT];
    bool hasB[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int t = threadIdx.x + it * F::THREADS;
      int j, q;
      coords(t < nitem ? t : 0, j, q);
      const int bA = b0 + 2 * q;
      offs[it] = (t < nitem && bA <= nm1) ? abase + bA * sb + j * es : -1;
      hasB[it] = bA + 1 <= nm1;
      const Cx<float> Z = sm[q * LP + padi(j)];
      vals[it] = {-0.5f * Z.y, 0.5f * Z.x};
    }
    if (A.dstfix) {
      long long oldA[NIT], oldB[NIT];
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        oldA[it] = offs[it] >= 0 ? A.dstfix[offs[it]] : 0ll;
        oldB[it] = (offs[it] >= 0 && hasB[it]) ? A.dstfix[offs[it] + sb] : 0ll;
      }
      const float fa = A.fixf[0], fb = A.fixf[1], ia = A.fixf[2], ib = A.fixf[3];
      const double isc = A.uout ? A.fixd[1] : 0.0;
      // max|u| for the convergence check from the high words of u_fix alone
      // (|u_fix| ~ 2^52, so to 2^-20 relative), converted once per thread
      unsigned umi = 0u;
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (offs[it] >= 0) {
          const long long nA = add64(oldA[it], f2ll((vals[it].x * fa) * fb));
          A.dstfix[offs[it]] = nA;
          if (A.uout) A.uout[offs[it]] = ll2d(nA) * isc;
          dmx = fmax_nan(dmx, fabsf(vals[it].x));
          umi = max(umi, (unsigned)abs((int)(nA >> 32)));
          if (hasB[it]) {
            const long long nB = add64(oldB[it], f2ll((vals[it].y * fa) * fb));
            A.dstfix[offs[it] + sb] = nB;
            if (A.uout) A.uout[offs[it] + sb] = ll2d(nB) * isc;
            dmx = fmax_nan(dmx, fabsf(vals[it].y));
            umi = max(umi, (unsigned)abs((int)(nB >> 32)));
          }
        }
      }
      umx = ((fmaf(u16f(umi >> 16), 65536.f, u16f(umi & 0xffffu)) * 4294967296.f) * ia) * ib;
    } else if (A.dst64) {
      double* o = static_cast<double*>(A.dst);
      double oldA[NIT], oldB[NIT];
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        const bool acc = offs[it] >= 0 && A.accumulate;
        oldA[it] = acc ? o[offs[it]] : 0.0;
        oldB[it] = (acc && hasB[it]) ? o[offs[it] + sb] : 0.0;
      }
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (offs[it] >= 0) {
          const double nA = oldA[it] + (double)vals[it].x;
          o[offs[it]] = nA;
          dmx = fmax_nan(dmx, fabsf(vals[it].x));
          umx = fmax_nan(umx, fabsf((float)nA));
          if (hasB[it]) {
            const double nB = oldB[it] + (double)vals[it].y;
            o[offs[it] + sb] = nB;
            dmx = fmax_nan(dmx, fabsf(vals[it].y));
            umx = fmax_nan(umx, fabsf((float)nB));
          }
        }
      }
    } else {
      float* o = static_cast<float*>(A.dst);
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        if (offs[it] >= 0) {
          o[offs[it]] = vals[it].x;
          dmx = fmax_nan(dmx, fabsf(vals[it].x));
          if (hasB[it]) {
            o[offs[it] + sb] = vals[it].y;
            dmx = fmax_nan(dmx, fabsf(vals[it].y));
          }
        }
      }
      umx = dmx;
    }
  }
  if (A.corr_max) {
    for (int o = 16; o > 0; o >>= 1) {
      dmx = fmax_nan(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
      umx = fmax_nan(umx, __shfl_xor_sync(0xffffffffu, umx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (!(dmx <= 0.f)) atomicMax(A.corr_max, (unsigned long long)__double_as_longlong((double)dmx));
      if (!(umx <= 0.f)) atomicMax(A.corr_max + 1, (unsigned long long)__double_as_longlong((double)umx));
    }
  }
}

template <int LOGL, int P>
__global__ void __launch_bounds__(Reg<LOGL, P>::THREADS) k_dst32(PassArgs A) {
  if (A.skip && *A.skip) return;
  extern __shared__ unsigned char smraw[];
  dst32_body<LOGL, P>(A, blockIdx.x, blockIdx.y, reinterpret_cast<Cx<float>*>(smraw));
}

// Each length compiled on its own (not inlined into the dispatching kernel, so
// that the register allocation of one length does not spill another).
template <int LOGL>
__device__ __noinline__ void dst32_item(const PassArgs& A, int bx, int by, Cx<float>* sm) {
  dst32_body<LOGL, reg_pairs(LOGL)>(A, bx, by, sm);
}

// Persistent FP32 pass over many independent grids: every transform length
// up to L = 2048 uses 128 threads and 17.4 KB per work item (P L / 16 = 128
// with P = reg_pairs(LOGL)), so one kernel takes the work items of all
// instances (item -> instance by binary search in `start`) and dispatches on
// the instance's LOGL.
__global__ void __launch_bounds__(128) k_dst32_batched(const PassArgs* __restrict__ args,
                                                       const int* __restrict__ start, int ninst) {
  extern __shared__ unsigned char smraw[];
  Cx<float>* sm = reinterpret_cast<Cx<float>*>(smraw);
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
    const int p = reg_pairs(A.logL);
    const int nbx = (A.n / 2 + p - 1) / p;
    const int bx = local % nbx, by = local / nbx;
    switch (A.logL) {
      case 4: dst32_item<4>(A, bx, by, sm); break;
      case 5: dst32_item<5>(A, bx, by, sm); break;
      case 6: dst32_item<6>(A, bx, by, sm); break;
      case 7: dst32_item<7>(A, bx, by, sm); break;
      case 8: dst32_item<8>(A, bx, by, sm); break;
      case 9: dst32_item<9>(A, bx, by, sm); break;
      case 10: dst32_item<10>(A, bx, by, sm); break;
      default: dst32_item<11>(A, bx, by, sm); break;
    }
    __syncthreads();
  }
}

// The check after refinement step `step` (0: the first FP32 solve): stop when
// the last correction max|delta| <= tol max|u|.  After the first solve there
// is no correction yet; it stops there only when ten times the relative size
// of the first correction observed in an earlier solve on this grid (nrm[8],
// an estimate of the FP32 solve's error, 1 until one is observed) is within
// tol, which a relaxed GMRES tolerance can reach.  The first correction of
// every solve updates that estimate.
__device__ __forceinline__ void check_body(unsigned long long* nrm, const double* tolp, int* conv, int step) {
  const double tol = tolp[0];
  if (*conv) return;
  double dm = __longlong_as_double((long long)nrm[3]);
  double um = __longlong_as_double((long long)nrm[4]);
  nrm[2] = nrm[3];
  nrm[5] = nrm[4];
  bool stop = dm <= tol * um;
  if (step == 0 && 10.0 * __longlong_as_double((long long)nrm[8]) <= tol) stop = true;
  if (step == 1 && um > 0.0) nrm[8] = (unsigned long long)__double_as_longlong(dm / um);
  if (stop) {
    *conv = 1;
  } else {
    nrm[6] += 1ull;   // one more refinement step will run
    nrm[7] += 1ull;
  }
  nrm[3] = 0ull;
  nrm[4] = 0ull;
}

__global__ void k_check(unsigned long long* nrm, const double* tol, int* conv, int step) {
  check_body(nrm, tol, conv, step);
}


// ---- exact residual of the mixed path (fixed point) -------------------------
// After the first FP32 solve u0, F is chosen so that max|u0| 2^F ~ 2^52; then
// u_fix = round(u 2^F) and R_fix = round(mult h^2 R 2^F) are int64, the
// integer part S of mult h^2 A_h is applied exactly in int64 (|S u_fix| <
// 2^61), and only the kappa part (relative size kappa h^2) goes through one
// FP64 product.  The residual is then exact for the stored u_fix, with no
// FP64 stencil arithmetic, and is handed to the next FP32 solve as FP32.
// Scales beyond the FP32 exponent range are applied as two factors
// 2^Fa 2^Fb (Fa + Fb = F).
__device__ __forceinline__ void fix_scale_body(const unsigned long long* __restrict__ umax, double multh2,
                                               double kc, double* __restrict__ fixd, float* __restrict__ fixf) {
  // U = u 2^F / (mult h^2) with max|U| ~ 2^52; R_fix = R 2^F (an exact power of two)
  const double um = __longlong_as_double((long long)umax[0]) / multh2;
  int F = 0;
  if (um > 0.0) F = 52 - (int)ceil(log2(um));
  F = max(-120, min(F, 240));
  const int Fa = F / 2, Fb = F - Fa;
  fixd[1] = ldexp(multh2, -F);                  // u = U mult h^2 2^-F
  fixd[2] = kc;
  fixd[3] = (double)F;
  fixf[0] = ldexpf(1.f, Fa);                    // U = (u 2^Fa) (2^Fb / mult h^2)
  fixf[1] = (float)(ldexp(1.0, Fb) / multh2);
  fixf[2] = ldexpf(1.f, -Fa);                   // u = (U 2^-Fa) (mult h^2 2^-Fb); r = (r_fix 2^-Fa) 2^-Fb
  fixf[3] = (float)ldexp(multh2, -Fb);
  fixf[4] = ldexpf(1.f, -Fb);
  if (!(um <= 1.7976931348623157e308)) {
    // a NaN or infinite first solve (non-finite data): the integer
    // conversions would turn it into finite values, so every conversion back
    // to floating point yields NaN instead and the caller sees a non-finite
    // result
    const double qn = __longlong_as_double(0x7ff8000000000000LL);
    fixd[1] = qn;
    fixf[2] = __int_as_float(0x7fc00000);
    fixf[3] = __int_as_float(0x7fc00000);
    fixf[4] = __int_as_float(0x7fc00000);
  }
}

__global__ void k_fix_scale(const unsigned long long* __restrict__ umax, double multh2, double kc,
                            double* __restrict__ fixd, float* __restrict__ fixf) {
  fix_scale_body(umax, multh2, kc, fixd, fixf);
}

// the check after the first FP32 solve and the fixed-point scale from its max|u|
__global__ void k_check_scale(unsigned long long* nrm, const double* tol, int* conv, double multh2, double kc,
                              double* __restrict__ fixd, float* __restrict__ fixf) {
  check_body(nrm, tol, conv, 0);
  fix_scale_body(nrm + 5, multh2, kc, fixd, fixf);
}

// u_fix = round(u0 2^F / (mult h^2)), R_fix = round(R 2^F); with u, also the
// FP64 solution of the fixed-point u_fix (u0 is 0 on the boundary layer)
__global__ void k_fix0(long long tot, const float* __restrict__ u0, const double* __restrict__ R, Grid g,
                       const double* __restrict__ fixd, const float* __restrict__ fixf,
                       long long* __restrict__ ufix, long long* __restrict__ rfix, double* __restrict__ u) {
  const int F = (int)fixd[3];
  const double isc = fixd[1];
  const float fa = fixf[0], fb = fixf[1];
  const int n1 = g.n + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (int)tot;
       t += gridDim.x * blockDim.x) {
    const long long uf = f2ll((u0[t] * fa) * fb);
    ufix[t] = uf;
    if (u) u[t] = ll2d(uf) * isc;
    int r = t;
    bool interior = true;
    for (int k = 0; k < g.d; ++k) {
      const int q = r / n1;
      const int i = r - q * n1;
      r = q;
      interior = interior && i >= 1 && i < g.n;
    }
    rfix[t] = interior ? d2ll_pow2(R[t], F) : 0ll;
  }
}

struct FixStencil {
  int w0, w1, w2, w3, kA, kB;
};

// S U of the integer stencil and the kappa combination kA U_P + kB e, with
// the weights of the three operators as shifts and adds on 32-bit pieces
__device__ __forceinline__ long long fix_apply(const FixStencil& W, long long c, long long e, long long k2,
                                               long long k3, long long& m) {
  if (W.w0 == -20) {          // 2D 4th order: -20 c + 4 e + k2; kappa: 8 c + e
    m = add64(shl64<3>(c), e);
    return add64(shl64<2>(sub64(e, add64(shl64<2>(c), c))), k2);
  }
  if (W.w0 == -200) {         // 3D 4th order: -200 c + 20 e + 6 k2 + k3; kappa: 6 c + e
    m = add64(add64(shl64<2>(c), shl64<1>(c)), e);
    const long long fifty_c = add64(add64(shl64<5>(c), shl64<4>(c)), shl64<1>(c));
    const long long t = sub64(add64(shl64<2>(e), e), fifty_c);           // 5 e - 50 c
    return add64(add64(shl64<2>(t), add64(shl64<2>(k2), shl64<1>(k2))), k3);
  }
  m = c;                      // 2nd order: -2 d c + e; kappa: c
  return W.w0 == -4 ? sub64(e, shl64<2>(c)) : sub64(e, add64(shl64<2>(c), shl64<1>(c)));
}

// the 9/27 neighbour sums of a fixed-point grid at index t (32-bit indices)
#define FIX_NEIGHBOURS(U)                                                                                       \
  const long long c = U(0);                                                                                     \
  long long e, k2 = 0, k3 = 0;                                                                                  \
  if (g.d == 2) {                                                                                               \
    e = add64(add64(U(-1), U(1)), add64(U(-n1), U(n1)));                                                        \
    if (W.w2) k2 = add64(add64(U(-n1 - 1), U(-n1 + 1)), add64(U(n1 - 1), U(n1 + 1)));                           \
  } else {                                                                                                      \
    const int s3 = n1 * n1;                                                                                     \
    e = add64(add64(add64(U(-1), U(1)), add64(U(-n1), U(n1))), add64(U(-s3), U(s3)));                           \
    if (W.w2)                                                                                                   \
      k2 = add64(add64(add64(add64(U(-n1 - 1), U(-n1 + 1)), add64(U(n1 - 1), U(n1 + 1))),                       \
                       add64(add64(U(-s3 - 1), U(-s3 + 1)), add64(U(s3 - 1), U(s3 + 1)))),                      \
                 add64(add64(U(-s3 - n1), U(-s3 + n1)), add64(U(s3 - n1), U(s3 + n1))));                        \
    if (W.w3)                                                                                                   \
      k3 = add64(add64(add64(U(-s3 - n1 - 1), U(-s3 - n1 + 1)), add64(U(-s3 + n1 - 1), U(-s3 + n1 + 1))),       \
                 add64(add64(U(s3 - n1 - 1), U(s3 - n1 + 1)), add64(U(s3 + n1 - 1), U(s3 + n1 + 1))));          \
  }


// round(kc m), the kappa part of the fixed-point residual, in integers:
// kc = K 2^-S with K the 64-bit left-aligned significand of kc (exact), so
// kc m is the 128-bit product K |m| scaled by 2^-S and rounded at bit S (round
// half away from zero).  No FP64 arithmetic: as an int64 -> FP64 conversion,
// product and conversion back it cost three FP64-pipe instructions per node
// (~80 us of FP64 pipe per 256^3 sweep), and as an inline FP64 branch the
// compiler evaluated it even when kc = 0.
struct KappaFix {
  unsigned long long K;
  int S, neg, zero;
};
__device__ __forceinline__ KappaFix kappa_fix(double kc) {
  KappaFix f;
  const unsigned long long b = (unsigned long long)__double_as_longlong(kc);
  const int E = (int)((b >> 52) & 0x7ff);
  f.zero = (b & 0x7fffffffffffffffull) == 0ull || E == 0;
  f.neg = (int)(b >> 63);
  f.K = ((b & 0xfffffffffffffull) | 0x10000000000000ull) << 11;
  f.S = 1086 - E;   // |kc| = K 2^(E - 1086)
  return f;
}
// |kc| < 1 (kappa h^2 scaled by at most 4), so S > 64 and the quotient fits
__device__ __forceinline__ long long kappa_int(const KappaFix& f, long long m) {
  if (f.zero || m == 0) return 0ll;
  const bool mneg = m < 0;
  const unsigned long long a = mneg ? (unsigned long long)(-m) : (unsigned long long)m;
  const unsigned long long hi = __umul64hi(a, f.K), lo = a * f.K;
  const int S = f.S;
  unsigned long long q;
  if (S >= 128) {
    q = 0ull;
  } else if (S >= 64) {
    const unsigned long long rb = S - 1 >= 64 ? (hi >> (S - 65)) & 1ull : (lo >> 63) & 1ull;
    q = (S - 64 >= 64 ? 0ull : hi >> (S - 64)) + rb;
  } else {
    const unsigned long long rb = (lo >> (S - 1)) & 1ull;
    q = ((hi << (64 - S)) | (lo >> S)) + rb;
  }
  const long long v = (long long)q;
  return mneg != (bool)f.neg ? -v : v;
}


// The exact residual of the mixed box solve,
//   r32 = (R_fix - S u_fix + round(kc (kA u + kB sum_edges))) 2^-F / (mult h^2),
// in 2D: a thread per column marching over kResRows rows with a three-row
// window of centre values and horizontal pair sums (three int64 loads per
// node instead of nine; integer sums are exact, so the grouping of the
// stencil sums does not change the result).  Grid: x over the columns 0..N, y over
// row chunks of 0..N; with uout and the convergence flag set, it writes the
// FP64 solution at every node instead.
constexpr int kResRows = 4;
__global__ void k_res_fix2(Grid g, FixStencil W, const long long* __restrict__ R, const long long* __restrict__ u,
                           const double* __restrict__ fixd, const float* __restrict__ fixf,
                           float* __restrict__ r32, const int* skip, double* __restrict__ uout) {
  const int n = g.n, n1 = n + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n) return;
  const int i0 = blockIdx.y * kResRows, i1 = min(n1, i0 + kResRows);
  if (skip && *skip) {
    if (uout)
      for (int i = i0; i < i1; ++i) uout[i * n1 + j] = ll2d(u[i * n1 + j]) * fixd[1];
    return;
  }
  if (j < 1 || j >= n) return;   // boundary columns of r are never read
  const int a = max(i0, 1), b = min(i1, n);
  if (a >= b) return;
  const KappaFix kf = kappa_fix(fixd[2]);
  const float f2 = fixf[2], f4 = fixf[4];
  const long long* p = u + (a - 1) * n1 + j;
  long long mC = p[0], mH = add64(p[-1], p[1]);
  p += n1;
  long long cC = p[0], cH = add64(p[-1], p[1]);
#pragma unroll
  for (int k = 0; k < kResRows; ++k) {
    const int i = a + k;
    if (i >= b) break;
    p += n1;
    const long long qC = p[0], qH = add64(p[-1], p[1]);
    const long long Ri = R[i * n1 + j];
    const long long e = add64(cH, add64(mC, qC));   // edge neighbours
    const long long k2 = add64(mH, qH);             // corners
    long long m;
    long long r = sub64(Ri, fix_apply(W, cC, e, k2, 0, m));
    if (!kf.zero) r = add64(r, kappa_int(kf, m));
    r32[i * n1 + j] = (ll2f(r) * f2) * f4;
    mC = cC;
    mH = cH;
    cC = qC;
    cH = qH;
  }
}

// The same residual in 3D, a thread per x-column and kR3 y-rows marching
// along z over kz slices, with a three-slice window of int64 slice sums per
// row (centre C, in-plane edge sum S1, in-plane corner sum S2): the 27-point
// sums are e = S1 + C(z-1) + C(z+1), k2 = S2 + S1(z-1) + S1(z+1),
// k3 = S2(z-1) + S2(z+1).  The next slice of u and R is loaded before the
// current one is computed.  Integer sums are exact, so the grouping does not
// change the result (checked bit for bit against the one-node 27-point form).  The grid covers every node 0..N per axis: interior nodes get
// the residual; with uout and the convergence flag set, every node gets u.
constexpr int kR3 = 2, kR3X = 32, kR3Y = 4, kR3Threads = kR3X * kR3Y;
__global__ void __launch_bounds__(kR3Threads, 5) k_res_fix3(Grid g, FixStencil W, const long long* __restrict__ R,
                                                            const long long* __restrict__ u,
                                                            const double* __restrict__ fixd,
                                                            const float* __restrict__ fixf, float* __restrict__ r32,
                                                            const int* skip, double* __restrict__ uout, int kz) {
  const int n = g.n, n1 = n + 1, plane = n1 * n1;
  const int x = blockIdx.x * kR3X + (threadIdx.x % kR3X);
  const int yb = blockIdx.y * (kR3Y * kR3) + (threadIdx.x / kR3X) * kR3;
  if (x > n || yb > n) return;
  const int z0 = blockIdx.z * kz, z1 = min(n1, z0 + kz);
  if (skip && *skip) {
    if (uout) {
      const double isc = fixd[1];
      for (int z = z0; z < z1; ++z)
#pragma unroll
        for (int r = 0; r < kR3; ++r)
          if (yb + r <= n) {
            const int t = z * plane + (yb + r) * n1 + x;
            uout[t] = ll2d(u[t]) * isc;
          }
    }
    return;
  }
  if (x < 1 || x >= n) return;   // boundary nodes of r are never read
  const int za = max(z0, 1), zb = min(z1, n);
  if (za >= zb) return;
  const KappaFix kf = kappa_fix(fixd[2]);
  const float f2 = fixf[2], f4 = fixf[4];
  // rows yb - 1 .. yb + kR3 (outside 0..N read as 0 and feed no output)
  int roff[kR3 + 2];
  bool rok[kR3 + 2];
#pragma unroll
  for (int r = 0; r < kR3 + 2; ++r) {
    const int y = yb - 1 + r;
    rok[r] = y >= 0 && y <= n;
    roff[r] = y * n1 + x;
  }
  bool out_ok[kR3];
#pragma unroll
  for (int r = 0; r < kR3; ++r) out_ok[r] = yb + r >= 1 && yb + r < n;
  long long raw[kR3 + 2][3];
  auto load = [&](int z) {
    const long long* s = u + z * plane;
#pragma unroll
    for (int r = 0; r < kR3 + 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) raw[r][c] = rok[r] ? __ldg(s + roff[r] + c - 1) : 0ll;
  };
  long long Rcur[kR3], Rnext[kR3];
  auto loadR = [&](int z, long long* dst) {
#pragma unroll
    for (int r = 0; r < kR3; ++r) dst[r] = out_ok[r] ? __ldg(R + z * plane + roff[r + 1]) : 0ll;
  };
  long long mC[kR3], mS1[kR3], mS2[kR3], cC[kR3], cS1[kR3], cS2[kR3];
  auto sums = [&](long long* C, long long* S1, long long* S2) {
    long long H[kR3 + 2];
#pragma unroll
    for (int r = 0; r < kR3 + 2; ++r) H[r] = add64(raw[r][0], raw[r][2]);
#pragma unroll
    for (int r = 0; r < kR3; ++r) {
      C[r] = raw[r + 1][1];
      S1[r] = add64(H[r + 1], add64(raw[r][1], raw[r + 2][1]));
      S2[r] = add64(H[r], H[r + 2]);
    }
  };
  loadR(za, Rcur);
  load(za - 1);
  sums(mC, mS1, mS2);
  load(za);
  sums(cC, cS1, cS2);
  load(za + 1);
  for (int z = za; z < zb; ++z) {
    long long qC[kR3], qS1[kR3], qS2[kR3];
    sums(qC, qS1, qS2);
    if (z + 1 < zb) {
      load(z + 2);
      loadR(z + 1, Rnext);
    }
    const int tb = z * plane + yb * n1 + x;
#pragma unroll
    for (int r = 0; r < kR3; ++r) {
      if (out_ok[r]) {
        const long long e = add64(cS1[r], add64(mC[r], qC[r]));
        const long long k2 = add64(cS2[r], add64(mS1[r], qS1[r]));
        const long long k3 = add64(mS2[r], qS2[r]);
        long long m;
        long long res = sub64(Rcur[r], fix_apply(W, cC[r], e, k2, k3, m));
        if (!kf.zero) res = add64(res, kappa_int(kf, m));
        r32[tb + r * n1] = (ll2f(res) * f2) * f4;
      }
      mC[r] = cC[r];
      mS1[r] = cS1[r];
      mS2[r] = cS2[r];
      cC[r] = qC[r];
      cS1[r] = qS1[r];
      cS2[r] = qS2[r];
      Rcur[r] = Rnext[r];
    }
  }
}

// launch of the fixed-point residual for the grid's dimension
void launch_res_fix(kfbi_problem* p, const Grid& g, const FixStencil& W, const long long* R, const long long* u,
                    const double* fixd, const float* fixf, float* r32, const int* skip, double* uout,
                    cudaStream_t st) {
  if (g.d == 2) {
    const dim3 grid((unsigned)div_up(g.n + 1, 128), (unsigned)div_up(g.n + 1, kResRows), 1u);
    KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_res_fix2<<<grid, 128, 0, st>>>(g, W, R, u, fixd, fixf, r32, skip, uout));
  } else {
    const int kz = 16;
    const dim3 grid((unsigned)div_up(g.n + 1, kR3X), (unsigned)div_up(g.n + 1, kR3Y * kR3),
                    (unsigned)div_up(g.n + 1, kz));
    KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_res_fix3<<<grid, kR3Threads, 0, st>>>(g, W, R, u, fixd, fixf, r32, skip,
                                                                               uout, kz));
  }
}

// u = U mult h^2 2^-F
__global__ void k_unfix(long long tot, const long long* __restrict__ ufix, const double* __restrict__ fixd,
                        double* __restrict__ u) {
  const double isc = fixd[1];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (int)tot;
       t += gridDim.x * blockDim.x)
    u[t] = ll2d(ufix[t]) * isc;
}

// u_fix += round(e 2^F) over a grid; max|e| -> corr[0], max|u| -> corr[1]
__global__ void k_fix_add(long long tot, const float* __restrict__ e, long long* __restrict__ ufix,
                          const float* __restrict__ fixf, unsigned long long* __restrict__ corr, const int* skip) {
  if (skip && *skip) return;
  const float fa = fixf[0], fb = fixf[1], ia = fixf[2], ib = fixf[3];
  float em = 0.f;
  unsigned umi = 0u;   // max|u| from the high words of u_fix, as in the DST passes
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (int)tot;
       t += gridDim.x * blockDim.x) {
    const float ev = e[t];
    const long long nv = add64(ufix[t], f2ll((ev * fa) * fb));
    ufix[t] = nv;
    em = fmax_nan(em, fabsf(ev));
    umi = max(umi, (unsigned)abs((int)(nv >> 32)));
  }
  float um = ((fmaf(u16f(umi >> 16), 65536.f, u16f(umi & 0xffffu)) * 4294967296.f) * ia) * ib;
  for (int o = 16; o > 0; o >>= 1) {
    em = fmax_nan(em, __shfl_xor_sync(0xffffffffu, em, o));
    um = fmax_nan(um, __shfl_xor_sync(0xffffffffu, um, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (!(em <= 0.f)) atomicMax(corr, (unsigned long long)__double_as_longlong((double)em));
    if (!(um <= 0.f)) atomicMax(corr + 1, (unsigned long long)__double_as_longlong((double)um));
  }
}

// max|x| of an FP32 grid as FP64 bits -> out[0]
__global__ void k_absmax32(long long tot, const float* __restrict__ x, unsigned long long* __restrict__ out,
                           const int* skip) {
  if (skip && *skip) return;
  float m = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (int)tot;
       t += gridDim.x * blockDim.x)
    m = fmax_nan(m, fabsf(x[t]));
  for (int o = 16; o > 0; o >>= 1) m = fmax_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && !(m <= 0.f)) atomicMax(out, (unsigned long long)__double_as_longlong((double)m));
}

template <typename T, int P>
void launch_pass_p(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st) {
  dim3 grid((unsigned)((npairs_b + P - 1) / P), (unsigned)na);
  size_t smem = sizeof(Cx<T>) * (size_t)(2 * A.n) * P * 2;
  KFBI_LAUNCH(p, KFBI_KC_DST, k_dst_pass<T, P><<<grid, 256, smem, st>>>(A));
}

template <int LOGL, int P>
void launch_reg(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st) {
  using F = Reg<LOGL, P>;
  dim3 grid((unsigned)((npairs_b + P - 1) / P), (unsigned)na);
  KFBI_LAUNCH(p, KFBI_KC_DST, k_dst32<LOGL, P><<<grid, F::THREADS, F::SMEM, st>>>(A));
}

// FP32 pass: P = reg_pairs(LOGL) line pairs per CTA (128-thread CTAs)
void launch_pass32(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st) {
  switch (A.logL) {
    case 4: launch_reg<4, reg_pairs(4)>(p, A, npairs_b, na, st); break;
    case 5: launch_reg<5, reg_pairs(5)>(p, A, npairs_b, na, st); break;
    case 6: launch_reg<6, reg_pairs(6)>(p, A, npairs_b, na, st); break;
    case 7: launch_reg<7, reg_pairs(7)>(p, A, npairs_b, na, st); break;
    case 8: launch_reg<8, reg_pairs(8)>(p, A, npairs_b, na, st); break;
    case 9: launch_reg<9, reg_pairs(9)>(p, A, npairs_b, na, st); break;
    case 10: launch_reg<10, reg_pairs(10)>(p, A, npairs_b, na, st); break;
    case 11: launch_reg<11, reg_pairs(11)>(p, A, npairs_b, na, st); break;
    case 12: launch_reg<12, reg_pairs(12)>(p, A, npairs_b, na, st); break;
    default: launch_reg<13, reg_pairs(13)>(p, A, npairs_b, na, st); break;
  }
}

template <int LOGL>
cudaError_t set_smem_reg(int max_optin) {
  return cudaFuncSetAttribute(k_dst32<LOGL, reg_pairs(LOGL)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_optin);
}

// pairs per CTA: enough butterflies for 256 threads (P L / 4 >= 256), at least
// `pmin` (strided passes read 2 P adjacent lines per row)
template <typename T>
void launch_pass(kfbi_problem* p, const PassArgs& A, int npairs_b, int na, cudaStream_t st, int pmin) {
  if (sizeof(T) == 4) {
    launch_pass32(p, A, npairs_b, na, st);
    return;
  }
  const int L = 2 * A.n;
  int P = std::max(pmin, 1024 / L);
  if (sizeof(T) == 8 && L >= 2048) P = std::min(P, 1);
  // small grids: fewer pairs per CTA until the pass has two CTAs per SM (a
  // 64^2 grid otherwise runs on 4 CTAs, each bound by one SM's FP64 rate)
  while (P > pmin && (long long)((npairs_b + P - 1) / P) * na < 2 * 152) P /= 2;
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
  A.twst = B->twst;
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
  {
    const std::vector<float> ts = stage_twiddles(B->logL);
    KFBI_CUDA(p, dalloc(&B->twst, ts.size()));
    KFBI_CUDA(p, cudaMemcpy(B->twst, ts.data(), sizeof(float) * ts.size(), cudaMemcpyHostToDevice));
  }
  KFBI_CUDA(p, cudaMemcpy(B->cosv, cs.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice));
  const long long nodes = g.nodes();
  if (p->cfg.precision == KFBI_MIXED) {
    KFBI_CUDA(p, dalloc(&B->work32, nodes));
    KFBI_CUDA(p, cudaMemset(B->work32, 0, sizeof(float) * nodes));
    KFBI_CUDA(p, dalloc(&B->res, nodes));
    KFBI_CUDA(p, cudaMemset(B->res, 0, sizeof(double) * nodes));
    KFBI_CUDA(p, dalloc(&B->ufix, nodes));
    KFBI_CUDA(p, dalloc(&B->rfix, nodes));
    KFBI_CUDA(p, dalloc(&B->fixd, 4));
    KFBI_CUDA(p, dalloc(&B->fixf, 8));
    // mult h^2 A_h = S - kappa h^2 kscale (kA u_P + kB sum of edge neighbours)
    const int order = p->cfg.order;
    double mult, kscale;
    if (order == 2) {
      mult = 1.0;
      B->w[0] = -2 * g.d; B->w[1] = 1; B->w[2] = 0; B->w[3] = 0;
      B->kA = 1; B->kB = 0; kscale = 1.0;
    } else if (g.d == 2) {   // 6 h^2 x eq. (9p-cds)
      mult = 6.0;
      B->w[0] = -20; B->w[1] = 4; B->w[2] = 1; B->w[3] = 0;
      B->kA = 8; B->kB = 1; kscale = 0.5;
    } else {                 // 48 h^2 x eq. (27p-cds)
      mult = 48.0;
      B->w[0] = -200; B->w[1] = 20; B->w[2] = 6; B->w[3] = 1;
      B->kA = 6; B->kB = 1; kscale = 4.0;
    }
    B->multh2 = mult * g.h * g.h;
    B->kc = kscale * p->kt * g.h * g.h;

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
  KFBI_CUDA(p, dalloc(&B->nrm, 9));
  {
    unsigned long long init[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double one = 1.0;   // no FP32 error estimate yet
    memcpy(&init[8], &one, sizeof(one));
    KFBI_CUDA(p, cudaMemcpy(B->nrm, init, sizeof(init), cudaMemcpyHostToDevice));
  }
  KFBI_CUDA(p, dalloc(&B->conv, 1));
  KFBI_CUDA(p, dalloc(&B->tol_dev, 1));
  B->tol = p->cfg.box_rtol > 0 ? p->cfg.box_rtol : 1e-13;
  KFBI_CUDA(p, cudaMemcpy(B->tol_dev, &B->tol, sizeof(double), cudaMemcpyHostToDevice));
  B->refine_steps = p->cfg.box_max_iters > 0 ? std::min(p->cfg.box_max_iters, 8) : 5;
  int dev = 0, optin = 0;
  KFBI_CUDA(p, cudaGetDevice(&dev));
  KFBI_CUDA(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // shared memory per CTA: the FP64 passes hold two length-2N buffers per
  // line pair; the FP32 register passes one padded buffer per pair
  const size_t need = p->cfg.precision == KFBI_MIXED
                          ? sizeof(Cx<float>) * (size_t)reg_pairs(B->logL) * (size_t)(2 * n + (2 * n) / 16)
                          : sizeof(Cx<double>) * (size_t)(2 * n) * 2 * std::max(1, 1024 / (2 * n));
  if ((size_t)optin < need)
    return fail(p, KFBI_ERR_UNSUPPORTED,
                p->cfg.precision == KFBI_MIXED ? "N too large for the shared-memory DST on this device"
                                               : "N too large for the FP64 shared-memory DST on this device "
                                                 "(2D: N <= 2048; the mixed path goes to 4096)");
  KFBI_CUDA(p, (set_smem<double, 1>(optin)));
  KFBI_CUDA(p, (set_smem<double, 2>(optin)));
  KFBI_CUDA(p, (set_smem<double, 4>(optin)));
  KFBI_CUDA(p, (set_smem<double, 8>(optin)));
  KFBI_CUDA(p, (set_smem<float, 1>(optin)));
  KFBI_CUDA(p, (set_smem<float, 2>(optin)));
  KFBI_CUDA(p, (set_smem<float, 4>(optin)));
  KFBI_CUDA(p, (set_smem<float, 8>(optin)));
  KFBI_CUDA(p, set_smem_reg<4>(optin));
  KFBI_CUDA(p, set_smem_reg<5>(optin));
  KFBI_CUDA(p, set_smem_reg<6>(optin));
  KFBI_CUDA(p, set_smem_reg<7>(optin));
  KFBI_CUDA(p, set_smem_reg<8>(optin));
  KFBI_CUDA(p, set_smem_reg<9>(optin));
  KFBI_CUDA(p, set_smem_reg<10>(optin));
  KFBI_CUDA(p, set_smem_reg<11>(optin));
  KFBI_CUDA(p, set_smem_reg<12>(optin));
  KFBI_CUDA(p, set_smem_reg<13>(optin));
  return KFBI_OK;
}

void box_destroy(kfbi_problem* p) {
  mg_destroy(p);
  BoxSolver* B = p->box;
  if (!B) return;
  cudaFree(B->tw64);
  cudaFree(B->tw32);
  cudaFree(B->twst);
  cudaFree(B->cosv);
  cudaFree(B->s64);
  cudaFree(B->s32);
  cudaFree(B->scale64);
  cudaFree(B->work64);
  cudaFree(B->work32);
  cudaFree(B->res);
  cudaFree(B->ufix);
  cudaFree(B->rfix);
  cudaFree(B->fixd);
  cudaFree(B->fixf);
  cudaFree(B->nrm);
  cudaFree(B->conv);
  cudaFree(B->tol_dev);
  delete B;
  p->box = nullptr;
}

namespace {
__global__ void k_set_double(double* __restrict__ p, double v) { *p = v; }
}  // namespace

// The refinement tolerance of the mixed sine-transform solve as the checks
// read it (device); null for the FP64 transform and the multigrid.
double* mg_tol_dev(kfbi_problem* p);
double mg_tol(const kfbi_problem* p);

double* box_tol_dev(kfbi_problem* p) {
  if (p->mg) return mg_tol_dev(p);
  return (p->box && p->cfg.precision == KFBI_MIXED) ? p->box->tol_dev : nullptr;
}
double box_tol(const kfbi_problem* p) {
  if (p->mg) return mg_tol(p);
  return p->box ? p->box->tol : 0.0;
}
kfbi_status box_tol_reset(kfbi_problem* p) {
  double* t = box_tol_dev(p);
  if (t) KFBI_LAUNCH(p, KFBI_KC_OTHER, k_set_double<<<1, 1, 0, p->stream>>>(t, box_tol(p)));
  return KFBI_OK;
}
// correction steps run by the mixed sine-transform solves since the reset
kfbi_status box_steps_reset(kfbi_problem* p) {
  if (box_tol_dev(p) && !p->mg)
    KFBI_CUDA(p, cudaMemsetAsync(p->box->nrm + 7, 0, sizeof(unsigned long long), p->stream));
  return KFBI_OK;
}
kfbi_status box_steps_total(kfbi_problem* p, long long* out) {
  *out = 0;
  if (!box_tol_dev(p) || p->mg) return KFBI_OK;
  unsigned long long c = 0;
  KFBI_CUDA(p, cudaMemcpyAsync(&c, p->box->nrm + 7, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  *out = (long long)c;
  return KFBI_OK;
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
  // mixed: u0 = DST32^{-1}(R) (FP32, in place in the work grid); fixed-point
  // scale from max|u0|; then repeat { r = R - A_h u exactly (int64 -> FP32);
  // u += DST32^{-1}(r) } until the correction is below tol max|u|.  The FP64
  // output u is written once: by the last step's final pass, or, when the
  // convergence flag stops the refinement earlier, by the next residual
  // kernel in place of its skipped step (by the conversion kernel when there
  // is no refinement step).  The check of the last step is left to the
  // host-side diagnostics (box_last_residual), which read its maxima.
  cudaStream_t st = p->stream;
  const long long nodes = g.nodes();
  const int eb = (int)std::min<long long>(div_up(nodes, 256), 152 * 8);
  {
    PassPlan P0 = plan_passes<float>(p, rhs, 1, u, 0, nullptr, B->nrm + 3);
    P0.args[0].zero_nrm = B->nrm;
    P0.args[0].zero_conv = B->conv;
    PassArgs& last = P0.args[P0.npass - 1];
    last.dst = B->work32;
    last.dst64 = 0;
    last.accumulate = 0;
    last.corr_max = B->nrm + 3;
    for (int k = 0; k < P0.npass; ++k) launch_pass<float>(p, P0.args[k], P0.npairs, P0.na, st, P0.pmin[k]);
  }
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_check_scale<<<1, 1, 0, st>>>(B->nrm, B->tol_dev, B->conv, B->multh2, B->kc,
                                                                      B->fixd, B->fixf));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_fix0<<<eb, 256, 0, st>>>(nodes, B->work32, rhs, g, B->fixd, B->fixf,
                                                                 B->ufix, B->rfix,
                                                                 B->refine_steps > 1 ? nullptr : u));
  float* r32 = reinterpret_cast<float*>(B->res);
  PassPlan PK = plan_passes<float>(p, r32, 0, u, 0, B->conv, B->nrm + 3);
  {
    PassArgs& last = PK.args[PK.npass - 1];
    last.dst = nullptr;
    last.dst64 = 0;
    last.accumulate = 1;
    last.dstfix = B->ufix;
    last.fixf = B->fixf;
    last.fixd = B->fixd;
    last.corr_max = B->nrm + 3;
  }
  PassPlan PL = PK;   // the last step's final pass also writes the FP64 solution
  PL.args[PL.npass - 1].uout = u;
  const FixStencil W{B->w[0], B->w[1], B->w[2], B->w[3], B->kA, B->kB};
  for (int it = 1; it < B->refine_steps; ++it) {
    launch_res_fix(p, g, W, B->rfix, B->ufix, B->fixd, B->fixf, r32, B->conv, u, st);
    const PassPlan& P = it + 1 < B->refine_steps ? PK : PL;
    for (int k = 0; k < P.npass; ++k) launch_pass<float>(p, P.args[k], P.npairs, P.na, st, P.pmin[k]);
    if (it + 1 < B->refine_steps)
      KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_check<<<1, 1, 0, st>>>(B->nrm, B->tol_dev, B->conv, it));
  }
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

// ---- exact fixed-point refinement for other FP32 inner solvers (multigrid) ----
struct FixState {
  long long* ufix = nullptr;
  long long* rfix = nullptr;
  double* fixd = nullptr;
  float* fixf = nullptr;
  unsigned long long* umax = nullptr;
  FixStencil W{};
  double multh2 = 0.0, kc = 0.0;
};

kfbi_status fix_create(kfbi_problem* p, FixState** out) {
  FixState* F = new FixState();
  *out = F;
  const Grid g = p->g;
  const long long nodes = g.nodes();
  KFBI_CUDA(p, dalloc(&F->ufix, nodes));
  KFBI_CUDA(p, dalloc(&F->rfix, nodes));
  KFBI_CUDA(p, dalloc(&F->fixd, 4));
  KFBI_CUDA(p, dalloc(&F->fixf, 8));
  KFBI_CUDA(p, dalloc(&F->umax, 1));
  double mult, kscale;
  if (p->cfg.order == 2) {
    mult = 1.0;
    F->W = FixStencil{-2 * g.d, 1, 0, 0, 1, 0};
    kscale = 1.0;
  } else if (g.d == 2) {
    mult = 6.0;
    F->W = FixStencil{-20, 4, 1, 0, 8, 1};
    kscale = 0.5;
  } else {
    mult = 48.0;
    F->W = FixStencil{-200, 20, 6, 1, 6, 1};
    kscale = 4.0;
  }
  F->multh2 = mult * g.h * g.h;
  F->kc = kscale * p->kt * g.h * g.h;
  return KFBI_OK;
}

void fix_destroy(FixState* F) {
  if (!F) return;
  cudaFree(F->ufix);
  cudaFree(F->rfix);
  cudaFree(F->fixd);
  cudaFree(F->fixf);
  cudaFree(F->umax);
  delete F;
}

// scale from max|u0|, then u_fix = round(u0 2^F), R_fix = round(mult h^2 R 2^F)
kfbi_status fix_init(kfbi_problem* p, FixState* F, const float* u0, const double* R, cudaStream_t st) {
  const long long nodes = p->g.nodes();
  const int eb = (int)std::min<long long>(div_up(nodes, 256), 152 * 8);
  KFBI_CUDA(p, cudaMemsetAsync(F->umax, 0, sizeof(unsigned long long), st));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_absmax32<<<eb, 256, 0, st>>>(nodes, u0, F->umax, nullptr));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_fix_scale<<<1, 1, 0, st>>>(F->umax, F->multh2, F->kc, F->fixd, F->fixf));
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_fix0<<<eb, 256, 0, st>>>(nodes, u0, R, p->g, F->fixd, F->fixf, F->ufix,
                                                                 F->rfix, nullptr));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status fix_residual(kfbi_problem* p, FixState* F, float* r32, const int* skip, cudaStream_t st) {
  const Grid g = p->g;
  launch_res_fix(p, g, F->W, F->rfix, F->ufix, F->fixd, F->fixf, r32, skip, nullptr, st);
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status fix_add(kfbi_problem* p, FixState* F, const float* e, unsigned long long* corr, const int* skip,
                    cudaStream_t st) {
  const long long nodes = p->g.nodes();
  const int eb = (int)std::min<long long>(div_up(nodes, 256), 152 * 8);
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_fix_add<<<eb, 256, 0, st>>>(nodes, e, F->ufix, F->fixf, corr, skip));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status fix_out(kfbi_problem* p, FixState* F, double* u, cudaStream_t st) {
  const long long nodes = p->g.nodes();
  const int eb = (int)std::min<long long>(div_up(nodes, 256), 152 * 8);
  KFBI_LAUNCH(p, KFBI_KC_RESIDUAL, k_unfix<<<eb, 256, 0, st>>>(nodes, F->ufix, F->fixd, u));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status mg_steps(kfbi_problem* p, int* steps, int* cycles);

// Refinement steps (FP32 solves) and V-cycles the last box solve executed:
// the FP64 sine transform is one step and no cycle; the mixed transform
// counts the first FP32 solve plus every correction step its convergence
// flag let run; the multigrid counts are kept by its check kernels.
kfbi_status box_steps(kfbi_problem* p, int* steps, int* cycles) {
  if (p->mg) return mg_steps(p, steps, cycles);
  *cycles = 0;
  *steps = 1;
  if (p->cfg.precision != KFBI_MIXED) return KFBI_OK;
  unsigned long long c = 0;
  KFBI_CUDA(p, cudaMemcpyAsync(&c, p->box->nrm + 6, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  KFBI_CUDA(p, cudaStreamSynchronize(p->stream));
  *steps = 1 + (int)std::min<unsigned long long>(c, (unsigned long long)p->box->refine_steps - 1);
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
  // the device checks every step but the last: with the flag unset after
  // more than one step, the last step's maxima are still in h[3], h[4]
  double dm, um;
  const bool last_open = p->cfg.precision == KFBI_MIXED && !c && B->refine_steps > 1;
  memcpy(&dm, &h[last_open ? 3 : 2], 8);
  memcpy(&um, &h[last_open ? 4 : 5], 8);
  if (last_open) c = dm <= B->tol * um ? 1 : 0;
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
  {
    // u is cleared before rhs is read: overlapping grids would lose the input
    const unsigned long long bytes =
        sizeof(double) * (dim == 2 ? 1ULL * (n + 1) * (n + 1) : 1ULL * (n + 1) * (n + 1) * (n + 1));
    const unsigned long long a = reinterpret_cast<uintptr_t>(rhs), b = reinterpret_cast<uintptr_t>(u);
    if (a < b + bytes && b < a + bytes) return KFBI_ERR_ARG;
  }
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
// Batched mixed-precision box solve: many independent grids (different N),
// the same steps as the single solve (FP32 solve, fixed-point scale, exact
// residual, FP32 corrections), each step one launch over all instances: the
// passes by persistent CTAs over all instances' line pairs, the grid kernels
// over all instances' rows, with per-instance convergence flags.
// ---------------------------------------------------------------------------
namespace kfbi {
namespace {

struct BoxDesc {
  Grid g;
  FixStencil W;
  double multh2, kc, tol;
  const double* R;         // right-hand side (FP64 grid)
  double* u;               // solution (FP64 grid)
  const float* u0;         // first FP32 solve (the work grid)
  long long* ufix;
  long long* rfix;
  float* r32;
  double* fixd;
  float* fixf;
  unsigned long long* nrm;
  int* conv;
  const double* tolp;      // per-instance refinement tolerance on the device (null: tol)
};

__device__ __forceinline__ int find_inst(const int* start, int ninst, int item) {
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// instance state reset; instances flagged in `done` (outer iteration
// finished) start as converged, so every pass and residual skips them
__global__ void k_zero_batched(const BoxDesc* __restrict__ D, int ninst, const int* __restrict__ done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  for (int k = 0; k < 6; ++k) D[i].nrm[k] = 0ull;
  *D[i].conv = done ? done[i] : 0;
}

// the batched check after refinement step `step`, with the rules of
// check_body (the first FP32 solve stops on the observed error estimate)
__global__ void k_check_batched(const BoxDesc* __restrict__ D, int ninst, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  unsigned long long* nrm = D[i].nrm;
  if (*D[i].conv) return;
  const double tol = D[i].tolp ? D[i].tolp[0] : D[i].tol;
  const double dm = __longlong_as_double((long long)nrm[3]);
  const double um = __longlong_as_double((long long)nrm[4]);
  nrm[2] = nrm[3];
  nrm[5] = nrm[4];
  bool stop = dm <= tol * um;
  if (step == 0 && 10.0 * __longlong_as_double((long long)nrm[8]) <= tol) stop = true;
  if (step == 1 && um > 0.0) nrm[8] = (unsigned long long)__double_as_longlong(dm / um);
  if (stop) *D[i].conv = 1;
  nrm[3] = 0ull;
  nrm[4] = 0ull;
}

__global__ void k_fix_scale_batched(const BoxDesc* __restrict__ D, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  fix_scale_body(D[i].nrm + 5, D[i].multh2, D[i].kc, D[i].fixd, D[i].fixf);
}

// grid kernels over all instances' rows (one row of the last axis per item);
// mode 0: u_fix = round(u0 2^F), R_fix = round(mult h^2 R 2^F);
// mode 1: exact residual -> r32 (skips converged instances);
// mode 2: u = u_fix 2^-F.
__global__ void k_rows_batched(const BoxDesc* __restrict__ D, const int* __restrict__ rstart, int ninst, int mode) {
  const int total = rstart[ninst];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int inst = find_inst(rstart, ninst, item);
    const BoxDesc& B = D[inst];
    if (mode == 1 && *B.conv) continue;
    const Grid g = B.g;
    const int n1 = g.n + 1;
    const int row = item - rstart[inst];
    const int i1 = row % n1, i0 = row / n1;   // 2D: i0 = 0
    const bool row_in = i1 >= 1 && i1 < g.n && (g.d == 2 || (i0 >= 1 && i0 < g.n));
    const int base = g.d == 2 ? i1 * n1 : (i0 * n1 + i1) * n1;
    for (int j = threadIdx.x; j <= g.n; j += blockDim.x) {
      const int t = base + j;
      const bool interior = row_in && j >= 1 && j < g.n;
      if (mode == 0) {
        const float* ff = B.fixf;
        B.ufix[t] = f2ll((B.u0[t] * ff[0]) * ff[1]);
        B.rfix[t] = interior ? d2ll_pow2(B.R[t], (int)B.fixd[3]) : 0ll;
      } else if (mode == 2) {
        B.u[t] = ll2d(B.ufix[t]) * B.fixd[1];
      } else {
        if (!interior) {
          B.r32[t] = 0.f;
          continue;
        }
        const FixStencil W = B.W;
        const long long* ub = B.ufix;
#define UP(o) ub[t + (o)]
        FIX_NEIGHBOURS(UP)
#undef UP
        long long m;
        long long r = sub64(B.rfix[t], fix_apply(W, c, e, k2, k3, m));
        const KappaFix kf = kappa_fix(B.fixd[2]);
        if (!kf.zero) r = add64(r, kappa_int(kf, m));
        B.r32[t] = (ll2f(r) * B.fixf[2]) * B.fixf[4];
      }
    }
  }
}

}  // namespace

struct BatchBox {
  int ninst = 0, npass = 0, steps = 3;
  PassArgs* dargs = nullptr;   // [2 npass][ninst]: step 0 passes, then refinement-step passes
  int* dstart = nullptr;       // [ninst + 1] pass work items
  BoxDesc* dbox = nullptr;     // [ninst]
  int* drstart = nullptr;      // [ninst + 1] grid rows
  int grid = 0, rgrid = 0;
};

void batch_box_copy_tiles(BatchBox* dst, const BatchBox* src) {
  dst->grid = src->grid;
  dst->rgrid = src->rgrid;
}

kfbi_status batch_box_create(kfbi_problem* p0, kfbi_problem* const* ps, int ninst,
                             double* const* rhs, BatchBox** out, const double* tol_dev) {
  BatchBox* bb = new BatchBox();
  *out = bb;
  bb->ninst = ninst;
  const int d = ps[0]->g.d;
  std::vector<PassPlan> plan0(ninst), plank(ninst);
  std::vector<int> start(ninst + 1, 0), rstart(ninst + 1, 0);
  std::vector<BoxDesc> box(ninst);
  for (int i = 0; i < ninst; ++i) {
    kfbi_problem* p = ps[i];
    if (p->g.d != d || p->cfg.precision != KFBI_MIXED || p->box == nullptr || p->mg != nullptr ||
        p->box->logL > 11)
      return fail(p0, KFBI_ERR_UNSUPPORTED,
                  "batched solves need mixed-precision DST problems of one dimension with N <= 1024");
    BoxSolver* B = p->box;
    float* r32 = reinterpret_cast<float*>(B->res);
    plan0[i] = plan_passes<float>(p, rhs[i], 1, p->ugrid, 0, B->conv, B->nrm + 3);
    {
      PassArgs& last = plan0[i].args[plan0[i].npass - 1];
      last.dst = B->work32;
      last.dst64 = 0;
      last.accumulate = 0;
      last.corr_max = B->nrm + 3;
    }
    plank[i] = plan_passes<float>(p, r32, 0, p->ugrid, 0, B->conv, B->nrm + 3);
    {
      PassArgs& last = plank[i].args[plank[i].npass - 1];
      last.dst = nullptr;
      last.dst64 = 0;
      last.accumulate = 1;
      last.dstfix = B->ufix;
      last.fixf = B->fixf;
      last.corr_max = B->nrm + 3;
    }
    const int pp = reg_pairs(B->logL);
    start[i + 1] = start[i] + ((plan0[i].npairs + pp - 1) / pp) * plan0[i].na;
    const int n1 = p->g.n + 1;
    rstart[i + 1] = rstart[i] + (d == 2 ? n1 : n1 * n1);
    box[i] = BoxDesc{p->g, FixStencil{B->w[0], B->w[1], B->w[2], B->w[3], B->kA, B->kB}, B->multh2, B->kc, B->tol,
                     rhs[i], p->ugrid, B->work32, B->ufix, B->rfix, r32, B->fixd, B->fixf, B->nrm, B->conv,
                     tol_dev ? tol_dev + i : nullptr};
  }
  bb->steps = 0;
  for (int i = 0; i < ninst; ++i) bb->steps = std::max(bb->steps, ps[i]->box->refine_steps);
  bb->npass = plan0[0].npass;
  std::vector<PassArgs> args;
  for (int v = 0; v < 2 * bb->npass; ++v)
    for (int i = 0; i < ninst; ++i)
      args.push_back(v < bb->npass ? plan0[i].args[v] : plank[i].args[v - bb->npass]);
  KFBI_CUDA(p0, dalloc(&bb->dargs, args.size()));
  KFBI_CUDA(p0, dalloc(&bb->dstart, ninst + 1));
  KFBI_CUDA(p0, dalloc(&bb->dbox, ninst));
  KFBI_CUDA(p0, dalloc(&bb->drstart, ninst + 1));
  KFBI_CUDA(p0, cudaMemcpy(bb->dargs, args.data(), sizeof(PassArgs) * args.size(), cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->dstart, start.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->dbox, box.data(), sizeof(BoxDesc) * ninst, cudaMemcpyHostToDevice));
  KFBI_CUDA(p0, cudaMemcpy(bb->drstart, rstart.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
  int dev = 0, sms = 0;
  KFBI_CUDA(p0, cudaGetDevice(&dev));
  KFBI_CUDA(p0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  KFBI_CUDA(p0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dst32_batched, 128, Reg<11, 1>::SMEM));
  bb->grid = sms * std::max(1, per_sm);
  bb->rgrid = sms * 8;
  return KFBI_OK;
}

namespace {
// a deterministic non-zero right-hand side for timing (values in [-0.5, 0.5))
__global__ void k_fill_pattern(long long tot, double* __restrict__ R) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x)
    R[t] = (double)((unsigned)(t * 2654435761ull) % 1000u) * 1e-3 - 0.5;
}
}  // namespace

// Autotuner of the batched box solve's launch shapes: the CTA count of the
// persistent transform pass (half, once or twice the CTAs resident on the
// GPU) and of the row kernel (4, 8, 16 or 32 CTAs per SM), each timed on the
// batch's own grids (a synthetic right-hand side, one warm-up and two timed
// box solves per candidate, CUDA events) and the fastest kept.  The shapes
// change only how the work items are spread, not the arithmetic.  rhs is
// zeroed again afterwards.
kfbi_status batch_box_autotune(kfbi_problem* p0, BatchBox* bb, kfbi_problem* const* ps, double* const* rhs,
                               const int* done, cudaStream_t st) {
  int dev = 0, sms = 0;
  KFBI_CUDA(p0, cudaGetDevice(&dev));
  KFBI_CUDA(p0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int i = 0; i < bb->ninst; ++i) {
    const long long tot = ps[i]->g.nodes();
    k_fill_pattern<<<std::min(div_up(tot, 256), 8 * sms), 256, 0, st>>>(tot, rhs[i]);
  }
  KFBI_CUDA(p0, cudaGetLastError());
  cudaEvent_t e0, e1;
  KFBI_CUDA(p0, cudaEventCreate(&e0));
  KFBI_CUDA(p0, cudaEventCreate(&e1));
  auto time_solve = [&](float* ms) -> kfbi_status {
    KFBI_TRY(batch_box_solve(p0, bb, done, st));
    KFBI_CUDA(p0, cudaEventRecord(e0, st));
    for (int r = 0; r < 2; ++r) KFBI_TRY(batch_box_solve(p0, bb, done, st));
    KFBI_CUDA(p0, cudaEventRecord(e1, st));
    KFBI_CUDA(p0, cudaEventSynchronize(e1));
    KFBI_CUDA(p0, cudaEventElapsedTime(ms, e0, e1));
    return KFBI_OK;
  };
  const int resident = bb->grid;   // batch_box_create: SMs x resident CTAs per SM
  kfbi_status s = KFBI_OK;
  float best = 1e30f;
  int best_grid = resident;
  for (int g : {std::max(1, resident / 2), resident, 2 * resident}) {
    bb->grid = g;
    float ms = 0.f;
    if ((s = time_solve(&ms)) != KFBI_OK) break;
    if (ms < best) {
      best = ms;
      best_grid = g;
    }
  }
  bb->grid = best_grid;
  best = 1e30f;
  int best_rgrid = 8 * sms;
  for (int per : {4, 8, 16, 32}) {
    if (s != KFBI_OK) break;
    bb->rgrid = per * sms;
    float ms = 0.f;
    if ((s = time_solve(&ms)) != KFBI_OK) break;
    if (ms < best) {
      best = ms;
      best_rgrid = per * sms;
    }
  }
  bb->rgrid = best_rgrid;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < bb->ninst; ++i)
    KFBI_CUDA(p0, cudaMemsetAsync(rhs[i], 0, sizeof(double) * ps[i]->g.nodes(), st));
  KFBI_CUDA(p0, cudaStreamSynchronize(st));
  return s;
}

void batch_box_tiles(const BatchBox* bb, int* pass_ctas, int* row_ctas) {
  *pass_ctas = bb->grid;
  *row_ctas = bb->rgrid;
}

void batch_box_destroy(BatchBox* bb) {
  if (!bb) return;
  cudaFree(bb->dargs);
  cudaFree(bb->dstart);
  cudaFree(bb->dbox);
  cudaFree(bb->drstart);
  delete bb;
}

// All instances not flagged in `done` (may be null): u_i = A_i^{-1} rhs_i by the
// mixed-precision steps of box_solve, every step one launch over all instances.
kfbi_status batch_box_solve(kfbi_problem* p0, BatchBox* bb, const int* done, cudaStream_t st) {
  const int ni = bb->ninst;
  const size_t smem = Reg<11, 1>::SMEM;
  const int cb = div_up(ni, 128);
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_zero_batched<<<cb, 128, 0, st>>>(bb->dbox, ni, done));
  for (int v = 0; v < bb->npass; ++v)
    KFBI_LAUNCH(p0, KFBI_KC_DST, k_dst32_batched<<<bb->grid, 128, smem, st>>>(bb->dargs + (size_t)v * ni,
                                                                               bb->dstart, ni));
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_check_batched<<<cb, 128, 0, st>>>(bb->dbox, ni, 0));
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_fix_scale_batched<<<cb, 128, 0, st>>>(bb->dbox, ni));
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_rows_batched<<<bb->rgrid, 128, 0, st>>>(bb->dbox, bb->drstart, ni, 0));
  for (int it = 1; it < bb->steps; ++it) {
    KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_rows_batched<<<bb->rgrid, 128, 0, st>>>(bb->dbox, bb->drstart, ni, 1));
    for (int v = 0; v < bb->npass; ++v)
      KFBI_LAUNCH(p0, KFBI_KC_DST, k_dst32_batched<<<bb->grid, 128, smem, st>>>(
          bb->dargs + (size_t)(bb->npass + v) * ni, bb->dstart, ni));
    KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_check_batched<<<cb, 128, 0, st>>>(bb->dbox, ni, it));
  }
  KFBI_LAUNCH(p0, KFBI_KC_RESIDUAL, k_rows_batched<<<bb->rgrid, 128, 0, st>>>(bb->dbox, bb->drstart, ni, 2));
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
