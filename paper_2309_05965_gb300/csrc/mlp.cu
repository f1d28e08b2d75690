// Learned initial density for GMRES (Algorithm 1, Step 4 from a learned
// start instead of zero): a small fully connected network evaluated at every
// DOF, trained on the GPU on densities that the method itself computes.
//
//   z1 = W1 x + b1, a1 = tanh z1;  z2 = W2 a1 + b2, a2 = tanh z2;
//   y = W3 a2 + b3 + WL x
//
// Precision: FP32 master weights; the products with W1, W2, W3 use those
// weights rounded to bfloat16 (kept in a BF16 copy refreshed after each
// update); the linear skip WL, activations and all sums are FP32, so the
// linear part of the map is resolved beyond bfloat16 precision.  Gradients are those at the rounded weights and update the
// FP32 masters with Adam (Kingma & Ba 2015, bias-corrected moments).
//
// The contractions (K = 16 or 256, N = 256; the weight gradients K = rows) run
// on the tensor cores: mma.sync bf16 with FP32 accumulation, FP32 operands
// split into bf16 parts so that the products keep FP32 precision (k_gemm).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kfbi_internal.cuh"

struct kfbi_mlp {
  int n_in = 0, width = 0, nparam = 0;
  int oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, oWL = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  float* theta = nullptr;          // FP32 masters
  float* grad = nullptr;
  float* mom1 = nullptr;
  float* mom2 = nullptr;
  __nv_bfloat16* wbf = nullptr;    // rounded copy, master layout
  float* shift = nullptr;          // [n_in] input normalisation x~ = (x - shift) * scale
  float* scale = nullptr;
  double out_shift = 0.0, out_scale = 1.0;
  long long step = 0;
  int train_lo = 0, train_hi = 0;  // parameters that Adam updates: [train_lo, train_hi)
  // per-row scratch
  int cap = 0;
  float* X = nullptr;     // normalised input [cap][n_in]
  float* a1 = nullptr;    // [cap][width]
  float* a2 = nullptr;
  float* d1 = nullptr;    // back-propagated signals [cap][width]
  float* d2 = nullptr;
  float* y = nullptr;     // [cap]
  float* dy = nullptr;
  float* tb = nullptr;    // gathered targets [cap]
  float* loss = nullptr;  // [1]
};

namespace kfbi {
namespace {

kfbi_status mfail(kfbi_mlp* m, kfbi_status s, const std::string& msg) {
  if (m) m->err = msg;
  return s;
}

#define MLP_CUDA(m, call)                                                         \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return mfail((m), KFBI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
__device__ __forceinline__ float tof(T v);
template <>
__device__ __forceinline__ float tof<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- tensor-core GEMM: mma.sync m16n8k16, bf16 operands, FP32 accumulation --
// An FP32 operand enters as a sum of bfloat16 parts, x = hi + mid + lo with
// each part the bf16 rounding of what the previous parts leave; every product
// of two bf16 values is exact in FP32, so three parts carry an FP32 value's
// 24 bits.  Weights already rounded to bf16 are one exact part.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  // a in the low half: the element of the smaller k (or row) index
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (M x N) = A (M x K) B (K x N) with element (i, k) of A at A[i sam + k sak]
// and (k, j) of B at B[k sbk + j sbn].  blockIdx.z splits K into chunks.
// mode 0: C = act(acc + bias) [* (1 - gate^2)];  mode 1: C += acc (atomic).
// 64 x 64 tiles, four warps of 32 x 32 (2 x 4 mma tiles), K steps of 16
// staged in shared memory as FP32.  A is split in three bf16 parts; B is one
// part when it is the bf16 weight copy, three when it is an FP32 array.
template <typename TB>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, int kchunk, const float* __restrict__ A,
                                              long long sam, long long sak, const TB* __restrict__ B,
                                              long long sbk, long long sbn, float* __restrict__ C, long long ldc,
                                              const float* __restrict__ bias, int act, const float* __restrict__ gate,
                                              int mode) {
  constexpr bool BEXACT = sizeof(TB) == 2;
  __shared__ float As[16][64 + 4];   // As[k][i]
  __shared__ float Bs[16][64 + 4];   // Bs[k][j]
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 128) {
      int i, k;
      if (sam == 1) {
        i = e & 63;
        k = e >> 6;
      } else {
        i = e >> 4;
        k = e & 15;
      }
      const int gi = m0 + i, gk = k0 + k;
      As[k][i] = (gi < M && gk < ke) ? A[gi * sam + gk * sak] : 0.f;
      int j, kk;
      if (sbn == 1) {
        j = e & 63;
        kk = e >> 6;
      } else {
        j = e >> 4;
        kk = e & 15;
      }
      const int gj = n0 + j, gk2 = k0 + kk;
      Bs[kk][j] = (gj < N && gk2 < ke) ? tof<TB>(B[gk2 * sbk + gj * sbn]) : 0.f;
    }
    __syncthreads();
    // A fragments (rows g, g + 8; k pairs 2tq, 2tq + 8) in three parts
    uint32_t af[3][2][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16 + g;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = r + ((q & 1) ? 8 : 0);
        const int kk = 2 * tq + ((q & 2) ? 8 : 0);
        __nv_bfloat16 h0, m0b, l0, h1, m1b, l1;
        split3(As[kk][rr], h0, m0b, l0);
        split3(As[kk + 1][rr], h1, m1b, l1);
        af[0][mi][q] = pack2(h0, h1);
        af[1][mi][q] = pack2(m0b, m1b);
        af[2][mi][q] = pack2(l0, l1);
      }
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int col = wn + ni * 8 + g;
      uint32_t bf[3][2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int kk = 2 * tq + (q ? 8 : 0);
        __nv_bfloat16 h0, m0b, l0, h1, m1b, l1;
        split3(Bs[kk][col], h0, m0b, l0);
        split3(Bs[kk + 1][col], h1, m1b, l1);
        bf[0][q] = pack2(h0, h1);
        bf[1][q] = pack2(m0b, m1b);
        bf[2][q] = pack2(l0, l1);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        // small terms first: lo, mid, then hi
        if (BEXACT) {
          mma16816(acc[mi][ni], af[2][mi], bf[0]);
          mma16816(acc[mi][ni], af[1][mi], bf[0]);
          mma16816(acc[mi][ni], af[0][mi], bf[0]);
        } else {
          mma16816(acc[mi][ni], af[2][mi], bf[0]);
          mma16816(acc[mi][ni], af[0][mi], bf[2]);
          mma16816(acc[mi][ni], af[1][mi], bf[1]);
          mma16816(acc[mi][ni], af[1][mi], bf[0]);
          mma16816(acc[mi][ni], af[0][mi], bf[1]);
          mma16816(acc[mi][ni], af[0][mi], bf[0]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = m0 + wm + mi * 16 + g + (e >= 2 ? 8 : 0);
        const int j = n0 + wn + ni * 8 + 2 * tq + (e & 1);
        if (i >= M || j >= N) continue;
        float* o = C + (long long)i * ldc + j;
        if (mode == 1) {
          atomicAdd(o, acc[mi][ni][e]);
        } else {
          float v = acc[mi][ni][e] + (bias ? bias[j] : 0.f);
          if (act) v = tanhf(v);
          if (gate) {
            const float gt = gate[(long long)i * ldc + j];
            v *= 1.f - gt * gt;
          }
          *o = v;
        }
      }
}

// X[i, :] = (raw[r_i, :] - shift) * scale with r_i = rows[i] (i when rows is
// null); the targets of the selected rows are gathered alongside.
__global__ void k_normalise(int n, int n_in, const float* __restrict__ raw, const int32_t* __restrict__ rows,
                            const float* __restrict__ shift, const float* __restrict__ scale,
                            float* __restrict__ X, const float* __restrict__ t_in, float* __restrict__ t_out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n_in) return;
  const int k = (int)(t % n_in);
  const long long i = t / n_in;
  const long long r = rows ? (long long)rows[i] : i;
  X[t] = (raw[r * n_in + k] - shift[k]) * scale[k];
  if (t_in && k == 0) t_out[i] = t_in[r];
}

// y_i = W3 a2_i + b3 (a warp per row); with targets: dy_i = (y_i - t_i)/n and
// the loss sum 1/(2n) sum e^2.
__global__ void k_output(int n, int W, const float* __restrict__ a2, const __nv_bfloat16* __restrict__ w3,
                         const float* __restrict__ b3, int n_in, const float* __restrict__ X,
                         const float* __restrict__ wl, float* __restrict__ y, const float* __restrict__ t,
                         float* __restrict__ dy, float* __restrict__ loss) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float s = 0.f;
  for (int k = lane; k < W; k += 32) s = fmaf(a2[(long long)row * W + k], __bfloat162float(w3[k]), s);
  if (lane < n_in) s = fmaf(X[(long long)row * n_in + lane], wl[lane], s);
  s = warp_sum(s);
  if (lane == 0) {
    const float v = s + b3[0];
    y[row] = v;
    if (t) {
      const float e = v - t[row];
      dy[row] = e / (float)n;
      atomicAdd(loss, 0.5f * e * e / (float)n);
    }
  }
}

// d2 = dy_i W3_k (1 - a2^2)
__global__ void k_back_out(int n, int W, const float* __restrict__ dy, const __nv_bfloat16* __restrict__ w3,
                           const float* __restrict__ a2, float* __restrict__ d2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * W) return;
  const int k = (int)(t % W);
  const long long i = t / W;
  const float g = a2[t];
  d2[t] = dy[i] * __bfloat162float(w3[k]) * (1.f - g * g);
}

// out_k += sum_i w_i X[i, k] (w = 1 when null); rows split over blocks
__global__ void k_colsum(int n, int c, const float* __restrict__ w, const float* __restrict__ X, float* __restrict__ out,
                         int rows_per_block) {
  const int k = threadIdx.x + blockIdx.y * blockDim.x;
  if (k >= c) return;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  float s = 0.f;
  for (int i = r0; i < r1; ++i) s = fmaf(w ? w[i] : 1.f, X[(long long)i * c + k], s);
  atomicAdd(out + k, s);
}

__global__ void k_round(int np, const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < np) wbf[t] = __float2bfloat16_rn(theta[t]);
}

__global__ void k_adam(int lo, int hi, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                       __nv_bfloat16* __restrict__ wbf) {
  const int t = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= hi) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float th = theta[t] - lr * (mt / bc1) / (sqrtf(vt / bc2) + eps);
  theta[t] = th;
  wbf[t] = __float2bfloat16_rn(th);
}

// Per-DOF raw features: [g1, g2, n (3), x (3), level-set parameters p0..p5,
// log10(sigma_in/sigma_out) (0 for a boundary value problem), 0].  The data
// are not rescaled per problem: the network's input normalisation (from its
// training set) brings each feature to unit size, and a problem family whose
// data share fields (the same sources with different geometries and
// coefficients) keeps its density a function of the DOF's features alone.
__global__ void k_features(int nb, int d, const double* __restrict__ x0, const double* __restrict__ x1,
                           const double* __restrict__ x2, const double* __restrict__ n0,
                           const double* __restrict__ n1, const double* __restrict__ n2,
                           const double* __restrict__ g1, const double* __restrict__ g2, LevelSet ls,
                           float lcontrast, float* __restrict__ F, const double* __restrict__ dens,
                           float* __restrict__ target) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  if (target) target[j] = (float)dens[j];
  float* f = F + (long long)j * KFBI_WS_FEATURES;
  f[0] = g1 ? (float)g1[j] : 0.f;
  f[1] = g2 ? (float)g2[j] : 0.f;
  f[2] = (float)n0[j];
  f[3] = (float)n1[j];
  f[4] = d == 3 ? (float)n2[j] : 0.f;
  f[5] = (float)x0[j];
  f[6] = (float)x1[j];
  f[7] = d == 3 ? (float)x2[j] : 0.f;
  for (int k = 0; k < 6; ++k) f[8 + k] = k < ls.np ? (float)ls.p[k] : 0.f;
  f[14] = lcontrast;
  f[15] = 0.f;
}

__global__ void k_to_density(int n, const float* __restrict__ y, double shift, double scale,
                             double* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = (double)y[j] * scale + shift;
}

kfbi_status ensure(kfbi_mlp* m, int n) {
  if (n <= m->cap) return KFBI_OK;
  MLP_CUDA(m, cudaStreamSynchronize(m->stream));
  float** bufs[] = {&m->X, &m->a1, &m->a2, &m->d1, &m->d2, &m->y, &m->dy, &m->tb};
  for (float** b : bufs) {
    cudaFree(*b);
    *b = nullptr;
  }
  const int cap = std::max(n, 1024);
  const size_t W = m->width;
  MLP_CUDA(m, dalloc(&m->X, (size_t)cap * m->n_in));
  MLP_CUDA(m, dalloc(&m->a1, (size_t)cap * W));
  MLP_CUDA(m, dalloc(&m->a2, (size_t)cap * W));
  MLP_CUDA(m, dalloc(&m->d1, (size_t)cap * W));
  MLP_CUDA(m, dalloc(&m->d2, (size_t)cap * W));
  MLP_CUDA(m, dalloc(&m->y, (size_t)cap));
  MLP_CUDA(m, dalloc(&m->dy, (size_t)cap));
  MLP_CUDA(m, dalloc(&m->tb, (size_t)cap));
  m->cap = cap;
  return KFBI_OK;
}

template <typename TB>
void gemm(cudaStream_t st, int M, int N, int K, const float* A, long long sam, long long sak, const TB* B,
          long long sbk, long long sbn, float* C, long long ldc, const float* bias, int act, const float* gate,
          int mode) {
  int splits = 1, chunk = K;
  if (mode == 1) {   // weight gradients: long K (the rows), few output tiles
    const int tiles = div_up(M, 64) * div_up(N, 64);
    splits = std::max(1, std::min(div_up(K, 256), div_up(152 * 8, tiles)));
    chunk = div_up(div_up(K, splits), 16) * 16;
    splits = div_up(K, chunk);
  }
  dim3 grid(div_up(N, 64), div_up(M, 64), splits);
  k_gemm<TB><<<grid, 128, 0, st>>>(M, N, K, chunk, A, sam, sak, B, sbk, sbn, C, ldc, bias, act, gate, mode);
}

// forward on rows already normalised into m->X
kfbi_status forward_rows(kfbi_mlp* m, int n, const float* t) {
  const int W = m->width, ni = m->n_in;
  cudaStream_t st = m->stream;
  const __nv_bfloat16* wb = m->wbf;
  gemm<__nv_bfloat16>(st, n, W, ni, m->X, ni, 1, wb + m->oW1, 1, ni, m->a1, W, m->theta + m->ob1, 1, nullptr, 0);
  gemm<__nv_bfloat16>(st, n, W, W, m->a1, W, 1, wb + m->oW2, 1, W, m->a2, W, m->theta + m->ob2, 1, nullptr, 0);
  k_output<<<div_up(n, 8), 256, 0, st>>>(n, W, m->a2, wb + m->oW3, m->theta + m->ob3, ni, m->X,
                                         m->theta + m->oWL, m->y, t, m->dy, m->loss);
  MLP_CUDA(m, cudaGetLastError());
  return KFBI_OK;
}

}  // namespace
}  // namespace kfbi

using namespace kfbi;

extern "C" {

const char* kfbi_mlp_last_error(const kfbi_mlp* m) { return m ? m->err.c_str() : ""; }

kfbi_status kfbi_mlp_destroy(kfbi_mlp* m) {
  if (!m) return KFBI_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  void* bufs[] = {m->theta, m->grad, m->mom1, m->mom2, m->wbf, m->shift, m->scale, m->X,
                  m->a1,    m->a2,   m->d1,   m->d2,   m->y,   m->dy,    m->tb,    m->loss};
  for (void* b : bufs) cudaFree(b);
  delete m;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_create(int n_in, int width, void* cuda_stream, kfbi_mlp** out) {
  if (!out || n_in < 1 || n_in > KFBI_WS_FEATURES || width < 1 || width > 1024) return KFBI_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return KFBI_ERR_CUDA;
  kfbi_mlp* m = new kfbi_mlp();
  m->n_in = n_in;
  m->width = width;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  m->oW1 = 0;
  m->ob1 = width * n_in;
  m->oW2 = m->ob1 + width;
  m->ob2 = m->oW2 + width * width;
  m->oW3 = m->ob2 + width;
  m->ob3 = m->oW3 + width;
  m->oWL = m->ob3 + 1;
  m->nparam = m->oWL + n_in;
  m->train_lo = 0;
  m->train_hi = m->nparam;
  const size_t np = m->nparam;
  bool ok = dalloc(&m->theta, np) == cudaSuccess && dalloc(&m->grad, np) == cudaSuccess &&
            dalloc(&m->mom1, np) == cudaSuccess && dalloc(&m->mom2, np) == cudaSuccess &&
            dalloc(&m->wbf, np) == cudaSuccess && dalloc(&m->shift, n_in) == cudaSuccess &&
            dalloc(&m->scale, n_in) == cudaSuccess && dalloc(&m->loss, 1) == cudaSuccess;
  if (ok) {
    std::vector<float> one(n_in, 1.f);
    ok = cudaMemset(m->theta, 0, np * 4) == cudaSuccess && cudaMemset(m->mom1, 0, np * 4) == cudaSuccess &&
         cudaMemset(m->mom2, 0, np * 4) == cudaSuccess && cudaMemset(m->grad, 0, np * 4) == cudaSuccess &&
         cudaMemset(m->wbf, 0, np * 2) == cudaSuccess && cudaMemset(m->shift, 0, n_in * 4) == cudaSuccess &&
         cudaMemcpy(m->scale, one.data(), n_in * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    kfbi_mlp_destroy(m);
    return KFBI_ERR_CUDA;
  }
  *out = m;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_num_params(const kfbi_mlp* m, int* count) {
  if (!m || !count) return KFBI_ERR_ARG;
  *count = m->nparam;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_set_params(kfbi_mlp* m, const float* params) {
  if (!m || !params) return KFBI_ERR_ARG;
  MLP_CUDA(m, cudaMemcpyAsync(m->theta, params, sizeof(float) * m->nparam, cudaMemcpyDeviceToDevice, m->stream));
  MLP_CUDA(m, cudaMemsetAsync(m->mom1, 0, sizeof(float) * m->nparam, m->stream));
  MLP_CUDA(m, cudaMemsetAsync(m->mom2, 0, sizeof(float) * m->nparam, m->stream));
  m->step = 0;
  k_round<<<div_up(m->nparam, 256), 256, 0, m->stream>>>(m->nparam, m->theta, m->wbf);
  MLP_CUDA(m, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status kfbi_mlp_set_trainable(kfbi_mlp* m, int groups) {
  if (!m || groups < 0 || groups > 3) return KFBI_ERR_ARG;
  // the nonlinear branch [W1, b1, W2, b2, W3] precedes the linear part [b3, WL]
  m->train_lo = (groups & 1) ? 0 : m->ob3;
  m->train_hi = (groups & 2) ? m->nparam : m->ob3;
  if (groups == 0) m->train_lo = m->train_hi = 0;
  MLP_CUDA(m, cudaMemsetAsync(m->mom1, 0, sizeof(float) * m->nparam, m->stream));
  MLP_CUDA(m, cudaMemsetAsync(m->mom2, 0, sizeof(float) * m->nparam, m->stream));
  m->step = 0;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_get_params(const kfbi_mlp* mc, float* params, float* grads) {
  kfbi_mlp* m = const_cast<kfbi_mlp*>(mc);
  if (!m) return KFBI_ERR_ARG;
  if (params)
    MLP_CUDA(m, cudaMemcpyAsync(params, m->theta, sizeof(float) * m->nparam, cudaMemcpyDeviceToDevice, m->stream));
  if (grads)
    MLP_CUDA(m, cudaMemcpyAsync(grads, m->grad, sizeof(float) * m->nparam, cudaMemcpyDeviceToDevice, m->stream));
  return KFBI_OK;
}

kfbi_status kfbi_mlp_set_affine(kfbi_mlp* m, const float* in_shift, const float* in_scale, double out_shift,
                                double out_scale) {
  if (!m || !in_shift || !in_scale || !std::isfinite(out_shift) || !std::isfinite(out_scale)) return KFBI_ERR_ARG;
  MLP_CUDA(m, cudaMemcpy(m->shift, in_shift, sizeof(float) * m->n_in, cudaMemcpyHostToDevice));
  MLP_CUDA(m, cudaMemcpy(m->scale, in_scale, sizeof(float) * m->n_in, cudaMemcpyHostToDevice));
  m->out_shift = out_shift;
  m->out_scale = out_scale;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_forward(kfbi_mlp* m, const float* X, int n, float* y) {
  if (!m || n < 0 || (n > 0 && (!X || !y))) return KFBI_ERR_ARG;
  if (n == 0) return KFBI_OK;
  KFBI_TRY(ensure(m, n));
  const long long tot = (long long)n * m->n_in;
  k_normalise<<<div_up(tot, 256), 256, 0, m->stream>>>(n, m->n_in, X, nullptr, m->shift, m->scale, m->X,
                                                        nullptr, nullptr);
  KFBI_TRY(forward_rows(m, n, nullptr));
  MLP_CUDA(m, cudaMemcpyAsync(y, m->y, sizeof(float) * n, cudaMemcpyDeviceToDevice, m->stream));
  return KFBI_OK;
}

kfbi_status kfbi_mlp_loss_grad(kfbi_mlp* m, const float* X, const float* t, const int32_t* rows, int n,
                               float* loss) {
  if (!m || !X || !t || n < 1) return KFBI_ERR_ARG;
  KFBI_TRY(ensure(m, n));
  cudaStream_t st = m->stream;
  const int W = m->width, ni = m->n_in;
  const long long tot = (long long)n * ni;
  MLP_CUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  MLP_CUDA(m, cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparam, st));
  k_normalise<<<div_up(tot, 256), 256, 0, st>>>(n, ni, X, rows, m->shift, m->scale, m->X, t, m->tb);
  KFBI_TRY(forward_rows(m, n, m->tb));
  const __nv_bfloat16* wb = m->wbf;
  float* g = m->grad;
  // output layer: dW3 = dy^T a2, db3 = sum dy
  const int rpb = 256;
  k_colsum<<<dim3(div_up(n, rpb), div_up(W, 256)), 256, 0, st>>>(n, W, m->dy, m->a2, g + m->oW3, rpb);
  k_colsum<<<dim3(div_up(n, rpb), 1), 32, 0, st>>>(n, 1, nullptr, m->dy, g + m->ob3, rpb);
  k_colsum<<<dim3(div_up(n, rpb), 1), 32, 0, st>>>(n, ni, m->dy, m->X, g + m->oWL, rpb);
  // d2 = dy W3 (1 - a2^2); dW2 = d2^T a1, db2 = sum d2
  k_back_out<<<div_up((long long)n * W, 256), 256, 0, st>>>(n, W, m->dy, wb + m->oW3, m->a2, m->d2);
  gemm<float>(st, W, W, n, m->d2, 1, W, m->a1, W, 1, g + m->oW2, W, nullptr, 0, nullptr, 1);
  k_colsum<<<dim3(div_up(n, rpb), div_up(W, 256)), 256, 0, st>>>(n, W, nullptr, m->d2, g + m->ob2, rpb);
  // d1 = (d2 W2) (1 - a1^2); dW1 = d1^T x~, db1 = sum d1
  gemm<__nv_bfloat16>(st, n, W, W, m->d2, W, 1, wb + m->oW2, W, 1, m->d1, W, nullptr, 0, m->a1, 0);
  gemm<float>(st, W, ni, n, m->d1, 1, W, m->X, ni, 1, g + m->oW1, ni, nullptr, 0, nullptr, 1);
  k_colsum<<<dim3(div_up(n, rpb), div_up(W, 256)), 256, 0, st>>>(n, W, nullptr, m->d1, g + m->ob1, rpb);
  MLP_CUDA(m, cudaGetLastError());
  if (loss) MLP_CUDA(m, cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return KFBI_OK;
}

kfbi_status kfbi_mlp_adam(kfbi_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return KFBI_ERR_ARG;
  m->step += 1;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)m->step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)m->step));
  const int cnt = m->train_hi - m->train_lo;
  if (cnt <= 0) return KFBI_OK;
  k_adam<<<div_up(cnt, 256), 256, 0, m->stream>>>(m->train_lo, m->train_hi, m->theta, m->grad, m->mom1, m->mom2,
                                                   lr, beta1, beta2, eps, bc1, bc2, m->wbf);
  MLP_CUDA(m, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status kfbi_warm_start_features(kfbi_problem* p, const kfbi_data* data, const double* density,
                                     float* features, float* target) {
  if (!p || !data || !features || !data->g1 || (!density != !target)) return KFBI_ERR_ARG;
  const Grid g = p->g;
  const bool iface = p->cfg.kind == KFBI_INTERFACE_MU || p->cfg.kind == KFBI_INTERFACE_GENERAL;
  const float lcontrast = iface ? (float)std::log10(p->cfg.sigma_in / p->cfg.sigma_out) : 0.f;
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_features<<<div_up(p->nb, 128), 128, 0, p->stream>>>(
      p->nb, g.d, p->x[0], p->x[1], g.d == 3 ? p->x[2] : p->x[0], p->nrm[0], p->nrm[1],
      g.d == 3 ? p->nrm[2] : p->nrm[0], data->g1, data->g2, p->ls, lcontrast, features, density, target));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status kfbi_warm_start(kfbi_problem* p, kfbi_mlp* m, const kfbi_data* data, double* x0) {
  if (!p || !m || !data || !x0 || !data->g1) return KFBI_ERR_ARG;
  if (p->nx != p->nb) return fail(p, KFBI_ERR_UNSUPPORTED, "the learned start predicts one density per DOF");
  if (m->n_in != KFBI_WS_FEATURES) return fail(p, KFBI_ERR_ARG, "the network must take KFBI_WS_FEATURES inputs");
  if (m->stream != p->stream) return fail(p, KFBI_ERR_ARG, "network and problem must share a stream");
  if (m->width < KFBI_WS_FEATURES) return fail(p, KFBI_ERR_ARG, "the network width must be >= KFBI_WS_FEATURES");
  const int nb = p->nb;
  {
    kfbi_status s = ensure(m, nb);
    if (s != KFBI_OK) return fail(p, s, m->err);
  }
  // features straight into the network's input scratch, then normalise in place
  KFBI_TRY(kfbi_warm_start_features(p, data, nullptr, m->d1, nullptr));
  const long long tot = (long long)nb * m->n_in;
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_normalise<<<div_up(tot, 256), 256, 0, p->stream>>>(
      nb, m->n_in, m->d1, nullptr, m->shift, m->scale, m->X, nullptr, nullptr));
  {
    kfbi_status s = forward_rows(m, nb, nullptr);
    if (s != KFBI_OK) return fail(p, s, m->err);
  }
  KFBI_LAUNCH(p, KFBI_KC_OTHER, k_to_density<<<div_up(nb, 256), 256, 0, p->stream>>>(nb, m->y, m->out_shift,
                                                                                         m->out_scale, x0));
  KFBI_CUDA(p, cudaGetLastError());
  return KFBI_OK;
}

kfbi_status kfbi_warm_start_batch(kfbi_batch* b, kfbi_mlp* m, const kfbi_data* data, double* const* x0s) {
  if (!b || !m || !data || !x0s) return KFBI_ERR_ARG;
  const int n = batch_size(b);
  kfbi_problem* p0 = batch_problem(b, 0);
  if (m->n_in != KFBI_WS_FEATURES) return fail(p0, KFBI_ERR_ARG, "the network must take KFBI_WS_FEATURES inputs");
  if (m->stream != p0->stream) return fail(p0, KFBI_ERR_ARG, "network and batch must share a stream");
  if (m->width < KFBI_WS_FEATURES) return fail(p0, KFBI_ERR_ARG, "the network width must be >= KFBI_WS_FEATURES");
  std::vector<long long> off(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    kfbi_problem* p = batch_problem(b, k);
    if (!x0s[k] || !data[k].g1) return fail(p0, KFBI_ERR_ARG, "missing data or start for an instance");
    if (p->nx != p->nb) return fail(p0, KFBI_ERR_UNSUPPORTED, "the learned start predicts one density per DOF");
    off[k + 1] = off[k] + p->nb;
  }
  if (off[n] > INT32_MAX / KFBI_WS_FEATURES) return fail(p0, KFBI_ERR_UNSUPPORTED, "too many DOFs in the batch");
  const int rows = (int)off[n];
  {
    kfbi_status s = ensure(m, rows);
    if (s != KFBI_OK) return fail(p0, s, m->err);
  }
  // every instance's features into one matrix, one normalisation and one
  // forward pass over all rows, then each instance's densities
  for (int k = 0; k < n; ++k)
    KFBI_TRY(kfbi_warm_start_features(batch_problem(b, k), &data[k], nullptr, m->d1 + off[k] * m->n_in, nullptr));
  const long long tot = (long long)rows * m->n_in;
  KFBI_LAUNCH(p0, KFBI_KC_OTHER, k_normalise<<<div_up(tot, 256), 256, 0, p0->stream>>>(
      rows, m->n_in, m->d1, nullptr, m->shift, m->scale, m->X, nullptr, nullptr));
  {
    kfbi_status s = forward_rows(m, rows, nullptr);
    if (s != KFBI_OK) return fail(p0, s, m->err);
  }
  for (int k = 0; k < n; ++k) {
    const int nb = batch_problem(b, k)->nb;
    KFBI_LAUNCH(p0, KFBI_KC_OTHER, k_to_density<<<div_up(nb, 256), 256, 0, p0->stream>>>(
        nb, m->y + off[k], m->out_shift, m->out_scale, x0s[k]));
  }
  KFBI_CUDA(p0, cudaGetLastError());
  return KFBI_OK;
}

}  // extern "C"
