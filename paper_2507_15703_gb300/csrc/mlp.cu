// Learned inversion of the angular spectrum: an MLP maps log C_l (l = lmin..lmax)
// to log P_inf at fixed k nodes, standing in for the iterative non-negative
// least-squares inversion of cmb3d_set_spectrum(CMB3D_SPEC_CL).
//
// Training needs no labels: the loss is the method's own forward relation
// (paper Sec. II.A, C_l = sum_j A[l, j] P(k_j) for P linear between nodes),
//     loss = mean over spectra and l of (log (A exp(y))_l - log C_l)^2,
// where y is the network output.  exp keeps P positive.  Steps are Adam with
// the gradient clipped to global norm 1.
//
// Everything runs in this file's kernels: a tcgen05 BF16 x BF16 -> FP32 GEMM
// with strided (so also transposed) FP32 operands and a bias / GELU epilogue,
// elementwise kernels for the loss and the GELU derivative, column sums for
// bias gradients, and Adam on FP32 master weights.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "cmb3d.h"
#include "tcgen05.cuh"

namespace {

constexpr int kTile = 128;                         // output tile 128 x 128
constexpr int kKc = 64;                            // K chunk per MMA round
constexpr uint32_t kLbo = 128, kSbo = (kKc / 8) * 128;
constexpr uint32_t kSpin = 1u << 24;
constexpr float kClip = 1.0f;                      // global gradient-norm clip of the Adam steps
constexpr int kGemmSmem = 48 * 1024;               // 32 KB used; 48 KB caps residency at 4 blocks/SM,
                                                   // so 4 x 128 TMEM columns always fit

// Element (i, j) of a strided FP32 matrix.
struct Mat {
  const float* p;
  long long s0, s1;
};

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143267794f * expf(-0.5f * x * x);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(a))) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(b))) << 16);
}

// out[m, n] = f(alpha sum_k A(m, k) B(n, k) + bias[n]), operands rounded to
// BF16, FP32 accumulation in tensor memory; zout (optional) receives the value
// before the GELU.  One 128-thread block per 128 x 128 output tile.
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, Mat A, Mat B, float alpha,
                                              const float* __restrict__ bias, float* __restrict__ zout,
                                              float* __restrict__ out, long long os0, long long os1, int gelu,
                                              unsigned* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sA = sm;
  unsigned char* sB = sm + kTile * kKc * 2;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t slot;
  const int t = threadIdx.x, warp = t / 32, lane = t % 32;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  if (t == 0) cmb3d::tc::mbar_init(&mbar, 1);
  if (warp == 0) cmb3d::tc::tmem_alloc(&slot, 128);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  cmb3d::tc::fence_before_sync();
  __syncthreads();
  cmb3d::tc::fence_after_sync();
  const uint32_t taddr = slot;
  const uint32_t idesc = cmb3d::tc::idesc_f16(128, 128, true);
  uint32_t phase = 0;
  bool ok = true;
  const int ma = m0 + t, nb = n0 + t;
  for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
    for (int kc = 0; kc < kKc / 8; ++kc) {
      float va[8], vb[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + 8 * kc + e;
        va[e] = (ma < M && k < K) ? A.p[ma * A.s0 + k * A.s1] : 0.f;
        vb[e] = (nb < N && k < K) ? B.p[nb * B.s0 + k * B.s1] : 0.f;
      }
      *reinterpret_cast<uint4*>(sA + cmb3d::tc::kmajor_offset(t, 8 * kc, kLbo, kSbo)) =
          make_uint4(pack_bf16(va[0], va[1]), pack_bf16(va[2], va[3]), pack_bf16(va[4], va[5]), pack_bf16(va[6], va[7]));
      *reinterpret_cast<uint4*>(sB + cmb3d::tc::kmajor_offset(t, 8 * kc, kLbo, kSbo)) =
          make_uint4(pack_bf16(vb[0], vb[1]), pack_bf16(vb[2], vb[3]), pack_bf16(vb[4], vb[5]), pack_bf16(vb[6], vb[7]));
    }
    cmb3d::tc::fence_async_shared();
    cmb3d::tc::fence_before_sync();
    __syncthreads();
    cmb3d::tc::fence_after_sync();
    if (t == 0) {
      const uint32_t a0 = cmb3d::tc::smem_addr(sA), b0 = cmb3d::tc::smem_addr(sB);
#pragma unroll
      for (int ks = 0; ks < kKc / 16; ++ks)
        cmb3d::tc::mma_f16(taddr, cmb3d::tc::smem_desc(a0 + 2 * ks * kLbo, kLbo, kSbo),
                           cmb3d::tc::smem_desc(b0 + 2 * ks * kLbo, kLbo, kSbo), idesc, (k0 > 0 || ks > 0) ? 1u : 0u);
      cmb3d::tc::mma_commit(&mbar);
    }
    if (!cmb3d::tc::mbar_wait(&mbar, phase, kSpin)) ok = false;   // the tile is reused only after the MMAs end
    phase ^= 1u;
    cmb3d::tc::fence_after_sync();
  }
  if (!ok && lane == 0) atomicOr(err, 1u);
  const int m = m0 + 32 * warp + lane;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    float d[32];
    cmb3d::tc::tmem_ld32(taddr + (static_cast<uint32_t>(32 * warp) << 16) + 32u * c, d);
    if (m < M) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = n0 + 32 * c + j;
        if (n < N) {
          float v = alpha * d[j] + (bias ? bias[n] : 0.f);
          if (zout) zout[m * os0 + n * os1] = v;
          out[m * os0 + n * os1] = gelu ? gelu_f(v) : v;
        }
      }
    }
  }
  cmb3d::tc::fence_before_sync();
  __syncthreads();
  cmb3d::tc::fence_after_sync();
  if (warp == 0) cmb3d::tc::tmem_dealloc(taddr, 128);
}

__global__ void k_gather_rows(const float* __restrict__ src, const long long* __restrict__ rows, int B, int d,
                              const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ raw,
                              float* __restrict__ norm) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(B) * d) return;
  const int b = static_cast<int>(i / d), l = static_cast<int>(i % d);
  const float v = src[rows[b] * d + l];
  raw[i] = v;
  norm[i] = (v - mu[l]) / sd[l];
}

// Row maxima of y (B x n): the forward relation is evaluated as the shifted
// log-sum-exp log(A exp(y))_l = ymax + log(A exp(y - ymax))_l, which neither
// overflows nor changes the loss or its gradient.
__global__ void k_rowmax(const float* __restrict__ y, int B, int n, float* __restrict__ ymax) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float m = -INFINITY;
  for (int j = 0; j < n; ++j) m = fmaxf(m, y[static_cast<long long>(b) * n + j]);
  ymax[b] = m;
}

__global__ void k_exp(const float* __restrict__ y, const float* __restrict__ ymax, int n, float* __restrict__ e,
                      long long total) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < total) e[i] = expf(y[i] - ymax[i / n]);
}

// d = log P - log C with log P = ymax + log P'; loss += d^2; dP' = 2 d / (count P')
__global__ void k_loss(const float* __restrict__ P, const float* __restrict__ ymax, int L,
                       const float* __restrict__ logc, long long n, float inv_count, float* __restrict__ dP,
                       double* __restrict__ loss) {
  __shared__ double part[256];
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    const float p = fmaxf(P[i], 1e-30f);
    const float d = logf(p) + ymax[i / L] - logc[i];
    acc = static_cast<double>(d) * d;
    if (dP) dP[i] = 2.0f * d * inv_count / p;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, part[0]);
}

__global__ void k_mul(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ c, long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] * b[i];
}

__global__ void k_gelu_back(const float* __restrict__ dg, const float* __restrict__ z, float* __restrict__ dz,
                            long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dz[i] = dg[i] * gelu_d(z[i]);
}

__global__ void k_colsum(const float* __restrict__ x, int M, int N, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += x[static_cast<long long>(m) * N + n];
  out[n] = s;
}

// Sum of squares of the gradient (for global-norm clipping).
__global__ void k_sqnorm(const float* __restrict__ g, long long n, double* __restrict__ out) {
  __shared__ double part[256];
  double acc = 0.0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    acc += static_cast<double>(g[i]) * g[i];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, part[0]);
}

// Adam with the gradient scaled to global norm <= clip.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2, const double* __restrict__ sqnorm, float clip) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double nrm = sqrt(*sqnorm);
  const float scale = nrm > clip ? static_cast<float>(clip / nrm) : 1.0f;
  const float gi = g[i] * scale;
  const float a = b1 * m1[i] + (1.f - b1) * gi, b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// ---- refinement of a predicted P (cmb3d_mlp_refine) ------------------------
// Minimises f(P) = 1/2 sum_l ((A P)_l / C_l - 1)^2 over P >= 0, the objective
// of the NNLS inversion, by accelerated projected gradient (FISTA) in the
// scaled variable y = P / s, s_j = 1 / || column j of diag(1/C) A ||.

__global__ void k_ref_weights(const float* __restrict__ logc, long long n, float* __restrict__ w,
                              float* __restrict__ w2) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = expf(-logc[i]);
  w[i] = v;
  w2[i] = v * v;
}

__global__ void k_square(const float* __restrict__ a, float* __restrict__ a2, long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a2[i] = a[i] * a[i];
}

// s = 1 / sqrt(column norms^2); the iterate starts at y = P0 / s, and x = s y = P0.
__global__ void k_ref_start(const float* __restrict__ colsq, const float* __restrict__ logp0, long long n,
                            float* __restrict__ sc, float* __restrict__ z, float* __restrict__ y,
                            float* __restrict__ x) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = rsqrtf(fmaxf(colsq[i], 1e-30f));
  const float p0 = expf(logp0[i]);
  sc[i] = s;
  z[i] = p0 / s;
  y[i] = p0 / s;
  x[i] = p0;
}

// The iterate back at the start (after the power iteration used y and x).
__global__ void k_ref_reset(const float* __restrict__ logp0, const float* __restrict__ sc, long long n,
                            float* __restrict__ z, float* __restrict__ y, float* __restrict__ x) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float p0 = expf(logp0[i]);
  z[i] = p0 / sc[i];
  y[i] = p0 / sc[i];
  x[i] = p0;
}

// r = w (w ap - 1) (gradient of f with respect to A P), or with `power` w^2 ap.
__global__ void k_ref_resid(const float* __restrict__ ap, const float* __restrict__ w, long long n, int power,
                            float* __restrict__ r) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float wi = w[i];
  r[i] = power ? wi * wi * ap[i] : wi * fmaf(wi, ap[i], -1.0f);
}

// One row per block: v = s g (the power-iteration image), its norm into lip[b]
// (times 1.05) and, normalised, into y and x = s y.
__global__ void k_ref_power(const float* __restrict__ g, const float* __restrict__ sc, int n_out,
                            float* __restrict__ y, float* __restrict__ x, float* __restrict__ lip) {
  __shared__ float part[256];
  const long long o = static_cast<long long>(blockIdx.x) * n_out;
  float acc = 0.f;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    const float v = sc[o + j] * g[o + j];
    acc += v * v;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) part[threadIdx.x] += part[threadIdx.x + st];
    __syncthreads();
  }
  const float nrm = sqrtf(part[0]);
  if (threadIdx.x == 0) lip[blockIdx.x] = 1.05f * nrm;
  const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    const float v = sc[o + j] * g[o + j] * inv;
    y[o + j] = v;
    x[o + j] = sc[o + j] * v;
  }
}

// FISTA step: z' = max(y - s g / L, 0), y = z' + mom (z' - z), z = z', x = s y.
__global__ void k_ref_step(const float* __restrict__ g, const float* __restrict__ sc, const float* __restrict__ lip,
                           int n_out, long long n, float mom, float* __restrict__ z, float* __restrict__ y,
                           float* __restrict__ x) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = sc[i];
  const float zn = fmaxf(y[i] - s * g[i] / lip[i / n_out], 0.0f);
  const float yn = fmaf(mom, zn - z[i], zn);
  z[i] = zn;
  y[i] = yn;
  x[i] = s * yn;
}

__global__ void k_ref_out(const float* __restrict__ z, const float* __restrict__ sc, long long n,
                          float* __restrict__ pk) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) pk[i] = sc[i] * z[i];
}

unsigned blocks_for(long long n, int threads = 256) { return static_cast<unsigned>((n + threads - 1) / threads); }

thread_local std::string g_mlp_detail;

}  // namespace

struct cmb3d_mlp_s {
  int n_in = 0, width = 0, depth = 0, n_out = 0, cap = 0, device = 0;
  std::vector<long long> w_off, b_off, in_dim, out_dim;
  long long nparam = 0;
  float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;   // params, grads, Adam moments
  float *afwd = nullptr, *mu = nullptr, *sd = nullptr;              // forward matrix n_in x n_out, normalisation
  std::vector<float*> z, act;                                       // per hidden layer: pre-activation, output
  float *xraw = nullptr, *xn = nullptr, *y = nullptr, *e = nullptr, *p = nullptr, *dp = nullptr, *de = nullptr;
  float *dy = nullptr, *dg = nullptr, *dz = nullptr, *ymax = nullptr;
  long long* rows = nullptr;
  double* loss = nullptr;
  double* gnorm = nullptr;
  unsigned* err = nullptr;
  long long step = 0;
  // refinement (cmb3d_mlp_refine), allocated on first use: A (.) A, and per
  // spectrum of a chunk the weights 1/C, column scales, FISTA iterates,
  // Lipschitz bounds and squared norms
  float *a2 = nullptr, *rw = nullptr, *rs = nullptr, *rz = nullptr, *ry = nullptr, *rx = nullptr, *rlip = nullptr;
  float* rnorm = nullptr;
};

namespace {

int mfail(int st, const std::string& msg) {
  g_mlp_detail = msg;
  return st;
}

cudaError_t gemm(cmb3d_mlp_s* h, int M, int N, int K, Mat A, Mat B, float alpha, const float* bias, float* zout,
                 float* out, long long os0, long long os1, bool gelu, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  k_gemm<<<grid, 128, kGemmSmem, s>>>(M, N, K, A, B, alpha, bias, zout, out, os0, os1, gelu ? 1 : 0, h->err);
  return cudaGetLastError();
}

// Forward pass of B normalised rows in h->xn: hidden layers into z/act, output into y.
cudaError_t forward(cmb3d_mlp_s* h, int B, cudaStream_t s) {
  const float* in = h->xn;
  long long ld = h->n_in;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < h->depth && e == cudaSuccess; ++l) {
    e = gemm(h, B, h->width, static_cast<int>(ld), Mat{in, ld, 1}, Mat{h->w + h->w_off[l], ld, 1}, 1.f,
             h->w + h->b_off[l], h->z[l], h->act[l], h->width, 1, true, s);
    in = h->act[l];
    ld = h->width;
  }
  if (e == cudaSuccess)
    e = gemm(h, B, h->n_out, h->width, Mat{in, h->width, 1}, Mat{h->w + h->w_off[h->depth], h->width, 1}, 1.f,
             h->w + h->b_off[h->depth], nullptr, h->y, h->n_out, 1, false, s);
  return e;
}

// Loss of the B rows (raw log C in h->xraw) and, if grads, all parameter gradients into h->g.
cudaError_t loss_and_grad(cmb3d_mlp_s* h, int B, bool grads, cudaStream_t s) {
  const long long ny = static_cast<long long>(B) * h->n_out, np = static_cast<long long>(B) * h->n_in;
  cudaError_t e = forward(h, B, s);
  if (e == cudaSuccess) {
    k_rowmax<<<blocks_for(B, 128), 128, 0, s>>>(h->y, B, h->n_out, h->ymax);
    k_exp<<<blocks_for(ny), 256, 0, s>>>(h->y, h->ymax, h->n_out, h->e, ny);
  }
  // P = E A^T: (B x n_out) times A (n_in x n_out) as the (n = l, k = j) operand
  if (e == cudaSuccess)
    e = gemm(h, B, h->n_in, h->n_out, Mat{h->e, h->n_out, 1}, Mat{h->afwd, h->n_out, 1}, 1.f, nullptr, nullptr, h->p,
             h->n_in, 1, false, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->loss, 0, sizeof(double), s);
  if (e == cudaSuccess)
    k_loss<<<blocks_for(np), 256, 0, s>>>(h->p, h->ymax, h->n_in, h->xraw, np, 1.0f / static_cast<float>(np),
                                          grads ? h->dp : nullptr, h->loss);
  if (e != cudaSuccess || !grads) return e == cudaSuccess ? cudaGetLastError() : e;
  // dE = dP A ; dY = dE * E
  e = gemm(h, B, h->n_out, h->n_in, Mat{h->dp, h->n_in, 1}, Mat{h->afwd, 1, h->n_out}, 1.f, nullptr, nullptr, h->de,
           h->n_out, 1, false, s);
  if (e != cudaSuccess) return e;
  k_mul<<<blocks_for(ny), 256, 0, s>>>(h->de, h->e, h->dy, ny);
  // output layer: dW = dY^T act, db = colsum(dY), dG = dY W
  const int L = h->depth;
  const float* a_in = L > 0 ? h->act[L - 1] : h->xn;
  const long long in_w = L > 0 ? h->width : h->n_in;
  e = gemm(h, h->n_out, static_cast<int>(in_w), B, Mat{h->dy, 1, h->n_out}, Mat{a_in, 1, in_w}, 1.f, nullptr, nullptr,
           h->g + h->w_off[L], in_w, 1, false, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<blocks_for(h->n_out, 128), 128, 0, s>>>(h->dy, B, h->n_out, h->g + h->b_off[L]);
  if (L == 0) return cudaGetLastError();
  e = gemm(h, B, h->width, h->n_out, Mat{h->dy, h->n_out, 1}, Mat{h->w + h->w_off[L], 1, h->width}, 1.f, nullptr,
           nullptr, h->dg, h->width, 1, false, s);
  for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
    const long long nh = static_cast<long long>(B) * h->width;
    k_gelu_back<<<blocks_for(nh), 256, 0, s>>>(h->dg, h->z[l], h->dz, nh);
    const float* xin = l > 0 ? h->act[l - 1] : h->xn;
    const long long iw = l > 0 ? h->width : h->n_in;
    e = gemm(h, h->width, static_cast<int>(iw), B, Mat{h->dz, 1, h->width}, Mat{xin, 1, iw}, 1.f, nullptr, nullptr,
             h->g + h->w_off[l], iw, 1, false, s);
    if (e != cudaSuccess) break;
    k_colsum<<<blocks_for(h->width, 128), 128, 0, s>>>(h->dz, B, h->width, h->g + h->b_off[l]);
    if (l > 0)
      e = gemm(h, B, h->width, h->width, Mat{h->dz, h->width, 1}, Mat{h->w + h->w_off[l], 1, h->width}, 1.f, nullptr,
               nullptr, h->dg, h->width, 1, false, s);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

void free_mlp(cmb3d_mlp_s* h) {
  if (!h) return;
  for (void* p : {static_cast<void*>(h->w), static_cast<void*>(h->g), static_cast<void*>(h->m1),
                  static_cast<void*>(h->m2), static_cast<void*>(h->afwd), static_cast<void*>(h->mu),
                  static_cast<void*>(h->sd), static_cast<void*>(h->xraw), static_cast<void*>(h->xn),
                  static_cast<void*>(h->y), static_cast<void*>(h->e), static_cast<void*>(h->p),
                  static_cast<void*>(h->dp), static_cast<void*>(h->de), static_cast<void*>(h->dy),
                  static_cast<void*>(h->dg), static_cast<void*>(h->dz), static_cast<void*>(h->rows),
                  static_cast<void*>(h->loss), static_cast<void*>(h->err), static_cast<void*>(h->ymax),
                  static_cast<void*>(h->gnorm), static_cast<void*>(h->a2), static_cast<void*>(h->rw),
                  static_cast<void*>(h->rs), static_cast<void*>(h->rz), static_cast<void*>(h->ry),
                  static_cast<void*>(h->rx), static_cast<void*>(h->rlip), static_cast<void*>(h->rnorm)})
    cudaFree(p);
  for (float* p : h->z) cudaFree(p);
  for (float* p : h->act) cudaFree(p);
  delete h;
}

int check_err(cmb3d_mlp_s* h) {
  unsigned v = 0;
  if (cudaMemcpy(&v, h->err, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(CMB3D_ECUDA, "error word read");
  if (v) {
    cudaMemset(h->err, 0, sizeof(unsigned));
    return mfail(CMB3D_ETIMEOUT, "a bounded wait for MMA completion gave up");
  }
  return CMB3D_OK;
}

}  // namespace

extern "C" {

const char* cmb3d_mlp_error_detail(void) { return g_mlp_detail.c_str(); }

int cmb3d_mlp_create(cmb3d_mlp_t* out, int n_in, int width, int depth, int n_out, const double* afwd,
                     const float* mu, const float* sd, const float* out_bias, int batch_cap, uint64_t seed) {
  if (!out) return mfail(CMB3D_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || width < 1 || depth < 0 || depth > 16 || n_out < 1 || !afwd || batch_cap < 1 ||
      batch_cap > (1 << 16) || n_in > (1 << 20) || width > 4096 || n_out > 8192)
    return mfail(CMB3D_EINVAL, "bad MLP shape or NULL forward matrix");
  cmb3d_mlp_s* h = new (std::nothrow) cmb3d_mlp_s;
  if (!h) return mfail(CMB3D_ENOMEM, "host allocation");
  h->n_in = n_in, h->width = width, h->depth = depth, h->n_out = n_out, h->cap = batch_cap;
  cudaGetDevice(&h->device);
  long long off = 0;
  for (int l = 0; l <= depth; ++l) {
    const long long di = l == 0 ? n_in : width, dout = l == depth ? n_out : width;
    h->in_dim.push_back(di);
    h->out_dim.push_back(dout);
    h->w_off.push_back(off);
    off += di * dout;
    h->b_off.push_back(off);
    off += dout;
  }
  h->nparam = off;
  std::vector<float> w(static_cast<size_t>(off), 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l <= depth; ++l) {
    std::normal_distribution<float> nd(0.f, 1.0f / std::sqrt(static_cast<float>(h->in_dim[l])));
    for (long long i = 0; i < h->in_dim[l] * h->out_dim[l]; ++i) w[static_cast<size_t>(h->w_off[l] + i)] = nd(rng);
  }
  if (out_bias)
    for (int j = 0; j < n_out; ++j) w[static_cast<size_t>(h->b_off[depth] + j)] = out_bias[j];
  std::vector<float> a(static_cast<size_t>(n_in) * n_out), m(n_in, 0.f), s(n_in, 1.f);
  for (size_t i = 0; i < a.size(); ++i) a[i] = static_cast<float>(afwd[i]);
  if (mu) std::copy(mu, mu + n_in, m.begin());
  if (sd) std::copy(sd, sd + n_in, s.begin());
  const long long B = batch_cap;
  bool ok = cudaMalloc(&h->w, off * 4) == cudaSuccess && cudaMalloc(&h->g, off * 4) == cudaSuccess &&
            cudaMalloc(&h->m1, off * 4) == cudaSuccess && cudaMalloc(&h->m2, off * 4) == cudaSuccess &&
            cudaMalloc(&h->afwd, a.size() * 4) == cudaSuccess && cudaMalloc(&h->mu, n_in * 4) == cudaSuccess &&
            cudaMalloc(&h->sd, n_in * 4) == cudaSuccess && cudaMalloc(&h->xraw, B * n_in * 4) == cudaSuccess &&
            cudaMalloc(&h->xn, B * n_in * 4) == cudaSuccess && cudaMalloc(&h->y, B * n_out * 4) == cudaSuccess &&
            cudaMalloc(&h->e, B * n_out * 4) == cudaSuccess && cudaMalloc(&h->p, B * n_in * 4) == cudaSuccess &&
            cudaMalloc(&h->dp, B * n_in * 4) == cudaSuccess && cudaMalloc(&h->de, B * n_out * 4) == cudaSuccess &&
            cudaMalloc(&h->dy, B * n_out * 4) == cudaSuccess && cudaMalloc(&h->dg, B * width * 4) == cudaSuccess &&
            cudaMalloc(&h->dz, B * width * 4) == cudaSuccess && cudaMalloc(&h->rows, B * 8) == cudaSuccess &&
            cudaMalloc(&h->loss, 8) == cudaSuccess && cudaMalloc(&h->err, 4) == cudaSuccess &&
            cudaMalloc(&h->ymax, B * 4) == cudaSuccess && cudaMalloc(&h->gnorm, 8) == cudaSuccess;
  for (int l = 0; l < depth && ok; ++l) {
    float *zl = nullptr, *al = nullptr;
    ok = cudaMalloc(&zl, B * width * 4) == cudaSuccess && cudaMalloc(&al, B * width * 4) == cudaSuccess;
    h->z.push_back(zl);
    h->act.push_back(al);
  }
  ok = ok && cudaMemcpy(h->w, w.data(), off * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->m1, 0, off * 4) == cudaSuccess && cudaMemset(h->m2, 0, off * 4) == cudaSuccess &&
       cudaMemset(h->g, 0, off * 4) == cudaSuccess && cudaMemset(h->err, 0, 4) == cudaSuccess &&
       cudaMemcpy(h->afwd, a.data(), a.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->mu, m.data(), n_in * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->sd, s.data(), n_in * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_mlp(h);
    return mfail(CMB3D_ENOMEM, "device allocation or upload of the MLP");
  }
  *out = h;
  return CMB3D_OK;
}

int cmb3d_mlp_loss_grad(cmb3d_mlp_t h, const float* logcl_dev, int64_t n, double* loss_host, float* grad_dev,
                        void* stream) {
  if (!h || !logcl_dev || n < 1 || n > h->cap || !loss_host) return mfail(CMB3D_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<long long> rows(static_cast<size_t>(n));
  for (long long i = 0; i < n; ++i) rows[static_cast<size_t>(i)] = i;
  cudaError_t e = cudaMemcpyAsync(h->rows, rows.data(), n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_gather_rows<<<blocks_for(n * h->n_in), 256, 0, s>>>(logcl_dev, h->rows, static_cast<int>(n), h->n_in, h->mu,
                                                         h->sd, h->xraw, h->xn);
    e = loss_and_grad(h, static_cast<int>(n), grad_dev != nullptr, s);
  }
  double l = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_dev) e = cudaMemcpyAsync(grad_dev, h->g, h->nparam * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
  *loss_host = l / (static_cast<double>(n) * h->n_in);
  return check_err(h);
}

int cmb3d_mlp_train(cmb3d_mlp_t h, const float* logcl_dev, int64_t n, int epochs, int batch, float lr, uint64_t seed,
                    float* epoch_loss_host, void* stream) {
  if (!h || !logcl_dev || n < 1 || epochs < 0 || batch < 1 || batch > h->cap || !(lr > 0))
    return mfail(CMB3D_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::mt19937_64 rng(seed);
  std::vector<long long> perm(static_cast<size_t>(n));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (long long i = 0; i < n; ++i) perm[static_cast<size_t>(i)] = i;
    std::shuffle(perm.begin(), perm.end(), rng);
    double sum = 0.0;
    long long seen = 0;
    for (long long b0 = 0; b0 + batch <= n; b0 += batch) {
      cudaError_t e = cudaMemcpyAsync(h->rows, perm.data() + b0, static_cast<size_t>(batch) * 8,
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
      k_gather_rows<<<blocks_for(static_cast<long long>(batch) * h->n_in), 256, 0, s>>>(
          logcl_dev, h->rows, batch, h->n_in, h->mu, h->sd, h->xraw, h->xn);
      e = loss_and_grad(h, batch, true, s);
      if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
      ++h->step;
      const float c1 = 1.f - std::pow(b1, static_cast<float>(h->step)), c2 = 1.f - std::pow(b2, static_cast<float>(h->step));
      e = cudaMemsetAsync(h->gnorm, 0, sizeof(double), s);
      if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
      k_sqnorm<<<304, 256, 0, s>>>(h->g, h->nparam, h->gnorm);
      k_adam<<<blocks_for(h->nparam), 256, 0, s>>>(h->w, h->g, h->m1, h->m2, h->nparam, lr, b1, b2, eps, c1, c2,
                                                     h->gnorm, kClip);
      double l = 0.0;
      e = cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
      sum += l;
      seen += batch;
    }
    if (epoch_loss_host) epoch_loss_host[ep] = static_cast<float>(sum / (static_cast<double>(seen) * h->n_in));
  }
  return check_err(h);
}

int cmb3d_mlp_predict(cmb3d_mlp_t h, const float* logcl_dev, int64_t n, float* logpk_dev, void* stream) {
  if (!h || n < 0 || (n > 0 && (!logcl_dev || !logpk_dev))) return mfail(CMB3D_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<long long> rows(static_cast<size_t>(h->cap));
  for (long long b0 = 0; b0 < n; b0 += h->cap) {
    const int B = static_cast<int>(std::min<long long>(h->cap, n - b0));
    for (int i = 0; i < B; ++i) rows[static_cast<size_t>(i)] = b0 + i;
    cudaError_t e = cudaMemcpyAsync(h->rows, rows.data(), static_cast<size_t>(B) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_gather_rows<<<blocks_for(static_cast<long long>(B) * h->n_in), 256, 0, s>>>(logcl_dev, h->rows, B, h->n_in,
                                                                                   h->mu, h->sd, h->xraw, h->xn);
      e = forward(h, B, s);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(logpk_dev + b0 * h->n_out, h->y, static_cast<size_t>(B) * h->n_out * 4,
                          cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // rows[] is reused by the next chunk
    if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
  }
  return check_err(h);
}

int cmb3d_mlp_params(cmb3d_mlp_t h, float* get_host, const float* set_host, int64_t* count) {
  if (!h) return mfail(CMB3D_EINVAL, "NULL MLP");
  if (count) *count = h->nparam;
  if (get_host && cudaMemcpy(get_host, h->w, h->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(CMB3D_ECUDA, "parameter read");
  if (set_host && cudaMemcpy(h->w, set_host, h->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return mfail(CMB3D_ECUDA, "parameter write");
  return CMB3D_OK;
}

void cmb3d_mlp_destroy(cmb3d_mlp_t h) { free_mlp(h); }

int cmb3d_mlp_refine(cmb3d_mlp_t h, const float* logcl_dev, const float* logpk_dev, int64_t n, int iters,
                     int power_iters, float* pk_dev, void* stream) {
  if (!h || n < 0 || iters < 0 || power_iters < 1 || (n > 0 && (!logcl_dev || !logpk_dev || !pk_dev)))
    return mfail(CMB3D_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long cap = h->cap, ni = h->n_in, no = h->n_out;
  if (!h->a2) {
    bool ok = cudaMalloc(&h->a2, ni * no * 4) == cudaSuccess && cudaMalloc(&h->rw, cap * ni * 4) == cudaSuccess &&
              cudaMalloc(&h->rs, cap * no * 4) == cudaSuccess && cudaMalloc(&h->rz, cap * no * 4) == cudaSuccess &&
              cudaMalloc(&h->ry, cap * no * 4) == cudaSuccess && cudaMalloc(&h->rx, cap * no * 4) == cudaSuccess &&
              cudaMalloc(&h->rlip, cap * 4) == cudaSuccess && cudaMalloc(&h->rnorm, cap * ni * 4) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return mfail(CMB3D_ENOMEM, "refinement buffers");
    }
    k_square<<<blocks_for(ni * no), 256, 0, s>>>(h->afwd, h->a2, ni * no);
  }
  const Mat a_t{h->afwd, no, 1};          // (n = l, k = j): A[l][j]
  const Mat a_n{h->afwd, 1, no};          // (n = j, k = l): A[l][j]
  for (long long b0 = 0; b0 < n; b0 += cap) {
    const int B = static_cast<int>(std::min(cap, n - b0));
    const long long nb_in = static_cast<long long>(B) * ni, nb_out = static_cast<long long>(B) * no;
    const float* lc = logcl_dev + b0 * ni;
    float* w2 = h->rnorm;
    k_ref_weights<<<blocks_for(nb_in), 256, 0, s>>>(lc, nb_in, h->rw, w2);
    // squared column norms of diag(1/C) A: (w^2) (A . A)
    cudaError_t e = gemm(h, B, static_cast<int>(no), static_cast<int>(ni), Mat{w2, ni, 1}, Mat{h->a2, 1, no}, 1.f,
                         nullptr, nullptr, h->de, no, 1, false, s);
    if (e == cudaSuccess)
      k_ref_start<<<blocks_for(nb_out), 256, 0, s>>>(h->de, logpk_dev + b0 * no, nb_out, h->rs, h->rz, h->ry, h->rx);
    // Lipschitz bound of the scaled gradient: power iteration on S A^T W^2 A S
    // from x = P0 (y and x serve as the iteration vector, then are reset)
    for (int it = 0; it < power_iters && e == cudaSuccess; ++it) {
      e = gemm(h, B, static_cast<int>(ni), static_cast<int>(no), Mat{h->rx, no, 1}, a_t, 1.f, nullptr, nullptr, h->p,
               ni, 1, false, s);
      if (e != cudaSuccess) break;
      k_ref_resid<<<blocks_for(nb_in), 256, 0, s>>>(h->p, h->rw, nb_in, 1, h->dp);
      e = gemm(h, B, static_cast<int>(no), static_cast<int>(ni), Mat{h->dp, ni, 1}, a_n, 1.f, nullptr, nullptr, h->de,
               no, 1, false, s);
      if (e != cudaSuccess) break;
      k_ref_power<<<B, 256, 0, s>>>(h->de, h->rs, static_cast<int>(no), h->ry, h->rx, h->rlip);
    }
    if (e == cudaSuccess) k_ref_reset<<<blocks_for(nb_out), 256, 0, s>>>(logpk_dev + b0 * no, h->rs, nb_out, h->rz, h->ry, h->rx);
    double t = 1.0;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
      e = gemm(h, B, static_cast<int>(ni), static_cast<int>(no), Mat{h->rx, no, 1}, a_t, 1.f, nullptr, nullptr, h->p,
               ni, 1, false, s);
      if (e != cudaSuccess) break;
      k_ref_resid<<<blocks_for(nb_in), 256, 0, s>>>(h->p, h->rw, nb_in, 0, h->dp);
      e = gemm(h, B, static_cast<int>(no), static_cast<int>(ni), Mat{h->dp, ni, 1}, a_n, 1.f, nullptr, nullptr, h->de,
               no, 1, false, s);
      if (e != cudaSuccess) break;
      const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
      k_ref_step<<<blocks_for(nb_out), 256, 0, s>>>(h->de, h->rs, h->rlip, static_cast<int>(no), nb_out,
                                                    static_cast<float>((t - 1.0) / tn), h->rz, h->ry, h->rx);
      t = tn;
    }
    if (e == cudaSuccess) k_ref_out<<<blocks_for(nb_out), 256, 0, s>>>(h->rz, h->rs, nb_out, pk_dev + b0 * no);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return mfail(CMB3D_ECUDA, "refinement");
  return check_err(h);
}

int cmb3d_mlp_gemm(int M, int N, int K, const float* a, int64_t as0, int64_t as1, const float* b, int64_t bs0,
                   int64_t bs1, float alpha, const float* bias, int gelu, float* out, int64_t os0, int64_t os1,
                   void* stream) {
  if (M < 1 || N < 1 || K < 1 || !a || !b || !out) return mfail(CMB3D_EINVAL, "bad GEMM shape or NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* err = nullptr;
  if (cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return mfail(CMB3D_ENOMEM, "error word");
  }
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  if (e == cudaSuccess) {
    dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    k_gemm<<<grid, 128, kGemmSmem, s>>>(M, N, K, Mat{a, as0, as1}, Mat{b, bs0, bs1}, alpha, bias, nullptr, out, os0,
                                        os1, gelu ? 1 : 0, err);
    e = cudaGetLastError();
  }
  unsigned v = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, err, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  if (e != cudaSuccess) return mfail(CMB3D_ECUDA, cudaGetErrorString(e));
  if (v) return mfail(CMB3D_ETIMEOUT, "a bounded wait for MMA completion gave up");
  return CMB3D_OK;
}

}  // extern "C"
