// The three passes of the inverse real 3-D FFT of one box realization, with
// the Gaussian draw of the Fourier coefficients fused into the first pass
// (paper Sec. II.D.1: every mode of the box receives a zero-mean complex normal
// number whose variance is the box power at |k|, and the inverse FFT of that
// array is the simulated field).
//
// Data layout in HBM: one packed half spectrum float2 [N][N][N/2] (4 N^3
// bytes), transformed in place:
//   pass 1  draw + FFT along z   columns (m_y, m_x'), tiles of T adjacent m_x'
//   pass 2  FFT along y          columns (z, m_x'),   tiles of T adjacent m_x'
//   pass 3  C2R FFT along x      rows (z, y) -> N reals float [z][y][x]
// The Hermitian planes m_x = 0 and m_x = N/2 both transform to real (y, z)
// planes, so they share the m_x' = 0 slot as T(0,.) + i T(N/2,.), which keeps
// every row a power of two long and the buffer exactly the size of the field.
#include "device_common.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

// Fourier coefficient of mode (mx, my, mz) on a Hermitian plane mx in {0, N/2}:
// the mode with the smaller index mz N + my of a conjugate pair draws from its
// own counter and its partner takes the conjugate; self-conjugate modes are
// real with variance P_box; the DC mode is zero.
template <int N>
__device__ __forceinline__ float2 draw_hermitian(int mx, int my, int mz, const float* __restrict__ amp,
                                                 uint2 key) {
  const int py = (N - my) & (N - 1), pz = (N - mz) & (N - 1);
  const int lin = mz * N + my, plin = pz * N + py;
  const int fy = my <= N / 2 ? my : my - N, fz = mz <= N / 2 ? mz : mz - N;
  const int q = mx * mx + fy * fy + fz * fz;
  const float a = __ldg(amp + q);
  if (lin == plin) {
    if (q == 0) return make_float2(0.f, 0.f);
    const uint4 w = philox4x32_10(make_uint4(mx >> 1, my, mz, 0u), key);
    const float2 g = box_muller(w.x, w.y);
    return make_float2(a * 1.41421356237309505f * g.x, 0.f);
  }
  const bool canon = lin < plin;
  const uint4 w = philox4x32_10(make_uint4(mx >> 1, canon ? my : py, canon ? mz : pz, 0u), key);
  const float2 g = box_muller(w.x, w.y);          // mx is even on both planes
  return make_float2(a * g.x, canon ? a * g.y : -a * g.y);
}

// Entry (m_x', m_y, m_z) of the packed half spectrum.
template <int N>
__device__ __forceinline__ float2 draw_packed(int xp, int my, int mz, const float* __restrict__ amp,
                                              uint2 key) {
  if (xp == 0) {
    const float2 A = draw_hermitian<N>(0, my, mz, amp, key);
    const float2 B = draw_hermitian<N>(N / 2, my, mz, amp, key);
    return make_float2(A.x - B.y, A.y + B.x);
  }
  const int fy = my <= N / 2 ? my : my - N, fz = mz <= N / 2 ? mz : mz - N;
  const int q = xp * xp + fy * fy + fz * fz;
  const float a = __ldg(amp + q);
  const uint4 w = philox4x32_10(make_uint4(xp >> 1, my, mz, 0u), key);
  const float2 g = (xp & 1) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
  return make_float2(a * g.x, a * g.y);
}

template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_draw_zfft(float2* __restrict__ buf, const float* __restrict__ amp,
                                                         const float2* __restrict__ tw, uint2 key) {
  constexpr int N2 = N / 2, NB = N / R;
  extern __shared__ float2 sm[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int xp = blockIdx.x * T + c;
  const int my = blockIdx.y;
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = draw_packed<N>(xp, my, j + r * NB, amp, key);
  float2* col = buf + static_cast<size_t>(my) * N2 + xp;   // (z, my, xp) at col[z N N2]
  stockham<N, R, N, false>(
      v, sm, tw, j, [&](int n) { return n * T + c; },
      [&](int n, float2 x) { col[static_cast<size_t>(n) * N * N2] = x; }, BlockSync{});
}

template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_yfft(float2* __restrict__ buf, const float2* __restrict__ tw) {
  constexpr int N2 = N / 2, NB = N / R;
  extern __shared__ float2 sm[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int xp = blockIdx.x * T + c;
  float2* col = buf + static_cast<size_t>(blockIdx.y) * N * N2 + xp;   // (z, y, xp) at col[y N2]
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = col[static_cast<size_t>(j + r * NB) * N2];
  stockham<N, R, N, false>(
      v, sm, tw, j, [&](int n) { return n * T + c; },
      [&](int n, float2 x) { col[static_cast<size_t>(n) * N2] = x; }, BlockSync{});
}

// Row pass: for k in [0, N/2) the half-length input is
//   Y[k] = (G[k] + conj(G[N/2-k])) + i w^k (G[k] - conj(G[N/2-k])),  w = e^{2 pi i/N},
// with G[0], G[N/2] the real and imaginary parts of the packed entry 0, so that
// the N/2-point inverse FFT y[n] = f(2n) + i f(2n+1) is the real row itself.
template <int N, int R, int ROWS>
__global__ void __launch_bounds__(ROWS*(N / 2 / R)) k_xc2r(float2* __restrict__ buf, const float2* __restrict__ tw) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int P = N2 + (N2 >> 4);            // row pitch: one pad slot per 16 entries
  extern __shared__ float2 sm[];
  const int j = threadIdx.x % NB, rl = threadIdx.x / NB;
  float2* g = buf + (static_cast<size_t>(blockIdx.x) * ROWS + rl) * N2;
  auto sidx = [&](int n) { return rl * P + n + (n >> 4); };
  for (int i = j; i < N2; i += NB) sm[sidx(i)] = g[i];
  __syncthreads();
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = j + r * NB;
    if (k == 0) {
      const float2 p = sm[sidx(0)];
      v[r] = make_float2(p.x + p.y, p.x - p.y);
    } else {
      const float2 a = sm[sidx(k)], b = cconj(sm[sidx(N2 - k)]);
      v[r] = cadd(cadd(a, b), cmul_i(cmul(__ldg(tw + k), csub(a, b))));
    }
  }
  stockham<N2, R, N, true>(v, sm, tw, j, sidx, [&](int n, float2 x) { g[n] = x; }, BlockSync{});
}

template <int N, int R, int T>
cudaError_t run_draw_zfft(float2* buf, const float* amp, const float2* tw, uint2 key, cudaStream_t s) {
  const size_t smem = sizeof(float2) * N * T;
  auto kern = k_draw_zfft<N, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N / 2 / T, N), T * (N / R), smem, s>>>(buf, amp, tw, key);
  return cudaGetLastError();
}

template <int N, int R, int T>
cudaError_t run_yfft(float2* buf, const float2* tw, cudaStream_t s) {
  const size_t smem = sizeof(float2) * N * T;
  auto kern = k_yfft<N, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N / 2 / T, N), T * (N / R), smem, s>>>(buf, tw);
  return cudaGetLastError();
}

template <int N, int R>
cudaError_t run_xc2r(float2* buf, const float2* tw, cudaStream_t s) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int ROWS0 = 256 / NB > 0 ? 256 / NB : 1;
  constexpr int ROWS = ROWS0 < N * N ? ROWS0 : N * N;
  constexpr int P = N2 + (N2 >> 4);
  const size_t smem = sizeof(float2) * P * ROWS;
  auto kern = k_xc2r<N, R, ROWS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N * N / ROWS), ROWS * NB, smem, s>>>(buf, tw);
  return cudaGetLastError();
}

// Diagnostic: the packed half spectrum [m_z][m_y][m_x'] with no transform.
template <int N>
__global__ void k_draw_only(float2* __restrict__ buf, const float* __restrict__ amp, uint2 key) {
  constexpr int N2 = N / 2;
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<size_t>(N) * N * N2) return;
  const int xp = static_cast<int>(i % N2), my = static_cast<int>((i / N2) % N), mz = static_cast<int>(i / (static_cast<size_t>(N2) * N));
  buf[i] = draw_packed<N>(xp, my, mz, amp, key);
}

template <int N>
cudaError_t run_draw_only(float2* buf, const float* amp, uint2 key, cudaStream_t s) {
  const size_t n = static_cast<size_t>(N) * N * (N / 2);
  k_draw_only<N><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(buf, amp, key);
  return cudaGetLastError();
}

inline uint2 key_of(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
}

}  // namespace

// Column-pass shapes (radix R, tile width T) and row-pass radix per box size.
cudaError_t launch_draw_zfft(int N, float2* buf, const float* amp, const float2* tw, uint64_t seed,
                             cudaStream_t s) {
  const uint2 key = key_of(seed);
  switch (N) {
    case 8: return run_draw_zfft<8, 8, 4>(buf, amp, tw, key, s);
    case 16: return run_draw_zfft<16, 8, 8>(buf, amp, tw, key, s);
    case 32: return run_draw_zfft<32, 8, 16>(buf, amp, tw, key, s);
    case 64: return run_draw_zfft<64, 8, 16>(buf, amp, tw, key, s);
    case 128: return run_draw_zfft<128, 8, 16>(buf, amp, tw, key, s);
    case 256: return run_draw_zfft<256, 8, 16>(buf, amp, tw, key, s);
    case 512: return run_draw_zfft<512, 8, 16>(buf, amp, tw, key, s);
    case 1024: return run_draw_zfft<1024, 16, 16>(buf, amp, tw, key, s);
    case 2048: return run_draw_zfft<2048, 16, 8>(buf, amp, tw, key, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_draw_only(int N, float2* buf, const float* amp, uint64_t seed, cudaStream_t s) {
  const uint2 key = key_of(seed);
  switch (N) {
    case 8: return run_draw_only<8>(buf, amp, key, s);
    case 16: return run_draw_only<16>(buf, amp, key, s);
    case 32: return run_draw_only<32>(buf, amp, key, s);
    case 64: return run_draw_only<64>(buf, amp, key, s);
    case 128: return run_draw_only<128>(buf, amp, key, s);
    case 256: return run_draw_only<256>(buf, amp, key, s);
    case 512: return run_draw_only<512>(buf, amp, key, s);
    case 1024: return run_draw_only<1024>(buf, amp, key, s);
    case 2048: return run_draw_only<2048>(buf, amp, key, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_yfft(int N, float2* buf, const float2* tw, cudaStream_t s) {
  switch (N) {
    case 8: return run_yfft<8, 8, 4>(buf, tw, s);
    case 16: return run_yfft<16, 8, 8>(buf, tw, s);
    case 32: return run_yfft<32, 8, 16>(buf, tw, s);
    case 64: return run_yfft<64, 8, 16>(buf, tw, s);
    case 128: return run_yfft<128, 8, 16>(buf, tw, s);
    case 256: return run_yfft<256, 8, 16>(buf, tw, s);
    case 512: return run_yfft<512, 8, 16>(buf, tw, s);
    case 1024: return run_yfft<1024, 16, 16>(buf, tw, s);
    case 2048: return run_yfft<2048, 16, 8>(buf, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xc2r(int N, float2* buf, const float2* tw, cudaStream_t s) {
  switch (N) {
    case 8: return run_xc2r<8, 4>(buf, tw, s);
    case 16: return run_xc2r<16, 8>(buf, tw, s);
    case 32: return run_xc2r<32, 8>(buf, tw, s);
    case 64: return run_xc2r<64, 8>(buf, tw, s);
    case 128: return run_xc2r<128, 8>(buf, tw, s);
    case 256: return run_xc2r<256, 8>(buf, tw, s);
    case 512: return run_xc2r<512, 8>(buf, tw, s);
    case 1024: return run_xc2r<1024, 8>(buf, tw, s);
    case 2048: return run_xc2r<2048, 16>(buf, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cmb3d
