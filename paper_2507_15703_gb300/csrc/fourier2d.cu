// Draw of the 2-D Fourier method (paper Sec. II.D.2): the hybrid layers
// T^(m_x, m_y, z_j), j < h, Fourier space in x and y, real space in z.  For
// each (m_x, m_y) the h values are S c, with S the symmetric square root of
// the z-covariance of that (m_x, m_y) (a host table indexed by
// q = m_x^2 + m_y^2) and c normals from the mode's own Philox counters
// (m_x, m_y, i / 2, 1), i < h: words (0, 1) for even i, (2, 3) for odd i,
// Box-Muller (g1, g2), c_i = (g1 + i g2) / sqrt 2.
//
// Hermitian symmetry of the real layers: on m_x in {0, N/2} the mode with the
// smaller m_y of the pair (m_y, -m_y mod N) draws and its partner takes the
// conjugate; self-conjugate modes (m_y in {0, N/2}) are real, S g1.  The
// output is packed like the 3-D half spectrum, [z][m_y][m_x'] with m_x' < N/2
// and slot m_x' = 0 holding T^(0, m_y, z) + i T^(N/2, m_y, z), so the 3-D
// method's y and x passes turn it into real layers.
#include "device_common.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

constexpr float kRsqrt2 = 0.70710678118654752f;

// Normals of mode (mx, my): c[i] = (g1 + i g2) / sqrt 2, or (g1, 0) when real.
template <int HM>
__device__ __forceinline__ void mode_normals(int mx, int my, int h, uint2 key, bool real, float2 (&c)[HM]) {
#pragma unroll
  for (int ip = 0; ip < HM / 2; ++ip) {
    if (2 * ip < h) {
      const uint4 w = philox4x32_10(make_uint4(mx, my, ip, 1u), key);
      const float2 ga = box_muller(w.x, w.y), gb = box_muller(w.z, w.w);
      c[2 * ip] = real ? make_float2(ga.x, 0.f) : make_float2(ga.x * kRsqrt2, ga.y * kRsqrt2);
      c[2 * ip + 1] = real ? make_float2(gb.x, 0.f) : make_float2(gb.x * kRsqrt2, gb.y * kRsqrt2);
    }
  }
}

// Row z of S times c (complex vector, real matrix).
template <int HM>
__device__ __forceinline__ float2 row_times(const float* __restrict__ S, int z, int h, const float2 (&c)[HM]) {
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < HM; ++i) {
    if (i < h) {
      const float sz = __ldg(S + z * h + i);
      acc.x = fmaf(sz, c[i].x, acc.x);
      acc.y = fmaf(sz, c[i].y, acc.y);
    }
  }
  return acc;
}

// The h values of a mode on a Hermitian line m_x in {0, N/2}, into v.
template <int HM>
__device__ __forceinline__ void hermitian_mode(int mx, int my, int N, int h, const float* __restrict__ tab,
                                               uint2 key, float2 (&v)[HM]) {
  const int py = (N - my) & (N - 1);
  const int fy = my <= N / 2 ? my : my - N;
  const float* S = tab + static_cast<size_t>(mx * mx + fy * fy) * h * h;
  float2 c[HM];
  const bool self = py == my, own = my < py;
  mode_normals<HM>(mx, self || own ? my : py, h, key, self, c);
#pragma unroll
  for (int z = 0; z < HM; ++z) {
    if (z < h) {
      const float2 a = row_times<HM>(S, z, h, c);
      v[z] = own || self ? a : make_float2(a.x, -a.y);
    }
  }
}

template <int HM>
__global__ void __launch_bounds__(256) k_draw2d(float2* __restrict__ buf, const float* __restrict__ tab, int N,
                                                int h, uint2 key) {
  const int N2 = N / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N2 * N) return;
  const int xp = t % N2, my = t / N2;
  float2* out = buf + static_cast<size_t>(my) * N2 + xp;       // (z, my, xp) at out[z N N2]
  const size_t plane = static_cast<size_t>(N) * N2;
  if (xp > 0) {
    const int fy = my <= N2 ? my : my - N;
    const float* S = tab + static_cast<size_t>(xp * xp + fy * fy) * h * h;
    float2 c[HM];
    mode_normals<HM>(xp, my, h, key, false, c);
#pragma unroll
    for (int z = 0; z < HM; ++z)
      if (z < h) out[z * plane] = row_times<HM>(S, z, h, c);
    return;
  }
  float2 a[HM], b[HM];
  hermitian_mode<HM>(0, my, N, h, tab, key, a);
  hermitian_mode<HM>(N2, my, N, h, tab, key, b);
#pragma unroll
  for (int z = 0; z < HM; ++z)
    if (z < h) out[z * plane] = make_float2(a[z].x - b[z].y, a[z].y + b[z].x);
}

template <int HM>
cudaError_t run_draw2d(int N, int h, float2* buf, const float* tab, uint2 key, cudaStream_t s) {
  const int n = N / 2 * N;
  k_draw2d<HM><<<(n + 255) / 256, 256, 0, s>>>(buf, tab, N, h, key);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_draw2d(int N, int h, float2* buf, const float* tab, uint64_t seed, cudaStream_t s) {
  if (N < 16 || (N & (N - 1)) || h < 1 || h > 32) return cudaErrorInvalidValue;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
  if (h <= 8) return run_draw2d<8>(N, h, buf, tab, key, s);
  if (h <= 16) return run_draw2d<16>(N, h, buf, tab, key, s);
  return run_draw2d<32>(N, h, buf, tab, key, s);
}

}  // namespace cmb3d
