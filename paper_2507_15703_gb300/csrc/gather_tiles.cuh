// Interpolation of the box field at one pixel (paper Sec. II.D.1), shared by
// the gather kernel (gather.cu) and the persistent batch kernel (batch.cu).
// Trilinear (2x2x2 taps) or Keys cubic convolution with a = -1/2 (4x4x4
// taps), periodic wrap.  The table entry holds the FP32 fractions and the base
// cell packed as bx | by << 11 | (bz & 1023) << 22 with bit 10 of bz in the
// sign of tz.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cmb3d {

template <int INTERP>
struct Weights;

template <>
struct Weights<1> {
  static constexpr int K = 2, OFF = 0;
  static __device__ __forceinline__ void run(float t, float* w) {
    w[0] = 1.0f - t;
    w[1] = t;
  }
};

template <>
struct Weights<3> {
  static constexpr int K = 4, OFF = -1;
  // Keys (1981) cubic convolution, a = -1/2, taps -1, 0, 1, 2.
  static __device__ __forceinline__ void run(float t, float* w) {
    const float t2 = t * t;
    w[0] = 0.5f * fmaf(2.0f - t, t, -1.0f) * t;
    w[1] = 0.5f * fmaf(fmaf(3.0f, t, -5.0f), t2, 2.0f);
    w[2] = 0.5f * fmaf(fmaf(-3.0f, t, 4.0f), t, 1.0f) * t;
    w[3] = 0.5f * (t - 1.0f) * t2;
  }
};

// Value at table entry e; `load(p)` reads one float of the field.
// One 64-bit pointer per z-plane of the stencil and 32-bit offsets within the
// plane (N^2 < 2^32); when the x-window does not wrap, the K taps of a row are
// loads from one address with immediate offsets.
template <int INTERP, class Load>
__device__ __forceinline__ float interpolate(const float* __restrict__ field, float4 e, int N, Load load) {
  using W = Weights<INTERP>;
  const uint32_t pk = __float_as_uint(e.w);
  const uint32_t bx = pk & 2047u, by = (pk >> 11) & 2047u;
  const uint32_t bz = (pk >> 22) | ((__float_as_uint(e.z) >> 31) << 10);
  const uint32_t n = static_cast<uint32_t>(N), m = n - 1u;
  float wx[W::K], wy[W::K], wz[W::K];
  W::run(e.x, wx);
  W::run(e.y, wy);
  W::run(fabsf(e.z), wz);
  uint32_t ro[W::K];                                   // row offsets within a z-plane
#pragma unroll
  for (int b = 0; b < W::K; ++b) ro[b] = ((by + static_cast<uint32_t>(b + W::OFF)) & m) * n;
  const uint32_t x0 = bx + static_cast<uint32_t>(W::OFF);   // wraps to 2^32-1 for bx = 0, OFF = -1
  auto run = [&](auto row_sum) {
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < W::K; ++c) {
      const float* plane = field + static_cast<size_t>((bz + static_cast<uint32_t>(c + W::OFF)) & m) * n * n;
      float accz = 0.0f;
#pragma unroll
      for (int b = 0; b < W::K; ++b) accz = fmaf(wy[b], row_sum(plane, ro[b]), accz);
      acc = fmaf(wz[c], accz, acc);
    }
    return acc;
  };
  if (x0 <= n - static_cast<uint32_t>(W::K)) {
    return run([&](const float* plane, uint32_t r) {
      const float* p = plane + (r + x0);
      float s = 0.0f;
#pragma unroll
      for (int a = 0; a < W::K; ++a) s = fmaf(wx[a], load(p + a), s);
      return s;
    });
  }
  return run([&](const float* plane, uint32_t r) {
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < W::K; ++a) s = fmaf(wx[a], load(plane + r + ((bx + static_cast<uint32_t>(a + W::OFF)) & m)), s);
    return s;
  });
}

}  // namespace cmb3d
