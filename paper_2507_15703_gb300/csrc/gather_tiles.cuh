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
    w[0] = 0.5f * ((2.0f - t) * t - 1.0f) * t;
    w[1] = 0.5f * ((3.0f * t - 5.0f) * t2 + 2.0f);
    w[2] = 0.5f * (((4.0f - 3.0f * t) * t) + 1.0f) * t;
    w[3] = 0.5f * (t - 1.0f) * t2;
  }
};

// Value at table entry e; `load(p)` reads one float of the field.
template <int INTERP, class Load>
__device__ __forceinline__ float interpolate(const float* __restrict__ field, float4 e, int N, Load load) {
  using W = Weights<INTERP>;
  const uint32_t pk = __float_as_uint(e.w);
  const uint32_t bx = pk & 2047u, by = (pk >> 11) & 2047u;
  const uint32_t bz = (pk >> 22) | ((__float_as_uint(e.z) >> 31) << 10);
  const uint32_t m = static_cast<uint32_t>(N) - 1u;
  float wx[W::K], wy[W::K], wz[W::K];
  W::run(e.x, wx);
  W::run(e.y, wy);
  W::run(fabsf(e.z), wz);
  uint32_t xs[W::K];
#pragma unroll
  for (int a = 0; a < W::K; ++a) xs[a] = (bx + static_cast<uint32_t>(a + W::OFF)) & m;
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < W::K; ++c) {
    const size_t zrow = static_cast<size_t>((bz + static_cast<uint32_t>(c + W::OFF)) & m) * N;
    float accz = 0.0f;
#pragma unroll
    for (int b = 0; b < W::K; ++b) {
      const float* row = field + (zrow + ((by + static_cast<uint32_t>(b + W::OFF)) & m)) * N;
      float s = 0.0f;
#pragma unroll
      for (int a = 0; a < W::K; ++a) s = fmaf(wx[a], load(row + xs[a]), s);
      accz = fmaf(wy[b], s, accz);
    }
    acc = fmaf(wz[c], accz, acc);
  }
  return acc;
}

}  // namespace cmb3d
