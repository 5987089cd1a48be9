// Sampling of the box field at the sky pixels (paper Sec. II.D.1: the box map
// is interpolated and evaluated at the pixel positions r n_hat, box centred on
// the sphere).  Trilinear (2x2x2 taps) or tricubic Keys cubic convolution with
// a = -1/2 (4x4x4 taps), periodic wrap.
//
// One thread per pixel.  The pixel table is precomputed on the host in FP64
// (base cell and FP32 fraction per axis, 16 bytes per pixel) and, unless the
// plan says otherwise, sorted by base cell so that neighbouring threads read
// neighbouring field rows; the result goes to the caller's pixel order
// through `perm` (the scattered 4-byte writes merge in L2).
#include "device_common.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

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

template <int INTERP>
__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ field, const float4* __restrict__ tab,
                                                const int32_t* __restrict__ perm, float* __restrict__ out,
                                                int npix, int N) {
  using W = Weights<INTERP>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const float4 e = __ldg(tab + i);
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
      for (int a = 0; a < W::K; ++a) s = fmaf(wx[a], __ldg(row + xs[a]), s);
      accz = fmaf(wy[b], s, accz);
    }
    acc = fmaf(wz[c], accz, acc);
  }
  out[perm ? perm[i] : i] = acc;
}

__global__ void k_philox(const uint4* __restrict__ ctr, uint2 key, uint4* __restrict__ out, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

}  // namespace

cudaError_t launch_gather(int N, int interp, const float* field, const float4* tab, const int32_t* perm,
                          float* out, int64_t npix, cudaStream_t s) {
  if (npix <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((npix + threads - 1) / threads);
  if (interp == 1)
    k_gather<1><<<blocks, threads, 0, s>>>(field, tab, perm, out, static_cast<int>(npix), N);
  else
    k_gather<3><<<blocks, threads, 0, s>>>(field, tab, perm, out, static_cast<int>(npix), N);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((n + threads - 1) / threads);
  k_philox<<<blocks, threads, 0, s>>>(reinterpret_cast<const uint4*>(ctr), key, reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

}  // namespace cmb3d
