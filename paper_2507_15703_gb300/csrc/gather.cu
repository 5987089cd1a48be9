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
#include "gather_tiles.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

template <int INTERP>
__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ field, const float4* __restrict__ tab,
                                                const int32_t* __restrict__ perm, float* __restrict__ out,
                                                int npix, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const float v = interpolate<INTERP>(field, __ldg(tab + i), N, [](const float* p) { return __ldg(p); });
  out[perm ? perm[i] : i] = v;
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
