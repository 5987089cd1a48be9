// Sampling of the box field at the sky pixels (paper Sec. II.D.1: the box map
// is interpolated and evaluated at the pixel positions r n_hat, box centred on
// the sphere).  Trilinear (2x2x2 taps) or tricubic Keys cubic convolution with
// a = -1/2 (4x4x4 taps), periodic wrap.
//
// One thread per pixel, or (sorted tables) one thread per run of pixels that
// share a base cell.  The pixel table is precomputed on the host in FP64
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

// One thread per run of at most kGatherRun pixels sharing a base cell (the
// table is sorted by cell, 13 pixels per cell on average at the paper's
// resolutions).  The cell's K^3 taps are loaded once into registers, the run's
// table entries and destinations up front, and each pixel is interpolated from
// the registers with exactly interpolate()'s loads and FMA order, so the map
// equals the one-pixel form bit for bit.  This cuts the instructions per pixel
// (the one-pixel form issues about 330, 64 of them loads) and the L1 requests.
template <int INTERP>
__global__ void __launch_bounds__(256) k_gather_runs(const float* __restrict__ field, const float4* __restrict__ tab,
                                                     const int32_t* __restrict__ perm, float* __restrict__ out,
                                                     const int2* __restrict__ runs, int nruns, int N) {
  using W = Weights<INTERP>;
  constexpr int K = W::K;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nruns) return;
  const int2 run = __ldg(runs + t);
  float4 es[kGatherRun];
  int32_t ds[kGatherRun];
#pragma unroll
  for (int k = 0; k < kGatherRun; ++k) {
    if (k < run.y) {
      es[k] = __ldg(tab + run.x + k);
      ds[k] = perm ? __ldg(perm + run.x + k) : run.x + k;
    }
  }
  const uint32_t pk = __float_as_uint(es[0].w);
  const uint32_t bx = pk & 2047u, by = (pk >> 11) & 2047u;
  const uint32_t bz = (pk >> 22) | ((__float_as_uint(es[0].z) >> 31) << 10);
  const uint32_t n = static_cast<uint32_t>(N), m = n - 1u;
  const uint32_t x0 = bx + static_cast<uint32_t>(W::OFF);
  float v[K][K][K];                                    // [z][y][x] taps of the cell's stencil
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const float* plane = field + static_cast<size_t>((bz + static_cast<uint32_t>(c + W::OFF)) & m) * n * n;
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const uint32_t r = ((by + static_cast<uint32_t>(b + W::OFF)) & m) * n;
      if (x0 <= n - static_cast<uint32_t>(K)) {
        const float* q = plane + (r + x0);
#pragma unroll
        for (int a = 0; a < K; ++a) v[c][b][a] = __ldg(q + a);
      } else {
#pragma unroll
        for (int a = 0; a < K; ++a) v[c][b][a] = __ldg(plane + r + ((bx + static_cast<uint32_t>(a + W::OFF)) & m));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kGatherRun; ++k) {
    if (k < run.y) {
      float wx[K], wy[K], wz[K];
      W::run(es[k].x, wx);
      W::run(es[k].y, wy);
      W::run(fabsf(es[k].z), wz);
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        float accz = 0.0f;
#pragma unroll
        for (int b = 0; b < K; ++b) {
          float s = 0.0f;
#pragma unroll
          for (int a = 0; a < K; ++a) s = fmaf(wx[a], v[c][b][a], s);
          accz = fmaf(wy[b], s, accz);
        }
        acc = fmaf(wz[c], accz, acc);
      }
      out[ds[k]] = acc;
    }
  }
}

__global__ void k_philox(const uint4* __restrict__ ctr, uint2 key, uint4* __restrict__ out, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

}  // namespace

cudaError_t launch_gather(int N, int interp, const float* field, const float4* tab, const int32_t* perm,
                          float* out, int64_t npix, cudaStream_t s, const int2* runs, int64_t nruns) {
  if (npix <= 0) return cudaSuccess;
  const int threads = 256;
  if (runs && nruns > 0) {
    const unsigned blocks = static_cast<unsigned>((nruns + threads - 1) / threads);
    if (interp == 1)
      k_gather_runs<1><<<blocks, threads, 0, s>>>(field, tab, perm, out, runs, static_cast<int>(nruns), N);
    else
      k_gather_runs<3><<<blocks, threads, 0, s>>>(field, tab, perm, out, runs, static_cast<int>(nruns), N);
    return cudaGetLastError();
  }
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
