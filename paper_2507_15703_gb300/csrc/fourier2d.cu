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
constexpr int kWarps = 8, kTile = 32;                 // 8 warps per block; up to 32 modes (m_x') per block

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Factor of mode (mx, my): the table entry of q = mx^2 + fy^2.
__device__ __forceinline__ const float* factor_of(int mx, int my, int N, int h, const float* __restrict__ tab) {
  const int fy = my <= N / 2 ? my : my - N;
  return tab + static_cast<size_t>(mx * mx + fy * fy) * h * h;
}

// Start copying a factor into sS (rows of h + 1 floats: lane z later reads
// row z without bank conflicts); lane i copies column i, one cp.async group.
__device__ __forceinline__ void stage_async(const float* __restrict__ S, float* sS, int h, int lane) {
  if (lane < h) {
#pragma unroll 8
    for (int z = 0; z < h; ++z) cp_async4(sS + z * (h + 1) + lane, S + z * h + lane);
  }
  cp_async_commit();
}

// Layer values of one mode, computed by a warp from its staged factor sS:
// lane z < h returns T^(mx, my, z).  Lanes ip < (h + 1)/2 draw the Philox
// block (mx, my', ip, 1) into sc[h].  On a Hermitian line (mx in {0, N/2})
// the partner of a drawing mode takes the conjugate of the drawing mode's
// values and self-conjugate modes are real.
__device__ __forceinline__ float2 warp_mode(int mx, int my, int N, int h, uint2 key, const float* sS, float2* sc,
                                            int lane) {
  const bool line = mx == 0 || mx == N / 2;
  const int py = (N - my) & (N - 1);
  const bool self = line && py == my, partner = line && !self && py < my;
  if (2 * lane < h) {
    const uint4 w = philox4x32_10(make_uint4(mx, partner ? py : my, lane, 1u), key);
    const float2 ga = box_muller(w.x, w.y), gb = box_muller(w.z, w.w);
    sc[2 * lane] = self ? make_float2(ga.x, 0.f) : make_float2(ga.x * kRsqrt2, ga.y * kRsqrt2);
    if (2 * lane + 1 < h) sc[2 * lane + 1] = self ? make_float2(gb.x, 0.f) : make_float2(gb.x * kRsqrt2, gb.y * kRsqrt2);
  }
  __syncwarp();
  float2 acc = make_float2(0.f, 0.f);
  if (lane < h) {
    const float* row = sS + lane * (h + 1);
#pragma unroll 8
    for (int i = 0; i < h; ++i) {                    // one accumulator, i ascending; loads run ahead
      const float si = row[i];
      acc.x = fmaf(si, sc[i].x, acc.x);
      acc.y = fmaf(si, sc[i].y, acc.y);
    }
  }
  __syncwarp();                                      // sc and sS are reused by the warp's next mode
  return partner ? make_float2(acc.x, -acc.y) : acc;
}

// Block (m_x' tile blockIdx.x, m_y = blockIdx.y): warp w takes the tile's
// modes w, w + 8, ...; while one mode is computed the next mode's factor is
// already on its way into the other staging buffer (cp.async).  The layers go
// through shared memory [z][mode] so each layer is stored as one row of
// consecutive m_x'.
__global__ void __launch_bounds__(kWarps * 32) k_draw2d(float2* __restrict__ buf, const float* __restrict__ tab,
                                                        int N, int h, uint2 key) {
  extern __shared__ float smem[];
  const int N2 = N / 2, tw = N2 < kTile ? N2 : kTile;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int xp0 = blockIdx.x * tw, my = blockIdx.y;
  constexpr int kPitch = kTile + 1;                  // odd pitch: lane z's stores fall in distinct banks
  float2* sout = reinterpret_cast<float2*>(smem);                          // [h][kPitch]
  float* region = smem + 2 * h * kPitch + warp * (2 * h * (h + 2));        // sc[h], then two sS[h][h + 1]
  float2* sc = reinterpret_cast<float2*>(region);
  float* const sb0 = region + 2 * h;                 // staging buffer b at sb0 + b h (h + 1)
  const int sbs = h * (h + 1);
  int m = warp;
  if (xp0 == 0 && m == 0) {                          // slot 0 packs T^(0, .) + i T^(N/2, .)
    stage_async(factor_of(0, my, N, h, tab), sb0, h, lane);
    stage_async(factor_of(N2, my, N, h, tab), sb0 + sbs, h, lane);
    cp_async_wait<0>();
    __syncwarp();
    const float2 a = warp_mode(0, my, N, h, key, sb0, sc, lane);
    const float2 b = warp_mode(N2, my, N, h, key, sb0 + sbs, sc, lane);
    if (lane < h) sout[lane * kPitch] = make_float2(a.x - b.y, a.y + b.x);
    m += kWarps;
  }
  if (m < tw) {
    stage_async(factor_of(xp0 + m, my, N, h, tab), sb0, h, lane);
    for (int it = 0; m < tw; ++it, m += kWarps) {
      const int cur = it & 1;
      const bool more = m + kWarps < tw;
      if (more) {
        stage_async(factor_of(xp0 + m + kWarps, my, N, h, tab), sb0 + (cur ^ 1) * sbs, h, lane);
        cp_async_wait<1>();                          // this mode's copies are done, the next one's in flight
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const float2 v = warp_mode(xp0 + m, my, N, h, key, sb0 + cur * sbs, sc, lane);
      if (lane < h) sout[lane * kPitch + m] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < h * tw; e += kWarps * 32) {
    const int z = e / tw, mm = e - z * tw;
    buf[(static_cast<size_t>(z) * N + my) * N2 + xp0 + mm] = sout[z * kPitch + mm];
  }
}

}  // namespace

cudaError_t launch_draw2d(int N, int h, float2* buf, const float* tab, uint64_t seed, cudaStream_t s) {
  if (N < 16 || (N & (N - 1)) || h < 1 || h > 32) return cudaErrorInvalidValue;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
  const int N2 = N / 2, tw = N2 < kTile ? N2 : kTile;
  const size_t smem = sizeof(float) * (2 * h * (kTile + 1) + kWarps * 2 * h * (h + 2));
  cudaError_t e = cudaFuncSetAttribute(k_draw2d, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_draw2d<<<dim3(N2 / tw, N), kWarps * 32, smem, s>>>(buf, tab, N, h, key);
  return cudaGetLastError();
}

}  // namespace cmb3d
