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
#include "fft_tiles.cuh"
#include "internal.h"

namespace cmb3d {
namespace {
// keyp != NULL: the Philox key is read from device memory (graph replays
// with new seeds); otherwise `key` is used.
template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_draw_zfft(float2* __restrict__ buf, const float* __restrict__ amp,
                                                         const float2* __restrict__ tw, uint2 key,
                                                         const uint2* __restrict__ keyp) {
  extern __shared__ float2 sm[];
  if (keyp) key = *keyp;
  draw_zfft_tile<N, R, T>(buf, amp, tw, key, blockIdx.x * T, blockIdx.y, sm);
}

template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_yfft(float2* __restrict__ buf, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  yfft_tile<N, R, T>(buf + static_cast<size_t>(blockIdx.y) * N * (N / 2), blockIdx.x * T, sm, tw);
}

template <int N, int R, int ROWS>
__global__ void __launch_bounds__(ROWS*(N / 2 / R)) k_xc2r(float2* __restrict__ buf, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  xc2r_rows<N, R, ROWS, false>(buf + static_cast<size_t>(blockIdx.x) * ROWS * (N / 2), sm, tw);
}

// Fused y + x passes: one thread-block cluster of C blocks owns one z-plane.
// Its blocks first transform the plane's N/2 columns along y (tiles of T
// columns, block b taking tiles b, b+C, ...), wait at the cluster barrier, and
// then transform the plane's N rows along x (block b taking rows
// [b N/C, (b+1) N/C)).  The y-transformed plane (4 N^2 bytes) is written and
// re-read through L2 while few planes are in flight, so HBM sees one read and
// one write of the box for both axes.
template <int N, int RY, int T, int RX, int C>
__global__ void __launch_bounds__(T*(N / RY)) k_yx_fused(float2* __restrict__ buf, const float2* __restrict__ tw) {
  constexpr int N2 = N / 2, NT = T * (N / RY), NBX = N2 / RX, ROWS = NT / NBX;
  static_assert(NT % NBX == 0 && (N / C) % ROWS == 0 && (N2 / T) % C == 0, "fused pass shape");
  extern __shared__ float2 sm[];
  const int crank = blockIdx.x % C;                 // rank in the (C,1,1) cluster
  float2* plane = buf + static_cast<size_t>(blockIdx.x / C) * N * N2;
  for (int tile = crank; tile < N2 / T; tile += C) {
    yfft_tile<N, RY, T>(plane, tile * T, sm, tw);
    __syncthreads();
  }
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  for (int r0 = crank * (N / C); r0 < (crank + 1) * (N / C); r0 += ROWS) {
    xc2r_rows<N, RX, ROWS>(plane + static_cast<size_t>(r0) * N2, sm, tw);
    __syncthreads();
  }
}

template <int N, int R, int T>
cudaError_t run_draw_zfft(float2* buf, const float* amp, const float2* tw, uint2 key, const uint2* keyp,
                          cudaStream_t s) {
  const size_t smem = sizeof(float2) * col_tile_elems<N, R, T>();
  auto kern = k_draw_zfft<N, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N / 2 / T, N), T * (N / R), smem, s>>>(buf, amp, tw, key, keyp);
  return cudaGetLastError();
}

template <int N, int R, int T>
cudaError_t run_yfft(float2* buf, const float2* tw, cudaStream_t s) {
  const size_t smem = sizeof(float2) * col_tile_elems<N, R, T>();
  auto kern = k_yfft<N, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N / 2 / T, N), T * (N / R), smem, s>>>(buf, tw);
  return cudaGetLastError();
}

template <int N, int R, int THREADS>
cudaError_t run_xc2r(float2* buf, const float2* tw, cudaStream_t s) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int ROWS0 = THREADS / NB > 0 ? THREADS / NB : 1;
  constexpr int ROWS = ROWS0 < N * N ? ROWS0 : N * N;
  constexpr int P = N2 + (N2 >> 4);
  const size_t smem = sizeof(float2) * P * ROWS;
  auto kern = k_xc2r<N, R, ROWS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N * N / ROWS), ROWS * NB, smem, s>>>(buf, tw);
  return cudaGetLastError();
}

// Diagnostic: the packed half spectrum [m_z][m_y][m_x'] with no transform;
// one thread per mode pair (mz, mz + N/2).
template <int N>
__global__ void k_draw_only(float2* __restrict__ buf, const float* __restrict__ amp, uint2 key) {
  constexpr int N2 = N / 2;
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<size_t>(N2) * N * N2) return;
  const int xp = static_cast<int>(i % N2), my = static_cast<int>((i / N2) % N);
  const int mz = static_cast<int>(i / (static_cast<size_t>(N2) * N));
  float2 lo, hi;
  draw_packed_pair<N>(xp, my, mz, amp, key, lo, hi);
  buf[(static_cast<size_t>(mz) * N + my) * N2 + xp] = lo;
  buf[(static_cast<size_t>(mz + N2) * N + my) * N2 + xp] = hi;
}

template <int N>
cudaError_t run_draw_only(float2* buf, const float* amp, uint2 key, cudaStream_t s) {
  const size_t n = static_cast<size_t>(N / 2) * N * (N / 2);
  k_draw_only<N><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(buf, amp, key);
  return cudaGetLastError();
}

template <int N, int RY, int T, int RX, int C>
cudaError_t run_yx_fused(float2* buf, const float2* tw, cudaStream_t s) {
  constexpr int N2 = N / 2, NT = T * (N / RY), NBX = N2 / RX, ROWS = NT / NBX;
  constexpr int P = N2 + (N2 >> 4);
  constexpr int CE = col_tile_elems<N, RY, T>();
  constexpr size_t smem = sizeof(float2) * (CE > ROWS * P ? CE : ROWS * P);
  auto kern = k_yx_fused<N, RY, T, RX, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * N);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, buf, tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

inline uint2 key_of(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
}

}  // namespace

// ---------------------------------------------------------------------------
// Variant tables.  Every box size has a default shape (variant 0); sizes from
// 256 up have alternatives (radix, tile width, threads per block) that the
// plan's autotuner times on the device.
//   column passes (draw + z, y):  (R, T), T * N / R threads, (N + N / R) * T * 8 B shared (T < 16)
//   row pass (x):                 (R, threads per block)
//   fused y+x pass:               (RY, T, RX, cluster size C)
// ---------------------------------------------------------------------------

int num_col_variants(int N) { return N >= 256 ? 3 : 1; }
int num_row_variants(int N) { return N >= 256 ? 3 : 1; }
int num_fused_variants(int N) { return N == 128 ? 1 : (N == 256 || N == 512 || N == 1024) ? 2 : 0; }

#define CMB3D_COL_SWITCH(RUN, ...)                                                        \
  switch (N * 4 + v) {                                                                  \
    case 8 * 4: return RUN<8, 8, 4>(__VA_ARGS__);                                          \
    case 16 * 4: return RUN<16, 8, 8>(__VA_ARGS__);                                        \
    case 32 * 4: return RUN<32, 8, 16>(__VA_ARGS__);                                       \
    case 64 * 4: return RUN<64, 8, 16>(__VA_ARGS__);                                       \
    case 128 * 4: return RUN<128, 8, 16>(__VA_ARGS__);                                     \
    case 256 * 4: return RUN<256, 8, 16>(__VA_ARGS__);                                     \
    case 256 * 4 + 1: return RUN<256, 16, 16>(__VA_ARGS__);                                \
    case 256 * 4 + 2: return RUN<256, 8, 8>(__VA_ARGS__);                                  \
    case 512 * 4: return RUN<512, 8, 16>(__VA_ARGS__);                                     \
    case 512 * 4 + 1: return RUN<512, 16, 16>(__VA_ARGS__);                                \
    case 512 * 4 + 2: return RUN<512, 8, 8>(__VA_ARGS__);                                  \
    case 1024 * 4: return RUN<1024, 16, 16>(__VA_ARGS__);                                  \
    case 1024 * 4 + 1: return RUN<1024, 16, 8>(__VA_ARGS__);                               \
    case 1024 * 4 + 2: return RUN<1024, 8, 8>(__VA_ARGS__);                                \
    case 2048 * 4: return RUN<2048, 16, 8>(__VA_ARGS__);                                   \
    case 2048 * 4 + 1: return RUN<2048, 16, 4>(__VA_ARGS__);                               \
    case 2048 * 4 + 2: return RUN<2048, 8, 4>(__VA_ARGS__);                                \
    default: return cudaErrorInvalidValue;                                              \
  }

cudaError_t launch_draw_zfft(int N, int v, float2* buf, const float* amp, const float2* tw, uint64_t seed,
                             cudaStream_t s, const uint2* key_dev) {
  const uint2 key = key_of(seed);
  CMB3D_COL_SWITCH(run_draw_zfft, buf, amp, tw, key, key_dev, s)
}

cudaError_t launch_yfft(int N, int v, float2* buf, const float2* tw, cudaStream_t s) {
  CMB3D_COL_SWITCH(run_yfft, buf, tw, s)
}

cudaError_t launch_xc2r(int N, int v, float2* buf, const float2* tw, cudaStream_t s) {
  switch (N * 4 + v) {
    case 8 * 4: return run_xc2r<8, 4, 256>(buf, tw, s);
    case 16 * 4: return run_xc2r<16, 8, 256>(buf, tw, s);
    case 32 * 4: return run_xc2r<32, 8, 256>(buf, tw, s);
    case 64 * 4: return run_xc2r<64, 8, 256>(buf, tw, s);
    case 128 * 4: return run_xc2r<128, 8, 256>(buf, tw, s);
    case 256 * 4: return run_xc2r<256, 8, 256>(buf, tw, s);
    case 256 * 4 + 1: return run_xc2r<256, 16, 256>(buf, tw, s);
    case 256 * 4 + 2: return run_xc2r<256, 8, 512>(buf, tw, s);
    case 512 * 4: return run_xc2r<512, 8, 256>(buf, tw, s);
    case 512 * 4 + 1: return run_xc2r<512, 16, 256>(buf, tw, s);
    case 512 * 4 + 2: return run_xc2r<512, 8, 512>(buf, tw, s);
    case 1024 * 4: return run_xc2r<1024, 8, 256>(buf, tw, s);
    case 1024 * 4 + 1: return run_xc2r<1024, 16, 256>(buf, tw, s);
    case 1024 * 4 + 2: return run_xc2r<1024, 8, 512>(buf, tw, s);
    case 2048 * 4: return run_xc2r<2048, 16, 256>(buf, tw, s);
    case 2048 * 4 + 1: return run_xc2r<2048, 16, 512>(buf, tw, s);
    case 2048 * 4 + 2: return run_xc2r<2048, 8, 512>(buf, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_yx_fused(int N, int v, float2* buf, const float2* tw, cudaStream_t s) {
  switch (N * 4 + v) {
    case 128 * 4: return run_yx_fused<128, 8, 16, 8, 4>(buf, tw, s);
    case 256 * 4: return run_yx_fused<256, 8, 16, 8, 8>(buf, tw, s);
    case 256 * 4 + 1: return run_yx_fused<256, 16, 16, 8, 8>(buf, tw, s);
    case 512 * 4: return run_yx_fused<512, 8, 16, 8, 8>(buf, tw, s);
    case 512 * 4 + 1: return run_yx_fused<512, 16, 16, 8, 8>(buf, tw, s);
    case 1024 * 4: return run_yx_fused<1024, 16, 16, 8, 8>(buf, tw, s);
    case 1024 * 4 + 1: return run_yx_fused<1024, 16, 8, 8, 8>(buf, tw, s);
    default: return cudaErrorNotSupported;
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

}  // namespace cmb3d
