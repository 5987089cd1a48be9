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
#include <atomic>

#include "fft_tiles.cuh"
#include "internal.h"

namespace cmb3d {
namespace {
// keyp != NULL: the Philox key is read from device memory (graph replays
// with new seeds); otherwise `key` is used.
// Blocks (x < N/2/T, y = m_y) draw the regular columns x T .. x T + T-1 of row
// m_y; the extra column of blocks x = N/2/T draws the packed Hermitian column
// m_x' = 0 of the T rows y T .. y T + T-1 (y < N/T), so that no warp mixes the
// Hermitian path with the regular one.
template <int N, int R, int T>
__device__ __forceinline__ void draw_block(float2* __restrict__ buf, const float* __restrict__ amp,
                                           const float2* __restrict__ tw, uint2 key, float2* sm,
                                           const uint32_t* __restrict__ zmask, int zlo, int zhi) {
  if (blockIdx.x == N / 2 / T) {
    if (static_cast<int>(blockIdx.y) * T >= N) return;
    draw_zfft_tile<N, R, T, kDrawHermitian>(buf, amp, tw, key, blockIdx.y * T, 0, sm, zmask, zlo, zhi);
  } else {
    draw_zfft_tile<N, R, T, kDrawRegular>(buf, amp, tw, key, blockIdx.x * T, blockIdx.y, sm, zmask, zlo, zhi);
  }
}

template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_draw_zfft(float2* __restrict__ buf, const float* __restrict__ amp,
                                                         const float2* __restrict__ tw, uint2 key,
                                                         const uint2* __restrict__ keyp,
                                                         const uint32_t* __restrict__ zmask, int zlo, int zhi) {
  extern __shared__ float2 sm[];
  // two copies of the body: with the key a kernel parameter its Philox round
  // keys stay in uniform registers, computed once per thread block
  if (keyp)
    draw_block<N, R, T>(buf, amp, tw, *keyp, sm, zmask, zlo, zhi);
  else
    draw_block<N, R, T>(buf, amp, tw, key, sm, zmask, zlo, zhi);
}

// The same kernel compiled for MINB resident blocks per SM: 256-thread tiles
// take 4 for radix 8 (64 registers a thread) or 2 for radix 16 (128
// registers) unless their draw variant names another count.
template <int N, int R, int T, int MINB>
__global__ void __launch_bounds__(T*(N / R), MINB) k_draw_zfft_mb(float2* __restrict__ buf, const float* __restrict__ amp,
                                                            const float2* __restrict__ tw, uint2 key,
                                                            const uint2* __restrict__ keyp,
                                                            const uint32_t* __restrict__ zmask, int zlo, int zhi) {
  extern __shared__ float2 sm[];
  if (keyp)
    draw_block<N, R, T>(buf, amp, tw, *keyp, sm, zmask, zlo, zhi);
  else
    draw_block<N, R, T>(buf, amp, tw, key, sm, zmask, zlo, zhi);
}

// MINB > 0: compiled for that many resident blocks; 0: 256-thread tiles get
// 4 (radix 8) or 2 (radix 16), larger tiles none.
template <int N, int R, int T, int MINB = 0>
constexpr auto draw_kernel() {
  if constexpr (MINB > 0)
    return k_draw_zfft_mb<N, R, T, MINB>;
  else if constexpr (T * (N / R) == 256)
    return k_draw_zfft_mb<N, R, T, (R == 8 ? 4 : 2)>;
  else
    return k_draw_zfft<N, R, T>;
}

// y pass over z-planes blockIdx.y, or with `planes` over planes[blockIdx.y];
// with `rowmask` (N bits per plane) only the marked rows are stored.
template <int N, int R, int T>
__global__ void __launch_bounds__(T*(N / R)) k_yfft(float2* __restrict__ buf, const float2* __restrict__ tw,
                                                    const int32_t* __restrict__ planes,
                                                    const uint32_t* __restrict__ rowmask) {
  extern __shared__ float2 sm[];
  constexpr int W = N / 32 > 0 ? N / 32 : 1;
  __shared__ uint32_t smask[W];
  const int z = planes ? __ldg(planes + blockIdx.y) : static_cast<int>(blockIdx.y);
  if (rowmask) {
    for (int i = threadIdx.x; i < W; i += blockDim.x) smask[i] = __ldg(rowmask + static_cast<size_t>(z) * W + i);
    __syncthreads();
  }
  yfft_tile<N, R, T>(buf + static_cast<size_t>(z) * N * (N / 2), blockIdx.x * T, sm, tw, rowmask ? smask : nullptr);
}

template <int N, int R, int ROWS>
__global__ void __launch_bounds__(ROWS*(N / 2 / R)) k_xc2r(float2* __restrict__ buf, const float2* __restrict__ tw,
                                                              const int32_t* __restrict__ rows,
                                                              const uint32_t* __restrict__ cols) {
  extern __shared__ float2 sm[];
  if (rows)
    xc2r_rows<N, R, ROWS, false>(buf, sm, tw, rows + static_cast<size_t>(blockIdx.x) * ROWS,
                                 cols ? cols + static_cast<size_t>(blockIdx.x) * ROWS : nullptr);
  else
    xc2r_rows<N, R, ROWS, false>(buf + static_cast<size_t>(blockIdx.x) * ROWS * (N / 2), sm, tw);
}

// The same row pass compiled for MINB resident blocks per SM (register cap
// 65536 / (MINB x threads)): more rows in flight per SM.
template <int N, int R, int ROWS, int MINB>
__global__ void __launch_bounds__(ROWS*(N / 2 / R), MINB) k_xc2r_mb(float2* __restrict__ buf,
                                                                       const float2* __restrict__ tw,
                                                                       const int32_t* __restrict__ rows,
                                                                       const uint32_t* __restrict__ cols) {
  extern __shared__ float2 sm[];
  if (rows)
    xc2r_rows<N, R, ROWS, false>(buf, sm, tw, rows + static_cast<size_t>(blockIdx.x) * ROWS,
                                 cols ? cols + static_cast<size_t>(blockIdx.x) * ROWS : nullptr);
  else
    xc2r_rows<N, R, ROWS, false>(buf + static_cast<size_t>(blockIdx.x) * ROWS * (N / 2), sm, tw);
}

template <int N, int R, int ROWS, int MINB>
constexpr auto xc2r_kernel() {
  if constexpr (MINB > 1)
    return k_xc2r_mb<N, R, ROWS, MINB>;
  else
    return k_xc2r<N, R, ROWS>;
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

// Fused y + x passes through distributed shared memory.  A cluster of
// C = N/32 thread blocks holds one z-plane (N rows of N/2 packed entries) in
// its shared memories, and the y transform is split four-step fashion as
// N = 32 C with input row y = c + C m and output row k = k1 + 32 k2:
//   1. block c loads its rows y = c + C m (m < 32) and transforms along m
//      (radix 16 in registers, radix 2 between lanes l and l + 16), then
//      multiplies entry k1 by w_N^(c k1);
//   2. after a cluster barrier, block b forms for k1 in [b K, (b+1) K)
//      (K = 32 / C) the C-point transforms over the C blocks' entries k1
//      (shared::cluster loads), i.e. rows k1 + 32 k2 of the y-transformed plane;
//   3. after a second cluster barrier (no block reads another's memory after
//      it) block b stores its 32 complete rows in its own shared memory and
//      runs the x pass (complex-to-real, as in xc2r_rows) on them, writing the
//      real rows to HBM.
// HBM sees one read and one write of the plane for both axes.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Load the float2 at the same shared-memory offset as `local` in the block of
// cluster rank `rank`.
__device__ __forceinline__ float2 ld_cluster(const float2* local, uint32_t rank) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local));
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(r) : "memory");
  return v;
}

template <int N>
struct DsmemShape {
  static constexpr int N2 = N / 2, M = 32, C = N / M, K = M / C, P = N2 + (N2 >> 4), NT = N;
  static constexpr int ITEMS = K * N2 / NT;          // step-2 transforms per thread
  static constexpr size_t SMEM = sizeof(float2) * M * P;
  static_assert(C >= 2 && C <= 16 && ITEMS * C == 16, "cluster shape");
};

template <int N>
__global__ void __launch_bounds__(N, 2) k_yx_dsmem(float2* __restrict__ buf, const float2* __restrict__ tw) {
  using D = DsmemShape<N>;
  constexpr int N2 = D::N2, M = D::M, C = D::C, K = D::K, P = D::P;
  extern __shared__ float2 A[];                      // 32 rows of pitch P; entry n at n + n/16
  auto at = [](int row, int n) { return row * P + n + (n >> 4); };
  const int t = threadIdx.x;
  const int crank = blockIdx.x % C;                  // rank in the (C,1,1) cluster
  float2* plane = buf + static_cast<size_t>(blockIdx.x / C) * N * N2;

  {  // step 1: lanes 0-15 take even m, lanes 16-31 odd m, of 16 columns
    const int lane = t & 31, j = lane >> 4, col = (t >> 5) * 16 + (lane & 15);
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = __ldcg(plane + static_cast<size_t>(crank + C * (j + 2 * r)) * N2 + col);
    IDft<16>::run(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v[q].x, 16), __shfl_xor_sync(0xffffffffu, v[q].y, 16));
      const float2 e0 = j ? o : v[q], e1 = cmul(j ? v[q] : o, __ldg(tw + (N / 32) * q));
      const int k1 = q + 16 * j;
      A[at(k1, col)] = cmul(j ? csub(e0, e1) : cadd(e0, e1), __ldg(tw + crank * k1));
    }
  }
  cluster_sync();
  float2 w[D::ITEMS][C];
#pragma unroll
  for (int u = 0; u < D::ITEMS; ++u) {                // step 2
    const int i = t + D::NT * u, k1 = crank * K + i / N2, col = i % N2;
    const float2* src = A + at(k1, col);
#pragma unroll
    for (int c = 0; c < C; ++c) w[u][c] = ld_cluster(src, c);
    IDft<C>::run(w[u]);
  }
  cluster_sync();
#pragma unroll
  for (int u = 0; u < D::ITEMS; ++u) {
    const int i = t + D::NT * u, k1l = i / N2, col = i % N2;
#pragma unroll
    for (int k2 = 0; k2 < C; ++k2) A[at(k1l + K * k2, col)] = w[u][k2];
  }
  __syncthreads();
  {  // step 3: x pass on local row rl = output row crank K + rl % K + 32 (rl / K)
    constexpr int R = 16, NB = N2 / R;
    static_assert(M * NB == D::NT, "one thread per butterfly");
    const int j = t % NB, rl = t / NB;
    float2* g = plane + static_cast<size_t>(crank * K + rl % K + M * (rl / K)) * N2;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = j + r * NB;
      if (k == 0) {
        const float2 p = A[at(rl, 0)];
        v[r] = make_float2(p.x + p.y, p.x - p.y);
      } else {
        const float2 a = A[at(rl, k)], b = cconj(A[at(rl, N2 - k)]);
        v[r] = cadd(cadd(a, b), cmul_i(cmul(__ldg(tw + k), csub(a, b))));
      }
    }
    stockham<N2, R, N, true>(
        v, A, tw, j, [&](int n) { return at(rl, n); }, [&](int n, float2 x) { g[n] = x; }, BlockSync{});
  }
}

template <int N>
cudaLaunchConfig_t dsmem_config(float2* buf, cudaStream_t s, cudaLaunchAttribute* attr) {
  using D = DsmemShape<N>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(D::C * N);
  cfg.blockDim = dim3(D::NT);
  cfg.dynamicSmemBytes = D::SMEM;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = D::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)buf;
  return cfg;
}

// Attributes set and the cluster shape checked against the device once per
// process and box size: 1 = can run, 0 = cannot (no launch is attempted).
template <int N>
int dsmem_ready() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> states[kMaxDevices];       // 0 unknown, 1 no, 2 yes
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  const int known = states[dev].load();
  if (known) return known - 1;
  using D = DsmemShape<N>;
  auto kern = k_yx_dsmem<N>;
  int ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(D::SMEM)) ==
           cudaSuccess;
  if (ok && D::C > 8) ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  int clusters = 0;
  if (ok) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = dsmem_config<N>(nullptr, nullptr, attr);
    ok = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0;
  }
  if (!ok) cudaGetLastError();
  states[dev].store(ok ? 2 : 1);
  return ok ? 1 : 0;
}

template <int N>
cudaError_t run_yx_dsmem(float2* buf, const float2* tw, cudaStream_t s) {
  if (!dsmem_ready<N>()) return cudaErrorNotSupported;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = dsmem_config<N>(buf, s, attr);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_yx_dsmem<N>, buf, tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int N, int R, int T, int MINB = 0>
cudaError_t run_draw_zfft(float2* buf, const float* amp, const float2* tw, uint2 key, const uint2* keyp,
                          cudaStream_t s, const uint32_t* zmask, int zlo, int zhi) {
  const size_t smem = sizeof(float2) * col_tile_elems<N, R, T>() + sizeof(float) * draw_amp_floats<N, T>();
  auto kern = draw_kernel<N, R, T, MINB>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(N / 2 / T + 1, N), T * (N / R), smem, s>>>(buf, amp, tw, key, keyp, zmask, zlo, zhi > 0 ? zhi : N);
  return cudaGetLastError();
}

template <int N, int R, int T>
cudaError_t run_yfft(float2* buf, const float2* tw, cudaStream_t s, const int32_t* planes, int nplanes,
                     const uint32_t* rowmask) {
  const size_t smem = sizeof(float2) * col_tile_elems<N, R, T>();
  auto kern = k_yfft<N, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int nz = planes ? nplanes : N;
  if (nz <= 0) return cudaSuccess;
  kern<<<dim3(N / 2 / T, nz), T * (N / R), smem, s>>>(buf, tw, planes, rowmask);
  return cudaGetLastError();
}

template <int N, int R, int THREADS, int MINB = 1>
cudaError_t run_xc2r(float2* buf, const float2* tw, cudaStream_t s, const int32_t* rows, int64_t nrows,
                     const uint32_t* cols) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int ROWS0 = THREADS / NB > 0 ? THREADS / NB : 1;
  constexpr int ROWS = ROWS0 < N * N ? ROWS0 : N * N;
  static_assert(N < 128 || kRowListPad % ROWS == 0, "pruned row lists are padded to whole blocks of every shape");
  constexpr int P = N2 + (N2 >> 4);
  const size_t smem = sizeof(float2) * P * ROWS;
  auto kern = xc2r_kernel<N, R, ROWS, MINB>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (rows && (nrows <= 0 || nrows % ROWS != 0)) return nrows == 0 ? cudaSuccess : cudaErrorInvalidValue;
  const int64_t nb = rows ? nrows / ROWS : static_cast<int64_t>(N) * N / ROWS;
  kern<<<dim3(static_cast<unsigned>(nb)), ROWS * NB, smem, s>>>(buf, tw, rows, rows ? cols : nullptr);
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
//   fused y+x pass:               (RY, T, RX, cluster size C); variant 2 (N = 256, 512): the
//                                 distributed-shared-memory form, cluster of N/32 blocks
// ---------------------------------------------------------------------------

int num_col_variants(int N) { return N >= 2048 ? 3 : N >= 256 ? 4 : 1; }
int num_draw_variants(int N) {
  return (N >= 1024 ? num_col_variants(N) + 2 : num_col_variants(N)) + (draw_tc_supported(N) ? 1 : 0);
}
int num_row_variants(int N) { return N >= 512 ? 4 : N >= 256 ? 3 : 1; }
int num_fused_variants(int N) { return N == 128 ? 1 : (N == 256 || N == 512) ? 3 : N == 1024 ? 2 : 0; }

bool fused_variant_available(int N, int v) {
  if (v < 0 || v >= num_fused_variants(N)) return false;
  if (v < 2) return true;
  return N == 256 ? dsmem_ready<256>() == 1 : N == 512 ? dsmem_ready<512>() == 1 : false;
}

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
    case 256 * 4 + 3: return RUN<256, 8, 4>(__VA_ARGS__);                                  \
    case 512 * 4: return RUN<512, 8, 16>(__VA_ARGS__);                                     \
    case 512 * 4 + 1: return RUN<512, 16, 16>(__VA_ARGS__);                                \
    case 512 * 4 + 2: return RUN<512, 8, 8>(__VA_ARGS__);                                  \
    case 512 * 4 + 3: return RUN<512, 8, 4>(__VA_ARGS__);                                  \
    case 1024 * 4: return RUN<1024, 16, 16>(__VA_ARGS__);                                  \
    case 1024 * 4 + 1: return RUN<1024, 16, 8>(__VA_ARGS__);                               \
    case 1024 * 4 + 2: return RUN<1024, 8, 8>(__VA_ARGS__);                                \
    case 1024 * 4 + 3: return RUN<1024, 8, 4>(__VA_ARGS__);                                \
    case 2048 * 4: return RUN<2048, 16, 8>(__VA_ARGS__);                                   \
    case 2048 * 4 + 1: return RUN<2048, 16, 4>(__VA_ARGS__);                               \
    case 2048 * 4 + 2: return RUN<2048, 8, 4>(__VA_ARGS__);                                \
    default: return cudaErrorInvalidValue;                                              \
  }

cudaError_t launch_draw_zfft(int N, int v, float2* buf, const float* amp, const float2* tw, uint64_t seed,
                             cudaStream_t s, const uint2* key_dev, const uint32_t* zmask, int zlo, int zhi,
                             unsigned* err) {
  if (draw_tc_supported(N) && v == num_draw_variants(N) - 1)
    return launch_draw_tc(N, buf, amp, tw, seed, s, err, key_dev, zmask, zlo, zhi);
  const uint2 key = key_of(seed);
  // at N = 1024 the 8-column radix-16 and the 4-column radix-8 tiles are compiled for 2
  // resident blocks, and two draw-only 256-thread radix-16 tiles of 4 columns follow the
  // column-pass table, compiled for 3 and for 4 resident blocks
  if (N == 1024 && v == 1) return run_draw_zfft<1024, 16, 8, 2>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  if (N == 1024 && v == 3) return run_draw_zfft<1024, 8, 4, 2>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  if (N == 1024 && v == 4) return run_draw_zfft<1024, 16, 4, 3>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  if (N == 1024 && v == 5) return run_draw_zfft<1024, 16, 4, 4>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  if (N == 2048 && v == 3) return run_draw_zfft<2048, 16, 2>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  if (N == 2048 && v == 4) return run_draw_zfft<2048, 8, 1>(buf, amp, tw, key, key_dev, s, zmask, zlo, zhi);
  CMB3D_COL_SWITCH(run_draw_zfft, buf, amp, tw, key, key_dev, s, zmask, zlo, zhi)
}

cudaError_t launch_yfft(int N, int v, float2* buf, const float2* tw, cudaStream_t s, const int32_t* planes,
                        int nplanes, const uint32_t* rowmask) {
  CMB3D_COL_SWITCH(run_yfft, buf, tw, s, planes, nplanes, rowmask)
}

cudaError_t launch_xc2r(int N, int v, float2* buf, const float2* tw, cudaStream_t s, const int32_t* rows,
                        int64_t nrows, const uint32_t* cols) {
  switch (N * 4 + v) {
    case 8 * 4: return run_xc2r<8, 4, 256>(buf, tw, s, rows, nrows, cols);
    case 16 * 4: return run_xc2r<16, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 32 * 4: return run_xc2r<32, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 64 * 4: return run_xc2r<64, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 128 * 4: return run_xc2r<128, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 256 * 4: return run_xc2r<256, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 256 * 4 + 1: return run_xc2r<256, 16, 256>(buf, tw, s, rows, nrows, cols);
    case 256 * 4 + 2: return run_xc2r<256, 8, 512>(buf, tw, s, rows, nrows, cols);
    case 512 * 4: return run_xc2r<512, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 512 * 4 + 1: return run_xc2r<512, 16, 256>(buf, tw, s, rows, nrows, cols);
    case 512 * 4 + 2: return run_xc2r<512, 8, 512>(buf, tw, s, rows, nrows, cols);
    case 512 * 4 + 3: return run_xc2r<512, 16, 256, 4>(buf, tw, s, rows, nrows, cols);
    case 1024 * 4: return run_xc2r<1024, 8, 256>(buf, tw, s, rows, nrows, cols);
    case 1024 * 4 + 1: return run_xc2r<1024, 16, 256>(buf, tw, s, rows, nrows, cols);
    case 1024 * 4 + 3: return run_xc2r<1024, 16, 256, 4>(buf, tw, s, rows, nrows, cols);
    case 1024 * 4 + 2: return run_xc2r<1024, 8, 512>(buf, tw, s, rows, nrows, cols);
    case 2048 * 4: return run_xc2r<2048, 16, 256>(buf, tw, s, rows, nrows, cols);
    case 2048 * 4 + 1: return run_xc2r<2048, 16, 512>(buf, tw, s, rows, nrows, cols);
    case 2048 * 4 + 2: return run_xc2r<2048, 8, 512>(buf, tw, s, rows, nrows, cols);
    case 2048 * 4 + 3: return run_xc2r<2048, 16, 256, 4>(buf, tw, s, rows, nrows, cols);
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
    case 256 * 4 + 2: return run_yx_dsmem<256>(buf, tw, s);
    case 512 * 4 + 2: return run_yx_dsmem<512>(buf, tw, s);
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
