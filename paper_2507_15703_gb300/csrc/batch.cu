// Many realizations in one persistent launch (the batched form of the 3-D
// Fourier method; the paper generates batches of maps that reuse one set of
// precomputed quantities, Sec. II.D.2 and Sec. IV).
//
// Every box contributes four kinds of work items:
//   D  draw + FFT along z of TPI column tiles,
//   Y  FFT along y of TPI column tiles,
//   X  complex-to-real FFT along x of TPI row blocks,
//   G  interpolation at GPI pixels.
// The host orders all items of all boxes in one list in which an item only
// depends on items listed before it: Y of box b waits for every D of box b,
// X for every Y, G for every X (per-box completion counters).  The list
// interleaves the ALU-bound D items of box b+1 with the memory-bound Y, X and
// G items of box b, so both kinds of work run side by side on the GPU.
// A box with a pruned transform (its pixels' stencils read only some z-planes
// and rows) has D items that store only those planes, Y items over those
// planes (storing the marked rows) and X items over those rows, as the
// single-box passes; each box carries its own Y and X item counts.
// Resident blocks take items in list order from an atomic counter; because
// all blocks are resident and dependencies point backwards, every wait ends.
// Each wait is nevertheless bounded: after `spin_limit` polls the block sets
// the error word and leaves, and the others notice and leave too.
#include "fft_tiles.cuh"
#include "gather_tiles.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

constexpr int kThreads = 512;

template <int N>
struct Shape;
// N = 256: radix 8 everywhere, 16-column tiles.
template <>
struct Shape<256> {
  static constexpr int RD = 8, TD = 16, RY = 8, TY = 16, RX = 8;
};
// N = 512: the autotuned single-box shapes that fit 512 threads.
template <>
struct Shape<512> {
  static constexpr int RD = 8, TD = 8, RY = 16, TY = 16, RX = 16;
};

template <int N>
struct Sizes {
  using S = Shape<N>;
  static constexpr int N2 = N / 2;
  static constexpr int NBX = N2 / S::RX, ROWS = kThreads / NBX, P = N2 + (N2 >> 4);
  static constexpr int D_TILES = (N2 / S::TD) * N, Y_TILES_PER_PLANE = N2 / S::TY;
  static constexpr int ND = D_TILES / kBatchTilesPerItem;
  static constexpr int DE = col_tile_elems<N, S::RD, S::TD>(), YE = col_tile_elems<N, S::RY, S::TY>();
  static constexpr int CE = DE > YE ? DE : YE;
  static constexpr int SMEM_ELEMS = CE > ROWS * P ? CE : ROWS * P;
  static_assert(S::TD * (N / S::RD) == kThreads && S::TY * (N / S::RY) == kThreads, "tile shapes");
  static_assert(D_TILES % kBatchTilesPerItem == 0 && kRowListPad % ROWS == 0, "item grouping, row blocks");
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int N, int INTERP, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_batch(const BatchBox* __restrict__ boxes,
                                                     const uint64_t* __restrict__ items, int nitems,
                                                     unsigned* __restrict__ ctr, const float2* __restrict__ tw,
                                                     unsigned spin_limit, int withhold_draw) {
  using S = Shape<N>;
  using Z = Sizes<N>;
  constexpr int N2 = N / 2;
  extern __shared__ float2 sm[];
  __shared__ unsigned s_k;
  __shared__ int s_abort;
  __shared__ uint32_t smask[N / 32];
  unsigned* next = ctr;
  unsigned* err = ctr + 1;
  unsigned* done = ctr + 2;
  for (;;) {
    if (threadIdx.x == 0) s_k = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned k = s_k;
    if (k >= static_cast<unsigned>(nitems)) return;
    const uint64_t it = items[k];
    const int b = static_cast<int>(it >> 40), type = static_cast<int>((it >> 32) & 0xF);
    const int idx = static_cast<int>(it & 0xFFFFFFFFu);
    const BatchBox bx = boxes[b];
    if (type != kBatchDraw) {
      if (threadIdx.x == 0) {
        const unsigned need = type == kBatchY ? static_cast<unsigned>(Z::ND) : type == kBatchX ? bx.nY : bx.nX;
        const unsigned* c = done + 4 * b + (type - 1);
        unsigned spins = 0;
        int ok = 1;
        while (ld_acquire(c) < need) {
          if (++spins > spin_limit || *reinterpret_cast<volatile unsigned*>(err)) {
            ok = 0;
            break;
          }
          __nanosleep(256);
        }
        if (!ok) atomicOr(err, 1u);
        s_abort = !ok;
      }
      __syncthreads();
      if (s_abort) return;
    }
    if (type == kBatchDraw) {
      const uint2 key = make_uint2(bx.key_lo, bx.key_hi);
      for (int t = idx * kBatchTilesPerItem; t < (idx + 1) * kBatchTilesPerItem; ++t) {
        const int my = t / (N2 / S::TD), xt = t % (N2 / S::TD);
        draw_zfft_tile<N, S::RD, S::TD>(bx.buf, bx.amp, tw, key, xt * S::TD, my, sm, bx.zmask, bx.zlo, bx.zhi);
        __syncthreads();
      }
    } else if (type == kBatchY) {
      const int end = min(bx.ny_tiles, (idx + 1) * kBatchTilesPerItem);
      for (int t = idx * kBatchTilesPerItem; t < end; ++t) {
        const int pi = t / Z::Y_TILES_PER_PLANE, xt = t % Z::Y_TILES_PER_PLANE;
        const int z = bx.planes ? __ldg(bx.planes + pi) : pi;
        if (bx.rowmask) {                              // the plane's stored rows, for the tile's last stage
          for (int i = threadIdx.x; i < N / 32; i += kThreads)
            smask[i] = __ldg(bx.rowmask + static_cast<size_t>(z) * (N / 32) + i);
          __syncthreads();
        }
        yfft_tile<N, S::RY, S::TY>(bx.buf + static_cast<size_t>(z) * N * N2, xt * S::TY, sm, tw,
                                   bx.rowmask ? smask : nullptr);
        __syncthreads();
      }
    } else if (type == kBatchX) {
      const int end = min(bx.nx_blocks, (idx + 1) * kBatchTilesPerItem);
      for (int t = idx * kBatchTilesPerItem; t < end; ++t) {
        if (bx.rows)
          xc2r_rows<N, S::RX, Z::ROWS>(bx.buf, sm, tw, bx.rows + static_cast<size_t>(t) * Z::ROWS,
                                       bx.cols ? bx.cols + static_cast<size_t>(t) * Z::ROWS : nullptr);
        else
          xc2r_rows<N, S::RX, Z::ROWS>(bx.buf + static_cast<size_t>(t) * Z::ROWS * N2, sm, tw);
        __syncthreads();
      }
    } else {
      const float* field = reinterpret_cast<const float*>(bx.buf);
      const int end = min(bx.npix, (idx + 1) * kBatchPixelsPerItem);
      for (int i = idx * kBatchPixelsPerItem + static_cast<int>(threadIdx.x); i < end; i += kThreads) {
        // the field was written by other blocks during this launch; the
        // gpu-scope acquire of the X counter and the block barrier order these
        // plain (L1-cacheable) loads after those writes
        const float v = interpolate<INTERP>(field, __ldg(bx.tab + i), N, [](const float* p) { return *p; });
        bx.out[bx.perm ? bx.perm[i] : i] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !(withhold_draw && type == kBatchDraw)) {
      __threadfence();
      atomicAdd(done + 4 * b + type, 1u);
    }
  }
}

template <int N, int INTERP, int MINB>
cudaError_t run_batch(int grid, const BatchBox* boxes, const uint64_t* items, int nitems, unsigned* ctr,
                      const float2* tw, unsigned spin_limit, int withhold, cudaStream_t s) {
  const size_t smem = sizeof(float2) * Sizes<N>::SMEM_ELEMS;
  auto kern = k_batch<N, INTERP, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(boxes, items, nitems, ctr, tw, spin_limit, withhold);
  return cudaGetLastError();
}

template <int N, int INTERP, int MINB>
cudaError_t grid_of(int* blocks) {
  const size_t smem = sizeof(float2) * Sizes<N>::SMEM_ELEMS;
  auto kern = k_batch<N, INTERP, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *blocks = per_sm * sms;
  return *blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace

bool batch_supported(int N) { return N == 256 || N == 512; }

int batch_draw_items(int N) { return N == 256 ? Sizes<256>::ND : Sizes<512>::ND; }

void batch_box_counts(int N, int64_t nplanes, int64_t nrows, int* ny_tiles, int* nx_blocks, int* nY, int* nX) {
  const int tpp = N == 256 ? Sizes<256>::Y_TILES_PER_PLANE : Sizes<512>::Y_TILES_PER_PLANE;
  const int rows = N == 256 ? Sizes<256>::ROWS : Sizes<512>::ROWS;
  *ny_tiles = static_cast<int>(nplanes) * tpp;
  *nx_blocks = static_cast<int>(nrows / rows);
  *nY = (*ny_tiles + kBatchTilesPerItem - 1) / kBatchTilesPerItem;
  *nX = (*nx_blocks + kBatchTilesPerItem - 1) / kBatchTilesPerItem;
}

// Variant v: 0 = two resident blocks per SM (64 registers per thread),
// 1 = one block per SM (no register cap, no spills).
int num_batch_variants() { return 2; }

#define CMB3D_BATCH_SWITCH(F, ...)                                                  \
  switch ((N == 256 ? 0 : N == 512 ? 4 : 8) + (interp == 1 ? 0 : 2) + (v ? 1 : 0)) { \
    case 0: return F<256, 1, 2>(__VA_ARGS__);                                       \
    case 1: return F<256, 1, 1>(__VA_ARGS__);                                       \
    case 2: return F<256, 3, 2>(__VA_ARGS__);                                       \
    case 3: return F<256, 3, 1>(__VA_ARGS__);                                       \
    case 4: return F<512, 1, 2>(__VA_ARGS__);                                       \
    case 5: return F<512, 1, 1>(__VA_ARGS__);                                       \
    case 6: return F<512, 3, 2>(__VA_ARGS__);                                       \
    case 7: return F<512, 3, 1>(__VA_ARGS__);                                       \
    default: return cudaErrorNotSupported;                                          \
  }

cudaError_t batch_grid(int N, int interp, int v, int* blocks) { CMB3D_BATCH_SWITCH(grid_of, blocks) }

cudaError_t launch_batch(int N, int interp, int v, int grid, const BatchBox* boxes, const uint64_t* items,
                         int nitems, unsigned* ctr, const float2* tw, unsigned spin_limit, int withhold,
                         cudaStream_t s) {
  CMB3D_BATCH_SWITCH(run_batch, grid, boxes, items, nitems, ctr, tw, spin_limit, withhold, s)
}

}  // namespace cmb3d
