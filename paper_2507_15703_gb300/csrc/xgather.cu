// The last inverse-FFT pass fused with the sampling at the sky pixels (paper
// Sec. II.D.1: the box field is interpolated at r n_hat after the inverse
// transform).  The real rows are formed in shared memory and never written:
// one block per entry (a tile of kXgTile x kXgTile (z, y) base cells, see
// internal.h) transforms the y-transformed rows its pixels' stencils read,
// keeping only the entry's needed x columns, then interpolates its pixels.
// The row transform is the x pass's own (xc2r_row_transform) and the tap
// arithmetic that of interpolate(): same operations in the same order, so the
// maps equal the separate x pass and gather bit for bit.
#include "device_common.cuh"
#include "fft_tiles.cuh"
#include "gather_tiles.cuh"
#include "internal.h"

namespace cmb3d {
namespace {

// Rows per batch and radix of the row transform (256 threads a block).
template <int N>
struct XgShape {
  static constexpr int R = N >= 1024 ? 16 : 8;
  static constexpr int NB = N / 2 / R;
  static constexpr int ROWS = 256 / NB;
  static constexpr int MINB = N >= 1024 ? 2 : 4;    // resident blocks a register budget allows
  static constexpr int P = N / 2 + (N / 2 >> 4);
};

// Row slots per axis of an entry's patch: the tile and the stencil's reach.
template <int INTERP>
struct XgSlots {
  static constexpr int value = kXgTile + Weights<INTERP>::K - 1;
};

// Patch row pitch: odd, so the lanes of a warp reading one column of
// different slots fall in different banks.
constexpr int kXgPitch = kXgCols + 1;

template <int N, int INTERP>
constexpr size_t xg_smem() {
  using S = XgShape<N>;
  constexpr int SL = XgSlots<INTERP>::value;
  return sizeof(float2) * S::ROWS * S::P + sizeof(float) * SL * SL * kXgPitch + sizeof(int16_t) * N;
}

template <int N, int INTERP>
__global__ void __launch_bounds__(256, XgShape<N>::MINB) k_xgather(const float2* __restrict__ buf, const float2* __restrict__ tw,
                                                 const XgEntry* __restrict__ entries,
                                                 const int32_t* __restrict__ row_slot,
                                                 const int32_t* __restrict__ row_glob,
                                                 const int16_t* __restrict__ cols, const float4* __restrict__ tab,
                                                 const int32_t* __restrict__ perm, float* __restrict__ out) {
  using S = XgShape<N>;
  using W = Weights<INTERP>;
  constexpr int N2 = N / 2, SL = XgSlots<INTERP>::value;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);                           // ROWS x P transform scratch
  float* patch = reinterpret_cast<float*>(sm + S::ROWS * S::P);           // SL*SL slots x kXgPitch
  int16_t* xmap = reinterpret_cast<int16_t*>(patch + SL * SL * kXgPitch);  // x -> patch column, or -1
  const XgEntry e = entries[blockIdx.x];
  for (int x = threadIdx.x; x < N; x += blockDim.x) xmap[x] = -1;
  __syncthreads();
  for (int c = threadIdx.x; c < e.ncols; c += blockDim.x) xmap[cols[e.col_begin + c]] = static_cast<int16_t>(c);
  __syncthreads();

  const int rl = threadIdx.x / S::NB;
  for (int rb = 0; rb < e.nrows; rb += S::ROWS) {
    if (rb > 0) __syncthreads();                     // the previous batch has read its scratch
    const int slot = __ldg(row_slot + e.row_begin + rb + rl);
    const float2* g = buf + static_cast<size_t>(__ldg(row_glob + e.row_begin + rb + rl)) * N2;
    float* prow = patch + (slot < 0 ? 0 : slot) * kXgPitch;
    xc2r_row_transform<N, S::R, S::ROWS, false>(g, sm, tw, [&](int n, float2 y) {
      if (slot < 0) return;
      const int c0 = xmap[2 * n], c1 = xmap[2 * n + 1];
      if (c0 >= 0) prow[c0] = y.x;
      if (c1 >= 0) prow[c1] = y.y;
    });
  }
  __syncthreads();

  for (int i = e.pix_begin + static_cast<int>(threadIdx.x); i < e.pix_end; i += blockDim.x) {
    const float4 t = __ldg(tab + i);
    const uint32_t pk = __float_as_uint(t.w);
    const int bx = static_cast<int>(pk & 2047u), by = static_cast<int>((pk >> 11) & 2047u);
    const int bz = static_cast<int>((pk >> 22) | ((__float_as_uint(t.z) >> 31) << 10));
    float wx[W::K], wy[W::K], wz[W::K];
    W::run(t.x, wx);
    W::run(t.y, wy);
    W::run(fabsf(t.z), wz);
    int xc[W::K];
#pragma unroll
    for (int a = 0; a < W::K; ++a) xc[a] = xmap[(bx + a + W::OFF) & (N - 1)];
    const float* base = patch + ((bz - e.z0) * SL + (by - e.y0)) * kXgPitch;
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < W::K; ++c) {
      float accz = 0.0f;
#pragma unroll
      for (int b = 0; b < W::K; ++b) {
        const float* row = base + (c * SL + b) * kXgPitch;
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < W::K; ++a) s = fmaf(wx[a], row[xc[a]], s);
        accz = fmaf(wy[b], s, accz);
      }
      acc = fmaf(wz[c], accz, acc);
    }
    out[perm ? __ldg(perm + i) : i] = acc;
  }
}

template <int N, int INTERP>
cudaError_t run_xgather(const float2* buf, const float2* tw, const XgEntry* entries, int nentries,
                        const int32_t* row_slot, const int32_t* row_glob, const int16_t* cols, const float4* tab,
                        const int32_t* perm, float* out, cudaStream_t s) {
  constexpr size_t smem = xg_smem<N, INTERP>();
  auto kern = k_xgather<N, INTERP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<dim3(static_cast<unsigned>(nentries)), 256, smem, s>>>(buf, tw, entries, row_slot, row_glob, cols, tab,
                                                                 perm, out);
  return cudaGetLastError();
}

}  // namespace

bool xgather_supported(int N) { return N >= 32 && N <= 2048 && (N & (N - 1)) == 0; }

int xgather_rows_per_block(int N) {
  switch (N) {
    case 32: return XgShape<32>::ROWS;
    case 64: return XgShape<64>::ROWS;
    case 128: return XgShape<128>::ROWS;
    case 256: return XgShape<256>::ROWS;
    case 512: return XgShape<512>::ROWS;
    case 1024: return XgShape<1024>::ROWS;
    case 2048: return XgShape<2048>::ROWS;
    default: return 0;
  }
}

cudaError_t launch_xgather(int N, int interp, const float2* buf, const float2* tw, const XgEntry* entries,
                           int nentries, const int32_t* row_slot, const int32_t* row_glob, const int16_t* cols,
                           const float4* tab, const int32_t* perm, float* out, cudaStream_t s) {
  if (nentries <= 0) return cudaSuccess;
#define CMB3D_XG_CASE(n)                                                                                  \
  case n:                                                                                                 \
    return interp == 1 ? run_xgather<n, 1>(buf, tw, entries, nentries, row_slot, row_glob, cols, tab, perm, out, s) \
                       : run_xgather<n, 3>(buf, tw, entries, nentries, row_slot, row_glob, cols, tab, perm, out, s);
  switch (N) {
    CMB3D_XG_CASE(32)
    CMB3D_XG_CASE(64)
    CMB3D_XG_CASE(128)
    CMB3D_XG_CASE(256)
    CMB3D_XG_CASE(512)
    CMB3D_XG_CASE(1024)
    CMB3D_XG_CASE(2048)
    default: return cudaErrorInvalidValue;
  }
#undef CMB3D_XG_CASE
}

}  // namespace cmb3d
