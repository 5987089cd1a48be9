// FFT along y with the radix-16 stages done as split-FP16 DFT-GEMMs on the
// tensor cores (tcgen05, FP32 accumulation in tensor memory).
//
// In each radix-16 Stockham stage every thread owns one butterfly: 16 complex
// inputs.  Its inputs are scaled by a power of two so the largest component is
// below 2^10, split into FP16 high and low parts (x = x_hi + x_lo to about 22
// bits) and written as row m = threadIdx.x of the matrix A = [x_hi | x_lo |
// x_hi] (32 reals each: 16 real parts then 16 imaginary parts).  With B the
// real form of the 16-point inverse DFT, split the same way as
// [W_hi | W_hi | W_lo], one chain of MMAs gives
//     x_hi W_hi + x_lo W_hi + x_hi W_lo
// (the x_lo W_lo term, about 2^-22 of the result, is dropped), read back by the
// same thread from tensor-memory lane m and unscaled.  Twiddles, the last
// radix-2/4 stage and all data movement stay in FP32.
#include <cuda_fp16.h>

#include "fft_tiles.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace cmb3d {
namespace {

constexpr int KDIM = 96;                              // [x_hi | x_lo | x_hi], 32 reals each
constexpr uint32_t kLbo = 128;                        // neighbouring core matrices along K
constexpr uint32_t kSbo = (KDIM / 8) * 128;           // neighbouring 8-row groups
constexpr uint32_t kSpinLimit = 1u << 24;             // polls of the MMA-completion wait
constexpr int kRowBytes = KDIM * 2;

// 2^e as a float, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
  return static_cast<uint32_t>(__half_as_ushort(a)) | (static_cast<uint32_t>(__half_as_ushort(b)) << 16);
}

// Row `row` of a K-major matrix of KDIM halves from vals[KDIM].
__device__ __forceinline__ void store_row(unsigned char* base, int row, const __half* vals) {
#pragma unroll
  for (int kc = 0; kc < KDIM / 8; ++kc) {
    const __half* h = vals + 8 * kc;
    const uint4 q = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
    *reinterpret_cast<uint4*>(base + tc::kmajor_offset(row, 8 * kc, kLbo, kSbo)) = q;
  }
}

struct GemmDft16 {
  unsigned char* sA;
  unsigned char* sB;
  uint64_t* mbar;
  uint32_t taddr;
  int mblocks;
  uint32_t* phase;
  unsigned* err;

  template <int R>
  __device__ __forceinline__ void operator()(float2 (&v)[R]) const {
    static_assert(R == 16, "the tensor-core stage is radix 16");
    const int m = threadIdx.x, warp = m / 32;
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < 16; ++r) mx = fmaxf(mx, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
    // mx < 2^e with e from the exponent field; scale so the largest part is below 2^10
    const int e = mx > 0.f ? ((__float_as_int(mx) >> 23) & 0xFF) - 126 : 0;
    const int sh = max(-120, min(120, 10 - e));
    const float up = pow2f(sh), down = pow2f(-sh);
    __half row[KDIM];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float a = v[r].x * up, b = v[r].y * up;
      const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
      row[r] = ah;
      row[16 + r] = bh;
      row[32 + r] = __float2half_rn(a - __half2float(ah));
      row[48 + r] = __float2half_rn(b - __half2float(bh));
      row[64 + r] = ah;
      row[80 + r] = bh;
    }
    store_row(sA, m, row);
    tc::fence_async_shared();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (m == 0) {
      const uint32_t idesc = tc::idesc_f16(128, 32, false);
      const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
      for (int mb = 0; mb < mblocks; ++mb)
#pragma unroll
        for (int ks = 0; ks < KDIM / 16; ++ks)
          tc::mma_f16(taddr + 32u * mb, tc::smem_desc(a0 + mb * 16 * kSbo + 2 * ks * kLbo, kLbo, kSbo),
                      tc::smem_desc(b0 + 2 * ks * kLbo, kLbo, kSbo), idesc, ks > 0);
      tc::mma_commit(mbar);
    }
    if (!tc::mbar_wait(mbar, *phase, kSpinLimit) && (m & 31) == 0) atomicOr(err, 1u);
    *phase ^= 1u;
    tc::fence_after_sync();
    float d[32];
    tc::tmem_ld32(taddr + (static_cast<uint32_t>(32 * (warp % 4)) << 16) + 32u * (warp / 4), d);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = make_float2(d[k] * down, d[16 + k] * down);
    tc::fence_before_sync();
  }
};

template <int N>
struct GemmShape {
  static constexpr int T = 8, R = 16, NT = T * (N / R), MB = NT / 128, N2 = N / 2, NB = N / R;
  static constexpr int TMEM_COLS = 32 * MB < 32 ? 32 : 32 * MB;
  static constexpr size_t SMEM =
      static_cast<size_t>(NT) * kRowBytes + 32 * kRowBytes + sizeof(float2) * col_tile_elems<N, R, T>();
  static_assert(NT % 128 == 0, "whole 128-row MMA blocks");
};

template <int N>
__global__ void __launch_bounds__(GemmShape<N>::NT) k_yfft_gemm(float2* __restrict__ buf,
                                                                const float2* __restrict__ tw, unsigned* err) {
  using G = GemmShape<N>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sA = smraw;
  unsigned char* sB = smraw + G::NT * kRowBytes;
  float2* sm = reinterpret_cast<float2*>(sB + 32 * kRowBytes);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t slot;
  const int t = threadIdx.x, warp = t / 32;
  if (t < 32) {
    // row n of B: output n (n < 16: real part of X_n, else imaginary part of
    // X_{n-16}) against inputs k (k < 16: real part of x_k, else imaginary
    // part of x_{k-16}); X_q = sum_p x_p exp(+2 pi i p q / 16)
    __half row[KDIM];
    const int q = t % 16, im_out = t / 16;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int p = k % 16, im_in = k / 16;
      float sn, cs;
      sincospif(static_cast<float>((p * q) % 16) / 8.0f, &sn, &cs);
      const float w = im_out ? (im_in ? cs : sn) : (im_in ? -sn : cs);
      const __half wh = __float2half_rn(w);
      row[k] = wh;
      row[32 + k] = wh;
      row[64 + k] = __float2half_rn(w - __half2float(wh));
    }
    store_row(sB, t, row);
  }
  if (t == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&slot, G::TMEM_COLS);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_async_shared();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = slot;
  uint32_t phase = 0;
  GemmDft16 dft{sA, sB, &mbar, taddr, G::MB, &phase, err};

  const int c = t % G::T, j = t / G::T;
  float2* col = buf + static_cast<size_t>(blockIdx.y) * N * G::N2 + blockIdx.x * G::T + c;
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldcg(col + static_cast<size_t>(j + r * G::NB) * G::N2);
  stockham<N, 16, N, false>(
      v, sm, tw, j, [&](int n) { return col_slot<G::R, G::T>(n, c); },
      [&](int n, float2 x) { __stcg(col + static_cast<size_t>(n) * G::N2, x); }, BlockSync{}, dft);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, G::TMEM_COLS);
}

template <int N>
cudaError_t run_yfft_gemm(float2* buf, const float2* tw, unsigned* err, cudaStream_t s) {
  using G = GemmShape<N>;
  auto kern = k_yfft_gemm<N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(G::SMEM));
  if (e != cudaSuccess) return e;
  kern<<<dim3(G::N2 / G::T, N), G::NT, G::SMEM, s>>>(buf, tw, err);
  return cudaGetLastError();
}

}  // namespace

bool yfft_gemm_supported(int N) { return N == 256 || N == 512 || N == 1024; }

cudaError_t launch_yfft_gemm(int N, float2* buf, const float2* tw, unsigned* err, cudaStream_t s) {
  switch (N) {
    case 256: return run_yfft_gemm<256>(buf, tw, err, s);
    case 512: return run_yfft_gemm<512>(buf, tw, err, s);
    case 1024: return run_yfft_gemm<1024>(buf, tw, err, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cmb3d
