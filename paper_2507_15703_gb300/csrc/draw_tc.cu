// The draw fused with the z-FFT, with the 1024-point transform of every column
// done as two 32-point DFT-GEMMs on the tensor cores (tcgen05, split FP16
// operands, FP32 accumulation in tensor memory).  Same result as the FP32
// Stockham draw (draw_zfft_tile) up to rounding: paper Sec. II.D.1 (a complex
// normal of variance P_box per mode, then the inverse FFT).
//
// Four-step form of X[k] = sum_n x[n] w^(nk), w = exp(+2 pi i / 1024), with
// n = n1 + 32 n2 and k = k2 + 32 k1 (n1, n2, k1, k2 < 32):
//   step 1  Y[n1][k2]  = sum_n2 x[n1 + 32 n2] v^(n2 k2),      v = exp(+2 pi i / 32)
//   twiddle Y'[n1][k2] = Y[n1][k2] w^(n1 k2)
//   step 2  X[k2 + 32 k1] = sum_n1 Y'[n1][k2] v^(n1 k1).
// A tile is T = 4 adjacent columns m_x' of one row m_y; thread t = 32 c + l
// owns GEMM row t in both steps: in step 1 the row (c, n1 = l), whose 32
// inputs it draws itself (the mode pairs (m_z, m_z + 512), m_z = l + 32 n2,
// n2 < 16, share one Philox block); in step 2 the row (c, k2 = l), gathered
// through a padded shared-memory transpose.  A row is 32 complex values, K =
// 64 reals (real and imaginary parts interleaved), times the real 64 x 64 form
// of the 32-point inverse DFT.
//
// Split operands: each value x (scaled) is x_hi + x_lo with x_hi = fp16(x),
// x_lo = fp16(x - x_hi) (about 22 bits), likewise the DFT matrix W; one MMA
// chain accumulates x_hi W_hi + x_lo W_hi + x_hi W_lo (x_lo W_lo, about 2^-22
// of the result, is dropped).  A column's values are scaled by one power of two
// s_c chosen from its largest amplitude so that every real and imaginary part
// is below 2^10 in step 1; step-1 outputs are then below 32 sqrt(2) 2^10, in
// FP16 range without rescaling, and the outputs are multiplied by 1/s_c.
//
// Persistent CTAs of 128 threads take tiles round-robin; the packed Hermitian
// column m_x' = 0 (lane group c = 0 of tile 0 of each row) is drawn by a
// second, small launch with the FP32 Stockham path (4 rows of the column per
// 256-thread block, radix 16).
// Every wait for MMA completion is bounded: after the limit the CTA sets the
// error word and carries on (the result is then wrong, and the host reports it).
#include <cuda_fp16.h>

#include "fft_tiles.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace cmb3d {
namespace {

constexpr int kTcN = 1024, kTcT = 4, kTcThreads = 128, kTcK = 64;
constexpr uint32_t kTcLbo = 128, kTcSbo = (kTcK / 8) * 128;     // K-major, unswizzled core matrices
constexpr int kTcABytes = kTcThreads * kTcK * 2;                 // one 128 x 64 FP16 operand: 16 KB
constexpr int kTcBBytes = 64 * kTcK * 2;                         // the 64 x 64 DFT matrix: 8 KB
constexpr int kTcXPitch = 33;                                    // transpose rows (float2), padded
constexpr int kTcXBytes = kTcThreads * kTcXPitch * 8;            // 33.8 KB, overlaps the A operands
constexpr int kTcAmpPitch = 520;                                 // >= 513 floats per column
// smem: [A_hi | A_lo] (or the transpose buffer, or the amplitude exchange) | B_hi | B_lo
constexpr int kTcOffB = kTcXBytes > 2 * kTcABytes ? ((kTcXBytes + 1023) / 1024) * 1024 : 2 * kTcABytes;
constexpr int kTcSmem = kTcOffB + 2 * kTcBBytes;
constexpr uint32_t kTcSpin = 1u << 24;
constexpr uint32_t kTcCols = 64;                                 // TMEM columns: one 128 x 64 FP32 block

static_assert(kTcSmem <= 227 * 1024, "shared memory");
static_assert(kTcT * kTcAmpPitch * 4 <= kTcOffB, "amplitude exchange fits");

__device__ __forceinline__ uint32_t h2bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// One value pair (re, im) split into FP16 high and low pairs.
__device__ __forceinline__ void split2(float re, float im, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(re, im);
  const float2 hf = __half22float2(h);
  hi = h2bits(h);
  lo = h2bits(__floats2half2_rn(re - hf.x, im - hf.y));
}

// Pairs 4 kc .. 4 kc + 3 (re|im packed in a uint32) of row `row` of a
// K-major operand: one 16-byte chunk.
__device__ __forceinline__ void store_chunk(unsigned char* base, int row, int kc, uint32_t p0, uint32_t p1,
                                            uint32_t p2, uint32_t p3) {
  *reinterpret_cast<uint4*>(base + tc::kmajor_offset(row, 8 * kc, kTcLbo, kTcSbo)) = make_uint4(p0, p1, p2, p3);
}


// The 12 MMAs of one 32-point DFT of all 128 rows: x_hi W_hi + x_lo W_hi + x_hi W_lo.
__device__ __forceinline__ void issue_dft(uint32_t taddr, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                          uint64_t* mbar) {
  constexpr uint32_t idesc = tc::idesc_f16(128, 64, false);
  const uint32_t as[3] = {a_hi, a_lo, a_hi}, bs[3] = {b_hi, b_hi, b_lo};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int ks = 0; ks < kTcK / 16; ++ks)
      tc::mma_f16(taddr, tc::smem_desc(as[p] + 2 * ks * kTcLbo, kTcLbo, kTcSbo),
                  tc::smem_desc(bs[p] + 2 * ks * kTcLbo, kTcLbo, kTcSbo), idesc, (p > 0 || ks > 0) ? 1u : 0u);
  tc::mma_commit(mbar);
}

template <bool KEYP>
__global__ void __launch_bounds__(kTcThreads) k_draw_tc(float2* __restrict__ buf, const float* __restrict__ amp,
                                                        const float2* __restrict__ tw, uint2 key_arg,
                                                        const uint2* __restrict__ keyp,
                                                        const uint32_t* __restrict__ zmask, int zlo, int zhi,
                                                        unsigned* err) {
  constexpr int N = kTcN, N2 = N / 2, H = N / 2;
  constexpr int XT = N2 / kTcT;                     // tiles per row
  constexpr int NREG = XT * N;                      // regular tiles
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  unsigned char* sAhi = smem;
  unsigned char* sAlo = smem + kTcABytes;
  unsigned char* sBhi = smem + kTcOffB;
  unsigned char* sBlo = smem + kTcOffB + kTcBBytes;
  float* sAmp = reinterpret_cast<float*>(smem);
  float2* sX = reinterpret_cast<float2*>(smem);
  const int t = threadIdx.x, c = t >> 5, l = t & 31;
  const uint2 key = KEYP ? *keyp : key_arg;

  // B: the real form of the 32-point inverse DFT, output o = 2 k + p against
  // input i = 2 n + q (p, q: 0 real, 1 imaginary), split into FP16 hi and lo
  if (t < 64) {
    const int k = t >> 1, p = t & 1;
#pragma unroll 1
    for (int kc = 0; kc < 8; ++kc) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int n = 4 * kc + i;
        float sn, cs;
        sincospif(static_cast<float>((n * k) & 31) / 16.0f, &sn, &cs);
        // coefficients of x_n's real and imaginary parts in output (k, p)
        const float wr = p ? sn : cs, wi = p ? cs : -sn;
        split2(wr, wi, hi[i], lo[i]);
      }
      store_chunk(sBhi, t, kc, hi[0], hi[1], hi[2], hi[3]);
      store_chunk(sBlo, t, kc, lo[0], lo[1], lo[2], lo[3]);
    }
  }
  if (t == 0) tc::mbar_init(&mbar, 1);
  if (c == 0) tc::tmem_alloc(&tslot, kTcCols);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_async_shared();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot + (static_cast<uint32_t>(32 * c) << 16);   // this warp's 32 lanes
  const uint32_t a_hi = tc::smem_addr(sAhi), a_lo = tc::smem_addr(sAlo);
  const uint32_t b_hi = tc::smem_addr(sBhi), b_lo = tc::smem_addr(sBlo);
  uint32_t phase = 0;
  bool ok = true;

  for (int tile = blockIdx.x; tile < NREG; tile += gridDim.x) {
    const int my = tile / XT, x0 = (tile % XT) * kTcT, xp = x0 + c;
    const bool live = xp != 0;                        // m_x' = 0 belongs to the Hermitian tiles
    const int fy = my <= H ? my : my - N;
    const int base = xp * xp + fy * fy;
    // amplitudes of the first modes m_z = l + 32 n2 (n2 < 16); those of the
    // second modes, |f_z| = 512 - m_z, come from the lane that owns it
    float alo[16];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) alo[n2] = __ldg(amp + base + (l + 32 * n2) * (l + 32 * n2));
    float* sa = sAmp + c * kTcAmpPitch;
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) sa[l + 32 * n2] = alo[n2];
    if (l == 0) sa[H] = __ldg(amp + base + H * H);
    __syncthreads();
    float ahi[16], mx = 0.0f;
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      ahi[n2] = sa[H - l - 32 * n2];
      mx = fmaxf(mx, fmaxf(alo[n2], ahi[n2]));
    }
    __syncthreads();                                  // the exchange area is reused by the operands
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // s = 2^sh with (largest amplitude x 5.8) 2^sh < 2^10; the Box-Muller radius is below 5.78
    const float big = mx * 5.8f;
    const int e = big > 0.0f ? ((__float_as_int(big) >> 23) & 0xFF) - 127 : 0;
    const int sh = max(-120, min(120, 9 - e));
    const float up = __int_as_float((127 + sh) << 23), down = __int_as_float((127 - sh) << 23);
    // step-1 row (c, n1 = l): pairs n2 (mode l + 32 n2) in chunks of four
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t hl[4], ll[4], hh[4], lh[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int n2 = 4 * g + i;
        const uint4 w = philox4x32_10(make_uint4(xp, my, l + 32 * n2, 0u), key);
        const float2 g0 = box_muller(w.x, w.y), g1 = box_muller(w.z, w.w);
        const float s0 = live ? alo[n2] * up : 0.0f, s1 = live ? ahi[n2] * up : 0.0f;
        split2(s0 * g0.x, s0 * g0.y, hl[i], ll[i]);
        split2(s1 * g1.x, s1 * g1.y, hh[i], lh[i]);
      }
      store_chunk(sAhi, t, g, hl[0], hl[1], hl[2], hl[3]);
      store_chunk(sAlo, t, g, ll[0], ll[1], ll[2], ll[3]);
      store_chunk(sAhi, t, g + 4, hh[0], hh[1], hh[2], hh[3]);
      store_chunk(sAlo, t, g + 4, lh[0], lh[1], lh[2], lh[3]);
    }
    tc::fence_async_shared();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_dft(tslot, a_hi, a_lo, b_hi, b_lo, &mbar);
    if (!tc::mbar_wait(&mbar, phase, kTcSpin)) ok = false;
    phase ^= 1u;
    tc::fence_after_sync();
    // step-1 row (c, n1 = l): Y[k2], twiddled by w^(l k2), into the transpose buffer
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      float d[32];
      tc::tmem_ld32(taddr + 32u * h, d);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k2 = 16 * h + i;
        sX[(32 * c + k2) * kTcXPitch + l] = cmul(make_float2(d[2 * i], d[2 * i + 1]), __ldg(tw + ((l * k2) & (N - 1))));
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // step-2 row (c, k2 = l): Y'[n1][k2] for n1 < 32, split in registers, then
    // stored once every thread has read its row (the buffers overlap)
    uint32_t hi[32], lo[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
      const float2 y = sX[t * kTcXPitch + n1];
      split2(y.x, y.y, hi[n1], lo[n1]);
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      store_chunk(sAhi, t, kc, hi[4 * kc], hi[4 * kc + 1], hi[4 * kc + 2], hi[4 * kc + 3]);
      store_chunk(sAlo, t, kc, lo[4 * kc], lo[4 * kc + 1], lo[4 * kc + 2], lo[4 * kc + 3]);
    }
    tc::fence_async_shared();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_dft(tslot, a_hi, a_lo, b_hi, b_lo, &mbar);
    if (!tc::mbar_wait(&mbar, phase, kTcSpin)) ok = false;
    phase ^= 1u;
    tc::fence_after_sync();
    // outputs X[k2 + 32 k1] of column c, k2 = l
    float2* col = buf + static_cast<size_t>(my) * N2 + xp;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      float d[32];
      tc::tmem_ld32(taddr + 32u * h, d);
      if (live) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int z = l + 32 * (16 * h + i);
          if (z >= zlo && z < zhi && (!zmask || ((__ldg(zmask + (z >> 5)) >> (z & 31)) & 1u)))
            col[static_cast<size_t>(z) * N * N2] = make_float2(d[2 * i] * down, d[2 * i + 1] * down);
        }
      }
    }
    tc::fence_before_sync();
  }
  if (!ok) atomicOr(err, 1u);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (c == 0) tc::tmem_dealloc(tslot, kTcCols);
}

// The packed Hermitian column m_x' = 0 of rows 4 b .. 4 b + 3.
__global__ void __launch_bounds__(256) k_draw_herm(float2* __restrict__ buf, const float* __restrict__ amp,
                                                   const float2* __restrict__ tw, uint2 key,
                                                   const uint2* __restrict__ keyp, const uint32_t* __restrict__ zmask,
                                                   int zlo, int zhi) {
  extern __shared__ float2 hsm[];
  draw_zfft_tile<kTcN, 16, 4, kDrawHermitian>(buf, amp, tw, keyp ? *keyp : key, 4 * blockIdx.x, 0, hsm, zmask, zlo,
                                               zhi);
}

// Persistent grid: as many CTAs as fit on every SM (shared memory allows four
// of 128 threads), after asking for the largest shared-memory carveout.
template <bool KEYP>
int tc_grid() {
  static int grid = 0;
  if (grid > 0) return grid;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(k_draw_tc<KEYP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_draw_tc<KEYP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_draw_tc<KEYP>, kTcThreads, kTcSmem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // the occupancy query can answer below what the shared memory allows (it
  // does not always see the carveout); count from the per-SM budget then
  int smem_sm = 0, reserved = 0;
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
    const int by_smem = smem_sm / (kTcSmem + reserved + 1024);   // 1 KB of static shared memory
    per = per > by_smem ? per : by_smem;
  }
  cudaGetLastError();
  grid = sms * (per > 0 ? (per < 4 ? per : 4) : 1);
  return grid;
}

}  // namespace

bool draw_tc_supported(int N) { return N == kTcN; }

cudaError_t launch_draw_tc(int N, float2* buf, const float* amp, const float2* tw, uint64_t seed, cudaStream_t s,
                           unsigned* err, const uint2* key_dev, const uint32_t* zmask, int zlo, int zhi) {
  if (N != kTcN || !err) return cudaErrorNotSupported;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xFFFFFFFFu), static_cast<uint32_t>(seed >> 32));
  const int hi_z = zhi > 0 ? zhi : N;
  {
    constexpr size_t hs = sizeof(float2) * col_tile_elems<kTcN, 16, 4>();
    static_assert(4 * (kTcN / 16) == 256 && hs <= 48 * 1024, "Hermitian tile: 256 threads, default shared memory");
    k_draw_herm<<<kTcN / 4, 256, hs, s>>>(buf, amp, tw, key, key_dev, zmask, zlo, hi_z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (key_dev) {
    const int g = tc_grid<true>();
    if (g <= 0) return cudaErrorLaunchFailure;
    k_draw_tc<true><<<g, kTcThreads, kTcSmem, s>>>(buf, amp, tw, key, key_dev, zmask, zlo, hi_z, err);
  } else {
    const int g = tc_grid<false>();
    if (g <= 0) return cudaErrorLaunchFailure;
    k_draw_tc<false><<<g, kTcThreads, kTcSmem, s>>>(buf, amp, tw, key, key_dev, zmask, zlo, hi_z, err);
  }
  return cudaGetLastError();
}

}  // namespace cmb3d
