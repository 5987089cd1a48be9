// Device bodies of the realization passes, shared by the per-pass kernels
// (fft_passes.cu) and the persistent batch kernel (batch.cu).
#pragma once

#include "device_common.cuh"

namespace cmb3d {

// Shared-memory slot of element n of column c in a tile of T columns
// transformed with radix R.  For T < 16 a 16-lane half-warp spans several
// butterflies; one pad slot per R elements puts their 64-bit accesses in
// distinct banks in every Stockham stage (neighbouring butterflies land R + 1
// slots apart in the first store, 1 slot apart afterwards).
template <int R, int T>
__host__ __device__ constexpr int col_slot(int n, int c) {
  return (T < 16 ? n + n / R : n) * T + c;
}
template <int N, int R, int T>
__host__ __device__ constexpr int col_tile_elems() {
  return (T < 16 ? N + N / R : N) * T;
}


// Fourier coefficients of the modes (mx, my, mz) and (mx, my, mz + N/2),
// mz < N/2, which share the Philox counter (mx, my, mz, 0): words (0, 1) draw
// the first, words (2, 3) the second.

// On a Hermitian plane mx in {0, N/2}: the mode with the smaller index
// mz N + my of a conjugate pair draws from its own counter and its partner
// takes the conjugate; self-conjugate modes are real with variance P_box; the
// DC mode is zero.  The partners of the two modes also share one counter.
template <int N>
__device__ __forceinline__ void draw_hermitian_pair(int mx, int my, int mz, const float* __restrict__ amp,
                                                    uint2 key, float2& lo, float2& hi) {
  constexpr int H = N / 2;
  const int py = (N - my) & (N - 1);
  const int pz_lo = (N - mz) & (N - 1), pz_hi = (pz_lo + H) & (N - 1);
  const int fy = my <= H ? my : my - N;
  const int q_lo = mx * mx + fy * fy + mz * mz;
  const int fz_hi = mz + H <= H ? mz + H : mz + H - N;
  const int q_hi = mx * mx + fy * fy + fz_hi * fz_hi;
  const uint4 own = philox4x32_10(make_uint4(mx, my, mz, 0u), key);
  const uint4 par = philox4x32_10(make_uint4(mx, py, pz_lo & (H - 1), 0u), key);
  // partner words: the partner of mode lo is pz_lo (lo words if pz_lo < H)
  const bool plo_is_lo = pz_lo < H;
  float2 out[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int z = h ? mz + H : mz, pz = h ? pz_hi : pz_lo, q = h ? q_hi : q_lo;
    const int lin = z * N + my, plin = pz * N + py;
    const float a = __ldg(amp + q);
    const float2 g_own = h ? box_muller(own.z, own.w) : box_muller(own.x, own.y);
    if (lin == plin) {
      out[h] = q == 0 ? make_float2(0.f, 0.f) : make_float2(a * 1.41421356237309505f * g_own.x, 0.f);
    } else if (lin < plin) {
      out[h] = make_float2(a * g_own.x, a * g_own.y);
    } else {
      const bool use_lo = (h == 0) == plo_is_lo;
      const float2 g = use_lo ? box_muller(par.x, par.y) : box_muller(par.z, par.w);
      out[h] = make_float2(a * g.x, -a * g.y);
    }
  }
  lo = out[0];
  hi = out[1];
}

// Entries (m_x', m_y, mz) and (m_x', m_y, mz + N/2) of the packed half spectrum.
template <int N>
__device__ __forceinline__ void draw_packed_pair(int xp, int my, int mz, const float* __restrict__ amp,
                                                 uint2 key, float2& lo, float2& hi) {
  constexpr int H = N / 2;
  if (xp == 0) {
    float2 A0, A1, B0, B1;
    draw_hermitian_pair<N>(0, my, mz, amp, key, A0, A1);
    draw_hermitian_pair<N>(H, my, mz, amp, key, B0, B1);
    lo = make_float2(A0.x - B0.y, A0.y + B0.x);
    hi = make_float2(A1.x - B1.y, A1.y + B1.x);
    return;
  }
  const int fy = my <= H ? my : my - N;
  const int fz_hi = mz + H <= H ? mz + H : mz + H - N;
  const int base = xp * xp + fy * fy;
  const float a_lo = __ldg(amp + base + mz * mz), a_hi = __ldg(amp + base + fz_hi * fz_hi);
  const uint4 w = philox4x32_10(make_uint4(xp, my, mz, 0u), key);
  const float2 g0 = box_muller(w.x, w.y), g1 = box_muller(w.z, w.w);
  lo = make_float2(a_lo * g0.x, a_lo * g0.y);
  hi = make_float2(a_hi * g1.x, a_hi * g1.y);
}

// Pitch (floats) of one column's amplitude row in the draw's exchange area:
// at least N/2 + 1, and = 32/T mod 32, so that the T columns x 32/T rows of a
// warp hit 32 distinct banks.
template <int N, int T>
__host__ __device__ constexpr int amp_pitch() {
  return (N / 2 + 1 + 31 - ((32 / T) % 32)) / 32 * 32 + (32 / T) % 32;
}
// Shared floats of the draw tile beyond its FFT tile (the amplitude exchange).
template <int N, int T>
__host__ __device__ constexpr int draw_amp_floats() {
  return T * amp_pitch<N, T>();
}

// Which columns a draw tile covers.
enum DrawTileKind {
  kDrawMixed = 0,     // T columns x0 .. x0+T-1 of row m_y; a lane on m_x' = 0 takes the Hermitian path
  kDrawRegular = 1,   // the same, but a lane on m_x' = 0 draws nothing and stores nothing
  kDrawHermitian = 2  // the packed Hermitian column m_x' = 0 of the T rows m_y = x0 .. x0+T-1
};

// Draw + inverse FFT along z of T columns (blockDim.x == T * N / R): one
// thread draws the mode pairs (m_z, m_z + N/2) of its column for its
// first-stage inputs.  Only output planes z in [zlo, zhi) are stored, and with
// `zmask` (N bits) only those whose bit is also set.
//
// kDrawRegular: the amplitude of mode (m_x', m_y, m_z) depends on |f_z| only
// through q = m_x'^2 + f_y^2 + f_z^2, and the thread drawing m_z < N/2 needs
// |f_z| = m_z for the first mode of a pair and N/2 - m_z for the second, which
// is the first mode's |f_z| of thread NB - j.  So each thread reads only its
// first modes' amplitudes from the table (one L2 sector each), shares them
// through shared memory (`sa`: draw_amp_floats<N, T>() floats past the FFT
// tile) and takes the second modes' from there: half the table traffic.
template <int N, int R, int T, int KIND = kDrawMixed>
__device__ __forceinline__ void draw_zfft_tile(float2* __restrict__ buf, const float* __restrict__ amp,
                                               const float2* __restrict__ tw, uint2 key, int x0, int my,
                                               float2* sm, const uint32_t* __restrict__ zmask = nullptr,
                                               int zlo = 0, int zhi = N) {
  constexpr int N2 = N / 2, NB = N / R, H = N / 2;
  static_assert(R < 32, "one bit per output of a thread");
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  float2 v[R];
  float2* col;
  bool store = true;
  if constexpr (KIND == kDrawRegular) {
    constexpr int P = amp_pitch<N, T>();
    const int xp = x0 + c;
    store = xp != 0;
    float* sa = reinterpret_cast<float*>(sm + col_tile_elems<N, R, T>()) + c * P;
    const int fy = my <= H ? my : my - N;
    const int base = xp * xp + fy * fy;
    float alo[R / 2];
#pragma unroll
    for (int r = 0; r < R / 2; ++r) alo[r] = __ldg(amp + base + (j + r * NB) * (j + r * NB));
    const float anyq = j == 0 ? __ldg(amp + base + H * H) : 0.0f;
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      const uint4 w = philox4x32_10(make_uint4(xp, my, j + r * NB, 0u), key);
      const float2 g0 = box_muller(w.x, w.y);
      v[r] = make_float2(alo[r] * g0.x, alo[r] * g0.y);
      v[r + R / 2] = box_muller(w.z, w.w);
      sa[j + r * NB] = alo[r];
    }
    if (j == 0) sa[H] = anyq;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      const float a = sa[H - j - r * NB];
      v[r + R / 2] = make_float2(a * v[r + R / 2].x, a * v[r + R / 2].y);
    }
    if (!store) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
    }
    col = buf + static_cast<size_t>(my) * N2 + xp;            // (z, my, xp) at col[z N N2]
  } else if constexpr (KIND == kDrawHermitian) {
    const int row = x0 + c;
#pragma unroll
    for (int r = 0; r < R / 2; ++r) draw_packed_pair<N>(0, row, j + r * NB, amp, key, v[r], v[r + R / 2]);
    col = buf + static_cast<size_t>(row) * N2;
  } else {
    const int xp = x0 + c;
#pragma unroll
    for (int r = 0; r < R / 2; ++r) draw_packed_pair<N>(xp, my, j + r * NB, amp, key, v[r], v[r + R / 2]);
    col = buf + static_cast<size_t>(my) * N2 + xp;
  }
  // The thread's outputs are n = j + k NB for k < R (in the engine's output
  // order), so the stored range zlo <= n < zhi is one run of k.  At radix 16
  // up to N = 1024 one mask per thread replaces two compares per output
  // (measured: 1.8 % faster at 1024^3; slower at radix 8, where a thread has
  // only eight outputs to spread the mask over, and at 2048^3).
  constexpr bool kMask = R >= 16 && N <= 1024;
  uint32_t kmask = 0u;
  if constexpr (kMask) {
    const int klo = min(R, max(0, (zlo - j + NB - 1) / NB)), khi = min(R, max(0, (zhi - j + NB - 1) / NB));
    kmask = store ? (((1u << khi) - 1u) & ~((1u << klo) - 1u)) : 0u;
  }
  stockham<N, R, N, false>(
      v, sm, tw, j, [&](int n) { return col_slot<R, T>(n, c); },
      [&](int n, float2 x) {
        bool in_range;
        if constexpr (kMask)
          in_range = (kmask >> ((n - j) / NB)) & 1u;
        else
          in_range = store && n >= zlo && n < zhi;
        if (in_range && (!zmask || ((__ldg(zmask + (n >> 5)) >> (n & 31)) & 1u)))
          col[static_cast<size_t>(n) * N * N2] = x;
      },
      BlockSync{});
}

// In-place inverse FFT along y of the T adjacent columns x0 .. x0+T-1 of one
// z-plane (plane points at element (z, 0, 0)); blockDim.x == T * N / R.
// Loads and stores go through L2 only (.cg), so the data may have been written
// by other thread blocks of the same cluster.  With `mask` (N bits, shared
// memory, visible to every thread) only rows y whose bit is set are stored.
template <int N, int R, int T>
__device__ __forceinline__ void yfft_tile(float2* __restrict__ plane, int x0, float2* sm,
                                          const float2* __restrict__ tw, const uint32_t* mask = nullptr) {
  constexpr int N2 = N / 2, NB = N / R;
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  float2* col = plane + x0 + c;                                   // (y, x0 + c) at col[y N2]
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = __ldcg(col + static_cast<size_t>(j + r * NB) * N2);
  stockham<N, R, N, false>(
      v, sm, tw, j, [&](int n) { return col_slot<R, T>(n, c); },
      [&](int n, float2 x) {
        if (!mask || ((mask[n >> 5] >> (n & 31)) & 1u)) __stcg(col + static_cast<size_t>(n) * N2, x);
      },
      BlockSync{});
}

// Row pass: for k in [0, N/2) the half-length input is
//   Y[k] = (G[k] + conj(G[N/2-k])) + i w^k (G[k] - conj(G[N/2-k])),  w = e^{2 pi i/N},
// with G[0], G[N/2] the real and imaginary parts of the packed entry 0, so that
// the N/2-point inverse FFT y[n] = f(2n) + i f(2n+1) is the real row itself.
// Thread j of a row holds G[j + r NB]; when a row's NB threads lie in one warp
// the partner G[N/2 - k] comes from lane (NB - j) mod NB by a shuffle (entry
// R-1-r there, or R-r for lane 0), otherwise through shared memory.
// FIRST_SYNC: shared memory may still be read by an earlier step of the block.
// `g` is the calling thread's row (N/2 packed entries, read through L2) and
// store(n, y) receives entry n of the transformed row, y = (f(2n), f(2n+1)).
template <int N, int R, int ROWS, bool FIRST_SYNC, class Store>
__device__ __forceinline__ void xc2r_row_transform(const float2* g, float2* sm,
                                                   const float2* __restrict__ tw, Store store) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int P = N2 + (N2 >> 4);            // row pitch: one pad slot per 16 entries
  const int j = threadIdx.x % NB, rl = threadIdx.x / NB;
  auto sidx = [&](int n) { return rl * P + n + (n >> 4); };
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = __ldcg(g + j + r * NB);     // all loads in flight at once
  if constexpr (NB <= 32) {
    const int src = (NB - j) & (NB - 1);
    float2 b[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float2 mine = j == 0 ? v[(R - r) % R] : v[R - 1 - r];
      b[r] = make_float2(__shfl_sync(0xffffffffu, mine.x, src, NB), __shfl_sync(0xffffffffu, mine.y, src, NB));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = j + r * NB;
      if (k == 0) {
        v[r] = make_float2(v[r].x + v[r].y, v[r].x - v[r].y);
      } else {
        const float2 a = v[r], c = cconj(b[r]);
        v[r] = cadd(cadd(a, c), cmul_i(cmul(__ldg(tw + k), csub(a, c))));
      }
    }
    stockham<N2, R, N, FIRST_SYNC>(v, sm, tw, j, sidx, store, BlockSync{});
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) sm[sidx(j + r * NB)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = j + r * NB;
      if (k == 0) {
        const float2 p = sm[sidx(0)];
        v[r] = make_float2(p.x + p.y, p.x - p.y);
      } else {
        const float2 a = sm[sidx(k)], c = cconj(sm[sidx(N2 - k)]);
        v[r] = cadd(cadd(a, c), cmul_i(cmul(__ldg(tw + k), csub(a, c))));
      }
    }
    stockham<N2, R, N, true>(v, sm, tw, j, sidx, store, BlockSync{});
  }
}

// The block's rows are rows[0 .. ROWS-1] (consecutive), or with `list` the rows
// rows + list[rl] * N/2 for rl < ROWS; each is transformed in place.  With
// `cols` (one word per listed row) an entry n, the reals 2n and 2n + 1, is
// stored only when bit 2n / (N/32) of the row's word is set.
template <int N, int R, int ROWS, bool FIRST_SYNC = true>
__device__ __forceinline__ void xc2r_rows(float2* __restrict__ rows, float2* sm, const float2* __restrict__ tw,
                                          const int32_t* __restrict__ list = nullptr,
                                          const uint32_t* __restrict__ cols = nullptr) {
  constexpr int N2 = N / 2, NB = N2 / R;
  constexpr int CSH = ilog2c(N) - 5 > 0 ? ilog2c(N) - 5 : 0;   // column blocks of N/32 reals
  static_assert(32 % R == 0, "whole column blocks per output step");
  const int rl = threadIdx.x / NB, j = threadIdx.x % NB;
  float2* g = rows + static_cast<size_t>(list ? __ldg(list + rl) : rl) * N2;
  if (list) {
    // the thread's outputs are n = j + k NB (k < R): entry n holds reals 2n, 2n+1
    // of block (2 j >> CSH) + k 32/R, since 2 k NB = k N/R is a whole number
    // of blocks; so the row's word is shifted once and each output tests one
    // fixed bit (one transform instance for listed rows, with or without cols)
    const uint32_t cmj = cols ? __ldg(cols + rl) >> ((2 * j) >> CSH) : ~0u;
    xc2r_row_transform<N, R, ROWS, FIRST_SYNC>(g, sm, tw, [&](int n, float2 x) {
      if ((cmj >> (((n - j) / NB) * (32 / R))) & 1u) g[n] = x;
    });
  } else {
    xc2r_row_transform<N, R, ROWS, FIRST_SYNC>(g, sm, tw, [&](int n, float2 x) { g[n] = x; });
  }
}

}  // namespace cmb3d
