// Device building blocks shared by the cmb3d kernels (sm_103a).
//
//  * complex arithmetic on float2;
//  * unnormalised inverse DFTs of radix 2, 4, 8, 16 in registers,
//    X[k] = sum_r v[r] exp(+2 pi i r k / R) (the inverse-transform sign of the
//    paper's Fourier series, Sec. I);
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the uniform /
//    Box-Muller mapping used by the draw;
//  * a Stockham auto-sort FFT engine (Govindaraju et al., SC'08 formulation)
//    that runs one length-NF transform per "column" of a shared-memory tile,
//    all radix-R stages but a final smaller radix, with the first stage's
//    inputs supplied in registers and the last stage's outputs handed to a
//    caller functor (so loads and stores to HBM happen outside the engine).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cmb3d {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// Device code is compiled without implicit contraction (-fmad=false), so the
// rounding of every expression is fixed by the source and identical in every
// kernel that inlines it; the complex product spells out its two FMAs.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }   // i * a
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// exp(+i pi k / 8) for k = 1..7: cos and sin of multiples of 22.5 degrees.
#define CMB3D_C1 0.92387953251128674f   // cos(pi/8)
#define CMB3D_S1 0.38268343236508978f   // sin(pi/8)
#define CMB3D_SQ 0.70710678118654752f   // sqrt(1/2)

template <int R> struct IDft;

template <> struct IDft<1> {
  static __device__ __forceinline__ void run(float2*) {}
};

template <> struct IDft<2> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <> struct IDft<4> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    float2 c = cadd(v[1], v[3]), d = cmul_i(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <> struct IDft<8> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    IDft<4>::run(e);
    IDft<4>::run(o);
    // o[k] *= exp(+i pi k / 4)
    o[1] = make_float2((o[1].x - o[1].y) * CMB3D_SQ, (o[1].x + o[1].y) * CMB3D_SQ);
    o[2] = cmul_i(o[2]);
    o[3] = make_float2((-o[3].x - o[3].y) * CMB3D_SQ, (o[3].x - o[3].y) * CMB3D_SQ);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <> struct IDft<16> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    IDft<8>::run(e);
    IDft<8>::run(o);
    // o[k] *= exp(+i pi k / 8)
    o[1] = cmul(o[1], make_float2(CMB3D_C1, CMB3D_S1));
    o[2] = make_float2((o[2].x - o[2].y) * CMB3D_SQ, (o[2].x + o[2].y) * CMB3D_SQ);
    o[3] = cmul(o[3], make_float2(CMB3D_S1, CMB3D_C1));
    o[4] = cmul_i(o[4]);
    o[5] = cmul(o[5], make_float2(-CMB3D_S1, CMB3D_C1));
    o[6] = make_float2((-o[6].x - o[6].y) * CMB3D_SQ, (o[6].x - o[6].y) * CMB3D_SQ);
    o[7] = cmul(o[7], make_float2(-CMB3D_C1, CMB3D_S1));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 8] = csub(e[k], o[k]);
    }
  }
};

// ---------------------------------------------------------------------------
// Random numbers
// ---------------------------------------------------------------------------

// Philox4x32-10: ten rounds of two 32x32->64 multiplies, XOR of the high
// halves with the round key into the other words, and a word swap; the key is
// bumped by the two Weyl constants between rounds.  Each multiply is one
// 64-bit product (high and low halves together).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ (k.x + i * 0x9E3779B9u), static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ (k.y + i * 0xBB67AE85u), static_cast<uint32_t>(p0));
  }
  return c;
}

// Uniform in (0,1): ((w >> 9) + 1/2) 2^-23, exact in binary32.  The top 23
// bits become the mantissa of 1 + (w >> 9) 2^-23 (the high word of w 2^23 is
// w >> 9, added to the bits of 1.0 by one multiply-add); subtracting
// 1 - 2^-24 is exact (Sterbenz), so no integer-to-float conversion is needed.
__device__ __forceinline__ float one_plus_mantissa(uint32_t w) { return __uint_as_float(__umulhi(w, 1u << 23) + 0x3F800000u); }
__device__ __forceinline__ float uniform_from_word(uint32_t w) {
  return one_plus_mantissa(w) - 0.99999994039535522f;
}

// -2 ln u for a uniform u of the draw (a positive normal binary32 below 1).
// u = 2^e f with f in [sqrt(1/2), sqrt(2)) by an integer split of its bits;
// ln f = 2 atanh(s) with s = (f - 1)/(f + 1), |s| <= 0.1716, and
// 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + s^6/7) with truncation below 8.5e-8
// (relative; it only lowers |atanh|, and a bias of the radius alone averages
// out against the sign-symmetric angle).  f - 1 is exact; the quotient takes
// the hardware reciprocal (rcp.approx.ftz.f32, about 1 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float neg2_log_uniform(float u) {
  const int ix = static_cast<int>(__float_as_uint(u)) - 0x3F3504F3;
  const float ef = static_cast<float>(ix >> 23);
  const float f = __uint_as_float(static_cast<uint32_t>((ix & 0x007FFFFF) + 0x3F3504F3));
  const float s = (f - 1.0f) * rcp_approx(f + 1.0f);
  const float z = s * s;
  // -4 (1 + z/3 + z^2/5 + z^3/7)
  float p = fmaf(z, -0.57142857142857143f, -0.8f);
  p = fmaf(z, p, -1.3333333333333333f);
  p = fmaf(z, p, -4.0f);
  return fmaf(ef, -1.3862943611198906f, s * p);   // -2 e ln 2 - 4 atanh(s)
}

__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller: two standard normals (g1, g2) = sqrt(-2 ln u0) (cos 2 pi u1,
// sin 2 pi u1).  The square root is s * rsqrt(s) (s > 0 since u0 < 1), within
// 2 ulp.  The angle is reduced by half turns: h = nearest integer to 2 u1 comes
// from the rounding of 2 u1 + 1.5 2^23 (no ties: 2 u1 is an odd multiple of
// 2^-23), r = u1 - h/2 in [-1/4, 1/4] is exact, the hardware sine and cosine
// (sin.approx / cos.approx) evaluate a = 2 pi r in [-pi/2, pi/2], and
// (cos, sin)(2 pi u1) = (-1)^h (cos a, sin a), the sign going onto the radius.
// Over all 2^23 uniforms the absolute error of cos and sin stays below 3.4e-7
// (measured against FP64), and it has no mean: the reduced arguments r of odd
// and of even h form the same set, so any systematic error of the hardware
// functions or of the FP32 2 pi cancels between the two signs.  (A plain
// centred angle 2 pi u1 - pi has the same per-value error but a mean of
// 3.5e-8 on the cosine, which the inverse FFT adds up coherently at the
// origin of the field, 1e-5 of its rms at 128^3.)
__device__ __forceinline__ float2 box_muller(uint32_t w0, uint32_t w1) {
  const float s2 = neg2_log_uniform(uniform_from_word(w0));
  const float rad = s2 * rsqrtf(s2);
  const float u1 = uniform_from_word(w1);
  const float t = fmaf(2.0f, u1, 12582912.0f);
  const float a = fmaf(-0.5f, t - 12582912.0f, u1) * 6.283185307179586f;
  const float rs = __uint_as_float(__float_as_uint(rad) ^ (__float_as_uint(t) << 31));   // (-1)^h rad
  return make_float2(rs * cos_approx(a), rs * sin_approx(a));
}

// ---------------------------------------------------------------------------
// Stockham engine
// ---------------------------------------------------------------------------
//
// One transform of length NF per participating thread group.  A thread is
// identified by its butterfly index j in [0, NF/R).  Stage t (sub-transform
// size Ns = R^t) reads elements j + r NF/R, multiplies element r by
// w^(r (j mod Ns)) with w = exp(+2 pi i / (Ns R)), applies the radix-R DFT and
// writes element r to (j div Ns) Ns R + (j mod Ns) + r Ns.  A final stage of
// radix R2 = NF / R^S (when NF is not a power of R) has NF/R2 butterflies,
// R/R2 per thread.  The last stage writes element n in natural order.
//
//   v     first-stage inputs, element r = x[j + r NF/R] (already loaded).
//   sidx  functor: element index n -> shared-memory index of this transform.
//   tw    twiddle table of TWN entries, tw[m] = exp(+2 pi i m / TWN), with
//         TWN a multiple of NF.
//   out   functor (n, value) receiving the final outputs.
//   sync  functor providing the barrier among the threads sharing the tile.
// If FIRST_SYNC, a barrier precedes the first shared-memory write (needed when
// the first-stage inputs were read from the same shared buffer).
struct RegisterDft {
  template <int R>
  __device__ __forceinline__ void operator()(float2 (&v)[R]) const {
    IDft<R>::run(v);
  }
};

// `dft` performs the radix-R transforms of the full stages (all threads call
// it together); the default does them in registers.
template <int NF, int R, int TWN, bool FIRST_SYNC, class SIdx, class Out, class Sync, class Dft = RegisterDft>
__device__ __forceinline__ void stockham(float2 (&v)[R], float2* sm, const float2* __restrict__ tw,
                                         int j, SIdx sidx, Out out, Sync sync, Dft dft = Dft()) {
  constexpr int LR = ilog2c(R), LN = ilog2c(NF);
  constexpr int S = LN / LR;                       // full radix-R stages
  constexpr int R2 = 1 << (LN - S * LR);           // remainder radix (1 = none)
  constexpr int NB = NF / R;                       // butterflies per radix-R stage
  static_assert(S >= 1, "transform shorter than the radix");
  static_assert(TWN % NF == 0, "twiddle table must cover the transform");
  constexpr int TWS = TWN / NF;                    // table stride of exp(2 pi i / NF)

#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int Ns = 1 << (s * LR);
    if (s > 0) {
      sync();
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = sm[sidx(j + r * NB)];
      const int k = j & (Ns - 1);
      const int step = TWS * (NF / (Ns * R)) * k;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + r * step));
    }
    dft(v);
    if (R2 == 1 && s == S - 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) out(j + r * NB, v[r]);
      return;
    }
    if (s > 0 || FIRST_SYNC) sync();
    const int base = (j >> (s * LR)) * (Ns * R) + (j & (Ns - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) sm[sidx(base + r * Ns)] = v[r];
  }
  if constexpr (R2 > 1) {
    constexpr int NB2 = NF / R2;
    constexpr int PER = R / R2;
    sync();
    float2 u[PER][R2];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int jj = j + i * NB;                   // jj < NB2 = Ns, so k = jj
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        float2 x = sm[sidx(jj + r * NB2)];
        if (r > 0) x = cmul(x, __ldg(tw + TWS * r * jj));
        u[i][r] = x;
      }
      IDft<R2>::run(u[i]);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i)
#pragma unroll
      for (int r = 0; r < R2; ++r) out(j + i * NB + r * NB2, u[i][r]);
  }
}

struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

}  // namespace cmb3d
