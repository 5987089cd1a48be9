// One partial-sky map without any device allocation.
//
// Who needs this: code that runs where cudaMalloc is not available to it --
// for example inside a host callback or a plugin of a larger runtime that owns
// every device allocation, or a caller whose memory pool forbids new
// allocations after start-up.  Such a caller can hand us its inputs and its
// output buffer but cannot let the library allocate the box it transforms.
//
// The box (4 N^3 bytes) and the twiddle tables live in one file-scope
// __device__ array of fixed size, sized for N <= CMB3D_NOALLOC_MAX_N (64):
// about 1 MiB.  The driver places it when it loads this module on a device;
// under lazy module loading (the CUDA runtime's default) that happens at the
// first call on that device, and the array then stays until the context is
// destroyed.  In host code the array's name only stands in for it; its device
// address is obtained once per device context with cudaGetSymbolAddress and
// passed to the kernels.  The set-up is redone when the device's context
// changes (cudaDeviceReset), detected by the context's unique id.  All calls
// share the array: each call overwrites the whole box before reading it, so no
// state carries over, but calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it.
#include <cmath>
#include <mutex>

#include "cmb3d.h"
#include "device_common.cuh"
#include "internal.h"

namespace {

constexpr int kMaxN = CMB3D_NOALLOC_MAX_N;
constexpr size_t kBoxBytes = 4ull * kMaxN * kMaxN * kMaxN;
constexpr int kNumSizes = 4;                          // N = 8, 16, 32, 64
constexpr int kTwEntries = 8 + 16 + 32 + 64;          // one exp(2 pi i m / N) table per size
constexpr size_t kTwBytes = 1024;
static_assert(kTwEntries * sizeof(float2) <= kTwBytes, "twiddle area too small");
static_assert(kMaxN == 64, "table layout assumes a 64^3 maximum");

__device__ __align__(256) unsigned char g_noalloc_scratch[kBoxBytes + kTwBytes];

struct DeviceState {
  bool ready = false;
  unsigned long long ctx_id = 0;                      // unique id of the context set up
  unsigned char* base = nullptr;                      // device address of g_noalloc_scratch
};
constexpr int kMaxDevices = 64;
DeviceState g_state[kMaxDevices];
std::mutex g_mu;
float2 g_host_tw[kTwEntries];                         // staging for the set-up upload

int tw_offset(int N) { return N == 8 ? 0 : N == 16 ? 8 : N == 32 ? 24 : 56; }

// Unique id of the calling thread's current context (CUDA driver entry points
// cuCtxGetCurrent and cuCtxGetId, looked up through the runtime so the library
// does not link libcuda).  0 if the driver does not provide them: the set-up
// is then kept for the life of the process.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Once per device context, with that device current: look up the array's
// device address and upload the twiddle tables (a synchronous host-to-device
// copy).  cudaSetDevice on the current device makes its primary context
// current first, so the context id is that of the context the kernels run in.
int setup(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_state[dev];
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  const unsigned long long id = current_context_id();
  if (!st.ready || id != st.ctx_id) {
    st.ready = false;
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return static_cast<int>(e);
    for (int s = 0, N = 8; s < kNumSizes; ++s, N *= 2)
      for (int m = 0; m < N; ++m) {
        const double ang = 2.0 * M_PI * static_cast<double>(m) / static_cast<double>(N);
        g_host_tw[tw_offset(N) + m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
      }
    e = cudaMemcpy(static_cast<unsigned char*>(ptr) + kBoxBytes, g_host_tw, sizeof(g_host_tw), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return static_cast<int>(e);
    st.base = static_cast<unsigned char*>(ptr);
    st.ctx_id = id;
    st.ready = true;
  }
  *base = st.base;
  return 0;
}

template <int INTERP>
struct W;
template <>
struct W<1> {
  static constexpr int K = 2, OFF = 0;
  static __device__ __forceinline__ void run(float t, float* w) {
    w[0] = 1.0f - t;
    w[1] = t;
  }
};
template <>
struct W<3> {
  static constexpr int K = 4, OFF = -1;
  static __device__ __forceinline__ void run(float t, float* w) {
    const float t2 = t * t;
    w[0] = 0.5f * fmaf(2.0f - t, t, -1.0f) * t;
    w[1] = 0.5f * fmaf(fmaf(3.0f, t, -5.0f), t2, 2.0f);
    w[2] = 0.5f * fmaf(fmaf(-3.0f, t, 4.0f), t, 1.0f) * t;
    w[3] = 0.5f * (t - 1.0f) * t2;
  }
};

// Interpolation at pixels given as FP64 unit vectors in device memory.  The
// grid coordinate u = (r n + L/2) / (L/N) is evaluated with IEEE
// round-to-nearest double operations in that order (no contraction), exactly
// as the plan does on the host, so base cells and FP32 fractions agree.
template <int INTERP>
__global__ void __launch_bounds__(256) k_gather_xyz(const float* __restrict__ field, const double* __restrict__ pix,
                                                    float* __restrict__ out, int npix, int N, double L, double r) {
  using Wt = W<INTERP>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const double dp = __ddiv_rn(L, static_cast<double>(N));
  const double half_l = 0.5 * L;
  uint32_t b[3];
  float t[3];
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double u = __ddiv_rn(__dadd_rn(__dmul_rn(r, pix[3 * static_cast<size_t>(i) + a]), half_l), dp);
    if (!(fabs(u) < 4.0e15)) {                        // not finite, or beyond exact integer cells
      finite = false;
      u = 0.0;
    }
    const double fl = floor(u);
    long long bi = static_cast<long long>(fl) % N;
    if (bi < 0) bi += N;
    b[a] = static_cast<uint32_t>(bi);
    t[a] = __double2float_rn(__dsub_rn(u, fl));
  }
  const uint32_t m = static_cast<uint32_t>(N) - 1u;
  float wx[Wt::K], wy[Wt::K], wz[Wt::K];
  Wt::run(t[0], wx);
  Wt::run(t[1], wy);
  Wt::run(t[2], wz);
  uint32_t xs[Wt::K];
#pragma unroll
  for (int a = 0; a < Wt::K; ++a) xs[a] = (b[0] + static_cast<uint32_t>(a + Wt::OFF)) & m;
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < Wt::K; ++c) {
    const size_t zrow = static_cast<size_t>((b[2] + static_cast<uint32_t>(c + Wt::OFF)) & m) * N;
    float accz = 0.0f;
#pragma unroll
    for (int q = 0; q < Wt::K; ++q) {
      const float* row = field + (zrow + ((b[1] + static_cast<uint32_t>(q + Wt::OFF)) & m)) * N;
      float s = 0.0f;
#pragma unroll
      for (int a = 0; a < Wt::K; ++a) s = fmaf(wx[a], row[xs[a]], s);
      accz = fmaf(wy[q], s, accz);
    }
    acc = fmaf(wz[c], accz, acc);
  }
  out[i] = finite ? acc : __int_as_float(0x7FC00000);  // NaN marks a pixel that cannot be placed
}

// Status of a rejected call; the reason is what cmb3d_error_detail() returns.
int fail(int status, const char* reason) {
  cmb3d::set_error_detail(reason);
  return status;
}

}  // namespace

extern "C" int cmb3d_realize_sample_noalloc(int N, double L, double r, const double* pix_dev, int64_t npix,
                                            int interp, const float* amp_dev, uint64_t seed, float* out_dev,
                                            void* stream) {
  if (N < 8 || N > 2048 || (N & (N - 1)) != 0) return fail(CMB3D_EUNSUPPORTED, "N must be a power of two");
  if (N > kMaxN)
    return fail(CMB3D_EUNSUPPORTED, "N exceeds CMB3D_NOALLOC_MAX_N (64), the size of the static scratch box");
  if (!(std::isfinite(L) && L > 0) || !(std::isfinite(r) && r > 0) || !(L > 2.0 * r))
    return fail(CMB3D_EINVAL, "L and r must be finite, positive, with L > 2r");
  if (npix < 0 || npix >= (int64_t(1) << 31)) return fail(CMB3D_EINVAL, "npix out of range");
  if (interp != CMB3D_TRILINEAR && interp != CMB3D_TRICUBIC) return fail(CMB3D_EINVAL, "interp must be 1 or 3");
  if (!amp_dev || (npix > 0 && (!pix_dev || !out_dev))) return fail(CMB3D_EINVAL, "NULL input or output pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(CMB3D_ECUDA, "no usable CUDA device");
  }
  unsigned char* base = nullptr;
  if (setup(dev, &base) != 0) {
    cudaGetLastError();
    return fail(CMB3D_ECUDA, "static scratch set-up failed (cudaGetSymbolAddress or twiddle upload)");
  }
  cmb3d::set_error_detail("");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2* box = reinterpret_cast<float2*>(base);
  const float2* tw = reinterpret_cast<const float2*>(base + kBoxBytes) + tw_offset(N);
  cudaError_t e = cmb3d::launch_draw_zfft(N, 0, box, amp_dev, tw, seed, s);
  if (e == cudaSuccess) e = cmb3d::launch_yfft(N, 0, box, tw, s);
  if (e == cudaSuccess) e = cmb3d::launch_xc2r(N, 0, box, tw, s);
  if (e == cudaSuccess && npix > 0) {
    const unsigned blocks = static_cast<unsigned>((npix + 255) / 256);
    const float* field = reinterpret_cast<const float*>(box);
    if (interp == CMB3D_TRILINEAR)
      k_gather_xyz<1><<<blocks, 256, 0, s>>>(field, pix_dev, out_dev, static_cast<int>(npix), N, L, r);
    else
      k_gather_xyz<3><<<blocks, 256, 0, s>>>(field, pix_dev, out_dev, static_cast<int>(npix), N, L, r);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(CMB3D_ECUDA, cudaGetErrorString(e));
  return CMB3D_OK;
}
