// Host side of the cmb3d C ABI: plans, tables, argument checks and the launch
// sequence of one realization.  Compiled with -ffp-contract=off so the FP64
// pixel mapping is evaluated exactly as written (no fused multiply-add).
#include "cmb3d.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "spectrum.h"

namespace {

thread_local std::string g_detail;

int fail(int status, const std::string& msg) {
  g_detail = msg;
  return status;
}

int fail_cuda(cudaError_t e, const char* where) {
  g_detail = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return CMB3D_ECUDA;
}

struct TimingRec {
  int stage;
  cudaEvent_t a, b;
};

constexpr size_t kMaxTimingRecs = 1 << 16;

// Kernel shapes of one realization: variant of the draw+z pass, of the y and
// x passes, or of the fused y+x pass (fused < 0: separate y and x passes).
struct Schedule {
  int draw = 0, y = 0, x = 0, fused = -1;
};

}  // namespace

struct cmb3d_plan_s {
  int N = 0;
  double L = 0, r = 0;
  int interp = 1;
  uint32_t flags = 0;
  int64_t npix = 0;
  int device = 0;
  float2* buf = nullptr;          // packed half spectrum / field, 4 N^3 bytes
  float* amp = nullptr;           // sqrt(P_box(q)/2), q = 0 .. 3 (N/2)^2
  float2* tw = nullptr;           // exp(+2 pi i m / N), m < N
  float4* tab = nullptr;          // pixel table in gather order
  int32_t* perm = nullptr;        // gather order -> caller order (NULL = identity)
  float* outbuf = nullptr;        // staging for cmb3d_realize_sample_to_host
  int64_t dev_bytes = 0;
  bool has_spec = false;
  std::vector<double> knodes, pnodes;
  std::vector<TimingRec> recs;
  size_t tnext = 0;
  Schedule sched;
  bool tuned = false;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <class T>
int dev_alloc(cmb3d_plan_s* p, T** ptr, size_t count, const char* what) {
  *ptr = nullptr;
  if (count == 0) return CMB3D_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? CMB3D_ENOMEM : CMB3D_ECUDA,
                std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
  }
  p->dev_bytes += static_cast<int64_t>(count * sizeof(T));
  return CMB3D_OK;
}

void free_plan(cmb3d_plan_s* p) {
  if (!p) return;
  DeviceGuard g(p->device);
  cudaFree(p->buf);
  cudaFree(p->amp);
  cudaFree(p->tw);
  cudaFree(p->tab);
  cudaFree(p->perm);
  cudaFree(p->outbuf);
  for (auto& r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete p;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Launch `f` on stream s, bracketed by CUDA events when the plan times stages.
template <class F>
cudaError_t timed(cmb3d_plan_s* p, int stage, cudaStream_t s, F f) {
  if (!(p->flags & CMB3D_FLAG_STAGE_TIMING) || p->tnext >= kMaxTimingRecs) return f();
  if (p->tnext == p->recs.size()) {
    TimingRec r{stage, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&r.a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&r.b);
    if (e != cudaSuccess) {
      cudaEventDestroy(r.a);
      return e;
    }
    p->recs.push_back(r);
  }
  TimingRec& r = p->recs[p->tnext++];
  r.stage = stage;
  cudaError_t e = cudaEventRecord(r.a, s);
  if (e != cudaSuccess) return e;
  e = f();
  if (e != cudaSuccess) return e;
  return cudaEventRecord(r.b, s);
}

// Autotuner: time every kernel variant of this box size once (1 warm-up and
// 3 timed launches each, CUDA events on the caller's stream) and keep the
// fastest draw, y and x variants and, where available, the fastest fused y+x
// variant if it beats the best separate pair.  Results are cached per
// (device, N, flag restriction) for the life of the process.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, Schedule> g_tune_cache;

template <class F>
float time_launches(cudaStream_t s, F f, bool* ok) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) {
    *ok = false;
    return 0.f;
  }
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    *ok = false;
    return 0.f;
  }
  float ms = 0.f;
  *ok = f() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess;
  for (int i = 0; i < 3 && *ok; ++i) *ok = f() == cudaSuccess;
  *ok = *ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!*ok) cudaGetLastError();
  return ms / 3.f;
}

int autotune(cmb3d_plan_s* p, cudaStream_t s) {
  const int N = p->N;
  const int restrict_bits = p->flags & (CMB3D_FLAG_THREE_PASS | CMB3D_FLAG_FUSED_YX);
  const std::pair<int, int> key(p->device, N * 16 + restrict_bits);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      p->sched = it->second;
      p->tuned = true;
      return CMB3D_OK;
    }
  }
  Schedule best;
  bool ok = true;
  float t_best = 1e30f;
  for (int v = 0; v < cmb3d::num_col_variants(N); ++v) {
    const float t = time_launches(s, [&] { return cmb3d::launch_draw_zfft(N, v, p->buf, p->amp, p->tw, 1, s); }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune draw_zfft");
    if (t < t_best) t_best = t, best.draw = v;
  }
  float t_y = 1e30f, t_x = 1e30f, t_f = 1e30f;
  for (int v = 0; v < cmb3d::num_col_variants(N); ++v) {
    const float t = time_launches(s, [&] { return cmb3d::launch_yfft(N, v, p->buf, p->tw, s); }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune yfft");
    if (t < t_y) t_y = t, best.y = v;
  }
  for (int v = 0; v < cmb3d::num_row_variants(N); ++v) {
    const float t = time_launches(s, [&] { return cmb3d::launch_xc2r(N, v, p->buf, p->tw, s); }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune xc2r");
    if (t < t_x) t_x = t, best.x = v;
  }
  if (!(p->flags & CMB3D_FLAG_THREE_PASS))
    for (int v = 0; v < cmb3d::num_fused_variants(N); ++v) {
      const float t = time_launches(s, [&] { return cmb3d::launch_yx_fused(N, v, p->buf, p->tw, s); }, &ok);
      if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune yx_fused");
      if (t < t_f) t_f = t, best.fused = v;
    }
  if (!(p->flags & CMB3D_FLAG_FUSED_YX) && t_y + t_x <= t_f) best.fused = -1;
  p->sched = best;
  p->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return CMB3D_OK;
}

// The FFT passes (draw fused into the first), leaving the real field in buf.
int run_field(cmb3d_plan_s* p, uint64_t seed, cudaStream_t s) {
  if ((p->flags & CMB3D_FLAG_AUTOTUNE) && !p->tuned) {
    int st = autotune(p, s);
    if (st != CMB3D_OK) return st;
  }
  const Schedule& sc = p->sched;
  cudaError_t e;
  e = timed(p, CMB3D_STAGE_DRAW_ZFFT, s,
            [&] { return cmb3d::launch_draw_zfft(p->N, sc.draw, p->buf, p->amp, p->tw, seed, s); });
  if (e != cudaSuccess) return fail_cuda(e, "draw_zfft launch");
  if (sc.fused >= 0) {
    e = timed(p, CMB3D_STAGE_YX_FUSED, s, [&] { return cmb3d::launch_yx_fused(p->N, sc.fused, p->buf, p->tw, s); });
    if (e != cudaSuccess) return fail_cuda(e, "yx_fused launch");
    return CMB3D_OK;
  }
  e = timed(p, CMB3D_STAGE_YFFT, s, [&] { return cmb3d::launch_yfft(p->N, sc.y, p->buf, p->tw, s); });
  if (e != cudaSuccess) return fail_cuda(e, "yfft launch");
  e = timed(p, CMB3D_STAGE_XC2R, s, [&] { return cmb3d::launch_xc2r(p->N, sc.x, p->buf, p->tw, s); });
  if (e != cudaSuccess) return fail_cuda(e, "xc2r launch");
  return CMB3D_OK;
}

int run_gather(cmb3d_plan_s* p, float* out, cudaStream_t s) {
  cudaError_t e = timed(p, CMB3D_STAGE_GATHER, s, [&] {
    return cmb3d::launch_gather(p->N, p->interp, reinterpret_cast<const float*>(p->buf), p->tab, p->perm, out,
                                p->npix, s);
  });
  if (e != cudaSuccess) return fail_cuda(e, "gather launch");
  return CMB3D_OK;
}

int check_ready(cmb3d_plan_s* p) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (!p->has_spec) return fail(CMB3D_ENOSPEC, "cmb3d_set_spectrum has not been called on this plan");
  return CMB3D_OK;
}

}  // namespace

extern "C" {

const char* cmb3d_strerror(int status) {
  switch (status) {
    case CMB3D_OK: return "CMB3D_OK";
    case CMB3D_EINVAL: return "CMB3D_EINVAL: invalid argument";
    case CMB3D_ENOMEM: return "CMB3D_ENOMEM: out of memory";
    case CMB3D_ECUDA: return "CMB3D_ECUDA: CUDA error";
    case CMB3D_ENOSPEC: return "CMB3D_ENOSPEC: spectrum not set";
    case CMB3D_ETIMEOUT: return "CMB3D_ETIMEOUT: device wait timed out";
    case CMB3D_EUNSUPPORTED: return "CMB3D_EUNSUPPORTED: unsupported request";
    default: return "unknown cmb3d status";
  }
}

const char* cmb3d_error_detail(void) { return g_detail.c_str(); }

int cmb3d_plan(cmb3d_plan_t* out, int N, double L, double r, const double* pix_xyz, int64_t npix, int interp,
               uint32_t flags) {
  if (!out) return fail(CMB3D_EINVAL, "out is NULL");
  *out = nullptr;
  if (!is_pow2(N) || N < 8 || N > 2048) return fail(CMB3D_EUNSUPPORTED, "N must be a power of two in [8, 2048]");
  if (!(std::isfinite(L) && L > 0) || !(std::isfinite(r) && r > 0)) return fail(CMB3D_EINVAL, "L and r must be finite and > 0");
  if (!(L > 2.0 * r) && !(flags & CMB3D_FLAG_ALLOW_WRAP))
    return fail(CMB3D_EINVAL, "L must exceed 2r (set CMB3D_FLAG_ALLOW_WRAP to allow wrapping)");
  if (npix < 0 || npix >= (int64_t(1) << 31)) return fail(CMB3D_EINVAL, "npix out of range");
  if (npix > 0 && !pix_xyz) return fail(CMB3D_EINVAL, "pix_xyz is NULL");
  if (interp != CMB3D_TRILINEAR && interp != CMB3D_TRICUBIC) return fail(CMB3D_EINVAL, "interp must be 1 or 3");
  if (flags & ~uint32_t(CMB3D_FLAG_NO_SORT | CMB3D_FLAG_ALLOW_WRAP | CMB3D_FLAG_STAGE_TIMING | CMB3D_FLAG_THREE_PASS |
                        CMB3D_FLAG_FUSED_YX | CMB3D_FLAG_AUTOTUNE))
    return fail(CMB3D_EINVAL, "unknown flag bits");
  if ((flags & CMB3D_FLAG_THREE_PASS) && (flags & CMB3D_FLAG_FUSED_YX))
    return fail(CMB3D_EINVAL, "CMB3D_FLAG_THREE_PASS and CMB3D_FLAG_FUSED_YX exclude each other");
  for (int64_t i = 0; i < 3 * npix; ++i)
    if (!std::isfinite(pix_xyz[i])) return fail(CMB3D_EINVAL, "pixel coordinates must be finite");

  cmb3d_plan_s* p = new (std::nothrow) cmb3d_plan_s;
  if (!p) return fail(CMB3D_ENOMEM, "host allocation of the plan");
  p->N = N;
  p->L = L;
  p->r = r;
  p->interp = interp;
  p->flags = flags;
  p->npix = npix;
  if ((flags & CMB3D_FLAG_FUSED_YX) && cmb3d::num_fused_variants(N) > 0) p->sched.fused = 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(CMB3D_ECUDA, "no CUDA device");
  }

  // ---- pixel table (FP64 mapping, then FP32 fractions) --------------------
  std::vector<float4> tab;
  std::vector<int32_t> perm;
  try {
    tab.resize(static_cast<size_t>(npix));
    std::vector<std::pair<uint64_t, int32_t>> order;
    const bool sort = !(flags & CMB3D_FLAG_NO_SORT);
    if (sort) order.resize(static_cast<size_t>(npix));
    const double dp = L / N;
    const double half_l = 0.5 * L;
    std::vector<float4> raw(static_cast<size_t>(npix));
    for (int64_t i = 0; i < npix; ++i) {
      uint32_t b[3];
      float t[3];
      for (int a = 0; a < 3; ++a) {
        const double u = (r * pix_xyz[3 * i + a] + half_l) / dp;
        const double fl = std::floor(u);
        const double frac = u - fl;
        int64_t bi = static_cast<int64_t>(fl) % N;
        if (bi < 0) bi += N;
        b[a] = static_cast<uint32_t>(bi);
        t[a] = static_cast<float>(frac);
      }
      float tz = t[2];
      if (b[2] & 1024u) tz = -tz;  // bit 10 of bz rides in the sign of tz (tz >= 0, -0.0f included)
      uint32_t packed = cmb3d::pack_cell(b[0], b[1], b[2]);
      float w;
      std::memcpy(&w, &packed, sizeof(w));
      raw[static_cast<size_t>(i)] = make_float4(t[0], t[1], tz, w);
      if (sort)
        order[static_cast<size_t>(i)] = {(static_cast<uint64_t>(b[2]) * N + b[1]) * N + b[0], static_cast<int32_t>(i)};
    }
    if (sort) {
      std::sort(order.begin(), order.end());
      perm.resize(static_cast<size_t>(npix));
      for (int64_t i = 0; i < npix; ++i) {
        perm[static_cast<size_t>(i)] = order[static_cast<size_t>(i)].second;
        tab[static_cast<size_t>(i)] = raw[static_cast<size_t>(order[static_cast<size_t>(i)].second)];
      }
    } else {
      tab.swap(raw);
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(CMB3D_ENOMEM, "host allocation of the pixel table");
  }

  // ---- twiddles exp(+2 pi i m / N), FP64 rounded once to FP32 -------------
  std::vector<float2> tw(static_cast<size_t>(N));
  for (int m = 0; m < N; ++m) {
    const double ang = 2.0 * M_PI * static_cast<double>(m) / static_cast<double>(N);
    tw[static_cast<size_t>(m)] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
  }

  const size_t nbuf = static_cast<size_t>(N) * N * (N / 2);
  const size_t nq = 3 * static_cast<size_t>(N / 2) * (N / 2) + 1;
  int st;
  if ((st = dev_alloc(p, &p->buf, nbuf, "box")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->amp, nq, "amplitude table")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->tw, static_cast<size_t>(N), "twiddles")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->tab, static_cast<size_t>(npix), "pixel table")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->outbuf, static_cast<size_t>(npix), "output staging")) != CMB3D_OK ||
      (!perm.empty() && (st = dev_alloc(p, &p->perm, perm.size(), "permutation")) != CMB3D_OK)) {
    free_plan(p);
    return st;
  }
  cudaError_t e = cudaMemcpy(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && npix > 0)
    e = cudaMemcpy(p->tab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !perm.empty())
    e = cudaMemcpy(p->perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_plan(p);
    return fail_cuda(e, "plan upload");
  }
  *out = p;
  return CMB3D_OK;
}

namespace {

int check_cl(const double* x, const double* y, int n, int nkbins) {
  if (!x || !y || n < 1) return fail(CMB3D_EINVAL, "ell, cl must be non-NULL with n >= 1");
  if (nkbins < 8 || nkbins > 4096) return fail(CMB3D_EINVAL, "nkbins must be in [8, 4096]");
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || y[i] <= 0 || x[i] < 2 || x[i] != std::floor(x[i]) ||
        x[i] > 100000)
      return fail(CMB3D_EINVAL, "l must be integers >= 2 and C_l finite and > 0");
    if (i > 0 && !(x[i] > x[i - 1])) return fail(CMB3D_EINVAL, "l must be strictly increasing");
  }
  return CMB3D_OK;
}

}  // namespace

int cmb3d_fit_pk(const double* ell, const double* cl, int n, int N, double L, double r, int nk,
                 double* knodes_out, double* pk_out, double* fit_err) {
  int st = check_cl(ell, cl, n, nk);
  if (st != CMB3D_OK) return st;
  if (!is_pow2(N) || N < 8 || N > 2048) return fail(CMB3D_EUNSUPPORTED, "N must be a power of two in [8, 2048]");
  if (!(std::isfinite(L) && L > 0) || !(std::isfinite(r) && r > 0)) return fail(CMB3D_EINVAL, "L and r must be finite and > 0");
  if (!knodes_out || !pk_out) return fail(CMB3D_EINVAL, "output arrays are NULL");
  std::vector<double> kn, pn;
  double err = 0.0;
  try {
    st = cmb3d::fit_pk_from_cl(ell, cl, n, N, L, r, nk, &kn, &pn, &err, &g_detail);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation in the inversion");
  }
  if (st != CMB3D_OK) return st;
  std::copy(kn.begin(), kn.end(), knodes_out);
  std::copy(pn.begin(), pn.end(), pk_out);
  if (fit_err) *fit_err = err;
  return CMB3D_OK;
}

int cmb3d_set_spectrum(cmb3d_plan_t p, int kind, const double* x, const double* y, int n, int nkbins,
                       double* fit_err) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (!x || !y || n < 1) return fail(CMB3D_EINVAL, "x, y must be non-NULL with n >= 1");
  std::vector<double> kn, pn;
  double err = 0.0;
  if (kind == CMB3D_SPEC_PK) {
    for (int i = 0; i < n; ++i) {
      if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || x[i] < 0 || y[i] < 0)
        return fail(CMB3D_EINVAL, "k and P(k) must be finite and >= 0");
      if (i > 0 && !(x[i] > x[i - 1])) return fail(CMB3D_EINVAL, "k nodes must be strictly increasing");
    }
    kn.assign(x, x + n);
    pn.assign(y, y + n);
  } else if (kind == CMB3D_SPEC_CL) {
    int st = check_cl(x, y, n, nkbins);
    if (st != CMB3D_OK) return st;
    try {
      st = cmb3d::fit_pk_from_cl(x, y, n, p->N, p->L, p->r, nkbins, &kn, &pn, &err, &g_detail);
    } catch (const std::bad_alloc&) {
      return fail(CMB3D_ENOMEM, "host allocation in the inversion");
    }
    if (st != CMB3D_OK) return st;
  } else {
    return fail(CMB3D_EINVAL, "kind must be CMB3D_SPEC_PK or CMB3D_SPEC_CL");
  }

  // Eq. (2.11) for the cubic box: P_box(q) = P_inf(k_f sqrt q) k_f^3, k_f = 2 pi / L.
  const int N = p->N;
  const size_t nq = 3 * static_cast<size_t>(N / 2) * (N / 2) + 1;
  const double kf = 2.0 * M_PI / p->L;
  std::vector<float> amp(nq);
  for (size_t q = 0; q < nq; ++q) {
    const double pb = cmb3d::pk_interp(kn, pn, kf * std::sqrt(static_cast<double>(q))) * kf * kf * kf;
    amp[q] = static_cast<float>(std::sqrt(pb / 2.0));
  }
  DeviceGuard g(p->device);
  cudaError_t e = cudaMemcpy(p->amp, amp.data(), nq * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(e, "amplitude upload");
  p->knodes.swap(kn);
  p->pnodes.swap(pn);
  p->has_spec = true;
  if (fit_err) *fit_err = err;
  return CMB3D_OK;
}

int cmb3d_get_pk(cmb3d_plan_t p, const double* k, double* pk, int n) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (!p->has_spec) return fail(CMB3D_ENOSPEC, "spectrum not set");
  if (n < 0 || (n > 0 && (!k || !pk))) return fail(CMB3D_EINVAL, "bad k/pk arrays");
  for (int i = 0; i < n; ++i) pk[i] = cmb3d::pk_interp(p->knodes, p->pnodes, k[i]);
  return CMB3D_OK;
}

int cmb3d_realize_sample(cmb3d_plan_t p, uint64_t seed, float* out_dev, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (p->npix > 0 && !out_dev) return fail(CMB3D_EINVAL, "out_dev is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = run_field(p, seed, s)) != CMB3D_OK) return st;
  return run_gather(p, out_dev, s);
}

int cmb3d_realize_sample_to_host(cmb3d_plan_t p, uint64_t seed, float* out_host, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (p->npix > 0 && !out_host) return fail(CMB3D_EINVAL, "out_host is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = run_field(p, seed, s)) != CMB3D_OK) return st;
  if ((st = run_gather(p, p->outbuf, s)) != CMB3D_OK) return st;
  if (p->npix > 0) {
    cudaError_t e = cudaMemcpyAsync(out_host, p->outbuf, static_cast<size_t>(p->npix) * sizeof(float),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e, "map download");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "stream synchronize");
  return CMB3D_OK;
}

int cmb3d_realize_sample_batch(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs_dev, int B,
                               void* stream) {
  if (B < 0 || (B > 0 && (!plans || !seeds || !outs_dev))) return fail(CMB3D_EINVAL, "bad batch arrays");
  for (int b = 0; b < B; ++b) {
    int st = check_ready(plans[b]);
    if (st != CMB3D_OK) return st;
    if (plans[b]->N != plans[0]->N || plans[b]->L != plans[0]->L || plans[b]->interp != plans[0]->interp)
      return fail(CMB3D_EINVAL, "batched plans must share N, L and interp");
    if (plans[b]->npix > 0 && !outs_dev[b]) return fail(CMB3D_EINVAL, "outs_dev entry is NULL");
  }
  for (int b = 0; b < B; ++b) {
    int st = cmb3d_realize_sample(plans[b], seeds[b], outs_dev[b], stream);
    if (st != CMB3D_OK) return st;
  }
  return CMB3D_OK;
}

int cmb3d_draw_spectrum(cmb3d_plan_t p, uint64_t seed, void* spec_dev, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (!spec_dev) return fail(CMB3D_EINVAL, "spec_dev is NULL");
  DeviceGuard g(p->device);
  cudaError_t e = cmb3d::launch_draw_only(p->N, static_cast<float2*>(spec_dev), p->amp, seed,
                                          static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "draw launch");
  return CMB3D_OK;
}

int cmb3d_realize_field(cmb3d_plan_t p, uint64_t seed, float* field_dev, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (!field_dev) return fail(CMB3D_EINVAL, "field_dev is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = run_field(p, seed, s)) != CMB3D_OK) return st;
  const size_t bytes = static_cast<size_t>(p->N) * p->N * p->N * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(field_dev, p->buf, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return fail_cuda(e, "field copy");
  return CMB3D_OK;
}

int cmb3d_philox4x32_10(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!ctr_dev || !out_dev))) return fail(CMB3D_EINVAL, "bad philox arguments");
  if ((reinterpret_cast<uintptr_t>(ctr_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15u)
    return fail(CMB3D_EINVAL, "counter and output arrays must be 16-byte aligned");
  cudaError_t e = cmb3d::launch_philox(ctr_dev, seed, out_dev, n, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "philox launch");
  return CMB3D_OK;
}

int cmb3d_stage_times(cmb3d_plan_t p, double* ms, int64_t* launches, int n, int reset) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (!(p->flags & CMB3D_FLAG_STAGE_TIMING)) return fail(CMB3D_EINVAL, "plan was made without CMB3D_FLAG_STAGE_TIMING");
  if (n < 0 || (n > 0 && !ms)) return fail(CMB3D_EINVAL, "bad output arrays");
  std::vector<double> acc(CMB3D_NUM_STAGES, 0.0);
  std::vector<int64_t> cnt(CMB3D_NUM_STAGES, 0);
  DeviceGuard g(p->device);
  for (size_t i = 0; i < p->tnext; ++i) {
    const TimingRec& r = p->recs[i];
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return fail_cuda(e, "event synchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return fail_cuda(e, "event elapsed time");
    acc[static_cast<size_t>(r.stage)] += t;
    cnt[static_cast<size_t>(r.stage)] += 1;
  }
  for (int i = 0; i < n; ++i) {
    ms[i] = i < CMB3D_NUM_STAGES ? acc[static_cast<size_t>(i)] : 0.0;
    if (launches) launches[i] = i < CMB3D_NUM_STAGES ? cnt[static_cast<size_t>(i)] : 0;
  }
  if (reset) p->tnext = 0;
  return CMB3D_OK;
}

int cmb3d_plan_schedule(cmb3d_plan_t p, int* sched) {
  if (!p || !sched) return fail(CMB3D_EINVAL, "plan or sched is NULL");
  sched[0] = p->sched.draw;
  sched[1] = p->sched.fused >= 0 ? -1 : p->sched.y;
  sched[2] = p->sched.fused >= 0 ? -1 : p->sched.x;
  sched[3] = p->sched.fused;
  return CMB3D_OK;
}

int cmb3d_plan_set_schedule(cmb3d_plan_t p, const int* sched) {
  if (!p || !sched) return fail(CMB3D_EINVAL, "plan or sched is NULL");
  const int N = p->N;
  Schedule sc;
  sc.draw = sched[0];
  sc.fused = sched[3];
  if (sc.draw < 0 || sc.draw >= cmb3d::num_col_variants(N)) return fail(CMB3D_EINVAL, "draw variant out of range");
  if (sc.fused >= 0) {
    if (sc.fused >= cmb3d::num_fused_variants(N)) return fail(CMB3D_EINVAL, "fused variant out of range");
    if (p->flags & CMB3D_FLAG_THREE_PASS) return fail(CMB3D_EINVAL, "plan is restricted to separate passes");
  } else {
    sc.fused = -1;
    sc.y = sched[1];
    sc.x = sched[2];
    if (sc.y < 0 || sc.y >= cmb3d::num_col_variants(N)) return fail(CMB3D_EINVAL, "y variant out of range");
    if (sc.x < 0 || sc.x >= cmb3d::num_row_variants(N)) return fail(CMB3D_EINVAL, "x variant out of range");
    if (p->flags & CMB3D_FLAG_FUSED_YX && cmb3d::num_fused_variants(N) > 0)
      return fail(CMB3D_EINVAL, "plan is restricted to the fused pass");
  }
  p->sched = sc;
  p->tuned = true;
  return CMB3D_OK;
}

int cmb3d_plan_info(cmb3d_plan_t p, int* N, int64_t* npix, int64_t* device_bytes) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (N) *N = p->N;
  if (npix) *npix = p->npix;
  if (device_bytes) *device_bytes = p->dev_bytes;
  return CMB3D_OK;
}

void cmb3d_destroy(cmb3d_plan_t p) { free_plan(p); }

}  // extern "C"
