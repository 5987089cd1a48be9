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
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

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

}  // namespace

void cmb3d::set_error_detail(const char* msg) { g_detail = msg ? msg : ""; }

namespace {

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

// State of the persistent batch path, kept in the first plan of a batch: the
// device work list and descriptors of the last plan set, and the CUDA graph
// (counter reset + persistent launch) captured for it.
// Forms: kBatchPersistent (variant = blocks-per-SM variant of the persistent
// kernel) or kBatchStreams (a graph of two streams: the draws of all boxes on
// one, each box's y, x and gather passes on a higher-priority one gated by its
// draw, so draws overlap earlier boxes' memory-bound passes).
enum { kBatchPersistent = 0, kBatchStreams = 1 };

struct BatchCtx {
  std::vector<const void*> plans;
  unsigned spin_limit = 0;
  int withhold = 0;
  int form = -1;
  int variant = 0;
  int grid = 0, nitems = 0;
  cmb3d::BatchBox* d_boxes = nullptr;
  uint64_t* d_items = nullptr;
  unsigned* d_ctr = nullptr;
  uint2* d_keys = nullptr;
  size_t ctr_words = 0;
  std::vector<cmb3d::BatchBox> h_boxes;
  std::vector<uint2> h_keys;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    cudaFree(d_boxes);
    cudaFree(d_items);
    cudaFree(d_ctr);
    cudaFree(d_keys);
    *this = BatchCtx();
  }
};

unsigned g_batch_spin_limit = 1u << 22;   // polls of a bounded wait (about 2 s)
int g_batch_withhold = 0;                 // fault injection: D items never report done
int g_batch_force = -1;                   // tests: 0, 1 persistent variant; 2 two-stream graph

}  // namespace

struct cmb3d_plan_s {
  int N = 0;
  double L = 0, r = 0;
  int interp = 1;
  uint32_t flags = 0;
  int64_t npix = 0;
  int device = 0;
  float2* buf = nullptr;          // packed half spectrum / field, 4 N^3 bytes
  size_t box_elems = 0;           // float2 entries of buf (and buf2): the box and its scratch row
  float* amp = nullptr;           // sqrt(P_box(q)/2), q = 0 .. 3 (N/2)^2
  float2* tw = nullptr;           // exp(+2 pi i m / N), m < N
  float4* tab = nullptr;          // pixel table in gather order
  int32_t* perm = nullptr;        // gather order -> caller order (NULL = identity)
  int2* d_runs = nullptr;         // sorted tables: runs (first pixel, count <= 8) of one base cell
  int64_t nruns = 0;
  float* outbuf = nullptr;        // staging for cmb3d_realize_sample_to_host
  // cmb3d_realize_samples_to_host: a second staging buffer and a copy stream,
  // so the download of map i overlaps the kernels of map i + 1; ev_mapped[k]:
  // staging k holds a finished map, ev_copied[k]: staging k has been read.
  float* outbuf2 = nullptr;
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_mapped[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  unsigned* d_err = nullptr;      // set by a kernel whose bounded wait gave up
  int64_t dev_bytes = 0;
  bool has_spec = false;
  std::vector<double> knodes, pnodes;
  std::vector<TimingRec> recs;
  size_t tnext = 0;
  Schedule sched;
  bool tuned = false;
  BatchCtx batch;
  std::vector<const void*> batch_tuned_sig;   // plan set + outputs the batch autotune ran on
  int batch_best_form = 0, batch_best_v = 0;
  // Pruned transform of the sky-map path: the z-planes and (z, y) rows the
  // pixels' interpolation stencils read.  buf holds one scratch row past the
  // box (row index N^2) that pads the row list.
  bool prune = false;
  int64_t nplanes = 0, nrows = 0, nrows_pad = 0;
  int32_t* d_planes = nullptr;
  int32_t* d_rows = nullptr;
  uint32_t* d_rowmask = nullptr;   // N bits per z-plane
  uint32_t* d_rowcols = nullptr;   // per listed row: the column blocks (N/32 columns each) the stencils read
  int64_t x_stored = 0;            // reals the pruned x pass stores (set column blocks x N/32)
  uint32_t* d_zmask = nullptr;     // N bits: the listed z-planes (the draw stores only these for maps)
  int zlo = 0, zhi = 0;            // listed z-planes as one range [zlo, zhi) when contiguous (then no mask)
  // CMB3D_FLAG_PIPELINE: a second box and two internal streams; the draw of a
  // map (dstream) overlaps the passes and gather of the previous map (pstream,
  // higher priority).  ev_free[k]: box k's last gather done; ev_call: the
  // caller's stream at the call.
  bool pipe = false;
  float2* buf2 = nullptr;
  cudaStream_t dstream = nullptr, pstream = nullptr;
  cudaEvent_t ev_drawn[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr}, ev_call = nullptr;
  int next_box = 0;
  // The 2-D Fourier method (method 2; 3 = the 3-D method): h layers of N x N,
  // z-period M, layer 0 at z0; the per-q square roots of the z-covariance
  // (sqt) replace the amplitude table, and the passes run on plane and row
  // lists that cover the layers (d_planes_all, d_rows_all) or, for sky maps,
  // the pruned lists.
  int method = 3;
  int M = 0, h = 0;
  // CMB3D_FLAG_FUSED_XG: sky maps run the x pass and the gather as one kernel
  // (xgather.cu) on these entries, with the pixel table and permutation in
  // entry order.
  bool xg = false;
  int xg_nentries = 0;
  cmb3d::XgEntry* d_xg_entries = nullptr;
  int32_t* d_xg_slot = nullptr;
  int32_t* d_xg_row = nullptr;
  int16_t* d_xg_cols = nullptr;
  float4* d_xg_tab = nullptr;
  int32_t* d_xg_perm = nullptr;
  double z0 = 0.0;
  float* sqt = nullptr;
  int32_t* d_planes_all = nullptr;
  int32_t* d_rows_all = nullptr;
  int64_t nrows_all_pad = 0;
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

// Test hook (cmb3d_debug_alloc_limit): a plan whose device memory would pass
// this many bytes fails as if the device were out of memory (0: no limit).
int64_t g_alloc_limit = 0;

template <class T>
int dev_alloc(cmb3d_plan_s* p, T** ptr, size_t count, const char* what) {
  *ptr = nullptr;
  if (count == 0) return CMB3D_OK;
  if (g_alloc_limit > 0 && p->dev_bytes + static_cast<int64_t>(count * sizeof(T)) > g_alloc_limit)
    return fail(CMB3D_ENOMEM, std::string("cudaMalloc(") + what + "): beyond the debug allocation limit");
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
  if (p->dstream) cudaStreamSynchronize(p->dstream);
  if (p->pstream) cudaStreamSynchronize(p->pstream);
  if (p->cstream) cudaStreamSynchronize(p->cstream);
  for (cudaEvent_t ev : {p->ev_drawn[0], p->ev_drawn[1], p->ev_free[0], p->ev_free[1], p->ev_call, p->ev_mapped[0],
                         p->ev_mapped[1], p->ev_copied[0], p->ev_copied[1]})
    if (ev) cudaEventDestroy(ev);
  if (p->dstream) cudaStreamDestroy(p->dstream);
  if (p->pstream) cudaStreamDestroy(p->pstream);
  if (p->cstream) cudaStreamDestroy(p->cstream);
  cudaFree(p->buf2);
  cudaFree(p->outbuf2);
  p->batch.release();
  cudaFree(p->buf);
  cudaFree(p->amp);
  cudaFree(p->tw);
  cudaFree(p->tab);
  cudaFree(p->perm);
  cudaFree(p->d_runs);
  cudaFree(p->outbuf);
  cudaFree(p->d_err);
  cudaFree(p->d_planes);
  cudaFree(p->d_rows);
  cudaFree(p->d_rowmask);
  cudaFree(p->d_rowcols);
  cudaFree(p->d_zmask);
  cudaFree(p->sqt);
  cudaFree(p->d_planes_all);
  cudaFree(p->d_rows_all);
  cudaFree(p->d_xg_entries);
  cudaFree(p->d_xg_slot);
  cudaFree(p->d_xg_row);
  cudaFree(p->d_xg_cols);
  cudaFree(p->d_xg_tab);
  cudaFree(p->d_xg_perm);
  for (auto& r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete p;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// y-pass variants: the butterfly shapes, then (where it exists) the
// tensor-core split-FP16 form.
int num_y_variants(int N) { return cmb3d::num_col_variants(N) + (cmb3d::yfft_gemm_supported(N) ? 1 : 0); }
int gemm_y_variant(int N) { return cmb3d::yfft_gemm_supported(N) ? cmb3d::num_col_variants(N) : -1; }

cudaError_t launch_y(cmb3d_plan_s* p, int v, cudaStream_t s, float2* box = nullptr) {
  if (!box) box = p->buf;
  if (v == gemm_y_variant(p->N)) return cmb3d::launch_yfft_gemm(p->N, box, p->tw, p->d_err, s);
  return cmb3d::launch_yfft(p->N, v, box, p->tw, s);
}

// Make stream s wait for everything the plan's internal streams have queued
// (pipelined plans), before work on s that uses the plan's boxes.
cudaError_t join_pipeline(cmb3d_plan_s* p, cudaStream_t s) {
  if (!p->pipe) return cudaSuccess;
  cudaError_t e = cudaStreamWaitEvent(s, p->ev_free[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_free[1], 0);
  return e;
}

// After work on stream s that used box 0 outside the pipeline: the next
// pipelined draw into box 0 waits for it.
cudaError_t mark_box0_used(cmb3d_plan_s* p, cudaStream_t s) {
  return p->pipe ? cudaEventRecord(p->ev_free[0], s) : cudaSuccess;
}

// Wait on the host for the plan's internal streams (before host-side updates
// of device tables they read).
cudaError_t drain_pipeline(cmb3d_plan_s* p) {
  if (!p->pipe) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(p->dstream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->pstream);
  return e;
}

// Error word of the plan's kernels (synchronises); CMB3D_ETIMEOUT if set.
int check_device_error(cmb3d_plan_s* p) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda(e, "error word read");
  if (h) {
    cudaMemset(p->d_err, 0, sizeof(unsigned));
    return fail(CMB3D_ETIMEOUT, "a bounded wait for tensor-core MMA completion gave up");
  }
  return CMB3D_OK;
}

// An NVTX range named after the pass around each launch, for timeline tools
// (nsys, ncu's NVTX filters); inert when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(int stage) {
    static const char* const kNames[] = {"cmb3d draw+z", "cmb3d y pass", "cmb3d x pass", "cmb3d gather",
                                         "cmb3d y+x fused"};
    nvtxRangePushA(stage >= 0 && stage < 5 ? kNames[stage] : "cmb3d pass");
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Launch `f` on stream s inside an NVTX range, bracketed by CUDA events when
// the plan times stages.
template <class F>
cudaError_t timed(cmb3d_plan_s* p, int stage, cudaStream_t s, F f) {
  NvtxRange range(stage);
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

// Autotuner: time every kernel variant of this box size that can run on the
// device (median of 5 launches after 2 warm-ups, CUDA events on the caller's
// stream) and keep the fastest draw, y and x variants and, where available,
// the fastest fused y+x variant if it beats the best separate pair.  Results are cached per
// (device, N, flag restriction) for the life of the process.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, Schedule> g_tune_cache;

// Median of 5 individually timed launches after 2 warm-up launches.
template <class F>
float time_launches(cudaStream_t s, F f, bool* ok) {
  constexpr int kWarm = 2, kRuns = 5;
  cudaEvent_t ev[kRuns + 1];
  int made = 0;
  *ok = true;
  for (; made <= kRuns && *ok; ++made) *ok = cudaEventCreate(&ev[made]) == cudaSuccess;
  if (!*ok) --made;
  for (int i = 0; i < kWarm && *ok; ++i) *ok = f() == cudaSuccess;
  if (*ok) *ok = cudaEventRecord(ev[0], s) == cudaSuccess;
  for (int i = 0; i < kRuns && *ok; ++i) *ok = f() == cudaSuccess && cudaEventRecord(ev[i + 1], s) == cudaSuccess;
  float t[kRuns] = {};
  if (*ok) *ok = cudaEventSynchronize(ev[kRuns]) == cudaSuccess;
  for (int i = 0; i < kRuns && *ok; ++i) *ok = cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]) == cudaSuccess;
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  if (!*ok) {
    cudaGetLastError();
    return 0.f;
  }
  std::sort(t, t + kRuns);
  return t[kRuns / 2];
}

int autotune(cmb3d_plan_s* p, cudaStream_t s) {
  const int N = p->N;
  if (p->method == 2) {                               // y and x shapes on the layer lists
    Schedule best;
    bool ok = true;
    float ty = 1e30f, tx = 1e30f;
    for (int v = 0; v < cmb3d::num_col_variants(N); ++v) {
      const float t = time_launches(s, [&] {
        return cmb3d::launch_yfft(N, v, p->buf, p->tw, s, p->d_planes_all, p->h, nullptr);
      }, &ok);
      if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune yfft");
      if (t < ty) ty = t, best.y = v;
    }
    for (int v = 0; v < cmb3d::num_row_variants(N); ++v) {
      const float t = time_launches(s, [&] {
        return cmb3d::launch_xc2r(N, v, p->buf, p->tw, s, p->d_rows_all, p->nrows_all_pad);
      }, &ok);
      if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune xc2r");
      if (t < tx) tx = t, best.x = v;
    }
    p->sched = best;
    p->tuned = true;
    return CMB3D_OK;                                  // not cached: the layer count is per plan
  }
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
  for (int v = 0; v < cmb3d::num_draw_variants(N); ++v) {   // timed with the plan's stored-plane range
    const float t = time_launches(s, [&] {
      return cmb3d::launch_draw_zfft(N, v, p->buf, p->amp, p->tw, 1, s, nullptr,
                                     p->prune && p->zhi == 0 ? p->d_zmask : nullptr, p->prune ? p->zlo : 0,
                                     p->prune ? p->zhi : 0, p->d_err);
    }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune draw_zfft");
    if (t < t_best) t_best = t, best.draw = v;
  }
  float t_y = 1e30f, t_x = 1e30f, t_f = 1e30f;
  // the y and x shapes are timed on the plane and row lists a sky map of this
  // plan uses (the whole box when it does not prune)
  for (int v = 0; v < cmb3d::num_col_variants(N); ++v) {   // butterfly forms only: FP16 is opt-in
    const float t = time_launches(s, [&] {
      return p->prune ? cmb3d::launch_yfft(N, v, p->buf, p->tw, s, p->d_planes, static_cast<int>(p->nplanes),
                                           p->d_rowmask)
                      : cmb3d::launch_yfft(N, v, p->buf, p->tw, s);
    }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune yfft");
    if (t < t_y) t_y = t, best.y = v;
  }
  for (int v = 0; v < cmb3d::num_row_variants(N); ++v) {
    const float t = time_launches(s, [&] {
      return p->prune ? cmb3d::launch_xc2r(N, v, p->buf, p->tw, s, p->d_rows, p->nrows_pad, p->d_rowcols)
                      : cmb3d::launch_xc2r(N, v, p->buf, p->tw, s);
    }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune xc2r");
    if (t < t_x) t_x = t, best.x = v;
  }
  // fused forms transform the whole box: compared with the separate passes on it
  if (p->prune && !(p->flags & CMB3D_FLAG_THREE_PASS) && cmb3d::num_fused_variants(N) > 0) {
    t_y = t_x = 0.f;
    t_y = time_launches(s, [&] { return cmb3d::launch_yfft(N, best.y, p->buf, p->tw, s); }, &ok);
    if (ok) t_x = time_launches(s, [&] { return cmb3d::launch_xc2r(N, best.x, p->buf, p->tw, s); }, &ok);
    if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune separate passes");
  }
  if (!(p->flags & CMB3D_FLAG_THREE_PASS))
    for (int v = 0; v < cmb3d::num_fused_variants(N); ++v) {
      if (!cmb3d::fused_variant_available(N, v)) continue;
      const float t = time_launches(s, [&] { return cmb3d::launch_yx_fused(N, v, p->buf, p->tw, s); }, &ok);
      if (!ok) return fail_cuda(cudaErrorLaunchFailure, "autotune yx_fused");
      if (t < t_f) t_f = t, best.fused = v;
    }
  if (!(p->flags & CMB3D_FLAG_FUSED_YX) && t_y + t_x <= t_f) best.fused = -1;
  if ((p->flags & CMB3D_FLAG_FP16_GEMM) && gemm_y_variant(N) >= 0) best.fused = -1, best.y = gemm_y_variant(N);
  p->sched = best;
  p->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return CMB3D_OK;
}

int ensure_tuned(cmb3d_plan_s* p, cudaStream_t s) {
  if (!(p->flags & CMB3D_FLAG_AUTOTUNE) || p->tuned) return CMB3D_OK;
  if (cudaError_t e = join_pipeline(p, s); e != cudaSuccess) return fail_cuda(e, "pipeline join");
  return autotune(p, s);
}

// Draw fused with the z pass into `box`.  With `prune` (sky maps of a plan
// with a pruned transform) only the z-planes the y pass reads are stored.
int run_draw(cmb3d_plan_s* p, uint64_t seed, cudaStream_t s, float2* box, bool prune) {
  const Schedule& sc = p->sched;
  cudaError_t e = timed(p, CMB3D_STAGE_DRAW_ZFFT, s, [&] {
    if (p->method == 2) return cmb3d::launch_draw2d(p->N, p->h, box, p->sqt, seed, s);
    const bool pr = prune && p->prune;
    return cmb3d::launch_draw_zfft(p->N, sc.draw, box, p->amp, p->tw, seed, s, nullptr,
                                   pr && p->zhi == 0 ? p->d_zmask : nullptr, pr ? p->zlo : 0, pr ? p->zhi : 0,
                                   p->d_err);
  });
  if (e != cudaSuccess) return fail_cuda(e, "draw_zfft launch");
  return CMB3D_OK;
}

// The y and x passes on `box`, leaving the real field.  With `prune` (sky maps
// of a plan with a pruned transform) the y pass covers only the listed
// z-planes and stores only the marked rows, and the x pass covers only the
// listed rows, in the separate-pass shapes of the schedule.
int run_passes(cmb3d_plan_s* p, cudaStream_t s, bool prune, float2* box) {
  const Schedule& sc = p->sched;
  const bool no_x = prune && p->xg;                   // the gather kernel runs the x pass
  cudaError_t e;
  if (p->method == 2) {                               // the h layers: y and x passes on lists
    const bool pr = prune && p->prune;
    const int yv = sc.y >= 0 ? sc.y : 0, xv = sc.x >= 0 ? sc.x : 0;
    e = timed(p, CMB3D_STAGE_YFFT, s, [&] {
      return cmb3d::launch_yfft(p->N, yv, box, p->tw, s, pr ? p->d_planes : p->d_planes_all,
                                static_cast<int>(pr ? p->nplanes : p->h), pr ? p->d_rowmask : nullptr);
    });
    if (e != cudaSuccess) return fail_cuda(e, "yfft launch");
    if (no_x) return CMB3D_OK;
    e = timed(p, CMB3D_STAGE_XC2R, s, [&] {
      return cmb3d::launch_xc2r(p->N, xv, box, p->tw, s, pr ? p->d_rows : p->d_rows_all,
                                pr ? p->nrows_pad : p->nrows_all_pad, pr ? p->d_rowcols : nullptr);
    });
    if (e != cudaSuccess) return fail_cuda(e, "xc2r launch");
    return CMB3D_OK;
  }
  if (prune && p->prune) {
    const int yv = sc.y >= 0 ? sc.y : 0, xv = sc.x >= 0 ? sc.x : 0;
    e = timed(p, CMB3D_STAGE_YFFT, s, [&] {
      if (yv == gemm_y_variant(p->N)) return launch_y(p, yv, s, box);
      return cmb3d::launch_yfft(p->N, yv, box, p->tw, s, p->d_planes, static_cast<int>(p->nplanes), p->d_rowmask);
    });
    if (e != cudaSuccess) return fail_cuda(e, "yfft launch");
    if (no_x) return CMB3D_OK;
    e = timed(p, CMB3D_STAGE_XC2R, s,
              [&] { return cmb3d::launch_xc2r(p->N, xv, box, p->tw, s, p->d_rows, p->nrows_pad, p->d_rowcols); });
    if (e != cudaSuccess) return fail_cuda(e, "xc2r launch");
    return CMB3D_OK;
  }
  if (no_x) {                                         // whole-box y pass only
    e = timed(p, CMB3D_STAGE_YFFT, s, [&] { return launch_y(p, sc.y >= 0 ? sc.y : 0, s, box); });
    if (e != cudaSuccess) return fail_cuda(e, "yfft launch");
    return CMB3D_OK;
  }
  if (sc.fused >= 0) {
    e = timed(p, CMB3D_STAGE_YX_FUSED, s, [&] { return cmb3d::launch_yx_fused(p->N, sc.fused, box, p->tw, s); });
    if (e != cudaSuccess) return fail_cuda(e, "yx_fused launch");
    return CMB3D_OK;
  }
  e = timed(p, CMB3D_STAGE_YFFT, s, [&] { return launch_y(p, sc.y, s, box); });
  if (e != cudaSuccess) return fail_cuda(e, "yfft launch");
  e = timed(p, CMB3D_STAGE_XC2R, s, [&] { return cmb3d::launch_xc2r(p->N, sc.x, box, p->tw, s); });
  if (e != cudaSuccess) return fail_cuda(e, "xc2r launch");
  return CMB3D_OK;
}

// The whole realization into p->buf on stream s (after the pipeline, if any).
int run_field(cmb3d_plan_s* p, uint64_t seed, cudaStream_t s, bool prune) {
  int st = ensure_tuned(p, s);
  if (st != CMB3D_OK) return st;
  if (cudaError_t e = join_pipeline(p, s); e != cudaSuccess) return fail_cuda(e, "pipeline join");
  if ((st = run_draw(p, seed, s, p->buf, prune)) != CMB3D_OK) return st;
  return run_passes(p, s, prune, p->buf);
}

// Sampling of a sky map from `box`: the gather of the real field, or with the
// fused form (p->xg) the x pass and the gather of the y-transformed box.
int run_gather(cmb3d_plan_s* p, float* out, cudaStream_t s, const float2* box = nullptr) {
  const float2* b = box ? box : p->buf;
  cudaError_t e = timed(p, CMB3D_STAGE_GATHER, s, [&] {
    if (p->xg)
      return cmb3d::launch_xgather(p->N, p->interp, b, p->tw, p->d_xg_entries, p->xg_nentries, p->d_xg_slot,
                                   p->d_xg_row, p->d_xg_cols, p->d_xg_tab, p->d_xg_perm, out, s);
    return cmb3d::launch_gather(p->N, p->interp, reinterpret_cast<const float*>(b), p->tab, p->perm, out, p->npix, s,
                                p->d_runs, p->nruns);
  });
  if (e != cudaSuccess) return fail_cuda(e, "gather launch");
  return CMB3D_OK;
}

// One sky map into `out` through the pipelined plan: the draw on dstream into
// the next box once that box's previous gather is done, the passes and the
// gather on pstream after the draw and after the caller's stream at the call,
// and the caller's stream after the gather.
int run_map_pipelined(cmb3d_plan_s* p, uint64_t seed, float* out, cudaStream_t s) {
  const bool was_tuned = p->tuned;
  int st = ensure_tuned(p, s);
  if (st != CMB3D_OK) return st;
  if (p->tuned != was_tuned) {                        // the autotuner just used box 0 on s
    cudaError_t e = cudaEventRecord(p->ev_free[0], s);
    if (e != cudaSuccess) return fail_cuda(e, "pipeline order");
  }
  const int k = p->next_box;
  float2* box = k ? p->buf2 : p->buf;
  cudaError_t e = cudaStreamWaitEvent(p->dstream, p->ev_free[k], 0);
  if (e != cudaSuccess) return fail_cuda(e, "pipeline wait");
  if ((st = run_draw(p, seed, p->dstream, box, true)) != CMB3D_OK) return st;
  e = cudaEventRecord(p->ev_drawn[k], p->dstream);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_call, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->pstream, p->ev_call, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->pstream, p->ev_drawn[k], 0);
  if (e != cudaSuccess) return fail_cuda(e, "pipeline order");
  if ((st = run_passes(p, p->pstream, true, box)) != CMB3D_OK) return st;
  if ((st = run_gather(p, out, p->pstream, box)) != CMB3D_OK) return st;
  e = cudaEventRecord(p->ev_free[k], p->pstream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_free[k], 0);
  if (e != cudaSuccess) return fail_cuda(e, "pipeline order");
  p->next_box = k ^ 1;
  return CMB3D_OK;
}

// Host tables of a plan, built from the pixels alone (no device): the pixel
// table in gather order and its permutation, the gather runs, and the pruned
// transform's row mask, plane and row lists and per-row column blocks.
// Throws std::bad_alloc.
struct PixelTables {
  std::vector<float4> tab;
  std::vector<int32_t> perm;
  std::vector<uint32_t> rowmask;
  std::vector<int32_t> planes, rows, planes_all, rows_all;
  std::vector<int2> runs;
  std::vector<uint32_t> rowcols;   // per listed row: the column blocks (N/32 columns) the stencils read
  int64_t x_stored = 0;            // reals the pruned x pass stores
  bool outside = false;            // 2-D: a stencil leaves the layers
};

void build_pixel_tables(int N, int nz, int method, int h, double L, double r, double z0, const double* pix_xyz,
                        int64_t npix, int interp, uint32_t flags, PixelTables* t) {
  std::vector<float4>& tab = t->tab;
  std::vector<int32_t>& perm = t->perm;
  std::vector<uint32_t>& rowmask = t->rowmask;
  std::vector<int32_t>& planes = t->planes;
  std::vector<int32_t>& rows = t->rows;
  std::vector<int32_t>& planes_all = t->planes_all;
  std::vector<int32_t>& rows_all = t->rows_all;
  std::vector<int2>& runs = t->runs;
  std::vector<uint32_t>& rowcols = t->rowcols;
  std::vector<uint32_t> colmask;
  int64_t& x_stored = t->x_stored;
  bool& outside = t->outside;
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
      const double u = (r * pix_xyz[3 * i + a] + (method == 2 && a == 2 ? -z0 : half_l)) / dp;
      const double fl = std::floor(u);
      const double frac = u - fl;
      int64_t bi;
      if (method == 2 && a == 2) {                  // layers: no wrap, whole stencil inside
        bi = fl >= -2.0 && fl <= 2048.0 ? static_cast<int64_t>(fl) : -8;
        const int64_t lo = interp == CMB3D_TRICUBIC ? bi - 1 : bi, hi = interp == CMB3D_TRICUBIC ? bi + 2 : bi + 1;
        if (lo < 0 || hi > h - 1) {
          outside = true;
          bi = 0;
        }
      } else {
        bi = static_cast<int64_t>(fl) % N;
        if (bi < 0) bi += N;
      }
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
    // runs of at most kGatherRun pixels sharing one base cell (the key is the cell)
    for (int64_t i = 0; i < npix;) {
      int64_t j = i + 1;
      while (j < npix && j - i < cmb3d::kGatherRun &&
             order[static_cast<size_t>(j)].first == order[static_cast<size_t>(i)].first)
        ++j;
      runs.push_back(make_int2(static_cast<int>(i), static_cast<int>(j - i)));
      i = j;
    }
  } else {
    tab.swap(raw);
  }
  // rows (z, y) read by the interpolation stencils: z in bz + OFF .. bz + OFF + K - 1
  // (mod N), likewise y; consecutive pixels of one row are visited once
  const int K = interp == CMB3D_TRICUBIC ? 4 : 2, OFF = interp == CMB3D_TRICUBIC ? -1 : 0;
  const size_t words = static_cast<size_t>(N) * N / 32;
  if (!(flags & CMB3D_FLAG_NO_PRUNE) && N >= 128 && npix > 0) {
    rowmask.assign(words, 0u);
    colmask.assign(static_cast<size_t>(nz) * N, 0u);
    const int csh = cmb3d::ilog2i(N) - 5;            // column block: N / 32 columns
    uint64_t prev = ~uint64_t(0);
    uint32_t cur = 0;                               // column blocks of the current (z, y) group
    auto flush = [&](uint64_t key) {
      const int bz = static_cast<int>(key / static_cast<uint64_t>(N)), by = static_cast<int>(key % N);
      for (int c = 0; c < K; ++c) {
        const int z = (bz + c + OFF + N) & (N - 1);
        if (z >= nz) continue;
        for (int b = 0; b < K; ++b)
          colmask[static_cast<size_t>(z) * N + static_cast<size_t>((by + b + OFF + N) & (N - 1))] |= cur;
      }
    };
    for (int64_t i = 0; i < npix; ++i) {
      uint64_t key;
      int bx;
      if (sort) {
        key = order[static_cast<size_t>(i)].first / static_cast<uint64_t>(N);
        bx = static_cast<int>(order[static_cast<size_t>(i)].first % static_cast<uint64_t>(N));
      } else {
        uint32_t bits;
        const float4 e4 = tab[static_cast<size_t>(i)];
        std::memcpy(&bits, &e4.w, sizeof(bits));
        uint32_t sgn;
        std::memcpy(&sgn, &e4.z, sizeof(sgn));
        const uint64_t by = (bits >> 11) & 2047u, bz = (bits >> 22) | ((sgn >> 31) << 10);
        key = bz * static_cast<uint64_t>(N) + by;
        bx = static_cast<int>(bits & 2047u);
      }
      if (key != prev && prev != ~uint64_t(0)) {
        flush(prev);
        cur = 0;
      }
      for (int a = 0; a < K; ++a) cur |= 1u << (((bx + a + OFF + N) & (N - 1)) >> csh);
      if (key == prev) continue;
      prev = key;
      const int bz = static_cast<int>(key / static_cast<uint64_t>(N)), by = static_cast<int>(key % N);
      for (int c = 0; c < K; ++c) {
        const int z = (bz + c + OFF + N) & (N - 1);
        for (int b = 0; b < K; ++b) {
          const size_t row = static_cast<size_t>(z) * N + static_cast<size_t>((by + b + OFF + N) & (N - 1));
          rowmask[row >> 5] |= 1u << (row & 31);
        }
      }
    }
    if (prev != ~uint64_t(0)) flush(prev);
    for (int z = 0; z < N; ++z) {
      bool any = false;
      for (int w = 0; w < N / 32; ++w) {
        const uint32_t m = rowmask[static_cast<size_t>(z) * (N / 32) + w];
        any = any || m != 0;
        for (int bit = 0; bit < 32; ++bit)
          if ((m >> bit) & 1u) rows.push_back(z * N + w * 32 + bit);
      }
      if (any) planes.push_back(z);
    }
    if (static_cast<int64_t>(rows.size()) == static_cast<int64_t>(nz) * N) {   // nothing to prune
      rows.clear();
      planes.clear();
      rowmask.clear();
    } else {
      while (rows.size() % cmb3d::kRowListPad) rows.push_back(nz * N);   // scratch row past the box
      rowcols.resize(rows.size());
      for (size_t k = 0; k < rows.size(); ++k) {
        rowcols[k] = rows[k] < nz * N ? colmask[static_cast<size_t>(rows[k])] : 0u;   // scratch: store nothing
        x_stored += static_cast<int64_t>(__builtin_popcount(rowcols[k])) * (N / 32);
      }
    }
    colmask.clear();
    colmask.shrink_to_fit();
  }
  if (method == 2) {                                // every layer and row, for whole layers
    for (int z = 0; z < h; ++z) planes_all.push_back(z);
    for (int rr = 0; rr < h * N; ++rr) rows_all.push_back(rr);
    while (rows_all.size() % cmb3d::kRowListPadAny) rows_all.push_back(h * N);
  }
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

// Plan of the 3-D method (method 3) or of the 2-D Fourier method (method 2,
// with M, h, z0); the two share the pixel table, pruning and the passes.
namespace {

// Entries of the fused x pass + gather (internal.h): the pixels grouped by
// their tile of kXgTile x kXgTile (z, y) base cells, tiles in (z, y) order so
// that neighbouring entries share halo rows in L2; a tile whose stencils
// reach more than kXgCols distinct x is split into runs of increasing bx.
struct XgHost {
  std::vector<cmb3d::XgEntry> entries;
  std::vector<int32_t> slot, row;
  std::vector<int16_t> cols;
  std::vector<float4> tab;
  std::vector<int32_t> perm;
};

void build_xgather(int N, int nz, int interp, const std::vector<float4>& tab, const std::vector<int32_t>& perm,
                   XgHost* xg) {
  const int K = interp == CMB3D_TRICUBIC ? 4 : 2, OFF = interp == CMB3D_TRICUBIC ? -1 : 0;
  const int T = cmb3d::kXgTile, SL = T + K - 1, ROWS = cmb3d::xgather_rows_per_block(N);
  const int ntz = (nz + T - 1) / T, nty = N / T;
  const size_t npix = tab.size();
  std::vector<int32_t> bx(npix), by(npix), bz(npix);
  std::vector<int64_t> start(static_cast<size_t>(ntz) * nty + 1, 0);
  for (size_t i = 0; i < npix; ++i) {
    uint32_t w, z;
    std::memcpy(&w, &tab[i].w, sizeof(w));
    std::memcpy(&z, &tab[i].z, sizeof(z));
    bx[i] = static_cast<int32_t>(w & 2047u);
    by[i] = static_cast<int32_t>((w >> 11) & 2047u);
    bz[i] = static_cast<int32_t>((w >> 22) | ((z >> 31) << 10));
    ++start[static_cast<size_t>(bz[i] / T) * nty + by[i] / T + 1];
  }
  for (size_t t = 1; t < start.size(); ++t) start[t] += start[t - 1];
  std::vector<int32_t> order(npix);
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (size_t i = 0; i < npix; ++i)
      order[static_cast<size_t>(fill[static_cast<size_t>(bz[i] / T) * nty + by[i] / T]++)] = static_cast<int32_t>(i);
  }
  std::vector<int> stamp(static_cast<size_t>(N), -1);
  int group_id = 0;
  auto emit = [&](const int32_t* g, size_t n, int tz, int ty) {
    cmb3d::XgEntry e{};
    e.z0 = tz * T;
    e.y0 = ty * T;
    e.pix_begin = static_cast<int32_t>(xg->tab.size());
    e.col_begin = static_cast<int32_t>(xg->cols.size());
    e.row_begin = static_cast<int32_t>(xg->slot.size());
    std::vector<char> col(static_cast<size_t>(N), 0), used(static_cast<size_t>(SL) * SL, 0);
    for (size_t k = 0; k < n; ++k) {
      const size_t i = static_cast<size_t>(g[k]);
      xg->tab.push_back(tab[i]);
      xg->perm.push_back(perm.empty() ? static_cast<int32_t>(i) : perm[i]);
      for (int a = 0; a < K; ++a) col[static_cast<size_t>((bx[i] + a + OFF + N) & (N - 1))] = 1;
      const int lz = bz[i] - e.z0, ly = by[i] - e.y0;
      for (int c = 0; c < K; ++c)
        for (int b = 0; b < K; ++b) used[static_cast<size_t>((lz + c) * SL + ly + b)] = 1;
    }
    for (int x = 0; x < N; ++x)
      if (col[static_cast<size_t>(x)]) xg->cols.push_back(static_cast<int16_t>(x));
    for (int sl = 0; sl < SL * SL; ++sl) {
      if (!used[static_cast<size_t>(sl)]) continue;
      const int gz = ((e.z0 + sl / SL + OFF) % N + N) % N, gy = ((e.y0 + sl % SL + OFF) % N + N) % N;
      xg->slot.push_back(sl);
      xg->row.push_back(gz * N + gy);
    }
    while ((xg->slot.size() - static_cast<size_t>(e.row_begin)) % static_cast<size_t>(ROWS)) {
      xg->slot.push_back(-1);                         // padding: the scratch row past the box
      xg->row.push_back(nz * N);
    }
    e.pix_end = static_cast<int32_t>(xg->tab.size());
    e.ncols = static_cast<int32_t>(xg->cols.size()) - e.col_begin;
    e.nrows = static_cast<int32_t>(xg->slot.size()) - e.row_begin;
    xg->entries.push_back(e);
  };
  for (int tz = 0; tz < ntz; ++tz)
    for (int ty = 0; ty < nty; ++ty) {
      const size_t t = static_cast<size_t>(tz) * nty + ty;
      const int64_t b0 = start[t], b1 = start[t + 1];
      if (b0 == b1) continue;
      int ncols = 0;
      ++group_id;
      for (int64_t k = b0; k < b1; ++k)
        for (int a = 0; a < K; ++a) {
          int& st = stamp[static_cast<size_t>((bx[static_cast<size_t>(order[static_cast<size_t>(k)])] + a + OFF + N) &
                                              (N - 1))];
          if (st != group_id) st = group_id, ++ncols;
        }
      if (ncols <= cmb3d::kXgCols) {
        emit(order.data() + b0, static_cast<size_t>(b1 - b0), tz, ty);
        continue;
      }
      std::stable_sort(order.begin() + b0, order.begin() + b1,
                       [&](int32_t u, int32_t v) { return bx[static_cast<size_t>(u)] < bx[static_cast<size_t>(v)]; });
      int64_t g0 = b0;
      ncols = 0;
      ++group_id;
      for (int64_t k = b0; k < b1; ++k) {
        const int x0 = bx[static_cast<size_t>(order[static_cast<size_t>(k)])];
        int add = 0;
        for (int a = 0; a < K; ++a) add += stamp[static_cast<size_t>((x0 + a + OFF + N) & (N - 1))] != group_id;
        if (ncols + add > cmb3d::kXgCols) {           // close the run before this pixel
          emit(order.data() + g0, static_cast<size_t>(k - g0), tz, ty);
          g0 = k;
          ncols = 0;
          ++group_id;
        }
        for (int a = 0; a < K; ++a) {
          int& st = stamp[static_cast<size_t>((x0 + a + OFF + N) & (N - 1))];
          if (st != group_id) st = group_id, ++ncols;
        }
      }
      emit(order.data() + g0, static_cast<size_t>(b1 - g0), tz, ty);
    }
}

}  // namespace

static int create_plan(cmb3d_plan_t* out, int method, int N, int M, int h, double L, double r, double z0,
                       const double* pix_xyz, int64_t npix, int interp, uint32_t flags) {
  if (!out) return fail(CMB3D_EINVAL, "out is NULL");
  *out = nullptr;
  if (method == 2) {
    if (!is_pow2(N) || N < 16 || N > 2048) return fail(CMB3D_EUNSUPPORTED, "N must be a power of two in [16, 2048]");
    if (h < 1 || h > 32 || h > N) return fail(CMB3D_EUNSUPPORTED, "h must satisfy 1 <= h <= 32 and h <= N");
    if (M < 1 || M > 65536) return fail(CMB3D_EINVAL, "M must be in [1, 65536]");
    if (!std::isfinite(z0)) return fail(CMB3D_EINVAL, "z0 must be finite");
    if (flags & (CMB3D_FLAG_FUSED_YX | CMB3D_FLAG_FP16_GEMM))
      return fail(CMB3D_EUNSUPPORTED, "the 2-D method runs the separate FP32 y and x passes");
  } else if (!is_pow2(N) || N < 8 || N > 2048) {
    return fail(CMB3D_EUNSUPPORTED, "N must be a power of two in [8, 2048]");
  }
  if (!(std::isfinite(L) && L > 0) || !(std::isfinite(r) && r > 0)) return fail(CMB3D_EINVAL, "L and r must be finite and > 0");
  if (method == 3 && !(L > 2.0 * r) && !(flags & CMB3D_FLAG_ALLOW_WRAP))
    return fail(CMB3D_EINVAL, "L must exceed 2r (set CMB3D_FLAG_ALLOW_WRAP to allow wrapping)");
  if (npix < 0 || npix >= (int64_t(1) << 31)) return fail(CMB3D_EINVAL, "npix out of range");
  if (npix > 0 && !pix_xyz) return fail(CMB3D_EINVAL, "pix_xyz is NULL");
  if (interp != CMB3D_TRILINEAR && interp != CMB3D_TRICUBIC) return fail(CMB3D_EINVAL, "interp must be 1 or 3");
  if (flags & ~uint32_t(CMB3D_FLAG_NO_SORT | CMB3D_FLAG_ALLOW_WRAP | CMB3D_FLAG_STAGE_TIMING | CMB3D_FLAG_THREE_PASS |
                        CMB3D_FLAG_FUSED_YX | CMB3D_FLAG_AUTOTUNE | CMB3D_FLAG_FP16_GEMM |
                        CMB3D_FLAG_NO_PRUNE | CMB3D_FLAG_PIPELINE | CMB3D_FLAG_FUSED_XG))
    return fail(CMB3D_EINVAL, "unknown flag bits");
  if ((flags & CMB3D_FLAG_FP16_GEMM) && (flags & CMB3D_FLAG_FUSED_YX))
    return fail(CMB3D_EINVAL, "CMB3D_FLAG_FP16_GEMM uses separate y and x passes");
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
  p->method = method;
  p->M = M;
  p->h = h;
  p->z0 = z0;
  const int nz = method == 2 ? h : N;                 // z-planes of the box buffer
  if ((flags & CMB3D_FLAG_FUSED_YX) && cmb3d::num_fused_variants(N) > 0) p->sched.fused = 0;
  if (flags & CMB3D_FLAG_FP16_GEMM) {
    if (gemm_y_variant(N) < 0) {
      delete p;
      return fail(CMB3D_EUNSUPPORTED, "the tensor-core FFT stage exists for N = 256, 512, 1024");
    }
    p->sched.y = gemm_y_variant(N);
  }
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(CMB3D_ECUDA, "no CUDA device");
  }

  // ---- pixel table (FP64 mapping, then FP32 fractions) --------------------
  PixelTables pt;
  try {
    build_pixel_tables(N, nz, method, h, L, r, z0, pix_xyz, npix, interp, flags, &pt);
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(CMB3D_ENOMEM, "host allocation of the pixel table");
  }
  std::vector<float4>& tab = pt.tab;
  std::vector<int32_t>& perm = pt.perm;
  std::vector<uint32_t>& rowmask = pt.rowmask;
  std::vector<int32_t>& planes = pt.planes;
  std::vector<int32_t>& rows = pt.rows;
  std::vector<int32_t>& planes_all = pt.planes_all;
  std::vector<int32_t>& rows_all = pt.rows_all;
  std::vector<int2>& runs = pt.runs;
  std::vector<uint32_t>& rowcols = pt.rowcols;
  const int64_t x_stored = pt.x_stored;
  const bool outside = pt.outside;
  if (outside) {
    delete p;
    return fail(CMB3D_EINVAL, "a pixel's interpolation stencil leaves the h simulated layers");
  }

  // ---- twiddles exp(+2 pi i m / N), FP64 rounded once to FP32 -------------
  std::vector<float2> tw(static_cast<size_t>(N));
  for (int m = 0; m < N; ++m) {
    const double ang = 2.0 * M_PI * static_cast<double>(m) / static_cast<double>(N);
    tw[static_cast<size_t>(m)] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
  }

  const size_t nbuf = static_cast<size_t>(nz) * N * (N / 2) + (N / 2);   // + the scratch row
  const size_t nq = method == 2 ? 0 : 3 * static_cast<size_t>(N / 2) * (N / 2) + 1;
  int st;
  p->box_elems = nbuf;
  if ((st = dev_alloc(p, &p->buf, nbuf, "box")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->amp, nq, "amplitude table")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->d_planes_all, planes_all.size(), "layer list")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->d_rows_all, rows_all.size(), "layer row list")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->tw, static_cast<size_t>(N), "twiddles")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->tab, static_cast<size_t>(npix), "pixel table")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->outbuf, static_cast<size_t>(npix), "output staging")) != CMB3D_OK ||
      (st = dev_alloc(p, &p->d_err, 1, "error word")) != CMB3D_OK ||
      (!perm.empty() && (st = dev_alloc(p, &p->perm, perm.size(), "permutation")) != CMB3D_OK) ||
      (!runs.empty() && (st = dev_alloc(p, &p->d_runs, runs.size(), "gather runs")) != CMB3D_OK) ||
      (!rows.empty() && ((st = dev_alloc(p, &p->d_rows, rows.size(), "row list")) != CMB3D_OK ||
                         (st = dev_alloc(p, &p->d_planes, planes.size(), "plane list")) != CMB3D_OK ||
                         (st = dev_alloc(p, &p->d_rowmask, rowmask.size(), "row mask")) != CMB3D_OK ||
                         (st = dev_alloc(p, &p->d_rowcols, rowcols.size(), "row column blocks")) != CMB3D_OK ||
                         (st = dev_alloc(p, &p->d_zmask, static_cast<size_t>((N + 31) / 32), "plane mask")) != CMB3D_OK))) {
    free_plan(p);
    return st;
  }
  cudaError_t e = cudaMemcpy(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(unsigned));
  if (e == cudaSuccess && npix > 0)
    e = cudaMemcpy(p->tab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !perm.empty())
    e = cudaMemcpy(p->perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !runs.empty()) {
    e = cudaMemcpy(p->d_runs, runs.data(), runs.size() * sizeof(int2), cudaMemcpyHostToDevice);
    p->nruns = static_cast<int64_t>(runs.size());
  }
  if (e == cudaSuccess && !rows_all.empty()) {
    e = cudaMemcpy(p->d_planes_all, planes_all.data(), planes_all.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_rows_all, rows_all.data(), rows_all.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    p->nrows_all_pad = static_cast<int64_t>(rows_all.size());
  }
  if (e == cudaSuccess && !rows.empty()) {
    e = cudaMemcpy(p->d_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_planes, planes.data(), planes.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_rowmask, rowmask.data(), rowmask.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_rowcols, rowcols.data(), rowcols.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      std::vector<uint32_t> zmask(static_cast<size_t>((N + 31) / 32), 0u);
      for (int32_t z : planes) zmask[static_cast<size_t>(z) >> 5] |= 1u << (z & 31);
      e = cudaMemcpy(p->d_zmask, zmask.data(), zmask.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
      if (!planes.empty() && planes.back() - planes.front() + 1 == static_cast<int32_t>(planes.size())) {
        p->zlo = planes.front();                      // contiguous: a range test, no mask reads
        p->zhi = planes.back() + 1;
      }
    }
    p->prune = true;
    p->nplanes = static_cast<int64_t>(planes.size());
    p->nrows_pad = static_cast<int64_t>(rows.size());
    p->x_stored = x_stored;
    p->nrows = 0;
    for (int32_t rr : rows) p->nrows += rr < nz * N ? 1 : 0;
  }
  if (e == cudaSuccess && (flags & CMB3D_FLAG_FUSED_XG) && npix > 0 && cmb3d::xgather_supported(N)) {
    XgHost xg;
    try {
      build_xgather(N, nz, interp, tab, perm, &xg);
    } catch (const std::bad_alloc&) {
      free_plan(p);
      return fail(CMB3D_ENOMEM, "host allocation of the fused gather's entries");
    }
    if ((st = dev_alloc(p, &p->d_xg_entries, xg.entries.size(), "fused gather entries")) != CMB3D_OK ||
        (st = dev_alloc(p, &p->d_xg_slot, xg.slot.size(), "fused gather slots")) != CMB3D_OK ||
        (st = dev_alloc(p, &p->d_xg_row, xg.row.size(), "fused gather rows")) != CMB3D_OK ||
        (st = dev_alloc(p, &p->d_xg_cols, xg.cols.size(), "fused gather columns")) != CMB3D_OK ||
        (st = dev_alloc(p, &p->d_xg_tab, xg.tab.size(), "fused gather pixel table")) != CMB3D_OK ||
        (st = dev_alloc(p, &p->d_xg_perm, xg.perm.size(), "fused gather permutation")) != CMB3D_OK) {
      free_plan(p);
      return st;
    }
    e = cudaMemcpy(p->d_xg_entries, xg.entries.data(), xg.entries.size() * sizeof(cmb3d::XgEntry),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_xg_slot, xg.slot.data(), xg.slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_xg_row, xg.row.data(), xg.row.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_xg_cols, xg.cols.data(), xg.cols.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_xg_tab, xg.tab.data(), xg.tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_xg_perm, xg.perm.data(), xg.perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    p->xg_nentries = static_cast<int>(xg.entries.size());
    p->xg = e == cudaSuccess;
  }
  if (e == cudaSuccess && (flags & CMB3D_FLAG_PIPELINE)) {
    if ((st = dev_alloc(p, &p->buf2, nbuf, "second box")) != CMB3D_OK) {
      free_plan(p);
      return st;
    }
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->dstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->pstream, cudaStreamNonBlocking, hi);
    for (cudaEvent_t* ev : {&p->ev_drawn[0], &p->ev_drawn[1], &p->ev_free[0], &p->ev_free[1], &p->ev_call})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    p->pipe = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    free_plan(p);
    return fail_cuda(e, "plan upload");
  }
  *out = p;
  return CMB3D_OK;
}

int cmb3d_plan(cmb3d_plan_t* out, int N, double L, double r, const double* pix_xyz, int64_t npix, int interp,
               uint32_t flags) {
  return create_plan(out, 3, N, 0, 0, L, r, 0.0, pix_xyz, npix, interp, flags);
}

int cmb3d_plan_2d(cmb3d_plan_t* out, int N, int M, int h, double L, double r, double z0, const double* pix_xyz,
                  int64_t npix, int interp, uint32_t flags) {
  return create_plan(out, 2, N, M, h, L, r, z0, pix_xyz, npix, interp, flags);
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

int cmb3d_cl_matrix(const double* ell, int n, const double* knodes, int nk, double r, double* out) {
  if (!ell || !knodes || !out || n < 1 || nk < 2) return fail(CMB3D_EINVAL, "bad arrays");
  if (!(std::isfinite(r) && r > 0)) return fail(CMB3D_EINVAL, "r must be finite and > 0");
  for (int i = 0; i < n; ++i)
    if (!(ell[i] >= 0) || ell[i] != std::floor(ell[i]) || ell[i] > 100000) return fail(CMB3D_EINVAL, "bad l");
  for (int j = 0; j < nk; ++j)
    if (!std::isfinite(knodes[j]) || knodes[j] < 0 || (j > 0 && !(knodes[j] > knodes[j - 1])))
      return fail(CMB3D_EINVAL, "k nodes must be finite, >= 0 and increasing");
  try {
    std::vector<double> kn(knodes, knodes + nk);
    std::vector<double> A = cmb3d::cl_design_matrix(ell, n, kn, r, 16);
    std::copy(A.begin(), A.end(), out);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the design matrix");
  }
  return CMB3D_OK;
}

// The linear-programming inversion (paper Sec. II.B): argument checks, the
// grid, the targets and the matrix, shared by the two entry points below.
namespace {

int lp_setup(const double* ell, const double* cl, int nl, double R, double theta_max, double beam, double dr,
             double dk, double kmax, cmb3d::LpGrid* g, std::vector<double>* b, std::vector<double>* A) {
  if (!ell || !cl || nl < 1) return fail(CMB3D_EINVAL, "ell, cl must be non-NULL with n >= 1");
  for (int i = 0; i < nl; ++i) {
    if (!std::isfinite(ell[i]) || ell[i] < 0 || ell[i] != std::floor(ell[i]) || ell[i] > 100000 ||
        !std::isfinite(cl[i]) || cl[i] < 0)
      return fail(CMB3D_EINVAL, "l must be integers in [0, 100000] and C_l finite and >= 0");
    if (i > 0 && !(ell[i] > ell[i - 1])) return fail(CMB3D_EINVAL, "l must be strictly increasing");
  }
  int st = cmb3d::lp_grid(R, theta_max, beam, dr, dk, kmax, g, &g_detail);
  if (st != CMB3D_OK) return st;
  if (static_cast<double>(g->m) * g->n > 6.4e7 || static_cast<double>(g->n) * (g->m + 2.0 * g->n) > 6.4e7)
    return fail(CMB3D_EUNSUPPORTED, "linear program larger than 6.4e7 matrix or tableau entries");
  try {
    cmb3d::lp_targets(ell, cl, nl, beam, R, *g, b);
    if (A) {
      const unsigned hc = std::thread::hardware_concurrency();
      cmb3d::lp_matrix(*g, static_cast<int>(std::max(1u, std::min(hc, 32u))), A);
    }
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the linear program");
  }
  return CMB3D_OK;
}

}  // namespace

int cmb3d_lp_system(const double* ell, const double* cl, int n, double R, double theta_max, double beam,
                    double dr, double dk, double kmax, int* m_out, int* nk_out, double* r_out, double* knodes_out,
                    double* A_out, double* b_out) {
  if (!m_out || !nk_out) return fail(CMB3D_EINVAL, "m_out and nk_out must be non-NULL");
  cmb3d::LpGrid g;
  std::vector<double> b, A;
  int st = lp_setup(ell, cl, n, R, theta_max, beam, dr, dk, kmax, &g, &b, A_out ? &A : nullptr);
  if (st != CMB3D_OK) return st;
  *m_out = g.m;
  *nk_out = g.n;
  if (r_out)
    for (int i = 0; i < g.m; ++i) r_out[i] = i * g.dr;
  if (knodes_out)
    for (int j = 0; j <= g.n; ++j) knodes_out[j] = j * g.dk;
  if (b_out) std::copy(b.begin(), b.end(), b_out);
  if (A_out) std::copy(A.begin(), A.end(), A_out);
  return CMB3D_OK;
}

int cmb3d_fit_pk_lp(const double* ell, const double* cl, int n, double R, double theta_max, double beam,
                    double dr, double dk, double kmax, int cap, double* knodes_out, double* pk_out, int* nk_out,
                    double* objective, double* xi_err) {
  if (!knodes_out || !pk_out || !nk_out) return fail(CMB3D_EINVAL, "output arrays are NULL");
  cmb3d::LpGrid g;
  std::vector<double> b, A, x;
  int st = lp_setup(ell, cl, n, R, theta_max, beam, dr, dk, kmax, &g, &b, &A);
  if (st != CMB3D_OK) return st;
  if (cap < g.n + 1) return fail(CMB3D_EINVAL, "cap is smaller than the number of k nodes (nk + 1)");
  long pivots = 0;
  try {
    st = cmb3d::lp_solve(A, g.m, g.n, b, 100L * (g.m + g.n) + 10000, &x, &pivots, &g_detail);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the simplex tableau");
  }
  if (st != CMB3D_OK) return st;
  double obj = 0.0, worst = 0.0;
  for (int j = 0; j < g.n; ++j) {
    double c = 0.0;
    for (int i = 0; i < g.m; ++i) c += A[static_cast<size_t>(i) * g.n + j];
    obj += c * x[static_cast<size_t>(j)];
  }
  for (int i = 0; i < g.m; ++i) {
    double s = 0.0;
    for (int j = 0; j < g.n; ++j) s += A[static_cast<size_t>(i) * g.n + j] * x[static_cast<size_t>(j)];
    worst = std::max(worst, std::fabs(s - b[static_cast<size_t>(i)]));
  }
  for (int j = 0; j <= g.n; ++j) {
    knodes_out[j] = j * g.dk;
    pk_out[j] = j < g.n ? x[static_cast<size_t>(j)] : 0.0;
  }
  *nk_out = g.n + 1;
  if (objective) *objective = obj;
  if (xi_err) *xi_err = b[0] != 0.0 ? worst / std::fabs(b[0]) : worst;
  return CMB3D_OK;
}

// The 2-D method's per-q square roots of the z-covariance (host FP64, then
// FP32 on the device) from P_inf on the nodes (kn, pn).
static int set_spectrum_2d(cmb3d_plan_s* p, std::vector<double>& kn, std::vector<double>& pn, double err,
                           double* fit_err) {
  const int N = p->N, h = p->h;
  std::vector<float> table;
  try {
    const unsigned hc = std::thread::hardware_concurrency();
    cmb3d::sqrt_gamma_table(N, p->M, h, p->L, kn, pn, static_cast<int>(std::max(1u, std::min(hc, 32u))), &table);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the z-covariance table");
  }
  DeviceGuard g(p->device);
  cudaError_t e = drain_pipeline(p);                 // no draw of the plan still reads the table
  if (e != cudaSuccess) return fail_cuda(e, "pipeline drain");
  if (!p->sqt) {
    int st = dev_alloc(p, &p->sqt, table.size(), "z-covariance table");
    if (st != CMB3D_OK) return st;
  }
  e = cudaMemcpy(p->sqt, table.data(), table.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(e, "z-covariance table upload");
  p->knodes.swap(kn);
  p->pnodes.swap(pn);
  p->has_spec = true;
  if (fit_err) *fit_err = err;
  return CMB3D_OK;
}

int cmb3d_gamma_sqrt_table(int N, int M, int h, double L, const double* k, const double* pk, int n, float* out) {
  if (!is_pow2(N) || N < 2 || N > 2048 || M < 1 || M > 65536 || h < 1 || h > 64)
    return fail(CMB3D_EINVAL, "N (power of two), M or h out of range");
  if (!(std::isfinite(L) && L > 0) || !k || !pk || n < 1 || !out) return fail(CMB3D_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(k[i]) || !std::isfinite(pk[i]) || k[i] < 0 || pk[i] < 0 || (i > 0 && !(k[i] > k[i - 1])))
      return fail(CMB3D_EINVAL, "k must increase; k and P(k) finite and >= 0");
  try {
    std::vector<float> table;
    const unsigned hc = std::thread::hardware_concurrency();
    cmb3d::sqrt_gamma_table(N, M, h, L, std::vector<double>(k, k + n), std::vector<double>(pk, pk + n),
                            static_cast<int>(std::max(1u, std::min(hc, 32u))), &table);
    std::copy(table.begin(), table.end(), out);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the z-covariance table");
  }
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

  if (p->method == 2) return set_spectrum_2d(p, kn, pn, err, fit_err);
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
  cudaError_t e = drain_pipeline(p);                 // no draw of the plan still reads amp
  if (e == cudaSuccess) e = cudaMemcpy(p->amp, amp.data(), nq * sizeof(float), cudaMemcpyHostToDevice);
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
  if (p->pipe) return run_map_pipelined(p, seed, out_dev, s);
  if ((st = run_field(p, seed, s, true)) != CMB3D_OK) return st;
  return run_gather(p, out_dev, s);
}

int cmb3d_realize_sample_to_host(cmb3d_plan_t p, uint64_t seed, float* out_host, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (p->npix > 0 && !out_host) return fail(CMB3D_EINVAL, "out_host is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->pipe) {
    if ((st = run_map_pipelined(p, seed, p->outbuf, s)) != CMB3D_OK) return st;
  } else {
    if ((st = run_field(p, seed, s, true)) != CMB3D_OK) return st;
    if ((st = run_gather(p, p->outbuf, s)) != CMB3D_OK) return st;
  }
  if (p->npix > 0) {
    cudaError_t e = cudaMemcpyAsync(out_host, p->outbuf, static_cast<size_t>(p->npix) * sizeof(float),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e, "map download");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "stream synchronize");
  return check_device_error(p);
}

int cmb3d_realize_samples_to_host(cmb3d_plan_t p, const uint64_t* seeds, int count, float* const* outs_host,
                                  void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (count < 0 || (count > 0 && (!seeds || !outs_host))) return fail(CMB3D_EINVAL, "seeds or outs_host is NULL");
  for (int i = 0; i < count && p->npix > 0; ++i)
    if (!outs_host[i]) return fail(CMB3D_EINVAL, "an output pointer is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (p->npix > 0 && !p->outbuf2 &&               // first use: second staging buffer
      (st = dev_alloc(p, &p->outbuf2, static_cast<size_t>(p->npix), "second output staging")) != CMB3D_OK)
    return st;
  if (p->npix > 0 && !p->cstream) {               // ... the copy stream and its events
    e = cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      if (!p->ev_mapped[k]) e = cudaEventCreateWithFlags(&p->ev_mapped[k], cudaEventDisableTiming);
      if (e == cudaSuccess && !p->ev_copied[k]) e = cudaEventCreateWithFlags(&p->ev_copied[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      if (p->cstream) cudaStreamDestroy(p->cstream);
      p->cstream = nullptr;
      return fail_cuda(e, "copy stream setup");
    }
  }
  // On an error every download already queued is waited for, so that no copy
  // writes into the caller's host buffers after the call has returned.
  auto abort_with = [&](int status) {
    if (p->cstream) cudaStreamSynchronize(p->cstream);
    return status;
  };
  const size_t bytes = static_cast<size_t>(p->npix) * sizeof(float);
  for (int i = 0; i < count; ++i) {
    const int k = i & 1;
    float* staging = k ? p->outbuf2 : p->outbuf;
    if (p->npix > 0 && (e = cudaStreamWaitEvent(s, p->ev_copied[k], 0)) != cudaSuccess)
      return abort_with(fail_cuda(e, "staging order"));                     // map i - 2 has been read
    if (p->pipe) {
      if ((st = run_map_pipelined(p, seeds[i], staging, s)) != CMB3D_OK) return abort_with(st);
    } else {
      if ((st = run_field(p, seeds[i], s, true)) != CMB3D_OK) return abort_with(st);
      if ((st = run_gather(p, staging, s)) != CMB3D_OK) return abort_with(st);
    }
    if (p->npix == 0) continue;
    e = cudaEventRecord(p->ev_mapped[k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->cstream, p->ev_mapped[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(outs_host[i], staging, bytes, cudaMemcpyDeviceToHost, p->cstream);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_copied[k], p->cstream);
    if (e != cudaSuccess) return abort_with(fail_cuda(e, "map download"));
  }
  if (p->cstream) {
    e = cudaStreamWaitEvent(s, p->ev_copied[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_copied[1], 0);
    if (e != cudaSuccess) return abort_with(fail_cuda(e, "staging order"));
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return abort_with(fail_cuda(e, "stream synchronize"));
  return check_device_error(p);
}

namespace {

// Work list of a batch: round t lists the draw items of box t interleaved, by
// proportional position, with the y, x and gather items of box t-kLag, so the
// draws a pass waits for were handed out a full round earlier.
// Pruned extents of a box for the persistent kernel: (planes, rows) of its y
// and x passes, the whole box when the plan is not pruned.
void batch_extent(const cmb3d_plan_s* p, int* ny_tiles, int* nx_blocks, int* nY, int* nX) {
  const int64_t N = p->N;
  cmb3d::batch_box_counts(p->N, p->prune ? p->nplanes : N, p->prune ? p->nrows_pad : N * N, ny_tiles, nx_blocks,
                          nY, nX);
}

std::vector<uint64_t> batch_work_list(const cmb3d_plan_t* plans, int B, int N) {
  const int nD = cmb3d::batch_draw_items(N);
  constexpr int kLag = 2;
  std::vector<uint64_t> items;
  for (int t = 0; t < B + kLag; ++t) {
    std::vector<uint64_t> a, b;
    if (t < B)
      for (int i = 0; i < nD; ++i) a.push_back(cmb3d::batch_item(t, cmb3d::kBatchDraw, i));
    if (t >= kLag) {
      const int bx = t - kLag;
      const int nG = static_cast<int>((plans[bx]->npix + cmb3d::kBatchPixelsPerItem - 1) / cmb3d::kBatchPixelsPerItem);
      int nyt, nxb, nY, nX;
      batch_extent(plans[bx], &nyt, &nxb, &nY, &nX);
      for (int i = 0; i < nY; ++i) b.push_back(cmb3d::batch_item(bx, cmb3d::kBatchY, i));
      for (int i = 0; i < nX; ++i) b.push_back(cmb3d::batch_item(bx, cmb3d::kBatchX, i));
      for (int i = 0; i < nG; ++i) b.push_back(cmb3d::batch_item(bx, cmb3d::kBatchG, i));
    }
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
      const double ka = i < a.size() ? (i + 0.5) / a.size() : 2.0;
      const double kb = j < b.size() ? (j + 0.5) / b.size() : 2.0;
      items.push_back(ka <= kb ? a[i++] : b[j++]);
    }
  }
  return items;
}

int batch_persistent(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s,
                     int variant);
int batch_streams(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s);

int batch_form(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s, int form,
               int variant) {
  return form == kBatchStreams ? batch_streams(plans, seeds, outs, B, s)
                               : batch_persistent(plans, seeds, outs, B, s, variant);
}

// Form to use: the persistent kernel by default; with CMB3D_FLAG_AUTOTUNE on
// plans[0], each persistent variant and the two-stream graph are timed once
// on this plan set (build, then one timed run) and the fastest is kept.
int batch_run(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s) {
  cmb3d_plan_s* lead = plans[0];
  if (g_batch_force >= 0)
    return g_batch_force >= cmb3d::num_batch_variants() ? batch_streams(plans, seeds, outs, B, s)
                                                         : batch_persistent(plans, seeds, outs, B, s, g_batch_force);
  if (!(lead->flags & CMB3D_FLAG_AUTOTUNE)) return batch_persistent(plans, seeds, outs, B, s, 0);
  std::vector<const void*> sig(plans, plans + B);
  sig.insert(sig.end(), outs, outs + B);
  if (lead->batch_tuned_sig == sig) return batch_form(plans, seeds, outs, B, s, lead->batch_best_form, lead->batch_best_v);
  float best = 1e30f;
  int best_form = kBatchPersistent, best_v = 0;
  std::vector<std::pair<int, int>> cands;
  for (int v = 0; v < cmb3d::num_batch_variants(); ++v) cands.emplace_back(kBatchPersistent, v);
  cands.emplace_back(kBatchStreams, 0);
  for (const auto& c : cands) {
    int st = batch_form(plans, seeds, outs, B, s, c.first, c.second);    // builds the form
    if (st != CMB3D_OK) return st;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return fail_cuda(cudaErrorUnknown, "batch autotune event");
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return fail_cuda(cudaErrorUnknown, "batch autotune event");
    }
    cudaEventRecord(a, s);
    st = batch_form(plans, seeds, outs, B, s, c.first, c.second);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != CMB3D_OK) return st;
    if (ms < best) best = ms, best_form = c.first, best_v = c.second;
  }
  lead->batch_tuned_sig = sig;
  lead->batch_best_form = best_form;
  lead->batch_best_v = best_v;
  return batch_form(plans, seeds, outs, B, s, best_form, best_v);
}

int batch_streams(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s) {
  cmb3d_plan_s* lead = plans[0];
  BatchCtx& bc = lead->batch;
  const int N = lead->N;
  std::vector<const void*> sig(plans, plans + B);
  sig.insert(sig.end(), outs, outs + B);
  cudaError_t e = cudaSuccess;
  if (bc.form != kBatchStreams || bc.plans != sig) {
    bc.release();
    bc.form = kBatchStreams;
    bc.plans = sig;
    for (int b = 0; b < B; ++b)
      if ((plans[b]->flags & CMB3D_FLAG_AUTOTUNE) && !plans[b]->tuned) {
        int st = autotune(plans[b], s);
        if (st != CMB3D_OK) return st;
      }
    int lo = 0, hi = 0;
    std::vector<cudaEvent_t> ev(static_cast<size_t>(B) + 2, nullptr);
    bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&bc.d_keys), sizeof(uint2) * B) == cudaSuccess &&
              cudaStreamCreateWithFlags(&bc.cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithPriority(&bc.cap2, cudaStreamNonBlocking, hi) == cudaSuccess;
    for (auto& x : ev) ok = ok && cudaEventCreateWithFlags(&x, cudaEventDisableTiming) == cudaSuccess;
    if (ok && (e = cudaStreamBeginCapture(bc.cap, cudaStreamCaptureModeThreadLocal)) == cudaSuccess) {
      cudaError_t el = cudaEventRecord(ev[static_cast<size_t>(B)], bc.cap);
      if (el == cudaSuccess) el = cudaStreamWaitEvent(bc.cap2, ev[static_cast<size_t>(B)], 0);
      for (int b = 0; b < B && el == cudaSuccess; ++b) {
        cmb3d_plan_s* p = plans[b];
        const Schedule& sc = p->sched;
        // with the pruned passes below, only the listed z-planes are stored
        el = cmb3d::launch_draw_zfft(N, sc.draw, p->buf, p->amp, p->tw, 0, bc.cap, bc.d_keys + b,
                                     p->prune && p->zhi == 0 ? p->d_zmask : nullptr, p->prune ? p->zlo : 0,
                                     p->prune ? p->zhi : 0, p->d_err);
        if (el == cudaSuccess) el = cudaEventRecord(ev[static_cast<size_t>(b)], bc.cap);
        if (el == cudaSuccess) el = cudaStreamWaitEvent(bc.cap2, ev[static_cast<size_t>(b)], 0);
        if (el == cudaSuccess) {
          if (p->prune) {                         // the box's pruned transform (run_field)
            const int yv = sc.y >= 0 ? sc.y : 0, xv = sc.x >= 0 ? sc.x : 0;
            el = yv == gemm_y_variant(N) ? launch_y(p, yv, bc.cap2)
                                         : cmb3d::launch_yfft(N, yv, p->buf, p->tw, bc.cap2, p->d_planes,
                                                              static_cast<int>(p->nplanes), p->d_rowmask);
            if (el == cudaSuccess)
              el = cmb3d::launch_xc2r(N, xv, p->buf, p->tw, bc.cap2, p->d_rows, p->nrows_pad, p->d_rowcols);
          } else if (sc.fused >= 0) {
            el = cmb3d::launch_yx_fused(N, sc.fused, p->buf, p->tw, bc.cap2);
          } else {
            el = cmb3d::launch_yfft(N, sc.y, p->buf, p->tw, bc.cap2);
            if (el == cudaSuccess) el = cmb3d::launch_xc2r(N, sc.x, p->buf, p->tw, bc.cap2);
          }
        }
        if (el == cudaSuccess)
          el = cmb3d::launch_gather(N, p->interp, reinterpret_cast<const float*>(p->buf), p->tab, p->perm, outs[b],
                                    p->npix, bc.cap2, p->d_runs, p->nruns);
      }
      if (el == cudaSuccess) el = cudaEventRecord(ev[static_cast<size_t>(B) + 1], bc.cap2);
      if (el == cudaSuccess) el = cudaStreamWaitEvent(bc.cap, ev[static_cast<size_t>(B) + 1], 0);
      e = cudaStreamEndCapture(bc.cap, &bc.graph);
      if (e == cudaSuccess) e = el;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&bc.exec, bc.graph, 0);
    } else if (!ok) {
      e = cudaErrorMemoryAllocation;
    }
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bc.release();
      return fail_cuda(e, "batch stream-graph capture");
    }
    bc.h_keys.resize(static_cast<size_t>(B));
  }
  for (int b = 0; b < B; ++b)
    bc.h_keys[static_cast<size_t>(b)] = make_uint2(static_cast<uint32_t>(seeds[b] & 0xFFFFFFFFu),
                                                   static_cast<uint32_t>(seeds[b] >> 32));
  if ((e = cudaMemcpyAsync(bc.d_keys, bc.h_keys.data(), sizeof(uint2) * B, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaGraphLaunch(bc.exec, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail_cuda(e, "batch stream-graph launch");
  return CMB3D_OK;
}

int batch_persistent(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs, int B, cudaStream_t s,
                     int variant) {
  cmb3d_plan_s* lead = plans[0];
  BatchCtx& bc = lead->batch;
  const int N = lead->N;
  std::vector<const void*> sig(plans, plans + B);
  cudaError_t e;
  if (bc.form != kBatchPersistent || bc.plans != sig || bc.spin_limit != g_batch_spin_limit ||
      bc.withhold != g_batch_withhold || bc.variant != variant) {
    bc.release();
    bc.form = kBatchPersistent;
    bc.variant = variant;
    std::vector<uint64_t> items = batch_work_list(plans, B, N);
    bc.plans = sig;
    bc.spin_limit = g_batch_spin_limit;
    bc.withhold = g_batch_withhold;
    bc.nitems = static_cast<int>(items.size());
    bc.ctr_words = 2 + 4 * static_cast<size_t>(B);
    if ((e = cmb3d::batch_grid(N, lead->interp, variant, &bc.grid)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&bc.d_boxes), sizeof(cmb3d::BatchBox) * B)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&bc.d_items), sizeof(uint64_t) * items.size())) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&bc.d_ctr), sizeof(unsigned) * bc.ctr_words)) != cudaSuccess ||
        (e = cudaMemcpy(bc.d_items, items.data(), sizeof(uint64_t) * items.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&bc.cap, cudaStreamNonBlocking)) != cudaSuccess) {
      bc.release();
      return fail_cuda(e, "batch set-up");
    }
    // capture: reset the counters, run the persistent kernel
    if ((e = cudaStreamBeginCapture(bc.cap, cudaStreamCaptureModeThreadLocal)) == cudaSuccess) {
      cudaError_t e1 = cudaMemsetAsync(bc.d_ctr, 0, sizeof(unsigned) * bc.ctr_words, bc.cap);
      cudaError_t e2 = cmb3d::launch_batch(N, lead->interp, variant, bc.grid, bc.d_boxes, bc.d_items, bc.nitems,
                                           bc.d_ctr, lead->tw, bc.spin_limit, bc.withhold, bc.cap);
      e = cudaStreamEndCapture(bc.cap, &bc.graph);
      if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bc.exec, bc.graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bc.release();
      return fail_cuda(e, "batch graph capture");
    }
    bc.h_boxes.resize(static_cast<size_t>(B));
  }
  for (int b = 0; b < B; ++b) {
    const cmb3d_plan_s* p = plans[b];
    cmb3d::BatchBox bb{};
    bb.buf = p->buf;
    bb.amp = p->amp;
    bb.tab = p->tab;
    bb.perm = p->perm;
    bb.out = outs[b];
    bb.npix = static_cast<int>(p->npix);
    bb.key_lo = static_cast<uint32_t>(seeds[b] & 0xFFFFFFFFu);
    bb.key_hi = static_cast<uint32_t>(seeds[b] >> 32);
    bb.planes = p->prune ? p->d_planes : nullptr;
    bb.rowmask = p->prune ? p->d_rowmask : nullptr;
    bb.rows = p->prune ? p->d_rows : nullptr;
    bb.cols = p->prune ? p->d_rowcols : nullptr;
    bb.zmask = p->prune && p->zhi == 0 ? p->d_zmask : nullptr;
    bb.zlo = p->prune ? p->zlo : 0;
    bb.zhi = p->prune && p->zhi > 0 ? p->zhi : N;
    int nY, nX;
    batch_extent(p, &bb.ny_tiles, &bb.nx_blocks, &nY, &nX);
    bb.nY = static_cast<unsigned>(nY);
    bb.nX = static_cast<unsigned>(nX);
    bc.h_boxes[static_cast<size_t>(b)] = bb;
  }
  // descriptors from pageable memory: the call returns once they are staged
  if ((e = cudaMemcpyAsync(bc.d_boxes, bc.h_boxes.data(), sizeof(cmb3d::BatchBox) * B, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaGraphLaunch(bc.exec, s)) != cudaSuccess)
    return fail_cuda(e, "batch launch");
  unsigned h_err = 0;
  if ((e = cudaMemcpyAsync(&h_err, bc.d_ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail_cuda(e, "batch completion");
  if (h_err) return fail(CMB3D_ETIMEOUT, "a bounded wait in the persistent batch kernel gave up");
  return CMB3D_OK;
}

}  // namespace

int cmb3d_realize_sample_batch(const cmb3d_plan_t* plans, const uint64_t* seeds, float* const* outs_dev, int B,
                               void* stream) {
  if (B < 0 || (B > 0 && (!plans || !seeds || !outs_dev))) return fail(CMB3D_EINVAL, "bad batch arrays");
  if (B == 0) return CMB3D_OK;
  for (int b = 0; b < B; ++b) {
    int st = check_ready(plans[b]);
    if (st != CMB3D_OK) return st;
    if (plans[b]->N != plans[0]->N || plans[b]->L != plans[0]->L || plans[b]->interp != plans[0]->interp ||
        plans[b]->device != plans[0]->device || plans[b]->method != plans[0]->method)
      return fail(CMB3D_EINVAL, "batched plans must share the method, N, L, interp and device");
    if (plans[b]->npix > 0 && !outs_dev[b]) return fail(CMB3D_EINVAL, "outs_dev entry is NULL");
    for (int c = 0; c < b; ++c)
      if (plans[c] == plans[b]) return fail(CMB3D_EINVAL, "a plan appears twice in the batch (one box buffer each)");
  }
  DeviceGuard g(plans[0]->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool all3d = true;
  for (int b = 0; b < B; ++b) all3d = all3d && plans[b]->method == 3;
  if (all3d && cmb3d::batch_supported(plans[0]->N)) {
    for (int b = 0; b < B; ++b)
      if (cudaError_t e = join_pipeline(plans[b], s); e != cudaSuccess) return fail_cuda(e, "pipeline join");
    int st = batch_run(plans, seeds, outs_dev, B, s);
    for (int b = 0; b < B && st == CMB3D_OK; ++b)
      if (cudaError_t e = mark_box0_used(plans[b], s); e != cudaSuccess) return fail_cuda(e, "pipeline order");
    return st;
  }
  for (int b = 0; b < B; ++b) {
    int st = cmb3d_realize_sample(plans[b], seeds[b], outs_dev[b], stream);
    if (st != CMB3D_OK) return st;
  }
  return CMB3D_OK;
}

void cmb3d_debug_alloc_limit(int64_t bytes) { g_alloc_limit = bytes > 0 ? bytes : 0; }

int cmb3d_debug_poison_boxes(cmb3d_plan_t p) {
  if (!p) return fail(CMB3D_EINVAL, "NULL plan");
  DeviceGuard g(p->device);
  cudaError_t e = drain_pipeline(p);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const size_t bytes = p->box_elems * sizeof(float2);
  if (e == cudaSuccess) e = cudaMemset(p->buf, 0xFF, bytes);
  if (e == cudaSuccess && p->buf2) e = cudaMemset(p->buf2, 0xFF, bytes);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail_cuda(e, "poison boxes");
  return CMB3D_OK;
}

void cmb3d_batch_debug(uint32_t spin_limit, int withhold_draw, int force_form) {
  g_batch_spin_limit = spin_limit ? spin_limit : (1u << 22);
  g_batch_withhold = withhold_draw ? 1 : 0;
  g_batch_force = force_form >= 0 && force_form <= cmb3d::num_batch_variants() ? force_form : -1;
}

int cmb3d_draw_spectrum(cmb3d_plan_t p, uint64_t seed, void* spec_dev, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (!spec_dev) return fail(CMB3D_EINVAL, "spec_dev is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = p->method == 2 ? cmb3d::launch_draw2d(p->N, p->h, static_cast<float2*>(spec_dev), p->sqt, seed, s)
                                 : cmb3d::launch_draw_only(p->N, static_cast<float2*>(spec_dev), p->amp, seed, s);
  if (e != cudaSuccess) return fail_cuda(e, "draw launch");
  return CMB3D_OK;
}

int cmb3d_realize_field(cmb3d_plan_t p, uint64_t seed, float* field_dev, void* stream) {
  int st = check_ready(p);
  if (st != CMB3D_OK) return st;
  if (!field_dev) return fail(CMB3D_EINVAL, "field_dev is NULL");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = run_field(p, seed, s, false)) != CMB3D_OK) return st;
  const size_t bytes = static_cast<size_t>(p->method == 2 ? p->h : p->N) * p->N * p->N * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(field_dev, p->buf, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = mark_box0_used(p, s);
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
  return check_device_error(p);
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
  if (sc.draw < 0 || sc.draw >= cmb3d::num_draw_variants(N)) return fail(CMB3D_EINVAL, "draw variant out of range");
  if (sc.fused >= 0) {
    if (sc.fused >= cmb3d::num_fused_variants(N)) return fail(CMB3D_EINVAL, "fused variant out of range");
    if (!cmb3d::fused_variant_available(N, sc.fused))
      return fail(CMB3D_EUNSUPPORTED, "fused variant cannot run on this device (cluster shape)");
    if (p->flags & CMB3D_FLAG_THREE_PASS) return fail(CMB3D_EINVAL, "plan is restricted to separate passes");
  } else {
    sc.fused = -1;
    sc.y = sched[1];
    sc.x = sched[2];
    if (sc.y < 0 || sc.y >= num_y_variants(N)) return fail(CMB3D_EINVAL, "y variant out of range");
    if (sc.x < 0 || sc.x >= cmb3d::num_row_variants(N)) return fail(CMB3D_EINVAL, "x variant out of range");
    if (p->flags & CMB3D_FLAG_FUSED_YX && cmb3d::num_fused_variants(N) > 0)
      return fail(CMB3D_EINVAL, "plan is restricted to the fused pass");
  }
  p->sched = sc;
  p->tuned = true;
  return CMB3D_OK;
}

int cmb3d_batch_schedule(cmb3d_plan_t p, int* form, int* variant) {
  if (!p || !form || !variant) return fail(CMB3D_EINVAL, "NULL argument");
  *form = p->batch.form;
  *variant = p->batch.variant;
  return CMB3D_OK;
}

int cmb3d_plan_info(cmb3d_plan_t p, int* N, int64_t* npix, int64_t* device_bytes) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  if (N) *N = p->N;
  if (npix) *npix = p->npix;
  if (device_bytes) *device_bytes = p->dev_bytes;
  return CMB3D_OK;
}

int cmb3d_plan_prune_info(cmb3d_plan_t p, int64_t* planes, int64_t* rows) {
  if (!p) return fail(CMB3D_EINVAL, "plan is NULL");
  const int nz = p->method == 2 ? p->h : p->N;
  if (planes) *planes = p->prune ? p->nplanes : nz;
  if (rows) *rows = p->prune ? p->nrows : static_cast<int64_t>(nz) * p->N;
  return CMB3D_OK;
}

int cmb3d_pixel_tables_host(int N, double L, double r, const double* pix_xyz, int64_t npix, int interp,
                            uint32_t flags, int64_t* counts) {
  if (!counts) return fail(CMB3D_EINVAL, "counts is NULL");
  if (!is_pow2(N) || N < 8 || N > 2048) return fail(CMB3D_EUNSUPPORTED, "N must be a power of two in [8, 2048]");
  if (!(std::isfinite(L) && L > 0) || !(std::isfinite(r) && r > 0)) return fail(CMB3D_EINVAL, "L and r must be finite and > 0");
  if (!(L > 2.0 * r) && !(flags & CMB3D_FLAG_ALLOW_WRAP))
    return fail(CMB3D_EINVAL, "L must exceed 2r (set CMB3D_FLAG_ALLOW_WRAP to allow wrapping)");
  if (npix < 0 || npix >= (int64_t(1) << 31)) return fail(CMB3D_EINVAL, "npix out of range");
  if (npix > 0 && !pix_xyz) return fail(CMB3D_EINVAL, "pix_xyz is NULL");
  if (interp != CMB3D_TRILINEAR && interp != CMB3D_TRICUBIC) return fail(CMB3D_EINVAL, "interp must be 1 or 3");
  for (int64_t i = 0; i < 3 * npix; ++i)
    if (!std::isfinite(pix_xyz[i])) return fail(CMB3D_EINVAL, "pixel coordinates must be finite");
  PixelTables t;
  try {
    build_pixel_tables(N, N, 3, 0, L, r, 0.0, pix_xyz, npix, interp, flags, &t);
  } catch (const std::bad_alloc&) {
    return fail(CMB3D_ENOMEM, "host allocation of the pixel table");
  }
  const bool pruned = !t.rows.empty();
  int64_t listed = 0;
  for (int32_t rr : t.rows) listed += rr < N * N ? 1 : 0;
  counts[0] = pruned ? static_cast<int64_t>(t.planes.size()) : N;
  counts[1] = pruned ? listed : static_cast<int64_t>(N) * N;
  counts[2] = pruned ? t.x_stored : static_cast<int64_t>(N) * N * N;
  counts[3] = static_cast<int64_t>(t.runs.size());
  return CMB3D_OK;
}

int cmb3d_plan_x_stored(cmb3d_plan_t p, int64_t* reals) {
  if (!p || !reals) return fail(CMB3D_EINVAL, "plan or reals is NULL");
  const int nz = p->method == 2 ? p->h : p->N;
  *reals = p->prune ? p->x_stored : static_cast<int64_t>(nz) * p->N * p->N;
  return CMB3D_OK;
}

void cmb3d_destroy(cmb3d_plan_t p) { free_plan(p); }

}  // extern "C"
