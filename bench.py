"""Benchmark: partial-sky maps per second on the GB300 (3-D Fourier method;
the 2-D Fourier method with --workload fourier2d_box512_cap20).

One step = one complete map of the workload through the C ABI: Philox draw
fused with the z-FFT, y-FFT, x complex-to-real FFT and the tricubic gather at
the cap pixels.  Default workload: a 1024^3 box (L = 2.2 r) sampled at the
20,132,659 pixels of an f_sky = 0.4 polar cap of a 12*2048^2-point grid; the
512^3 box with the 5,033,165-pixel cap of a 12*1024^2-point grid is timed
after it and reported in config as a secondary figure.

The line printed by rank 0 carries maps/s (device-timed, inputs resident),
the end-to-end figure through the host-buffer entry point, the roofline of
the dominant kernel (algorithmic bytes / its CUDA-event time), the FP64
oracle timed on the host cores, clocks sampled during the timed region and
the number of kernel launches.

--impl reference runs the FP64 oracle on the host cores instead (the only
other place this script executes the oracle).

Multi-GPU: independent replicas (one process per GPU, seeds offset by rank),
no data-path collective; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS  # noqa: E402

DEFAULT_WORKLOAD = "box1024_cap0.4_tricubic"
SECONDARY_WORKLOAD = "box512_cap0.4_tricubic"
METRIC = "partial-sky maps/sec and achieved HBM GB/s at N^3 box, Npix pixels, 1 GB300"
L2_BYTES = 129 * 2 ** 20


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return

        def pump():
            for line in self.proc.stdout:
                self.lines.append(line.strip())
        self.thread = threading.Thread(target=pump, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


_FFT_SRC = ["paper_2507_15703_gb300/csrc/fft_passes.cu", "paper_2507_15703_gb300/csrc/fft_tiles.cuh",
            "paper_2507_15703_gb300/csrc/device_common.cuh"]
KERNEL_SOURCES = {
    "draw_zfft": _FFT_SRC,
    "yfft": _FFT_SRC,
    "xc2r": _FFT_SRC,
    "yx_fused": _FFT_SRC,
    "gather": ["paper_2507_15703_gb300/csrc/gather.cu", "paper_2507_15703_gb300/csrc/gather_tiles.cuh"],
    "batch": ["paper_2507_15703_gb300/csrc/batch.cu", "paper_2507_15703_gb300/csrc/fft_tiles.cuh"],
}
# the 2-D Fourier method draws with its own kernel
KERNEL_SOURCES_2D = dict(KERNEL_SOURCES, draw_zfft=["paper_2507_15703_gb300/csrc/fourier2d.cu",
                                                    "paper_2507_15703_gb300/csrc/device_common.cuh"])
# kernels whose limiter is instruction issue, not HBM (the draw: Philox,
# Box-Muller and the first FFT stages for every mode, one write of the box)
ALU_BOUND = {"draw_zfft"}


def ncu_counters(kernel: str, workload: str):
    """Per-launch counters of the kernel from the committed ncu summary
    (dram_bytes_per_launch, thread_inst_per_launch), or None when the kernel
    source changed since they were taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    srcs = KERNEL_SOURCES_2D if workload in WORKLOADS and WORKLOADS[workload].method == "2d" else KERNEL_SOURCES
    if not os.path.exists(p) or kernel not in srcs:
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != source_hash(srcs[kernel]):
        return None
    return e


def ncu_traffic(kernel: str, workload: str):
    e = ncu_counters(kernel, workload)
    return e.get("dram_bytes_per_launch") if e else None


def alu_peak_tinst(clk) -> tuple[float, str]:
    """Lane-instructions per second at full issue: SMs x 4 schedulers x 32
    lanes x the maximum SM clock (one warp instruction per scheduler per
    clock), in units of 1e12."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz"


def b_alg_bytes(N: int, npix: int) -> int:
    """The whole-map algorithmic minimum of the unpruned 3-D method: one write
    and one read of the complex half spectrum between the axes (2 H, H = 8 N^2
    (N/2 + 1) bytes), one write of the real field (4 N^3) and 20 B per pixel
    (16 B table + 4 B output)."""
    return 2 * 8 * N * N * (N // 2 + 1) + 4 * N ** 3 + 20 * npix


def algorithmic_bytes(N: int, npix: int, planes: int | None = None, rows: int | None = None,
                      nz: int | None = None, draw_planes: int | None = None, x_stored: int | None = None) -> dict:
    """Bytes each kernel must move per launch (the packed half spectrum and the
    real field are both 4 N^2 nz bytes for nz z-planes, N for the 3-D box and
    h layers for the 2-D method; a row is 4 N bytes): the draw writes the
    draw_planes z-planes it stores (default: all); yfft reads its z-planes and
    writes its rows; xc2r reads and writes its rows; gather reads 16 B of table
    + 4 B of permutation per pixel and writes 4 B per pixel (field reads are
    cache-dependent and not counted).  planes, rows: the pruned extent of the
    sky-map path (default: whole box); x_stored: the reals the x pass writes
    back (the column blocks the stencils read; default: whole rows)."""
    nz = N if nz is None else nz
    box, row = 4 * N * N * nz, 4 * N
    planes = nz if planes is None else planes
    rows = nz * N if rows is None else rows
    drawn = 4 * N * N * (nz if draw_planes is None else draw_planes)
    x_write = rows * row if x_stored is None else 4 * x_stored
    return {"draw_zfft": drawn, "yfft": planes * N * row + rows * row, "xc2r": rows * row + x_write,
            "gather": 24 * npix, "yx_fused": 2 * box}


# --------------------------------------------------------------------------
# the CUDA arm
# --------------------------------------------------------------------------

def run_cuda(args, rank, world, local):
    import torch
    from paper_2507_15703_gb300 import cmb3d

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    if w.batch > 1:
        return run_cuda_batch(args, rank, world, local, w)
    learned = train_learned_inversion(args, w, dev) if w.learned else None
    pix = w.pixels()
    npix = pix.shape[0]
    ell, cl = w.cl()

    t0 = time.time()
    flags = cmb3d.CMB3D_FLAG_STAGE_TIMING | cmb3d.CMB3D_FLAG_AUTOTUNE
    if args.three_pass:
        flags |= cmb3d.CMB3D_FLAG_THREE_PASS
    if args.fused:
        flags |= cmb3d.CMB3D_FLAG_FUSED_YX
    if args.fp16_gemm:
        flags |= cmb3d.CMB3D_FLAG_FP16_GEMM
    if args.no_prune:
        flags |= cmb3d.CMB3D_FLAG_NO_PRUNE
    if args.pipeline:
        flags |= cmb3d.CMB3D_FLAG_PIPELINE
    if args.fused_xg:
        flags |= cmb3d.CMB3D_FLAG_FUSED_XG
    if args.schedule:
        flags &= ~cmb3d.CMB3D_FLAG_AUTOTUNE
    if w.method == "2d":
        z0, nlayers = w.layers()
        make = lambda fl: cmb3d.Plan2D(w.N, w.M, nlayers, w.L, w.r, z0, pix, w.interp, fl)   # noqa: E731
    else:
        nlayers = w.N
        make = lambda fl: cmb3d.Plan(w.N, w.L, w.r, pix, w.interp, fl)   # noqa: E731
    plan = make(flags)
    if args.schedule:
        cmb3d.cmb3d_plan_set_schedule(plan.handle, tuple(int(v) for v in args.schedule.split(",")))
    if learned is not None:
        plan.set_pk(learned["knodes"], learned["pk_first_heldout"])
        fit_err = learned["summary"]["mlp_fwd_err_rms_median"]
    else:
        fit_err = plan.set_cl(ell, cl, w.nkbins)
        kn_fit = np.linspace(0.0, math.sqrt(3) * math.pi * w.N / w.L, w.nkbins)   # the fit's nodes
        plan_pk = (kn_fit, cmb3d.cmb3d_get_pk(plan.handle, kn_fit))
        rel_fit = (cmb3d.cmb3d_cl_matrix(ell, kn_fit, w.r) @ plan_pk[1] - cl) / cl
        fit_rms = float(np.sqrt(np.mean(rel_fit ** 2)))
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(npix, dtype=torch.float32, device=dev)
    seed0 = rank_seed_base(rank)

    dist = init_dist(world, dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for i in range(args.warmup):
        plan.realize_sample(seed0 + i, out, stream)
    torch.cuda.synchronize(dev)
    cmb3d.cmb3d_stage_times(plan.handle, reset=True)
    schedule = cmb3d.cmb3d_plan_schedule(plan.handle)
    if args.sweep and rank == 0:
        sweep(plan, out, stream, w.N, seed0)
        cmb3d.cmb3d_plan_set_schedule(plan.handle, schedule)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        plan.realize_sample(seed0 + args.warmup + i, out, stream)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    stage_ms, stage_n = cmb3d.cmb3d_stage_times(plan.handle, reset=True)
    t_max = max_over_ranks(dist, ms, dev)
    n_planes, n_rows = cmb3d.cmb3d_plan_prune_info(plan.handle)
    x_stored = cmb3d.cmb3d_plan_x_stored(plan.handle)

    # end to end through the host-output entry point: every map copied to
    # pinned host memory (a ring of 4 buffers), each download overlapping the
    # next map's kernels on the plan's copy stream
    ring = [torch.empty(npix, dtype=torch.float32).pin_memory().numpy() for _ in range(4)]
    host = ring[0]
    cmb3d.cmb3d_realize_samples_to_host(plan.handle, [seed0, seed0 + 1], ring[:2], stream)
    barrier()
    t1 = time.perf_counter()
    cmb3d.cmb3d_realize_samples_to_host(plan.handle, [seed0 + i for i in range(args.steps)],
                                        [ring[i % 4] for i in range(args.steps)], stream)
    barrier()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t1, dev)
    # one synchronous call per map (download not overlapped), for comparison
    t1 = time.perf_counter()
    for i in range(args.steps):
        cmb3d.cmb3d_realize_sample_to_host(plan.handle, seed0 + i, host, stream)
    barrier()
    e2e_sync_s = max_over_ranks(dist, time.perf_counter() - t1, dev)
    # the download alone (same pinned buffer, same stream), to separate the
    # host link from the map's own time in the end-to-end figure
    host_t = torch.from_numpy(host)
    ev0.record(stream)
    for i in range(args.steps):
        host_t.copy_(out, non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    d2h_ms = ev0.elapsed_time(ev1) / args.steps
    cmb3d.cmb3d_stage_times(plan.handle, reset=True)
    pipe_info = None
    if not args.pipeline and learned is None:
        # the same maps through a pipelined plan (second box, draw of map i+1
        # overlapping the passes and gather of map i); CUDA events, same stream
        pflags = (flags | cmb3d.CMB3D_FLAG_PIPELINE) & ~cmb3d.CMB3D_FLAG_STAGE_TIMING & ~cmb3d.CMB3D_FLAG_AUTOTUNE
        pplan = make(pflags)
        cmb3d.cmb3d_plan_set_schedule(pplan.handle, schedule)
        pplan.set_pk(*plan_pk)
        for i in range(args.warmup):
            pplan.realize_sample(seed0 + i, out, stream)
        barrier()
        ev0.record(stream)
        for i in range(args.steps):
            pplan.realize_sample(seed0 + args.warmup + i, out, stream)
        ev1.record(stream)
        barrier()
        p_ms = max_over_ranks(dist, ev0.elapsed_time(ev1), dev)
        pplan.close()
        pipe_info = {"maps_per_s": round(world * args.steps / (p_ms / 1e3), 3),
                     "ms_per_map": round(p_ms / args.steps, 5),
                     "note": "CMB3D_FLAG_PIPELINE: two boxes, each map's draw overlaps the previous map's "
                             "passes and gather (timed after the main run, same maps and stream)"}
    plan.close()

    secondary = None
    if rank == 0 and args.workload == DEFAULT_WORKLOAD and not args.no_secondary:
        secondary = secondary_figure(args, dev, stream, seed0)

    if rank != 0:
        finish_dist(dist)
        return

    maps = world * args.steps
    value = job_throughput(world, args.steps, t_max)
    # the 3-D draw stores only the z-planes the pruned y pass reads; the 2-D
    # draw writes all its layers
    ab = algorithmic_bytes(w.N, npix, n_planes, n_rows, nlayers, nlayers if w.method == "2d" else n_planes,
                           x_stored if not args.fused_xg else None)
    names = cmb3d.STAGE_NAMES
    kernels = {}
    for i, name in enumerate(names):
        n = int(stage_n[i])
        if n == 0:
            continue
        kernels[name] = kernel_entry(n, stage_ms[i], stage_ms.sum(), ab[name])
    dom = names[int(np.argmax(stage_ms))]
    per_map_bytes = sum(ab[k] for k in kernels)
    config = {"workload": args.workload, "N": w.N, "L_over_r": round(w.L / w.r, 4), "npix": npix, "fsky": w.fsky,
              "interp": "tricubic" if w.interp == 3 else "trilinear", "lmax": w.lmax, "nkbins": w.nkbins,
              "parallelism": f"replicas x{world}",
              "schedule": {"draw": schedule[0], "y": schedule[1], "x": schedule[2], "fused_yx": schedule[3],
                           "restriction": "three-pass" if args.three_pass else "fused" if args.fused else "autotuned",
                           "y_pass": "split-FP16 DFT-GEMM (tcgen05)" if args.fp16_gemm else "FP32 butterflies",
                           "pipelined": bool(args.pipeline), "fused_x_gather": bool(args.fused_xg)},
              "pruned_transform": {"z_planes": n_planes, "rows": n_rows, "x_stored_reals": x_stored,
                                   "of_planes": w.N, "of_rows": w.N ** 2,
                                   "note": "y pass on the z-planes, x pass on the (z, y) rows the "
                                           "interpolation stencils read, storing only the column blocks they "
                                           "read; maps equal the whole-box maps bit for bit"},
              "l2": f"no flush: per-map working set {per_map_bytes / 2**30:.2f} GiB > 129 MiB L2",
              "cl_fit_max_rel_err": fit_err,
              "cl_fit_rms_rel_err": None if learned is not None else round(fit_rms, 4),
              "cl_fit_note": None if learned is not None else
              "NNLS optimum of a P >= 0 on the nodes for this oscillating C_l family, not a solver failure",
              "plan_setup_s": round(setup_s, 2),
              "method": ({"name": "2-D Fourier method (Sec. II.D.2)", "M": w.M, "h": nlayers,
                          "z0": round(z0, 6), "dp": w.dp, "theta_max_deg": w.theta_max_deg}
                         if w.method == "2d" else {"name": "3-D Fourier method (Sec. II.D.1)"}),
              "pipelined_plan": pipe_info,
              "e2e_one_call_per_map_maps_per_s": round(world * args.steps / e2e_sync_s, 3),
              "e2e_d2h_ms_per_map": round(d2h_ms, 4),
              "e2e_d2h_gbs": round(4 * npix / (d2h_ms / 1e3) / 1e9, 1)}
    if w.method != "2d":
        ba = b_alg_bytes(w.N, npix)
        config["pipeline_bytes"] = {
            "b_alg_unpruned_per_map": ba,
            "b_alg_gbs": round(ba * value / world / 1e9, 1),
            "b_alg_frac_of_measured_hbm": round(ba * value / world / 1e9 / measured_peaks()[0], 4),
            "moved_pruned_per_map": per_map_bytes,
            "moved_gbs": round(per_map_bytes * value / world / 1e9, 1),
            "moved_frac_of_measured_hbm": round(per_map_bytes * value / world / 1e9 / measured_peaks()[0], 4),
            "note": "b_alg: the unpruned method's algorithmic minimum (write + read of the half spectrum, "
                    "field write, 20 B per pixel) per map at the measured map rate; moved: the bytes the "
                    "pruned kernels actually have to move (per-kernel algorithmic bytes summed)"}
    if secondary is not None:
        config["secondary"] = secondary
    if learned is not None:
        config["cl_fit_max_rel_err"] = None
        config["spectrum"] = "P(k) of held-out spectrum 0 from the learned inversion, refined on the GPU"
        s = learned["summary"]
        # a new spectrum per map: inversion time + the map's own time
        t_map = t_max / args.steps / 1e3
        s["maps_per_s_new_spectrum_each_map"] = {
            "learned": round(1.0 / (t_map + s["mlp_infer_ms_per_spectrum"] / 1e3), 3),
            "learned_refined": round(1.0 / (t_map + (s["mlp_infer_ms_per_spectrum"] + s["refine_ms_per_spectrum"])
                                                / 1e3), 3),
            "nnls": round(1.0 / (t_map + s["nnls_ms_per_spectrum"] / 1e3), 3),
            "note": "learned_refined reaches the NNLS optimum's accuracy (refined_fwd_err_rms_median_nnls_spectra "
                    "against nnls_fwd_err_rms_median on the same spectra)"}
        config["learned_inversion"] = s
    emit(args, w, value, t_max, world, config, per_map_bytes, kernels, dom, maps / e2e_s, 4 * npix,
         int(stage_n.sum()), clk)
    finish_dist(dist)


def secondary_figure(args, dev, stream, seed0, maps=50):
    """The 512^3 single-map workload timed on the same GPU after the main run
    (its own autotuned plan, CUDA events over `maps` maps): maps/s and the
    per-kernel times."""
    import torch
    from paper_2507_15703_gb300 import cmb3d
    w = WORKLOADS[SECONDARY_WORKLOAD]
    pix = w.pixels()
    ell, cl = w.cl()
    plan = cmb3d.Plan(w.N, w.L, w.r, pix, w.interp, cmb3d.CMB3D_FLAG_STAGE_TIMING | cmb3d.CMB3D_FLAG_AUTOTUNE)
    plan.set_cl(ell, cl, w.nkbins)
    out = torch.empty(pix.shape[0], dtype=torch.float32, device=dev)
    for i in range(max(args.warmup, 3)):
        plan.realize_sample(seed0 + i, out, stream)
    torch.cuda.synchronize(dev)
    cmb3d.cmb3d_stage_times(plan.handle, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(maps):
        plan.realize_sample(seed0 + 100 + i, out, stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    st_ms, st_n = cmb3d.cmb3d_stage_times(plan.handle, reset=True)
    plan.close()
    return {"workload": SECONDARY_WORKLOAD, "maps": maps, "maps_per_s": round(maps / (ms / 1e3), 1),
            "ms_per_map": round(ms / maps, 5),
            "kernel_ms": {name: round(float(st_ms[k] / st_n[k]), 5)
                          for k, name in enumerate(cmb3d.STAGE_NAMES) if st_n[k]}}


def train_learned_inversion(args, w, dev):
    """Train the MLP inversion on the GPU (own kernels) and compare it with
    the library's NNLS inversion on held-out spectra of the same family."""
    import torch
    from paper_2507_15703_gb300 import cmb3d
    from synth import random_cl_family
    ell = np.arange(2, w.lmax + 1, dtype=np.float64)
    n_hold, n_nnls = 64, 8
    _, cl = random_cl_family(np.random.default_rng(w.train_seed), w.n_train + n_hold, w.lmax)
    logc = np.log(cl).astype(np.float32)
    train, hold, cl_hold = logc[: w.n_train], logc[w.n_train:], cl[w.n_train:]
    kn = np.linspace(0.0, math.sqrt(3) * math.pi * w.N / w.L, w.nkbins)   # the NNLS nodes
    A = cmb3d.cmb3d_cl_matrix(ell, kn, w.r)
    mu, sd = train.mean(0), train.std(0) + 1e-3
    out_bias = np.full(kn.size, np.log(np.mean(cl[:1000]) / np.mean(A.sum(1))), dtype=np.float32)
    mlp = cmb3d.cmb3d_mlp_create(ell.size, 256, 3, kn.size, A, mu, sd, out_bias, batch_cap=1024, seed=w.train_seed)
    x = torch.tensor(train, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    # step schedule: (epochs, learning rate); Adam state carries across phases
    schedule = [(args.train_epochs * 6 // 12, 1e-3), (args.train_epochs * 4 // 12, 3e-4),
                (args.train_epochs - args.train_epochs * 10 // 12, 1e-4)]
    losses = np.concatenate([cmb3d.cmb3d_mlp_train(mlp, x, w.n_train, ep, 1024, lr, seed=w.train_seed + i)
                             for i, (ep, lr) in enumerate(schedule) if ep > 0])
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    xh = torch.tensor(hold, device=dev)
    yh = torch.empty((n_hold, kn.size), dtype=torch.float32, device=dev)
    cmb3d.cmb3d_mlp_predict(mlp, xh, n_hold, yh)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(10):
        cmb3d.cmb3d_mlp_predict(mlp, xh, n_hold, yh)
    torch.cuda.synchronize(dev)
    infer_ms = (time.perf_counter() - t0) / (10 * n_hold) * 1e3
    P = np.exp(yh.cpu().numpy().astype(np.float64))
    rel = np.abs(P @ A.T - cl_hold) / cl_hold
    # refined toward the NNLS optimum on the GPU (FISTA on the NNLS objective from the network's P)
    pr = torch.empty((n_hold, kn.size), dtype=torch.float32, device=dev)
    cmb3d.cmb3d_mlp_refine(mlp, xh, yh, n_hold, pr, iters=args.refine_iters)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    cmb3d.cmb3d_mlp_refine(mlp, xh, yh, n_hold, pr, iters=args.refine_iters)
    torch.cuda.synchronize(dev)
    refine_ms = (time.perf_counter() - t0) / n_hold * 1e3
    Pr = pr.cpu().numpy().astype(np.float64)
    rel_r = np.abs(Pr @ A.T - cl_hold) / cl_hold
    cmb3d.cmb3d_mlp_destroy(mlp)
    # the method without it: NNLS on the library's own nodes, same spectra
    nn_rms, nn_max = [], []
    t0 = time.perf_counter()
    for i in range(n_nnls):
        kk, pk, err = cmb3d.cmb3d_fit_pk(ell, cl_hold[i], w.N, w.L, w.r, w.nkbins)
        e = np.abs(cmb3d.cmb3d_cl_matrix(ell, kk, w.r) @ pk - cl_hold[i]) / cl_hold[i]
        nn_rms.append(float(np.sqrt(np.mean(e ** 2))))
        nn_max.append(float(e.max()))
    nnls_ms = (time.perf_counter() - t0) / n_nnls * 1e3
    summary = {"train_spectra": w.n_train, "epochs": args.train_epochs, "lr_schedule": schedule,
               "train_s": round(train_s, 2),
               "train_spectra_per_s": round(w.n_train * args.train_epochs / train_s, 1),
               "loss_first_last_epoch": [float(losses[0]), float(losses[-1])],
               "net": "2047 -> 3 x 256 GELU -> 512, BF16 GEMM operands, FP32 accumulate",
               "mlp_fwd_err_rms_median": float(np.median(np.sqrt(np.mean(rel ** 2, axis=1)))),
               "mlp_fwd_err_max_median": float(np.median(rel.max(axis=1))),
               "refined_fwd_err_rms_median": float(np.median(np.sqrt(np.mean(rel_r ** 2, axis=1)))),
               "refined_fwd_err_rms_median_nnls_spectra":
                   float(np.median(np.sqrt(np.mean(rel_r[:n_nnls] ** 2, axis=1)))),
               "refined_fwd_err_max_median": float(np.median(rel_r.max(axis=1))),
               "refine_iters": args.refine_iters, "refine_ms_per_spectrum": round(refine_ms, 4),
               "nnls_fwd_err_rms_median": float(np.median(nn_rms)),
               "nnls_fwd_err_max_median": float(np.median(nn_max)),
               "mlp_infer_ms_per_spectrum": round(infer_ms, 4), "nnls_ms_per_spectrum": round(nnls_ms, 1),
               "heldout": n_hold, "nnls_heldout": n_nnls}
    return {"knodes": kn, "pk_first_heldout": Pr[0], "summary": summary}


def run_cuda_batch(args, rank, world, local, w):
    """Batched workload: one step = B maps (each box its own pixel set) in one
    persistent launch replayed from a CUDA graph."""
    import torch
    from paper_2507_15703_gb300 import cmb3d

    dev = torch.device("cuda", local)
    pixs = w.batch_pixels()
    ell, cl = w.cl()
    t0 = time.time()
    plans = [cmb3d.Plan(w.N, w.L, w.r, p, w.interp, cmb3d.CMB3D_FLAG_AUTOTUNE) for p in pixs]
    fit_err = plans[0].set_cl(ell, cl, w.nkbins)
    kn = np.linspace(0.0, math.sqrt(3) * math.pi * w.N / w.L, w.nkbins)
    pk = cmb3d.cmb3d_get_pk(plans[0].handle, kn)
    for p in plans[1:]:
        p.set_pk(kn, pk)
    setup_s = time.time() - t0
    handles = [p.handle for p in plans]
    npix = [p.shape[0] for p in pixs]
    outs = [torch.empty(n, dtype=torch.float32, device=dev) for n in npix]
    stream = torch.cuda.current_stream(dev)
    dist = init_dist(world, dev)
    base = rank_seed_base(rank)

    def step(i):
        cmb3d.cmb3d_realize_sample_batch(handles, [base + i * w.batch + b for b in range(w.batch)], outs, stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(dist, ms, dev)

    form, variant = cmb3d.cmb3d_batch_schedule(handles[0])
    form_name = {0: f"persistent kernel ({2 - variant} blocks/SM) in a CUDA graph",
                 1: "two-stream CUDA graph (draws || passes)"}.get(form, "none")

    # every batch form on the same boxes (forced; the autotuner's pick is the main line)
    form_rates = {}
    for force, name in ((0, "persistent_2_blocks_per_sm"), (1, "persistent_1_block_per_sm"),
                        (2, "two_stream_graph")):
        cmb3d.cmb3d_batch_debug(0, False, force)
        try:
            for i in range(2):
                step(i)
            torch.cuda.synchronize(dev)
            fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            form_steps = max(1, min(args.steps, 5))
            fe0.record(stream)
            for i in range(form_steps):
                step(args.warmup + i)
            fe1.record(stream)
            torch.cuda.synchronize(dev)
            form_rates[name] = round(form_steps * w.batch / (fe0.elapsed_time(fe1) / 1e3), 1)
        finally:
            cmb3d.cmb3d_batch_debug(0, False, -1)

    # the plain form for comparison: the same boxes realized one after another
    for i in range(2):
        for b, p in enumerate(plans):
            cmb3d.cmb3d_realize_sample(handles[b], base + b, outs[b], stream)
    torch.cuda.synchronize(dev)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_steps = max(1, min(args.steps, 5))
    pe0.record(stream)
    for i in range(plain_steps):
        for b, p in enumerate(plans):
            cmb3d.cmb3d_realize_sample(handles[b], base + i * w.batch + b, outs[b], stream)
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    plain_value = plain_steps * w.batch / (pe0.elapsed_time(pe1) / 1e3)

    # end to end: the same batches with every map copied to pinned host memory
    hosts = [torch.empty(n, dtype=torch.float32).pin_memory() for n in npix]
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for i in range(args.steps):
        step(i)
        for h, o in zip(hosts, outs):
            h.copy_(o, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(dist, time.perf_counter() - t1, dev)
    # both forms run each box's pruned transform
    pruned = True
    extents = [cmb3d.cmb3d_plan_prune_info(p.handle) + (cmb3d.cmb3d_plan_x_stored(p.handle),) for p in plans]
    for p in plans:
        p.close()
    if rank != 0:
        finish_dist(dist)
        return
    maps = world * args.steps * w.batch
    value = job_throughput(world, args.steps * w.batch, t_max)
    batch_bytes = 24 * sum(npix)
    for zp, rw, xs in extents:
        ab = algorithmic_bytes(w.N, 0, zp, rw, None, zp if pruned else None, xs)   # pruned draws store zp planes
        batch_bytes += ab["draw_zfft"] + ab["yfft"] + ab["xc2r"]
    kernels = {"batch": kernel_entry(args.steps, ms, ms, batch_bytes)}
    kernels["batch"]["note"] = "one step = the whole batch (persistent kernel or graph), CUDA events"
    config = {"workload": args.workload, "N": w.N, "boxes_per_step": w.batch, "npix_total": int(sum(npix)),
              "npix_min": int(min(npix)), "npix_max": int(max(npix)), "fsky": "U[0.05, 0.5] per box",
              "interp": "tricubic" if w.interp == 3 else "trilinear", "lmax": w.lmax, "nkbins": w.nkbins,
              "parallelism": f"replicas x{world}", "schedule": f"autotuned: {form_name}",
              "l2": f"no flush: per-step working set {batch_bytes / 2**30:.1f} GiB > 129 MiB L2",
              "cl_fit_max_rel_err": fit_err, "plan_setup_s": round(setup_s, 2),
              "pruned_transform": {"z_planes_mean": round(float(np.mean([e[0] for e in extents])), 1),
                                   "rows_mean": round(float(np.mean([e[1] for e in extents])), 1),
                                   "of_planes": w.N, "of_rows": w.N ** 2},
              "plain_single_box_maps_per_s": round(plain_value, 1),
              "plain_note": "the same boxes, one cmb3d_realize_sample call per box on the stream (pruned "
                            "transform, same kernels: each map equals its batch map bit for bit)",
              "forms_maps_per_s": form_rates,
              "forms_note": "forced in turn on the same boxes, each box's pruned transform in every form; the "
                            "main line is the autotuner's pick"}
    emit(args, w, value, t_max, world, config, batch_bytes / w.batch, kernels, "batch", maps / e2e_s,
         4 * sum(npix), 2 * args.steps, clk)
    finish_dist(dist)


def init_dist(world, dev):
    """Process group of the replicas (RANK / WORLD_SIZE / MASTER_* from the
    environment): NCCL on the GPUs, gloo when dev is None (host-side tests)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if dev is None:
        dist.init_process_group("gloo")
    else:
        dist.init_process_group("nccl", device_id=dev)
    return dist


def finish_dist(dist):
    if dist is not None:
        dist.destroy_process_group()


def max_over_ranks(dist, v, dev):
    """The largest of every rank's v (the job's time is its slowest rank)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], device=dev if dev is not None else "cpu", dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


SEED_STRIDE = 1000003


def rank_seed_base(rank: int) -> int:
    """First seed of a replica: ranks draw disjoint seed ranges as long as a
    run uses fewer than SEED_STRIDE seeds per rank."""
    return SEED_STRIDE * rank


def job_throughput(world: int, units_per_rank: int, t_max_ms: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (t_max_ms / 1e3)


def kernel_entry(n, total_ms, all_ms, alg_bytes):
    peak, _ = measured_peaks()
    avg_ms = total_ms / max(n, 1)
    gbs = alg_bytes / (avg_ms / 1e3) / 1e9
    return {"launches": int(n), "avg_ms": round(float(avg_ms), 5), "share": round(float(total_ms / max(all_ms, 1e-12)), 4),
            "alg_bytes": int(alg_bytes), "alg_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peak, 4)}


ARGS_MODE: dict = {}                      # run options that change the kernels' work (set in main)


def roofline(dom, dk, workload, peak, peak_kind, clk):
    """Roofline of the dominant kernel.  HBM-bound kernels: algorithmic bytes
    per launch / CUDA-event time against the measured copy bandwidth.  The
    issue-bound draw: its executed lane-instructions per launch (a fixed
    property of the compiled kernel and N, from the committed ncu counters) /
    CUDA-event time against full issue; falls back to HBM if the counters are
    stale."""
    cnt = ncu_counters(dom, workload)
    if cnt and any(ARGS_MODE.values()):
        cnt = None                        # the counters were taken on the default pruned separate passes
    if dom in ALU_BOUND and cnt and cnt.get("thread_inst_per_launch"):
        p, src = alu_peak_tinst(clk)
        a = cnt["thread_inst_per_launch"] / (dk["avg_ms"] / 1e3) / 1e12
        return {"bound": "alu", "kernel": dom, "achieved": round(a, 2), "peak": round(p, 2), "unit": "Tinst/s",
                "frac": round(a / p, 4), "peak_source": src, "traffic": cnt.get("dram_bytes_per_launch"),
                "inst_per_launch": cnt["thread_inst_per_launch"], "hbm_frac": dk["frac_of_measured_hbm"]}
    return {"bound": "hbm", "kernel": dom, "achieved": dk["alg_gbs"], "peak": peak, "unit": "GB/s",
            "frac": dk["frac_of_measured_hbm"], "peak_source": peak_kind,
            "traffic": cnt.get("dram_bytes_per_launch") if cnt else None}


def emit(args, w, value, t_max, world, config, per_map_bytes, kernels, dom, e2e_value, d2h_bytes, launches, clk):
    peak, peak_kind = measured_peaks()
    dk = kernels[dom]
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "maps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if not getattr(args, "fp16_gemm", False) else "f32 (y pass: f16 hi+lo GEMM, f32 accumulate)",
        "data": "synthetic: Fibonacci-grid polar cap pixels, C_l family inverted to P(k) by the library's NNLS",
        "config": config,
        "achieved_gbs_alg_per_map": round(per_map_bytes * value / world / 1e9, 1),
        "roofline": roofline(dom, dk, args.workload, peak, peak_kind, clk),
        "kernels": kernels,
        "e2e": {"value": round(e2e_value, 3), "unit": "maps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(d2h_bytes)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args)
    print(json.dumps(line), flush=True)


def sweep(plan, out, stream, N, seed0, reps=20):
    """Time every kernel variant (stage events) and print one JSON line per
    schedule to stderr."""
    import torch
    from paper_2507_15703_gb300 import cmb3d
    scheds = [(d, 0, 0, -1) for d in range(7)] + [(0, y, 0, -1) for y in range(4)] + \
             [(0, 0, x, -1) for x in range(4)] + [(0, -1, -1, f) for f in range(4)]
    for sc in scheds:
        try:
            cmb3d.cmb3d_plan_set_schedule(plan.handle, sc)
        except cmb3d.Cmb3dError:
            continue
        for i in range(3):
            plan.realize_sample(seed0 + i, out, stream)
        torch.cuda.synchronize()
        cmb3d.cmb3d_stage_times(plan.handle, reset=True)
        for i in range(reps):
            plan.realize_sample(seed0 + i, out, stream)
        ms, n = cmb3d.cmb3d_stage_times(plan.handle, reset=True)
        per = {name: round(float(ms[k] / n[k]), 5) for k, name in enumerate(cmb3d.STAGE_NAMES) if n[k]}
        print(json.dumps({"sweep": list(sc), "avg_ms": per}), file=sys.stderr, flush=True)


# --------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------

def oracle_map_sample(w, seed):
    """One map of the workload computed by the FP64 oracle (draw, inverse FFT,
    interpolation at every pixel).  Returns (seconds, pixels done)."""
    from oracle import cmb3d_oracle as orc
    k = np.linspace(0.0, math.sqrt(3) * math.pi * w.N / w.L, w.nkbins)
    pk = 1e-3 / (1.0 + (k / 12.0) ** 3)
    pb = orc.p_box_of_q(w.N, w.L, k, pk)
    pix = w.batch_pixels()[seed % w.batch] if w.batch > 1 else w.pixels()
    t = time.perf_counter()
    vals = orc.realize_sample(w.N, w.L, w.r, pix, pb, seed, w.interp)
    return time.perf_counter() - t, vals.size


ORACLE_THREADS = 1   # numpy's pocketfft and its elementwise array operations run on the calling thread


ORACLE_BYTES_PER_CELL = 32   # peak host memory of one oracle map per box cell (31 measured at N = 64, 128)


def host_memory_bytes():
    """Memory this process may use: the available physical pages, capped by a
    cgroup limit where one is set."""
    avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    for f in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(f) as fh:
                v = fh.read().strip()
            if v.isdigit():
                avail = min(avail, int(v))
        except OSError:
            pass
    return avail


def cpu_baseline(w, args):
    """The oracle, as it stands, timed on one full map of the same workload on
    the host cores (numpy FP64; one map is the bounded sample).  A box whose
    FP64 oracle map does not fit the host memory gets no baseline."""
    need = ORACLE_BYTES_PER_CELL * w.N ** 3
    if need > 0.6 * host_memory_bytes():
        return {"value": None, "unit": "maps/s", "cores": ORACLE_THREADS, "kind": "oracle",
                "sample": f"none: one FP64 oracle map of the {w.N}^3 box needs about {need / 2**30:.0f} GiB of host "
                          f"memory, more than this host offers"}
    secs, _ = oracle_map_sample(w, 0)
    return {"value": round(1.0 / secs, 6), "unit": "maps/s", "cores": ORACLE_THREADS, "kind": "oracle",
            "sample": f"one full map of {args.workload} by the numpy FP64 oracle ({secs:.1f} s; "
                      f"{os.cpu_count()} host cores present, numpy's FFT and array operations use one)"}


def run_reference(args, rank, world):
    """The oracle arm: full maps of the workload by the FP64 oracle on the host
    cores.  Each step is one map; the run stops early once --ref-budget-s of
    timed work is spent (at least one warm-up and one timed map), and the line
    reports the number of maps actually timed."""
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    need = ORACLE_BYTES_PER_CELL * w.N ** 3
    if need > 0.6 * host_memory_bytes():
        print(json.dumps({"impl": "reference", "unavailable": f"one FP64 oracle map of the {w.N}^3 box needs about "
                                                              f"{need / 2**30:.0f} GiB of host memory, more than this "
                                                              f"host offers"}), flush=True)
        return
    warm = max(1, min(args.warmup, 1))
    for i in range(warm):
        oracle_map_sample(w, i)
    times = []
    t_start = time.perf_counter()
    for i in range(args.steps):
        s, _ = oracle_map_sample(w, warm + i)
        times.append(s)
        if time.perf_counter() - t_start > args.ref_budget_s:
            break
    total = sum(times)
    value = len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "maps/s", "n_gpus": world,
            "steps": len(times), "warmup": warm, "ms_per_step": round(1e3 * total / len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "N": w.N, "npix": int(w.pixels().shape[0])},
            "cpu_baseline": {"value": round(value, 6), "unit": "maps/s", "cores": ORACLE_THREADS, "kind": "oracle",
                             "sample": f"{len(times)} full map(s) of {args.workload} by the numpy FP64 oracle "
                                       f"(bounded to about {args.ref_budget_s:.0f} s)"},
            "e2e": {"value": round(value, 6), "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--ref-budget-s", type=float, default=90.0)
    ap.add_argument("--impl", default="cmb3d", choices=["cmb3d", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary 512^3 figure")
    ap.add_argument("--three-pass", action="store_true", help="only separate y and x passes")
    ap.add_argument("--fused", action="store_true", help="only the fused y+x pass")
    ap.add_argument("--no-prune", action="store_true", help="transform the whole box for every map")
    ap.add_argument("--fused-xg", action="store_true",
                    help="sky maps with the x pass fused into the gather (CMB3D_FLAG_FUSED_XG)")
    ap.add_argument("--pipeline", action="store_true",
                    help="time the pipelined plan (two boxes, each map's draw overlapping the previous map's "
                         "passes and gather); by default it is timed after the main run and reported in config")
    ap.add_argument("--sweep", action="store_true", help="also time every kernel variant (stderr)")
    ap.add_argument("--schedule", default="",
                    help="fixed kernel variants 'draw,y,x,fused' (fused -1: separate passes) instead of the autotuner")
    ap.add_argument("--train-epochs", type=int, default=120, help="learned-inversion workload: training epochs")
    ap.add_argument("--refine-iters", type=int, default=300,
                    help="learned-inversion workload: FISTA steps of the refinement toward the NNLS optimum")
    ap.add_argument("--fp16-gemm", action="store_true",
                    help="y pass with split-FP16 DFT-GEMM stages on the tensor cores")
    args = ap.parse_args()
    ARGS_MODE.update(no_prune=args.no_prune, fused_xg=args.fused_xg, fused=args.fused)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_cuda(args, rank, world, local)


if __name__ == "__main__":
    main()
