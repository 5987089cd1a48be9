"""The split-FP16 DFT-GEMM stage on the tensor cores (tcgen05, FP32 accumulate).

With CMB3D_FLAG_FP16_GEMM the y pass runs its radix-16 stages as GEMMs of
split (hi + lo) FP16 operands.  Bar for this path: max|T - T_oracle| / rms
<= 1e-3 against the FP64 oracle; the FP32-butterfly path keeps its 1e-5.
The 1024^3 study reports max and RMS errors for seeds 0..3 at the ~20M pixels
of the 1024^3 cap workload, both forms, and writes them as JSON.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import WORKLOADS, fibonacci_sphere  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def smooth_pk(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def errors(got, ref):
    d = np.asarray(got, np.float64) - ref
    rms = np.sqrt(np.mean(ref ** 2))
    return float(np.max(np.abs(d)) / rms), float(np.sqrt(np.mean(d ** 2)) / rms)


@pytest.mark.parametrize("N", [256, 512])
def test_fp16_gemm_stage_matches_oracle(N):
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(40000, 9001)
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_FP16_GEMM) as tc_plan, \
            cmb3d.Plan(N, L, 1.0, pix, 3) as fp32_plan:
        tc_plan.set_pk(kn, pk)
        fp32_plan.set_pk(kn, pk)
        d, y, x, f = cmb3d.cmb3d_plan_schedule(tc_plan.handle)
        assert f == -1 and y == 4                       # the tensor-core y variant follows the 4 butterfly shapes
        for seed in range(4):
            ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), seed, 3)
            mx, rms = errors(tc_plan.realize_sample(seed).cpu().numpy(), ref)
            assert mx <= 1e-3, (seed, mx, rms)
            mx32, _ = errors(fp32_plan.realize_sample(seed).cpu().numpy(), ref)
            assert mx32 <= 1e-5


def test_fp16_gemm_field_and_flag_rules():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    with cmb3d.Plan(N, L, 1.0, np.zeros((0, 3)), 1, cmb3d.CMB3D_FLAG_FP16_GEMM | cmb3d.CMB3D_FLAG_STAGE_TIMING) as p:
        p.set_pk(kn, pk)
        got = p.realize_field(7).cpu().numpy()
        cmb3d.cmb3d_stage_times(p.handle)             # also checks the device error word
    ref = orc.realize_field(N, orc.p_box_of_q(N, L, kn, pk), 7)
    mx, _ = errors(got, ref)
    assert mx <= 1e-3
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.Plan(128, L, 1.0, np.zeros((0, 3)), 1, cmb3d.CMB3D_FLAG_FP16_GEMM)
    assert e.value.status == cmb3d.CMB3D_EUNSUPPORTED
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.Plan(N, L, 1.0, np.zeros((0, 3)), 1, cmb3d.CMB3D_FLAG_FP16_GEMM | cmb3d.CMB3D_FLAG_FUSED_YX)


@pytest.mark.slow
def test_precision_study_box1024_seeds_0_to_3(tmp_path):
    """1024^3 box, ~20M tricubic cap pixels: max and RMS error of the split-FP16
    GEMM form and of the FP32-butterfly form against the FP64 oracle."""
    w = WORKLOADS["box1024_cap0.4_tricubic"]
    pix = w.pixels()
    kn, pk = smooth_pk(w.N, w.L, 256)
    pb = orc.p_box_of_q(w.N, w.L, kn, pk)
    b, t = orc.pixel_cells(pix, w.N, w.L, w.r)
    report = {"workload": w.name, "npix": int(pix.shape[0]), "seeds": {}}
    with cmb3d.Plan(w.N, w.L, w.r, pix, w.interp, cmb3d.CMB3D_FLAG_FP16_GEMM) as tc_plan, \
            cmb3d.Plan(w.N, w.L, w.r, pix, w.interp) as fp32_plan:
        tc_plan.set_pk(kn, pk)
        fp32_plan.set_pk(kn, pk)
        for seed in range(4):
            got_tc = tc_plan.realize_sample(seed).cpu().numpy()
            got_32 = fp32_plan.realize_sample(seed).cpu().numpy()
            ref = orc.sample(orc.realize_field(w.N, pb, seed), b, t, w.interp)
            e_tc, e_32 = errors(got_tc, ref), errors(got_32, ref)
            report["seeds"][seed] = {"fp16_gemm": {"max": e_tc[0], "rms": e_tc[1]},
                                     "fp32": {"max": e_32[0], "rms": e_32[1]}}
            assert e_tc[0] <= 1e-3 and e_32[0] <= 1e-5, report
    out = os.environ.get("CMB3D_PRECISION_REPORT", str(tmp_path / "precision_box1024.json"))
    with open(out, "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))
