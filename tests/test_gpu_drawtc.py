"""The draw with its 1024-point z-transform on the tensor cores.

At N = 1024 the last draw variant computes every column's z-transform as two
32-point DFT-GEMMs of split FP16 operands with FP32 accumulation (tcgen05).
Its maps and whole fields must equal those of the FP32 Stockham draw within
the FP32-path bar (max |d| / rms <= 1e-5), over pruned plane ranges, with the
Philox key in device memory (batch form), and (slow) against the FP64 oracle
itself.  The autotuner may pick it, so every schedule it can choose is a
parity case.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_pixels  # noqa: E402

pytestmark = pytest.mark.gpu
N, L, R = 1024, 2.2, 1.0
DRAW_TC = 6          # the last draw variant at N = 1024
DRAW_FP32 = 0        # the Stockham draw (radix 16, 16 columns)
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def spectrum():
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, 512)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3) * np.exp(-(k / 900.0) ** 2)


def rel(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2)))


def test_every_1024_variant_equals_default():
    """Every draw, y and x shape the autotuner may pick at N = 1024 (the
    tensor-core draw included) against the default shapes (the slow oracle
    test below pins the tensor-core draw, the y-pass study in
    test_gpu_tensorcore the default shapes, to the FP64 oracle)."""
    pix = cap_pixels(256, 0.4)
    kn, pk = spectrum()
    with cmb3d.Plan(N, L, R, pix, 3) as plan:
        plan.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (0, 0, 0, -1))
        ref = plan.realize_sample(21).cpu().numpy()
        scheds = [(d, 0, 0, -1) for d in range(1, DRAW_TC + 1)] + [(0, y, 0, -1) for y in range(1, 4)] + \
                 [(0, 0, x, -1) for x in range(1, 4)]
        for sc in scheds:
            cmb3d.cmb3d_plan_set_schedule(plan.handle, sc)
            assert rel(plan.realize_sample(21).cpu().numpy(), ref) <= TOL, sc


def test_tc_draw_is_a_draw_variant():
    pix = cap_pixels(64, 0.1)
    with cmb3d.Plan(N, L, R, pix, 3) as plan:
        plan.set_pk(*spectrum())
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (DRAW_TC, 0, 0, -1))
        assert cmb3d.cmb3d_plan_schedule(plan.handle)[0] == DRAW_TC
        with pytest.raises(cmb3d.Cmb3dError):
            cmb3d.cmb3d_plan_set_schedule(plan.handle, (DRAW_TC + 1, 0, 0, -1))


@pytest.mark.parametrize("fsky,nside,interp", [(0.4, 512, 3), (0.05, 1024, 1), (1.0, 256, 3)])
def test_tc_draw_maps_equal_fp32_draw(fsky, nside, interp):
    pix = cap_pixels(nside, fsky)
    kn, pk = spectrum()
    with cmb3d.Plan(N, L, R, pix, interp) as a, cmb3d.Plan(N, L, R, pix, interp) as b:
        a.set_pk(kn, pk)
        b.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(a.handle, (DRAW_TC, 0, 0, -1))
        cmb3d.cmb3d_plan_set_schedule(b.handle, (DRAW_FP32, 0, 0, -1))
        for seed in (0, 1, 2**40 + 3):
            ma = a.realize_sample(seed).cpu().numpy()
            mb = b.realize_sample(seed).cpu().numpy()
            assert rel(ma, mb) <= TOL, (fsky, seed, rel(ma, mb))


def test_tc_draw_whole_field_equals_fp32_draw():
    pix = cap_pixels(64, 0.1)
    kn, pk = spectrum()
    field = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    with cmb3d.Plan(N, L, R, pix, 3) as plan:
        plan.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (DRAW_FP32, 0, 0, -1))
        plan.realize_field(7, field)
        ref = field.cpu().numpy()
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (DRAW_TC, 0, 0, -1))
        plan.realize_field(7, field)
        got = field.cpu().numpy()
    assert rel(got, ref) <= TOL
    # the Hermitian column and its neighbours (tile 0 of each row) are in place
    z = got.reshape(N, N, N)[:, :, :8]
    assert np.all(np.isfinite(z)) and rel(z, ref.reshape(N, N, N)[:, :, :8]) <= TOL


def test_tc_draw_in_batch_graph():
    """The batch form reads the Philox key from device memory."""
    pixs = [cap_pixels(128, f) for f in (0.1, 0.3)]
    kn, pk = spectrum()
    plans = [cmb3d.Plan(N, L, R, p, 3) for p in pixs]
    try:
        for p in plans:
            p.set_pk(kn, pk)
            cmb3d.cmb3d_plan_set_schedule(p.handle, (DRAW_TC, 0, 0, -1))
        outs = [torch.empty(p.shape[0], dtype=torch.float32, device="cuda") for p in pixs]
        cmb3d.cmb3d_batch_debug(0, False, 2)                     # the two-stream graph form
        try:
            cmb3d.cmb3d_realize_sample_batch([p.handle for p in plans], [11, 12], outs)
        finally:
            cmb3d.cmb3d_batch_debug(0, False, -1)
        torch.cuda.synchronize()
        for p, o, s in zip(plans, outs, (11, 12)):
            cmb3d.cmb3d_plan_set_schedule(p.handle, (DRAW_FP32, 0, 0, -1))
            assert rel(o.cpu().numpy(), p.realize_sample(s).cpu().numpy()) <= TOL
    finally:
        for p in plans:
            p.close()


@pytest.mark.slow
def test_tc_draw_map_matches_oracle():
    pix = cap_pixels(256, 0.4)
    kn, pk = spectrum()
    with cmb3d.Plan(N, L, R, pix, 3) as plan:
        plan.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (DRAW_TC, 0, 0, -1))
        got = plan.realize_sample(5).cpu().numpy()
    ref = orc.realize_sample(N, L, R, pix, orc.p_box_of_q(N, L, kn, pk), 5, 3)
    assert rel(got, ref) <= TOL
