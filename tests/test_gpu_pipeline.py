"""Pipelined plans (CMB3D_FLAG_PIPELINE): two boxes and two internal streams,
the draw of a map overlapping the passes and gather of the previous one.

Every map must equal the map of a plain plan bit for bit (same kernels, same
arithmetic), whatever is interleaved: maps issued back to back without a
synchronisation, the whole field, a new spectrum, the host-output entry
point, the autotuner on the first call, and batches.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_pixels  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def smooth_pk(N, L, nk=96, amp=1e-3):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, amp / (1.0 + (k / 12.0) ** 3)


@pytest.mark.parametrize("N,flags", [(128, 0), (256, cmb3d.CMB3D_FLAG_STAGE_TIMING), (256, cmb3d.CMB3D_FLAG_NO_PRUNE)])
def test_back_to_back_maps_equal_plain_maps(N, flags):
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(128, 0.3)
    seeds = list(range(100, 109))
    with cmb3d.Plan(N, L, 1.0, pix, 3, flags | cmb3d.CMB3D_FLAG_PIPELINE) as piped, \
            cmb3d.Plan(N, L, 1.0, pix, 3, flags) as plain:
        piped.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        outs = [torch.empty(len(pix), dtype=torch.float32, device="cuda") for _ in seeds]
        for sd, o in zip(seeds, outs):                       # no synchronisation in between
            piped.realize_sample(sd, o)
        torch.cuda.synchronize()
        for sd, o in zip(seeds, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), plain.realize_sample(sd).cpu().numpy())
        if flags & cmb3d.CMB3D_FLAG_STAGE_TIMING:
            _, counts = cmb3d.cmb3d_stage_times(piped.handle)
            assert list(counts) == [len(seeds)] * 4 + [0]
        _, _, nbytes_piped = cmb3d.cmb3d_plan_info(piped.handle)
        _, _, nbytes_plain = cmb3d.cmb3d_plan_info(plain.handle)
        assert nbytes_piped - nbytes_plain == 4 * N ** 3 + 4 * N      # the second box


def test_interleaved_field_spectrum_and_host_output():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    kn2, pk2 = smooth_pk(N, L, amp=3e-3)
    pix = cap_pixels(128, 0.25)
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_PIPELINE) as piped, \
            cmb3d.Plan(N, L, 1.0, pix, 3) as plain:
        piped.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        a0 = piped.realize_sample(1)
        f = piped.realize_field(2)                           # whole field on the caller's stream
        a1 = piped.realize_sample(3)
        a2 = piped.realize_sample(4)
        np.testing.assert_array_equal(a0.cpu().numpy(), plain.realize_sample(1).cpu().numpy())
        np.testing.assert_array_equal(f.cpu().numpy(), plain.realize_field(2).cpu().numpy())
        np.testing.assert_array_equal(a1.cpu().numpy(), plain.realize_sample(3).cpu().numpy())
        np.testing.assert_array_equal(a2.cpu().numpy(), plain.realize_sample(4).cpu().numpy())
        piped.realize_sample(5)                              # still in flight when the spectrum changes
        piped.set_pk(kn2, pk2)
        plain.set_pk(kn2, pk2)
        b = piped.realize_sample(6)
        np.testing.assert_array_equal(b.cpu().numpy(), plain.realize_sample(6).cpu().numpy())
        host = np.empty(len(pix), np.float32)
        for sd in (7, 8, 9):
            cmb3d.cmb3d_realize_sample_to_host(piped.handle, sd, host)
            np.testing.assert_array_equal(host, plain.realize_sample(sd).cpu().numpy())


def test_autotune_on_first_pipelined_call():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(128, 0.3)
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_PIPELINE | cmb3d.CMB3D_FLAG_AUTOTUNE) as piped, \
            cmb3d.Plan(N, L, 1.0, pix, 3) as plain:
        piped.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        outs = [piped.realize_sample(sd) for sd in (11, 12, 13)]
        sched = cmb3d.cmb3d_plan_schedule(piped.handle)
        sep = (sched[0], sched[1] if sched[1] >= 0 else 0, sched[2] if sched[2] >= 0 else 0, -1)
        cmb3d.cmb3d_plan_set_schedule(plain.handle, sep)     # maps use the separate pruned passes
        for sd, o in zip((11, 12, 13), outs):
            np.testing.assert_array_equal(o.cpu().numpy(), plain.realize_sample(sd).cpu().numpy())


def test_batch_of_pipelined_plans():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    pixs = [cap_pixels(128, f) for f in (0.1, 0.3, 0.2)]
    plans = [cmb3d.Plan(N, L, 1.0, p, 1, cmb3d.CMB3D_FLAG_PIPELINE) for p in pixs]
    refs = [cmb3d.Plan(N, L, 1.0, p, 1) for p in pixs]
    try:
        for p in plans + refs:
            p.set_pk(kn, pk)
        first = plans[0].realize_sample(40)                  # pipelined work in flight
        outs = [torch.empty(len(p), dtype=torch.float32, device="cuda") for p in pixs]
        cmb3d.cmb3d_realize_sample_batch([p.handle for p in plans], [41, 42, 43], outs)
        after = plans[0].realize_sample(44)
        np.testing.assert_array_equal(first.cpu().numpy(), refs[0].realize_sample(40).cpu().numpy())
        for sd, o, r in zip((41, 42, 43), outs, refs):
            np.testing.assert_array_equal(o.cpu().numpy(), r.realize_sample(sd).cpu().numpy())
        np.testing.assert_array_equal(after.cpu().numpy(), refs[0].realize_sample(44).cpu().numpy())
    finally:
        for p in plans + refs:
            p.close()


@pytest.mark.parametrize("flags", [0, cmb3d.CMB3D_FLAG_PIPELINE, cmb3d.CMB3D_FLAG_STAGE_TIMING])
def test_many_maps_to_host_equal_single_maps(flags):
    """cmb3d_realize_samples_to_host: two staging buffers and a copy stream;
    every map equals the single-call map bit for bit, in pinned and pageable
    host memory, and a host buffer named twice holds its last map."""
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(128, 0.3)
    seeds = [21, 22, 23, 24, 25]
    with cmb3d.Plan(N, L, 1.0, pix, 3, flags) as plan, cmb3d.Plan(N, L, 1.0, pix, 3) as plain:
        plan.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        refs = [plain.realize_sample(sd).cpu().numpy() for sd in seeds]
        pinned = [torch.empty(len(pix), dtype=torch.float32).pin_memory().numpy() for _ in seeds]
        cmb3d.cmb3d_realize_samples_to_host(plan.handle, seeds, pinned)
        for o, r in zip(pinned, refs):
            np.testing.assert_array_equal(o, r)
        pageable = [np.empty(len(pix), np.float32) for _ in range(2)]
        cmb3d.cmb3d_realize_samples_to_host(plan.handle, seeds[:2], pageable)
        np.testing.assert_array_equal(pageable[1], refs[1])
        shared = np.empty(len(pix), np.float32)
        cmb3d.cmb3d_realize_samples_to_host(plan.handle, seeds[:3], [shared] * 3)
        np.testing.assert_array_equal(shared, refs[2])
        cmb3d.cmb3d_realize_samples_to_host(plan.handle, [], [])
        np.testing.assert_array_equal(plan.realize_sample(seeds[0]).cpu().numpy(), refs[0])   # still a plain plan
        if flags & cmb3d.CMB3D_FLAG_STAGE_TIMING:
            _, counts = cmb3d.cmb3d_stage_times(plan.handle)
            assert list(counts) == [11] * 4 + [0]


def test_many_maps_to_host_of_a_2d_plan():
    from synth import cap_layers
    N, M, dp = 128, 32, 0.0075
    z0, h = cap_layers(20.0, dp)
    kn, pk = smooth_pk(N, N * dp)
    pix = cap_pixels(128, 0.03)
    with cmb3d.Plan2D(N, M, h, N * dp, 1.0, z0, pix, 3, cmb3d.CMB3D_FLAG_PIPELINE) as plan:
        plan.set_pk(kn, pk)
        outs = [np.empty(len(pix), np.float32) for _ in range(3)]
        cmb3d.cmb3d_realize_samples_to_host(plan.handle, [4, 5, 6], outs)
        for sd, o in zip((4, 5, 6), outs):
            np.testing.assert_array_equal(o, plan.realize_sample(sd).cpu().numpy())


def test_many_maps_to_host_rejects_null_outputs():
    N, L = 128, 2.2
    kn, pk = smooth_pk(N, L)
    with cmb3d.Plan(N, L, 1.0, cap_pixels(64, 0.2), 1) as plan:
        plan.set_pk(kn, pk)
        lib = cmb3d.load()
        import ctypes as C
        seeds = (C.c_uint64 * 2)(1, 2)
        outs = (C.c_void_p * 2)(None, None)
        assert lib.cmb3d_realize_samples_to_host(plan.handle, seeds, 2, outs, None) == cmb3d.CMB3D_EINVAL
        assert lib.cmb3d_realize_samples_to_host(plan.handle, None, 2, outs, None) == cmb3d.CMB3D_EINVAL
