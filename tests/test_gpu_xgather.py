"""The x pass fused with the gather (CMB3D_FLAG_FUSED_XG): the real rows are
formed in shared memory per 8 x 8 tile of (z, y) base cells and never
written.  Its maps must equal, bit for bit, the maps of the separate x pass
(of the same radix: x variant 1 at N = 1024, else 0) and gather, for
every pixel order, interpolation, wrap, pruning, pipelining and method, and
match the oracle within 1e-5 of rms."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_layers, cap_pixels, fibonacci_sphere  # noqa: E402

pytestmark = pytest.mark.gpu
XG = cmb3d.CMB3D_FLAG_FUSED_XG


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def smooth_pk(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def same_radix_x(N):
    return 1 if N == 1024 else 0


def pair_maps(N, L, pix, interp, flags, seeds, r=1.0):
    kn, pk = smooth_pk(N, L)
    with cmb3d.Plan(N, L, r, pix, interp, flags | XG) as fused, cmb3d.Plan(N, L, r, pix, interp, flags) as plain:
        fused.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(plain.handle, (0, 0, same_radix_x(N), -1))
        cmb3d.cmb3d_plan_set_schedule(fused.handle, (0, 0, same_radix_x(N), -1))
        return ([fused.realize_sample(s).cpu().numpy() for s in seeds],
                [plain.realize_sample(s).cpu().numpy() for s in seeds])


@pytest.mark.parametrize("N,interp,flags", [
    (64, 3, 0), (64, 1, cmb3d.CMB3D_FLAG_NO_SORT), (128, 3, 0), (128, 1, 0), (256, 3, 0),
    (256, 3, cmb3d.CMB3D_FLAG_NO_SORT), (512, 3, 0), (512, 1, 0), (32, 3, 0),
    (256, 3, cmb3d.CMB3D_FLAG_NO_PRUNE), (256, 1, cmb3d.CMB3D_FLAG_PIPELINE),
])
def test_fused_maps_equal_separate_maps(N, interp, flags):
    pix = cap_pixels(128 if N <= 128 else 256, 0.3)
    got, ref = pair_maps(N, 2.2, pix, interp, flags, (3, 4))
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


def test_fused_maps_match_oracle():
    N, L = 128, 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(64, 0.4)
    with cmb3d.Plan(N, L, 1.0, pix, 3, XG) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(6).cpu().numpy()
    ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 6, 3)
    assert np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2)) <= 1e-5


def test_fused_maps_wrap_around_a_small_box():
    """The sphere is larger than the box: tiles at the box faces read rows
    across the periodic boundary in z and y, and columns across it in x."""
    N = 64
    pix = fibonacci_sphere(20000, 20000)
    got, ref = pair_maps(N, 1.5, pix, 3, cmb3d.CMB3D_FLAG_ALLOW_WRAP, (9,))
    np.testing.assert_array_equal(got[0], ref[0])


def test_fused_maps_split_long_limb_tiles():
    """Full sphere at 1024^3: tiles near the limb (where the surface runs along
    x) reach more than 64 columns and are split into runs of bx."""
    pix = fibonacci_sphere(3_000_000, 3_000_000)
    got, ref = pair_maps(1024, 2.2, pix, 3, 0, (2,))
    np.testing.assert_array_equal(got[0], ref[0])


def test_fused_2d_maps_equal_separate_maps():
    N, M, dp = 256, 64, 0.004
    z0, h = cap_layers(20.0, dp)
    kn, pk = smooth_pk(N, N * dp)
    pix = cap_pixels(256, (1 - math.cos(math.radians(20.0))) / 2)
    args = (N, M, h, N * dp, 1.0, z0, pix, 3)
    with cmb3d.Plan2D(*args, XG) as fused, cmb3d.Plan2D(*args) as plain:
        fused.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        for p in (fused, plain):
            cmb3d.cmb3d_plan_set_schedule(p.handle, (0, 0, 0, -1))
        for sd in (1, 2):
            np.testing.assert_array_equal(fused.realize_sample(sd).cpu().numpy(), plain.realize_sample(sd).cpu().numpy())


def test_fused_plan_keeps_the_whole_field_and_stage_counts():
    N, L = 128, 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(64, 0.2)
    with cmb3d.Plan(N, L, 1.0, pix, 1, XG | cmb3d.CMB3D_FLAG_STAGE_TIMING) as fused, \
            cmb3d.Plan(N, L, 1.0, pix, 1) as plain:
        fused.set_pk(kn, pk)
        plain.set_pk(kn, pk)
        np.testing.assert_array_equal(fused.realize_field(5).cpu().numpy(), plain.realize_field(5).cpu().numpy())
        cmb3d.cmb3d_stage_times(fused.handle, reset=True)
        fused.realize_sample(5)
        _, counts = cmb3d.cmb3d_stage_times(fused.handle)
        assert list(counts) == [1, 1, 0, 1, 0]                       # draw, y, (no x), fused gather
