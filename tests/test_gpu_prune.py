"""Pruned transform of the sky-map path.

A map only reads the field rows inside its pixels' interpolation stencils, so
the y pass covers only the z-planes holding such rows (and stores only those
rows) and the x pass only those rows.  The maps must equal the whole-box maps
bit for bit (same kernels, same arithmetic, fewer rows), the plane and row
counts must equal the ones counted here from the oracle's own pixel cells, and
the maps must match the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_pixels, fibonacci_sphere  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def smooth_pk(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def stencil_rows(pix, N, L, r, interp):
    """(z, y) rows read by the interpolation of every pixel, from the oracle's cells."""
    b, _ = orc.pixel_cells(pix, N, L, r)
    offs = (-1, 0, 1, 2) if interp == 3 else (0, 1)
    rows = set()
    for bz, by in set(zip(b[:, 2].tolist(), b[:, 1].tolist())):
        for c in offs:
            for d in offs:
                rows.add(((bz + c) % N, (by + d) % N))
    return rows


def stored_reals(pix, N, L, r, interp):
    """Reals the pruned x pass stores: per (z, y) row, every block of N/32
    columns holding an x that a stencil on that row reads (oracle cells)."""
    b, _ = orc.pixel_cells(pix, N, L, r)
    offs = np.array((-1, 0, 1, 2) if interp == 3 else (0, 1))
    z = (b[:, 2][:, None, None, None] + offs[:, None, None]) % N
    y = (b[:, 1][:, None, None, None] + offs[None, :, None]) % N
    x = (b[:, 0][:, None, None, None] + offs[None, None, :]) % N
    rowblk = (z * N + y) * 32 + x // (N // 32)
    return len(np.unique(rowblk)) * (N // 32)


@pytest.mark.parametrize("N,nside,fsky,interp,flags", [
    (128, 128, 0.4, 3, 0),
    (256, 256, 0.3, 3, 0),
    (256, 256, 0.1, 1, 0),
    (256, 128, 0.4, 3, cmb3d.CMB3D_FLAG_NO_SORT),
    (512, 256, 0.2, 3, 0),
])
def test_pruned_map_equals_whole_box_map(N, nside, fsky, interp, flags):
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(nside, fsky)
    with cmb3d.Plan(N, L, 1.0, pix, interp, flags | cmb3d.CMB3D_FLAG_STAGE_TIMING) as pruned, \
            cmb3d.Plan(N, L, 1.0, pix, interp, flags | cmb3d.CMB3D_FLAG_NO_PRUNE) as whole:
        pruned.set_pk(kn, pk)
        whole.set_pk(kn, pk)
        rows = stencil_rows(pix, N, L, 1.0, interp)
        planes = {z for z, _ in rows}
        assert cmb3d.cmb3d_plan_prune_info(pruned.handle) == (len(planes), len(rows))
        assert cmb3d.cmb3d_plan_prune_info(whole.handle) == (N, N * N)
        assert len(rows) < 0.5 * N * N
        # the x pass writes back only the column blocks the stencils read
        assert cmb3d.cmb3d_plan_x_stored(pruned.handle) == stored_reals(pix, N, L, 1.0, interp)
        assert cmb3d.cmb3d_plan_x_stored(whole.handle) == N ** 3
        assert cmb3d.cmb3d_plan_x_stored(pruned.handle) < 0.5 * len(rows) * N
        for seed in (0, 9):
            a = pruned.realize_sample(seed).cpu().numpy()
            b = whole.realize_sample(seed).cpu().numpy()
            np.testing.assert_array_equal(a, b)
        _, counts = cmb3d.cmb3d_stage_times(pruned.handle)
        assert list(counts) == [2, 2, 2, 2, 0]
        if N <= 256:
            ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 9, interp)
            assert float(np.max(np.abs(a - ref)) / np.sqrt(np.mean(ref ** 2))) <= TOL


@pytest.mark.parametrize("N", [256, 512])
def test_every_separate_variant_pruned(N):
    """Each y and x shape on the plane and row lists equals its whole-box run."""
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(256, 0.3)
    with cmb3d.Plan(N, L, 1.0, pix, 3) as pruned, \
            cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_NO_PRUNE) as whole:
        pruned.set_pk(kn, pk)
        whole.set_pk(kn, pk)
        for sc in [(0, y, 0, -1) for y in range(4)] + [(0, 0, x, -1) for x in range(4 if N >= 512 else 3)]:
            cmb3d.cmb3d_plan_set_schedule(pruned.handle, sc)
            cmb3d.cmb3d_plan_set_schedule(whole.handle, sc)
            np.testing.assert_array_equal(pruned.realize_sample(4).cpu().numpy(),
                                          whole.realize_sample(4).cpu().numpy(), err_msg=str(sc))
        # a fused schedule still gives the pruned separate passes for maps
        cmb3d.cmb3d_plan_set_schedule(pruned.handle, (0, -1, -1, 0))
        cmb3d.cmb3d_plan_set_schedule(whole.handle, (0, 0, 0, -1))
        np.testing.assert_array_equal(pruned.realize_sample(5).cpu().numpy(),
                                      whole.realize_sample(5).cpu().numpy())


def test_field_is_whole_and_tensor_core_y_pass_prunes_x():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    pix = cap_pixels(256, 0.3)
    with cmb3d.Plan(N, L, 1.0, pix, 3) as plan:
        plan.set_pk(kn, pk)
        field = plan.realize_field(21).cpu().numpy()
    assert float(np.max(np.abs(field - orc.realize_field(N, orc.p_box_of_q(N, L, kn, pk), 21)))
                 / np.sqrt(np.mean(field.astype(np.float64) ** 2))) <= TOL
    fl = cmb3d.CMB3D_FLAG_FP16_GEMM
    with cmb3d.Plan(N, L, 1.0, pix, 3, fl) as pruned, \
            cmb3d.Plan(N, L, 1.0, pix, 3, fl | cmb3d.CMB3D_FLAG_NO_PRUNE) as whole:
        pruned.set_pk(kn, pk)
        whole.set_pk(kn, pk)
        np.testing.assert_array_equal(pruned.realize_sample(3).cpu().numpy(), whole.realize_sample(3).cpu().numpy())


def test_no_pruning_when_stencils_cover_every_row():
    N, L = 128, 1.0
    pix = fibonacci_sphere(2_000_000)              # dense full sphere wrapping a small periodic box
    assert len(stencil_rows(pix, N, L, 1.0, 3)) == N * N
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_ALLOW_WRAP) as plan:
        assert cmb3d.cmb3d_plan_prune_info(plan.handle) == (N, N * N)
    with cmb3d.Plan(64, 2.2, 1.0, cap_pixels(64, 0.2), 3) as small:   # N < 128: whole box
        assert cmb3d.cmb3d_plan_prune_info(small.handle) == (64, 64 * 64)


def test_two_caps_store_two_plane_ranges():
    """Pixels of a north and a south cap: the listed z-planes form two ranges
    (the draw then tests a plane mask instead of one range); maps still equal
    the whole-box maps bit for bit, also through a pipelined plan."""
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    north = cap_pixels(128, 0.1)
    pix = np.concatenate([north, north * np.array([1.0, 1.0, -1.0])])
    with cmb3d.Plan(N, L, 1.0, pix, 3) as pruned, \
            cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_PIPELINE) as piped, \
            cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_NO_PRUNE) as whole:
        for p in (pruned, piped, whole):
            p.set_pk(kn, pk)
        planes, _ = cmb3d.cmb3d_plan_prune_info(pruned.handle)
        assert planes < N // 2
        for sd in (5, 6):
            ref = whole.realize_sample(sd).cpu().numpy()
            np.testing.assert_array_equal(pruned.realize_sample(sd).cpu().numpy(), ref)
            np.testing.assert_array_equal(piped.realize_sample(sd).cpu().numpy(), ref)
