"""The 2-D Fourier method (paper Sec. II.D.2) on the GPU against its FP64
oracle (oracle/fourier2d.py): the hybrid layers element by element, the real
layers and sky maps to 1e-5 of rms, pruned and pipelined maps bit for bit
equal to plain ones, and the argument checks that need a device."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fourier2d as f2  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_layers, cap_pixels, fibonacci_sphere  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def spectrum(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / np.sqrt(np.mean(ref ** 2)))


def packed(hyb):
    """Oracle hybrid layers [z, m_y, m_x <= N/2] in the kernel's packing."""
    N = hyb.shape[1]
    out = hyb[:, :, : N // 2].copy()
    out[:, :, 0] = hyb[:, :, 0] + 1j * hyb[:, :, N // 2]
    return out


@pytest.mark.parametrize("N,M,h", [(32, 16, 3), (32, 16, 8), (64, 32, 13), (32, 64, 32), (16, 8, 12)])
def test_hybrid_layers_match_oracle(N, M, h):
    L = 2.2
    kn, pk = spectrum(N, L)
    with cmb3d.Plan2D(N, M, h, L, 1.0, 0.0, np.zeros((0, 3))) as plan:
        plan.set_pk(kn, pk)
        got = plan.draw_spectrum(5).cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    table = f2.sqrt_gamma_table(N, M, h, L, kn, pk)
    ref = packed(f2.hybrid_from_normals(N, h, table, f2.normals_2d(N, h, 5)))
    scale = np.sqrt(np.mean(np.abs(ref) ** 2, axis=(1, 2)))[:, None, None]
    assert np.max(np.abs(got - ref) / scale) <= 2e-5


@pytest.mark.parametrize("N,M,h", [(32, 16, 5), (128, 32, 12), (256, 64, 22)])
def test_layers_match_oracle(N, M, h):
    L = 2.2
    kn, pk = spectrum(N, L)
    with cmb3d.Plan2D(N, M, h, L, 1.0, 0.0, np.zeros((0, 3))) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_field(9).cpu().numpy()
    ref = f2.realize_field_2d(N, M, h, L, kn, pk, 9)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("N,M,theta,dp,interp,flags", [
    (64, 32, 25.0, 0.02, 3, 0),
    (128, 32, 20.0, 0.0075, 1, 0),
    (128, 32, 20.0, 0.0075, 3, cmb3d.CMB3D_FLAG_NO_SORT),
    (256, 64, 15.0, 0.0034, 3, 0),
])
def test_maps_match_oracle(N, M, theta, dp, interp, flags):
    L = N * dp
    z0, h = cap_layers(theta, dp, 1.0, interp)
    kn, pk = spectrum(N, L)
    pix = fibonacci_sphere(400000, int(400000 * (1 - math.cos(math.radians(theta))) / 2))
    with cmb3d.Plan2D(N, M, h, L, 1.0, z0, pix, interp, flags) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(17).cpu().numpy()
    ref = f2.realize_sample_2d(N, M, h, L, 1.0, z0, pix, kn, pk, 17, interp)
    assert rel_err(got, ref) <= TOL


def test_pruned_pipelined_and_batched_maps_equal_plain_maps():
    N, M, theta, dp = 256, 64, 20.0, 0.004
    L = N * dp
    z0, h = cap_layers(theta, dp)
    kn, pk = spectrum(N, L)
    pix = cap_pixels(256, (1 - math.cos(math.radians(theta))) / 2)
    args = (N, M, h, L, 1.0, z0, pix, 3)
    with cmb3d.Plan2D(*args, cmb3d.CMB3D_FLAG_STAGE_TIMING) as pruned, \
            cmb3d.Plan2D(*args, cmb3d.CMB3D_FLAG_NO_PRUNE) as whole, \
            cmb3d.Plan2D(*args, cmb3d.CMB3D_FLAG_PIPELINE | cmb3d.CMB3D_FLAG_AUTOTUNE) as piped:
        for p in (pruned, whole, piped):
            p.set_pk(kn, pk)
        planes, rows = cmb3d.cmb3d_plan_prune_info(pruned.handle)
        assert planes <= h and rows < h * N
        assert cmb3d.cmb3d_plan_prune_info(whole.handle) == (h, h * N)
        outs = [piped.realize_sample(s) for s in (1, 2, 3)]          # back to back
        sched = cmb3d.cmb3d_plan_schedule(piped.handle)
        cmb3d.cmb3d_plan_set_schedule(pruned.handle, (0, sched[1], sched[2], -1))
        cmb3d.cmb3d_plan_set_schedule(whole.handle, (0, sched[1], sched[2], -1))
        for s, o in zip((1, 2, 3), outs):
            a = pruned.realize_sample(s).cpu().numpy()
            np.testing.assert_array_equal(a, whole.realize_sample(s).cpu().numpy())
            np.testing.assert_array_equal(a, o.cpu().numpy())
        _, counts = cmb3d.cmb3d_stage_times(pruned.handle)
        assert list(counts) == [3, 3, 3, 3, 0]
        batch_out = [torch.empty(len(pix), device="cuda") for _ in range(2)]
        cmb3d.cmb3d_realize_sample_batch([pruned.handle, whole.handle], [7, 8], batch_out)
        np.testing.assert_array_equal(batch_out[0].cpu().numpy(), pruned.realize_sample(7).cpu().numpy())
        np.testing.assert_array_equal(batch_out[1].cpu().numpy(), pruned.realize_sample(8).cpu().numpy())


def test_stencils_must_lie_in_the_layers():
    N, M, dp = 64, 32, 0.02
    z0, h = cap_layers(25.0, dp)
    pix = fibonacci_sphere(10000, int(10000 * (1 - math.cos(math.radians(25.0))) / 2))   # a 25-degree cap
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.Plan2D(N, M, h - 1, N * dp, 1.0, z0, pix, 3)                # one layer short
    assert e.value.status == cmb3d.CMB3D_EINVAL
    cmb3d.Plan2D(N, M, h, N * dp, 1.0, z0, pix, 3).close()
