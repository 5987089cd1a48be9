"""Fault handling without a GPU fault.

* A pruned sky map transforms only the z-planes and (z, y) rows its pixels'
  interpolation stencils read.  With every entry of the plan's box(es) set to
  NaN beforehand, the map must come out finite and equal, bit for bit, to the
  map of a clean box: no pass reads an entry that an earlier pass of the same
  map did not write.
* An allocation that would pass a (test) device-memory limit makes plan
  creation fail with CMB3D_ENOMEM and release what it had taken; the next plan
  works.
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


def spectrum(N, L):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, 128)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


@pytest.mark.parametrize("N,nside,fsky,interp,flags", [
    (256, 256, 0.1, 3, cmb3d.CMB3D_FLAG_NONE),
    (512, 512, 0.4, 3, cmb3d.CMB3D_FLAG_NONE),
    (256, 256, 0.05, 1, cmb3d.CMB3D_FLAG_PIPELINE),
    (1024, 512, 0.2, 3, cmb3d.CMB3D_FLAG_NONE),
])
def test_pruned_map_reads_no_stale_entries(N, nside, fsky, interp, flags):
    pix = cap_pixels(nside, fsky)
    with cmb3d.Plan(N, 2.2, 1.0, pix, interp, flags) as plan:
        plan.set_pk(*spectrum(N, 2.2))
        planes, rows = cmb3d.cmb3d_plan_prune_info(plan.handle)
        assert planes < N and rows < N * N            # the transform is pruned
        ref = [plan.realize_sample(s).cpu().numpy() for s in (3, 4)]
        cmb3d.cmb3d_debug_poison_boxes(plan.handle)
        got = [plan.realize_sample(s).cpu().numpy() for s in (3, 4)]
    for a, b in zip(got, ref):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


def test_allocation_limit_gives_enomem_and_frees():
    pix = cap_pixels(32, 0.2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    cmb3d.cmb3d_debug_alloc_limit(1 << 20)          # below one 64^3 box (1 MiB + a scratch row)
    try:
        with pytest.raises(cmb3d.Cmb3dError) as e:
            cmb3d.Plan(64, 2.2, 1.0, pix, 1)
        assert e.value.status == cmb3d.CMB3D_ENOMEM
        assert "limit" in cmb3d.load().cmb3d_error_detail().decode()
        # a plan with one box (1 MiB and about 0.1 MiB of tables) fits, a
        # pipelined plan's second box does not
        cmb3d.cmb3d_debug_alloc_limit((1 << 20) + (600 << 10))
        with cmb3d.Plan(64, 2.2, 1.0, pix, 1) as plan:
            info = cmb3d.cmb3d_plan_info(plan.handle)
            assert info[2] <= (1 << 20) + (600 << 10)
        with pytest.raises(cmb3d.Cmb3dError) as e:
            cmb3d.Plan(64, 2.2, 1.0, pix, 1, cmb3d.CMB3D_FLAG_PIPELINE)
        assert e.value.status == cmb3d.CMB3D_ENOMEM
    finally:
        cmb3d.cmb3d_debug_alloc_limit(0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= 4 << 20                 # nothing left behind (allocator granularity)
    with cmb3d.Plan(64, 2.2, 1.0, pix, 1) as plan:       # the library still works
        plan.set_pk(*spectrum(64, 2.2))
        assert np.all(np.isfinite(plan.realize_sample(1).cpu().numpy()))
