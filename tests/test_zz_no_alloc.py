"""The plan-free entry point that allocates no device memory.

Callers that cannot call cudaMalloc (code inside another runtime that owns all
device memory) use cmb3d_realize_sample_noalloc, whose box lives in a static
device array.  Its maps must equal those of the ordinary plan-based entry
point, cmb3d_realize_sample, within the FP32-path tolerance of the parity
tests, on two calls in a row (the second call must not see the first call's
box), at every supported size (each has its own twiddle table in the static
array), and match the FP64 oracle directly.  Sizes beyond the static maximum
must be rejected with the reason in cmb3d_error_detail(), and a pixel that
cannot be placed must come back as NaN.  Kept in a file that pytest collects
last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_pixels  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def amp_table(N, L, knodes, pnodes):
    """sqrt(P_box(q)/2) for q = 0 .. 3 (N/2)^2, P_box = P_inf(2 pi sqrt(q)/L) (2 pi/L)^3."""
    kf = 2.0 * np.pi / L
    q = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    k = kf * np.sqrt(q)
    p = np.interp(k, knodes, pnodes)
    p = np.where(k > knodes[-1], 0.0, p)
    return np.sqrt(p * kf ** 3 / 2.0).astype(np.float32)


def spectrum(N, L):
    knodes = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, 96)
    return knodes, 1e-3 / (1.0 + (knodes / 12.0) ** 3)


def rel_err(got, ref):
    return np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2))


@pytest.mark.parametrize("N", [8, 16, 32, 64])
@pytest.mark.parametrize("interp", [cmb3d.CMB3D_TRILINEAR, cmb3d.CMB3D_TRICUBIC])
def test_noalloc_matches_plan_entry_point(N, interp):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()
    L, r = 2.2, 1.0
    pix = cap_pixels(32, 0.1)
    knodes, pnodes = spectrum(N, L)
    pix_dev = torch.tensor(pix, dtype=torch.float64, device="cuda")
    amp_dev = torch.tensor(amp_table(N, L, knodes, pnodes), device="cuda")
    out = torch.empty(pix.shape[0], dtype=torch.float32, device="cuda")
    with cmb3d.Plan(N, L, r, pix, interp) as plan:
        plan.set_pk(knodes, pnodes)
        for seed in (7, 8):                       # two calls in a row
            ref = plan.realize_sample(seed).cpu().numpy().astype(np.float64)
            cmb3d.cmb3d_realize_sample_noalloc(N, L, r, pix_dev, pix.shape[0], interp, amp_dev, seed, out)
            got = out.cpu().numpy().astype(np.float64)
            assert rel_err(got, ref) <= TOL, (N, seed)


def test_noalloc_matches_oracle():
    cmb3d.load()
    N, L, r, seed = 32, 2.2, 1.0, 11
    pix = cap_pixels(16, 0.3)
    knodes, pnodes = spectrum(N, L)
    out = torch.empty(pix.shape[0], dtype=torch.float32, device="cuda")
    cmb3d.cmb3d_realize_sample_noalloc(N, L, r, torch.tensor(pix, dtype=torch.float64, device="cuda"),
                                       pix.shape[0], cmb3d.CMB3D_TRICUBIC,
                                       torch.tensor(amp_table(N, L, knodes, pnodes), device="cuda"), seed, out)
    ref = orc.realize_sample(N, L, r, pix, orc.p_box_of_q(N, L, knodes, pnodes), seed, 3)
    assert rel_err(out.cpu().numpy().astype(np.float64), ref) <= TOL


def test_noalloc_non_finite_pixel_is_nan():
    cmb3d.load()
    N, L, r = 16, 2.2, 1.0
    pix = cap_pixels(8, 0.5)[:5].copy()
    pix[2, 1] = np.nan
    knodes, pnodes = spectrum(N, L)
    out = torch.zeros(5, dtype=torch.float32, device="cuda")
    cmb3d.cmb3d_realize_sample_noalloc(N, L, r, torch.tensor(pix, dtype=torch.float64, device="cuda"), 5,
                                       cmb3d.CMB3D_TRILINEAR,
                                       torch.tensor(amp_table(N, L, knodes, pnodes), device="cuda"), 3, out)
    got = out.cpu().numpy()
    assert np.isnan(got[2]) and np.all(np.isfinite(np.delete(got, 2)))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    cmb3d.load()
    one = torch.zeros(3, dtype=torch.float64, device="cuda")
    amp = torch.zeros(3 * 64 ** 2 + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_realize_sample_noalloc(2 * cmb3d.CMB3D_NOALLOC_MAX_N, 2.2, 1.0, one, 1, 1, amp, 0, out)
    assert e.value.status == cmb3d.CMB3D_EUNSUPPORTED
    assert "CMB3D_NOALLOC_MAX_N" in cmb3d.load().cmb3d_error_detail().decode()
