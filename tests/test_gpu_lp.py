"""Maps from the spectrum of the linear-programming inversion (paper Sec. II.B)
through the CUDA path against the oracle fed the same spectrum: the 3-D
method on a 64^3 box and the 2-D method on 22 layers of a 20-degree cap.
The spectrum nodes come from the library's host LP (cmb3d_fit_pk_lp) and go
to both sides unchanged."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from oracle import fourier2d as f2  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_layers, cap_pixels, cl_family  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / np.sqrt(np.mean(ref ** 2)))


def test_lp_spectrum_3d_map_matches_oracle():
    N, L = 64, 2.2
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    theta = math.acos(1 - 2 * 0.1)                                          # the f_sky = 0.1 cap
    kn, pk, _, xi_err = cmb3d.cmb3d_fit_pk_lp(ell, cl, 1.0, theta, 0.0, 1 / 500, 0.0, math.sqrt(3) * math.pi * N / L)
    assert xi_err < 0.1                    # excess of xi_inf over xi_sph (no l = 0, 1 power in the C_l)
    pix = cap_pixels(32, 0.1)
    with cmb3d.Plan(N, L, 1.0, pix, 3) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(5).cpu().numpy()
    ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 5, 3)
    assert rel_err(got, ref) <= TOL


def test_lp_spectrum_2d_map_matches_oracle():
    N, M, theta, dp = 256, 64, 20.0, 0.0068
    L = N * dp
    z0, h = cap_layers(theta, dp)
    ell, cl = cl_family(384, 1e3, 22.0, 300.0)
    kn, pk, _, _ = cmb3d.cmb3d_fit_pk_lp(ell, cl, 1.0, math.radians(theta), 0.0, 1 / 1500, 0.0,
                                         math.sqrt(3) * math.pi / dp)
    pix = cap_pixels(256, (1 - math.cos(math.radians(theta))) / 2)
    with cmb3d.Plan2D(N, M, h, L, 1.0, z0, pix, 3) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(8).cpu().numpy()
    ref = f2.realize_sample_2d(N, M, h, L, 1.0, z0, pix, kn, pk, 8, 3)
    assert rel_err(got, ref) <= TOL
