"""The paper's decisive test (Sec. III.B) applied to the oracle's sky maps.

Maps of the 3-D Fourier method must be draws from a zero-mean Gaussian with a
known pixel covariance Gamma.  Here Gamma is the exact covariance of the
interpolated box field, sum over taps of w_a w_b C(x_a - x_b) with C the lattice
covariance of the box, so no noise has to be added to make it positive
definite.  Whitening each map with the Cholesky factor of Gamma must give
independent standard normals, which a Kolmogorov-Smirnov test checks.  A map
scaled by 1.05 must fail the same test (the test is not vacuous).
"""
import numpy as np
import pytest
from scipy import stats
from scipy.linalg import solve_triangular

from oracle import cmb3d_oracle as orc
from synth import fibonacci_sphere


def _taps(b, t, interp, N):
    offs = (0, 1) if interp == 1 else (-1, 0, 1, 2)
    wf = orc.trilinear_weights if interp == 1 else orc.keys_weights
    wx, wy, wz = wf(t[0]), wf(t[1]), wf(t[2])
    taps = []
    for iz, sz in enumerate(offs):
        for iy, sy in enumerate(offs):
            for ix, sx in enumerate(offs):
                taps.append(((b[0] + sx) % N, (b[1] + sy) % N, (b[2] + sz) % N,
                             wx[ix] * wy[iy] * wz[iz]))
    return taps


def exact_pixel_covariance(N, pb, b, t, interp):
    cov_lat = orc.box_covariance(N, pb)
    taps = [_taps(b[i], t[i], interp, N) for i in range(b.shape[0])]
    n = len(taps)
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            s = 0.0
            for (xa, ya, za, wa) in taps[i]:
                for (xb, yb, zb, wb) in taps[j]:
                    s += wa * wb * cov_lat[(za - zb) % N, (ya - yb) % N, (xa - xb) % N]
            G[i, j] = G[j, i] = s
    return G


@pytest.mark.parametrize("interp", [1, 3])
def test_whitened_maps_are_standard_normal(interp):
    N, L, r = 16, 2.2, 1.0
    q = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    pb = np.exp(-q / 12.0)
    pix = fibonacci_sphere(240, 40)          # a polar cap of 40 well-separated pixels
    b, t = orc.pixel_cells(pix, N, L, r)
    G = exact_pixel_covariance(N, pb, b, t, interp)
    Lc = np.linalg.cholesky(G)
    maps = np.array([orc.realize_sample(N, L, r, pix, pb, s, interp) for s in range(400)])
    x = solve_triangular(Lc, maps.T, lower=True).ravel()
    assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.var(x) - 1.0) < 5 * np.sqrt(2.0 / x.size)
    xbad = solve_triangular(Lc, 1.05 * maps.T, lower=True).ravel()
    assert stats.kstest(xbad, "norm").pvalue < 1e-3 or abs(np.var(xbad) - 1) > 5 * np.sqrt(2.0 / x.size)
