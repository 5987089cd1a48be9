"""Pins of the oracle's pixel mapping and interpolation (Sec. II.D.1 sampling).

Fixed by mathematics: interpolation returns grid values at grid points,
trilinear interpolation reproduces linear functions and the Keys kernel
(a = -1/2) reproduces quadratics, the weights sum to one, and the periodic
wrap equals sampling a periodically extended field.
"""
import numpy as np
import pytest

from oracle import cmb3d_oracle as orc
from synth import fibonacci_sphere, cap_pixels, cap_count


def test_weights_partition_of_unity():
    t = np.linspace(0, 1, 101)[:-1]
    for w in (orc.trilinear_weights(t), orc.keys_weights(t)):
        assert np.max(np.abs(sum(w) - 1.0)) < 1e-15


@pytest.mark.parametrize("interp", [1, 3])
def test_grid_points_return_grid_values(interp):
    N = 12
    rng = np.random.default_rng(0)
    field = rng.standard_normal((N, N, N))
    b = rng.integers(0, N, size=(200, 3))
    t = np.zeros((200, 3))
    got = orc.sample(field, b, t, interp)
    np.testing.assert_array_equal(got, field[b[:, 2], b[:, 1], b[:, 0]])


def _poly_field(N, coef, degree):
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    f = coef[0] + coef[1] * x + coef[2] * y + coef[3] * z
    if degree == 2:
        f = f + coef[4] * x * x + coef[5] * y * z + coef[6] * z * z + coef[7] * x * y
    return f.astype(np.float64), lambda p: (coef[0] + coef[1] * p[:, 0] + coef[2] * p[:, 1] + coef[3] * p[:, 2]
                                            + (0 if degree == 1 else
                                               coef[4] * p[:, 0] ** 2 + coef[5] * p[:, 1] * p[:, 2]
                                               + coef[6] * p[:, 2] ** 2 + coef[7] * p[:, 0] * p[:, 1]))


@pytest.mark.parametrize("interp,degree", [(1, 1), (3, 1), (3, 2)])
def test_polynomial_reproduction(interp, degree):
    N = 20
    rng = np.random.default_rng(1)
    coef = rng.standard_normal(8)
    field, exact = _poly_field(N, coef, degree)
    # interior points only, so no tap wraps around
    p = rng.uniform(2, N - 3, size=(500, 3))
    b = np.floor(p).astype(np.int64)
    t = p - b
    got = orc.sample(field, b, t, interp)
    assert np.max(np.abs(got - exact(p))) < 1e-11


def test_trilinear_does_not_reproduce_quadratics():
    # guards the test above against a vacuous pass
    N = 20
    field, exact = _poly_field(N, np.array([0, 0, 0, 0, 1.0, 0, 0, 0]), 2)
    p = np.array([[5.5, 6.0, 7.0]])
    b = np.floor(p).astype(np.int64)
    assert abs(orc.sample(field, b, p - b, 1)[0] - exact(p)[0]) > 0.2


@pytest.mark.parametrize("interp", [1, 3])
def test_periodic_wrap(interp):
    N = 10
    rng = np.random.default_rng(2)
    field = rng.standard_normal((N, N, N))
    big = np.tile(field, (3, 3, 3))            # periodic extension, offset N
    p = rng.uniform(0, N, size=(300, 3))
    p[:5, 0] = N - 0.3                          # cells at the upper edge
    p[5:10, 2] = 0.2                            # and at the lower edge
    b = np.floor(p).astype(np.int64)
    t = p - b
    got = orc.sample(field, b, t, interp)
    ref = orc.sample(big, b + N, t, interp)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_pixel_cells_geometry():
    N, L, r = 64, 2.2, 1.0
    pix = fibonacci_sphere(3000)
    b, t = orc.pixel_cells(pix, N, L, r)
    assert b.dtype == np.int64 and np.all((b >= 0) & (b < N))
    assert np.all((t >= 0) & (t < 1))
    pos = (b + t) * (L / N) - 0.5 * L
    np.testing.assert_allclose(pos, r * pix, atol=1e-12)
    # the pole maps onto the box's central column
    b0, t0 = orc.pixel_cells(np.array([[0.0, 0.0, 1.0]]), N, L, r)
    assert b0[0, 0] == N // 2 and t0[0, 0] == 0.0
    assert b0[0, 2] == int(np.floor((r + L / 2) / (L / N)))


def test_fibonacci_cap_is_equal_area():
    npix = 12 * 32 ** 2
    pix = fibonacci_sphere(npix)
    np.testing.assert_allclose(np.linalg.norm(pix, axis=1), 1.0, atol=1e-15)
    # equal area: z is uniform on (-1, 1)
    hist, _ = np.histogram(pix[:, 2], bins=16, range=(-1, 1))
    assert hist.min() == hist.max() == npix // 16
    cap = cap_pixels(32, 0.1)
    assert cap.shape[0] == cap_count(npix, 0.1) == 1229
    assert np.all(cap[:, 2] >= 1 - 2 * 0.1)
    assert pix[cap.shape[0], 2] < 1 - 2 * 0.1
