"""The oracle's sky maps reproduce the paper's angular correlation, Eq. (2.1).

Over many realizations, the pair average of T_i T_j of the oracle's maps
(draw, inverse FFT and Keys interpolation of a 64^3 box of side 2.2 r) must
match sum_l (2l+1) C_l P_l(cos theta) / 4 pi, with C_l the forward projection
of the box's P(k), at every angular bin to within 5 standard errors.  This ties
the whole map pipeline (the box power of Eq. 2.11, the draw's variance, the
transform, the pixel geometry of Sec. II.D.1) to the angular spectrum through
the chord relation of Eq. (2.3).  A map scaled by 1.05 (a 10 % error in xi)
and maps sampled on a sphere of radius 0.95 r (chords off by 5 %) must fail.

P(k) = k^2 exp(-(k/5)^2) has P(0) = 0 and no power near the 64^3 box's
Nyquist wavenumber (91); its correlation length (about 0.4 r) is far below
the 1.2 r that separates a pair with chord <= 0.85 r from its periodic images
(conditions in xi_check).
"""
import numpy as np

from oracle import cmb3d_oracle as orc
from synth import fibonacci_sphere
import xi_check

N, L, R = 64, 2.2, 1.0
NMAPS = 300
ZMAX = 5.0


def _setup():
    pix = fibonacci_sphere(12 * 32 * 32)
    knodes = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, 256)
    pnodes = knodes ** 2 * np.exp(-(knodes / 5.0) ** 2)
    bins = xi_check.pair_bins(pix, np.random.default_rng(2507))
    return pix, knodes, pnodes, bins


def _maps(pix, knodes, pnodes, radius):
    pbox = orc.p_box_of_q(N, L, knodes, pnodes)
    return np.stack([orc.realize_sample(N, L, radius, pix, pbox, 1000 + s, 3) for s in range(NMAPS)])


def test_oracle_maps_match_eq_2_1():
    pix, knodes, pnodes, bins = _setup()
    th = xi_check.theory(bins, knodes, pnodes, R, lmax=60)
    assert th[0] > 0 and np.min(th) < 0           # the correlation changes sign inside the bins
    maps = _maps(pix, knodes, pnodes, R)
    z, _ = xi_check.z_scores(maps, bins, th)
    assert np.max(np.abs(z)) < ZMAX, z
    zs, _ = xi_check.z_scores(1.05 * maps, bins, th)
    assert np.max(np.abs(zs)) > ZMAX, zs


def test_oracle_maps_on_a_smaller_sphere_fail():
    pix, knodes, pnodes, bins = _setup()
    th = xi_check.theory(bins, knodes, pnodes, R, lmax=60)
    z, _ = xi_check.z_scores(_maps(pix, knodes, pnodes, 0.95 * R), bins, th)
    assert np.max(np.abs(z)) > ZMAX, z
