"""Pins of the oracle's spectrum relations (Sec. II.A and II.C of the paper).

A Gaussian 3-D spectrum P(k) = A exp(-s^2 k^2) has closed forms for every
quantity the path needs:
  * Eq. (2.4): xi_inf(d) = A pi^{3/2} / s^3 exp(-d^2 / (4 s^2));
  * C_l = 16 pi^2 int k^2 P j_l(k r)^2 dk
        = 16 pi^2 A pi / (4 r s^2) exp(-r^2/(2 s^2)) I_{l+1/2}(r^2 / (2 s^2))
    (Weber's second exponential integral with j_l = sqrt(pi/2x) J_{l+1/2});
  * Eq. (2.1) with those C_l must equal xi_inf at the chord of Eq. (2.3).
Eq. (2.11) for the cubic box is pinned on a spectrum that is linear in k.
"""
import math

import numpy as np
import pytest
from scipy.special import ive

from oracle import cmb3d_oracle as orc

A, S, R = 3.0, 0.05, 1.0


def gaussian_nodes(nk=8001, kmax=200.0):
    k = np.linspace(0.0, kmax, nk)
    return k, A * np.exp(-(S * k) ** 2)


def cl_closed(ell):
    x = R * R / (2 * S * S)
    return 16 * np.pi ** 2 * A * np.pi / (4 * R * S * S) * ive(np.asarray(ell) + 0.5, x)


def xi_closed(d):
    return A * np.pi ** 1.5 / S ** 3 * np.exp(-np.asarray(d) ** 2 / (4 * S * S))


def test_xi_inf_closed_form():
    k, p = gaussian_nodes()
    d = np.array([0.0, 0.01, 0.05, 0.1, 0.2])
    np.testing.assert_allclose(orc.xi_inf(d, k, p), xi_closed(d), rtol=1e-5)


def test_cl_matrix_closed_form():
    k, p = gaussian_nodes()
    ell = np.arange(2, 60)
    A_ = orc.cl_matrix(ell, k, R)
    np.testing.assert_allclose(A_ @ p, cl_closed(ell), rtol=1e-5)


def test_xi_sph_equals_xi_inf_at_chord():
    """Eq. (2.1) evaluated with the C_l of a 3-D spectrum equals Eq. (2.4) at the
    chord (2.3): the relation the method relies on."""
    ell = np.arange(0, 400)
    cl = cl_closed(ell)
    theta = np.array([0.0, 0.02, 0.05, 0.1, 0.2])
    lhs = orc.xi_sph(theta, ell, cl)
    rhs = xi_closed(orc.chord(theta) * R)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * rhs[0])


def test_chord():
    assert orc.chord(np.pi) == pytest.approx(2.0)
    assert orc.chord(np.pi / 3) == pytest.approx(1.0)


def test_p_box_linear_spectrum():
    N, L = 16, 2.2
    kf = 2 * np.pi / L
    knodes = np.array([0.5, 10.0, 60.0])
    pnodes = 2.0 + 0.25 * knodes              # linear in k between the nodes
    pb = orc.p_box_of_q(N, L, knodes, pnodes)
    q = np.arange(pb.size)
    k = kf * np.sqrt(q)
    want = np.where(k < 0.5, 2.0 + 0.25 * 0.5, np.where(k > 60.0, 0.0, 2.0 + 0.25 * k)) * kf ** 3
    np.testing.assert_allclose(pb, want, rtol=1e-14)
    assert pb.size == 3 * (N // 2) ** 2 + 1


def test_box_variance_approximates_xi0():
    """Sec. III.A: the box variance sum_k P_box approximates xi_inf(0) = 4 pi
    int k^2 P dk when the box resolves the spectrum (L large, dk small)."""
    N, L = 64, 30.0
    s = 0.6
    k = np.linspace(0, 40, 4001)
    p = np.exp(-(s * k) ** 2)
    pb = orc.p_box_of_q(N, L, k, p)
    var = orc.box_variance(N, pb)
    xi0 = np.pi ** 1.5 / s ** 3
    assert abs(var - xi0) < 1e-3 * xi0


def test_invert_cl_recovers_forward_projection():
    """NNLS inversion of closed-form C_l: forward-projected C_l match to 1e-3."""
    ell = np.arange(2, 41)
    cl = cl_closed(ell)
    knodes, pnodes, err = orc.invert_cl(ell, cl, N=64, L=2.2, r=R, nk=128)
    assert np.all(pnodes >= 0)
    assert err < 1e-3
    fwd = orc.cl_matrix(ell, knodes, R) @ pnodes
    np.testing.assert_allclose(fwd, cl, rtol=1e-3)


def test_invert_cl_family_small_box():
    from synth import cl_family
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    knodes, pnodes, err = orc.invert_cl(ell, cl, N=64, L=2.2, r=1.0, nk=256)
    assert knodes[-1] == pytest.approx(math.sqrt(3) * math.pi * 64 / 2.2)
    assert np.all(pnodes >= 0) and err < 1e-2
