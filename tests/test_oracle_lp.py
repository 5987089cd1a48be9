"""Pins of the linear-programming inversion oracle (paper Sec. II.B).

* The matrix: each column is Eq. 2.4 of a hat spectrum, checked against
  scipy's adaptive quadrature of the same integral and against the oracle's
  xi_inf (interpolating a unit node vector, a different code path); applied
  to a sampled Gaussian P it reproduces the closed form of xi_inf.
* The LP: on a tiny instance the optimum equals the best basic feasible
  solution found by enumerating every basis; when b = A x_true for some
  x_true >= 0 the optimum is an exact solution with objective sum(b), the
  property Eq. 2.5 is chosen for.
* End to end: C_l of a Gaussian P (closed form) are exactly realisable, so
  the fitted P must reproduce xi_sph at the chord both on the constraint
  grid and between its points.
A wrong 4 pi, a k instead of k^2 at r = 0, a sign in the constraints, the
objective not summing A's columns, or a transposed hat fails one of these.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import ive

from oracle import cmb3d_oracle as orc
from oracle import lp_inversion as lp

A0, S, R = 3.0, 0.05, 1.0


def gaussian_cl(lmax=400):
    ell = np.arange(0, lmax + 1)
    x = R * R / (2 * S * S)
    return ell, 16 * np.pi ** 2 * A0 * np.pi / (4 * R * S * S) * ive(ell + 0.5, x)


def xi_closed(d):
    return A0 * np.pi ** 1.5 / S ** 3 * np.exp(-np.asarray(d) ** 2 / (4 * S * S))


def test_grid_follows_the_paper_defaults():
    theta = math.radians(25.0)
    r, th, kn = lp.lp_grid(1.0, theta, beam=0.01, dr=0.0, dk=0.0, kmax=60.0)
    rmax = 2 * math.sin(theta)
    assert r[1] == pytest.approx(0.002) and r[-1] <= rmax < r[-1] + 0.002
    assert kn[1] == pytest.approx(2 * math.pi / (3 * rmax)) and kn[-2] < 60.0 <= kn[-1] + kn[1]
    np.testing.assert_allclose(orc.chord(th), r, rtol=1e-14, atol=1e-16)
    assert lp.r_max_of_cap(1.0, math.radians(120.0)) == 2.0                  # the whole diameter


def test_matrix_columns_are_eq_2_4_of_hat_spectra():
    r = np.array([0.0, 0.013, 0.2, 0.77])
    kn = np.linspace(0.0, 40.0, 11)
    A = lp.lp_matrix(r, kn)
    for j in (0, 3, 9):
        hat = lambda k: np.interp(k, kn, np.eye(len(kn))[j])                # noqa: E731
        for i, ri in enumerate(r):
            f = (lambda k: k * k * hat(k)) if ri == 0 else (lambda k: k * np.sin(k * ri) / ri * hat(k))
            ref = 4 * np.pi * quad(f, 0.0, kn[-1], points=kn[1:-1], limit=200, epsabs=0, epsrel=1e-12)[0]
            assert A[i, j] == pytest.approx(ref, rel=1e-11, abs=1e-11 * np.max(np.abs(A[:, j])))
        unit = np.eye(len(kn))[j]
        np.testing.assert_allclose(A[:, j], orc.xi_inf(r, kn, unit), rtol=1e-12, atol=1e-12 * np.max(np.abs(A[:, j])))


def test_matrix_on_a_gaussian_spectrum_gives_the_closed_form():
    kn = np.linspace(0.0, 200.0, 4001)
    d = np.array([0.0, 0.01, 0.05, 0.1, 0.2])
    A = lp.lp_matrix(d, kn)
    np.testing.assert_allclose(A @ (A0 * np.exp(-(S * kn[:-1]) ** 2)), xi_closed(d), rtol=1e-5)


def test_tiny_lp_equals_the_best_vertex():
    rng = np.random.default_rng(3)
    A = rng.uniform(0.2, 1.0, (3, 3))
    b = rng.uniform(0.5, 1.0, 3)
    x, obj = lp.solve_lp(A, b)
    c = A.sum(axis=0)
    # standard form [A, -I] [x; s] = b, x, s >= 0: every basis of 3 of the 6 columns
    M = np.hstack([A, -np.eye(3)])
    best = np.inf
    for cols in itertools.combinations(range(6), 3):
        B = M[:, cols]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        xb = np.linalg.solve(B, b)
        if np.all(xb >= -1e-12):
            full = np.zeros(6)
            full[list(cols)] = xb
            best = min(best, c @ full[:3])
    assert obj == pytest.approx(best, rel=1e-10)
    assert np.all(A @ x >= b - 1e-9) and np.all(x >= -1e-12)


def test_lp_reaches_an_exact_solution_when_one_exists():
    rng = np.random.default_rng(4)
    r = np.linspace(0.0, 0.6, 40)
    kn = np.linspace(0.0, 60.0, 21)
    A = lp.lp_matrix(r, kn)
    x_true = rng.uniform(0.0, 1.0, 20) * (rng.uniform(size=20) < 0.5)
    b = A @ x_true
    x, obj = lp.solve_lp(A, b)
    assert obj == pytest.approx(b.sum(), rel=1e-9)
    assert np.max(np.abs(A @ x - b)) <= 1e-8 * np.max(np.abs(b))


def test_gaussian_cl_are_matched_on_and_between_the_grid():
    ell, cl = gaussian_cl()
    kn, pk, info = lp.invert_xi_lp(ell, cl, R, math.radians(30.0), beam=0.0, dr=0.01, kmax=150.0)
    assert np.all(pk >= 0) and pk[-1] == 0.0
    np.testing.assert_allclose(info["b"], xi_closed(info["r"]), rtol=0, atol=1e-13 * xi_closed(0.0))
    assert info["objective"] == pytest.approx(info["b"].sum(), rel=1e-9)
    xi0 = info["b"][0]
    assert np.max(np.abs(orc.xi_inf(info["r"], kn, pk) - info["b"])) <= 1e-9 * xi0
    rm = info["r"][:-1] + 0.005
    assert np.max(np.abs(orc.xi_inf(rm, kn, pk) - orc.xi_sph(2 * np.arcsin(rm / 2), ell, cl))) <= 1e-6 * xi0


def test_beam_smooths_the_targets():
    ell, cl = gaussian_cl(200)
    r, th, _ = lp.lp_grid(R, math.radians(10.0), beam=0.02, dr=0.0, dk=0.0, kmax=50.0)
    b = lp.lp_targets(th, ell, cl, 0.02)
    # the smoothed C_l equal the Gaussian C_l of the same sum over l with weights exp(-b^2 l^2)
    ref = orc.xi_sph(th, ell, cl * np.exp(-(0.02 * ell) ** 2))
    np.testing.assert_allclose(b, ref, rtol=1e-13)
    assert b[0] < orc.xi_sph(np.array([0.0]), ell, cl)[0]
