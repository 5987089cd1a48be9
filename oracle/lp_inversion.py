"""FP64 oracle of the paper's linear-programming inversion (Sec. II.B).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package.
Plain numpy / scipy in float64; library primitives used:
scipy.optimize.linprog (HiGHS) as the LP solver, numpy's Gauss-Legendre
nodes and scipy's Legendre polynomials (through cmb3d_oracle.xi_sph).

The method looks for a flat-space spectrum P_inf >= 0 whose correlation
function xi_inf(r) (Eq. 2.4) equals the sphere's xi_sph(theta) (Eq. 2.1, with
the beam-smoothed C_l of Eq. 2.2) at the chord r = 2 R sin(theta/2) (Eq. 2.3)
for every separation the cap holds.  Discretised in r and k this is a linear
program: minimise c^T x subject to A x >= b and x >= 0, with c_j = sum_i A_ij
(Eq. 2.5), so that the objective is sum_i (A x)_i and an exact solution
A x = b, when one exists, is the minimum.

Readings (where the paper is silent or leaves a choice):
 L1. Separations: r_i = i dr for i = 0 .. floor(r_max / dr), r_max the
     largest chord between two cap points, 2 R sin(theta_max) for
     theta_max <= pi/2 (the chord of the angle 2 theta_max) and 2 R beyond.
     Defaults from the paper: dr = b / 5 and dk = 2 pi / (3 r_max).
 L2. Targets: b_i = xi_sph(theta_i), theta_i = 2 arcsin(r_i / (2 R)), from
     C_l exp(-b^2 l^2) (b = 0: no smoothing).
 L3. Unknowns: x_j = P_inf(k_j) at k_j = j dk for j = 0 .. n - 1,
     n = floor(k_max / dk); P_inf is linear between nodes and zero from
     k_n = n dk on (a last node carrying P = 0), the interpolation the box
     spectrum uses, so the fitted nodes feed cmb3d_set_spectrum unchanged.
 L4. Matrix: A_ij = 4 pi int k phi_j(k) sin(k r_i) / r_i dk (4 pi int k^2
     phi_j dk at r = 0), phi_j the hat function of node j: column j is
     Eq. 2.4 applied to the spectrum that is 1 at node j and 0 at the others.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.cmb3d_oracle import xi_sph


def r_max_of_cap(R: float, theta_max: float) -> float:
    """L1: the largest separation between two points of a cap of polar
    half-angle theta_max (radians) on the sphere of radius R."""
    return 2.0 * R * math.sin(theta_max) if theta_max <= math.pi / 2 else 2.0 * R


def lp_grid(R: float, theta_max: float, beam: float, dr: float, dk: float, kmax: float):
    """L1, L3: separations r_i, their angles theta_i, and the k nodes
    (n unknown nodes plus the zero node k_n).  dr = 0 selects b/5 and
    dk = 0 selects 2 pi / (3 r_max)."""
    rmax = r_max_of_cap(R, theta_max)
    dr = beam / 5.0 if dr == 0.0 else dr
    dk = 2.0 * math.pi / (3.0 * rmax) if dk == 0.0 else dk
    if not (dr > 0.0 and dk > 0.0 and kmax >= dk):
        raise ValueError("need dr > 0 (or a beam), dk > 0 and kmax >= dk")
    m = int(math.floor(rmax / dr)) + 1
    n = int(math.floor(kmax / dk))
    r = dr * np.arange(m, dtype=np.float64)
    theta = 2.0 * np.arcsin(np.minimum(r / (2.0 * R), 1.0))
    knodes = dk * np.arange(n + 1, dtype=np.float64)
    return r, theta, knodes


def lp_targets(theta, ell, cl, beam: float) -> np.ndarray:
    """L2: xi_sph(theta_i) of the beam-smoothed C_l (Eq. 2.1, 2.2)."""
    ell = np.asarray(ell, dtype=np.float64)
    smooth = np.asarray(cl, dtype=np.float64) * np.exp(-(beam * ell) ** 2)
    return xi_sph(theta, ell.astype(np.int64), smooth)


def lp_matrix(r, knodes, nquad: int = 16) -> np.ndarray:
    """L4: A_ij = 4 pi int k phi_j(k) sin(k r_i)/r_i dk over each node interval
    [k_a, k_a+1] by Gauss-Legendre, where the hats of nodes a and a + 1 are
    (k_a+1 - k)/(k_a+1 - k_a) and (k - k_a)/(k_a+1 - k_a); the last node k_n
    carries P = 0 and has no column."""
    xg, wg = np.polynomial.legendre.leggauss(nquad)
    knodes = np.asarray(knodes, dtype=np.float64)
    n = len(knodes) - 1
    r = np.asarray(r, dtype=np.float64)[:, None]
    at0 = r == 0.0
    A = np.zeros((r.shape[0], n))
    for a in range(n):
        ka, kb = knodes[a], knodes[a + 1]
        k = 0.5 * (kb - ka) * xg + 0.5 * (kb + ka)
        w = 0.5 * (kb - ka) * wg
        kern = np.where(at0, k * k, k * np.sin(k * r) / np.where(at0, 1.0, r))
        A[:, a] += 4.0 * np.pi * np.sum(kern * w * (kb - k) / (kb - ka), axis=1)
        if a + 1 < n:
            A[:, a + 1] += 4.0 * np.pi * np.sum(kern * w * (k - ka) / (kb - ka), axis=1)
    return A


def solve_lp(A: np.ndarray, b: np.ndarray):
    """Eq. 2.5: minimise c^T x with c_j = sum_i A_ij subject to A x >= b and
    x >= 0 (HiGHS).  Returns (x, c^T x)."""
    from scipy.optimize import linprog
    c = A.sum(axis=0)
    res = linprog(c, A_ub=-A, b_ub=-b, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"linprog failed: {res.message}")
    return res.x, float(c @ res.x)


def invert_xi_lp(ell, cl, R: float, theta_max: float, beam: float = 0.0, dr: float = 0.0,
                 dk: float = 0.0, kmax: float = 0.0):
    """The whole inversion: returns the k nodes (n + 1), P_inf at the nodes
    (the last one 0), and a dict with r, theta, A, b and the objective."""
    r, theta, knodes = lp_grid(R, theta_max, beam, dr, dk, kmax)
    b = lp_targets(theta, ell, cl, beam)
    A = lp_matrix(r, knodes)
    x, obj = solve_lp(A, b)
    pk = np.append(np.maximum(x, 0.0), 0.0)           # the solver's rounding below 0 (P >= 0 is a bound)
    return knodes, pk, {"r": r, "theta": theta, "A": A, "b": b, "objective": obj}
