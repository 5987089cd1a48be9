"""Ensemble two-point correlation of sky maps against the paper's Eq. (2.1).

Test helper (no arithmetic of the simulation method): it samples pixel pairs
by angular separation, averages T_i T_j over the pairs of each bin and over
many realizations, and compares the result with

    xi(theta) = sum_l (2l+1) C_l P_l(cos theta) / (4 pi)            (Eq. 2.1)

for the C_l that the box's P(k) projects to, C_l = 16 pi^2 int k^2 P(k)
j_l(kr)^2 dk (the forward relation; its pins live in test_oracle_spectrum).

Conditions under which the periodic box reproduces Eq. (2.1) up to errors far
below the statistical ones, so that a z-test is meaningful:
  * P(0) = 0: the box has no k = 0 mode, so a P with power at k = 0 would
    lower every covariance by P(0) k_f^3;
  * P negligible beyond a few times the peak, far below the box's Nyquist
    wavenumber, so the lattice sum of P_box cos(k.d) equals the aliased
    sum over periodic images of xi_inf (Poisson summation), and so that Keys
    interpolation attenuates the variance by less than 1e-3 (k dp <= 0.4);
  * only chords d with L - d well beyond the correlation length, so every
    periodic image of a pair is uncorrelated with it.
"""
from __future__ import annotations

import numpy as np

from oracle import cmb3d_oracle as orc

# bin 0 holds the pixels themselves (theta = 0); the others are (lo, hi] degrees
THETA_EDGES_DEG = np.array([0.0, 4.0, 8.0, 12.0, 16.0, 20.0, 25.0, 30.0, 35.0, 40.0, 45.0, 50.0])


def pair_bins(pix: np.ndarray, rng: np.random.Generator, ncentre: int = 400, per_bin: int = 20000):
    """For bin 0 every pixel with itself; for each (lo, hi] bin up to per_bin
    pairs (centre, other) with the centres drawn at random.  Returns a list of
    (i, j, theta_rad) per bin."""
    npix = pix.shape[0]
    centres = rng.choice(npix, size=min(ncentre, npix), replace=False)
    cosang = np.clip(pix[centres] @ pix.T, -1.0, 1.0)
    theta = np.degrees(np.arccos(cosang))
    allp = np.arange(npix)
    bins = [(allp, allp, np.zeros(npix))]
    for lo, hi in zip(THETA_EDGES_DEG[:-1], THETA_EDGES_DEG[1:]):
        c, j = np.nonzero((theta > lo) & (theta <= hi))
        if c.size > per_bin:
            keep = rng.choice(c.size, size=per_bin, replace=False)
            c, j = c[keep], j[keep]
        bins.append((centres[c], j, np.radians(theta[c, j])))
    return bins


def theory(bins, knodes, pnodes, r: float, lmax: int) -> np.ndarray:
    """Eq. (2.1) with the forward-projected C_l (l = 0 .. lmax), averaged over
    each bin's sampled pairs."""
    ell = np.arange(0, lmax + 1)
    cl = orc.cl_matrix(ell, knodes, r) @ np.asarray(pnodes, dtype=np.float64)
    out = []
    for _, _, th in bins:
        u, inv = np.unique(np.round(th, 12), return_inverse=True)
        out.append(float(np.mean(orc.xi_sph(u, ell, cl)[inv])))
    return np.array(out)


def estimate(maps: np.ndarray, bins):
    """Per bin: mean over realizations of the pair-average of T_i T_j, and its
    standard error from the scatter between realizations."""
    maps = np.asarray(maps, dtype=np.float64)
    est, sem = [], []
    for i, j, _ in bins:
        per_map = np.mean(maps[:, i] * maps[:, j], axis=1)
        est.append(per_map.mean())
        sem.append(per_map.std(ddof=1) / np.sqrt(per_map.size))
    return np.array(est), np.array(sem)


def z_scores(maps, bins, th):
    est, sem = estimate(maps, bins)
    return (est - th) / sem, est
