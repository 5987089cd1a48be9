"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the simulation method itself: it only
builds the inputs a user would supply -- unit vectors of sky pixels, a target
angular power spectrum C_l, and the named workloads.  Both the FP64 oracle and
the CUDA path receive exactly these arrays.

Pixels.  The paper samples the box at HEALPix pixels, taking the first pixels of
a RING-ordered map as the polar cap (Sec. II.D.1).  HEALPix is not available
here, so an equal-area Fibonacci grid stands in for it: point i of Npix has
z_i = 1 - (2i+1)/Npix and azimuth 2*pi*frac(i*(sqrt(5)-1)/2).  Like RING order,
index order runs from the north pole southwards, so a polar cap of sky fraction
f_sky is the first round(f_sky*Npix) points.

Spectrum.  The target C_l family is
    C_l = A / (l(l+1)) * (1 + 0.5 cos(pi*l/p)) * exp(-(l/d)^2),
an l(l+1)-flat spectrum with an oscillation of period p (standing in for
acoustic peaks) and a Gaussian beam, which is the smoothing of Eq. (2.2) with
b = 1/d.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN_FRACTION = (math.sqrt(5.0) - 1.0) / 2.0


def fibonacci_sphere(npix: int, count: int | None = None) -> np.ndarray:
    """Unit vectors (count x 3, float64) of the first `count` points of an
    equal-area Fibonacci grid of `npix` points, ordered from the north pole."""
    if count is None:
        count = npix
    i = np.arange(count, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / npix
    frac = np.mod(i * GOLDEN_FRACTION, 1.0)
    phi = 2.0 * np.pi * frac
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    out = np.empty((count, 3), dtype=np.float64)
    out[:, 0] = s * np.cos(phi)
    out[:, 1] = s * np.sin(phi)
    out[:, 2] = z
    return out


def cap_count(npix: int, fsky: float) -> int:
    """Number of grid points with z >= 1 - 2 f_sky (a polar cap of area
    fraction f_sky): the first floor(f_sky*npix + 1/2) indices."""
    return int(math.floor(fsky * npix + 0.5))


def cap_pixels(nside: int, fsky: float) -> np.ndarray:
    """Polar-cap pixels of a 12*nside^2-point Fibonacci grid."""
    npix = 12 * nside * nside
    return fibonacci_sphere(npix, cap_count(npix, fsky))


def cl_family(lmax: int, amplitude: float = 1e3, period: float = 22.0,
              damping: float = 100.0, lmin: int = 2) -> tuple[np.ndarray, np.ndarray]:
    """(l, C_l) for l = lmin..lmax of the synthetic spectrum family."""
    ell = np.arange(lmin, lmax + 1, dtype=np.float64)
    cl = (amplitude / (ell * (ell + 1.0)) * (1.0 + 0.5 * np.cos(np.pi * ell / period))
          * np.exp(-(ell / damping) ** 2))
    return ell, cl


def random_cl_family(rng: np.random.Generator, n: int, lmax: int,
                     amp_range=(1e2, 1e4), period_range=(15.0, 30.0),
                     damping_range=(800.0, 2000.0)) -> tuple[np.ndarray, np.ndarray]:
    """n spectra of the family with log-uniform amplitude and uniform period
    and damping, drawn from `rng`.  Returns (ell, cl[n, len(ell)])."""
    amp = np.exp(rng.uniform(math.log(amp_range[0]), math.log(amp_range[1]), n))
    per = rng.uniform(*period_range, n)
    dmp = rng.uniform(*damping_range, n)
    ell = np.arange(2, lmax + 1, dtype=np.float64)
    cl = (amp[:, None] / (ell * (ell + 1.0)) * (1.0 + 0.5 * np.cos(np.pi * ell[None, :] / per[:, None]))
          * np.exp(-(ell[None, :] / dmp[:, None]) ** 2))
    return ell, cl


def batch_fsky(nbox: int, seed: int = 2507, lo: float = 0.05, hi: float = 0.5) -> np.ndarray:
    """Per-box sky fractions of the batched workload, uniform on [lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, nbox)


def cap_layers(theta_max_deg: float, dp: float, r: float = 1.0, interp: int = 3) -> tuple[float, int]:
    """Layers of the 2-D Fourier method that hold a polar cap of half-angle
    theta_max on the sphere of radius r with grid step dp: layer 0 at
    z0 = r cos(theta_max) - 1.5 dp (the cap's lowest pixels sit 1.5 steps up,
    so a tricubic stencil keeps one layer below), and h layers up to the pole
    with the stencil's margin above."""
    z0 = r * math.cos(math.radians(theta_max_deg)) - 1.5 * dp
    top = math.floor((r - z0) / dp)
    return z0, top + (3 if interp == 3 else 2)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: box, spectrum, pixels and interpolation."""
    name: str
    N: int                  # box points per axis
    nside: int              # pixel grid has 12*nside^2 points on the full sphere
    fsky: float             # polar-cap sky fraction sampled
    lmax: int               # C_l given for l = 2..lmax
    damping: float          # d in exp(-(l/d)^2)
    interp: int             # 1 = trilinear, 3 = tricubic
    nkbins: int = 256       # k nodes of the fitted P(k)
    r: float = 1.0          # sphere radius
    L_over_r: float = 2.2   # box side in units of r
    amplitude: float = 1e3
    period: float = 22.0
    batch: int = 1          # boxes per step; > 1: each box has its own cap
    fsky_seed: int = 2507   # seed of the per-box sky fractions (batch > 1)
    learned: bool = False   # P(k) from the learned inversion (trained per run)
    n_train: int = 100000   # training spectra of the learned inversion
    train_seed: int = 4     # seed of the training and held-out spectra
    method: str = "3d"      # "2d": the 2-D Fourier method on the cap's layers
    M: int = 0              # 2-D: z-period in grid steps
    theta_max_deg: float = 0.0   # 2-D: cap half-angle
    dp: float = 0.0         # 2-D: grid step (box side L = N dp)

    @property
    def L(self) -> float:
        return self.N * self.dp if self.method == "2d" else self.L_over_r * self.r

    def layers(self) -> tuple[float, int]:
        """2-D: (z0, h) of the layers that hold the cap."""
        return cap_layers(self.theta_max_deg, self.dp, self.r, self.interp)

    def pixels(self) -> np.ndarray:
        return cap_pixels(self.nside, self.fsky)

    def batch_pixels(self) -> list[np.ndarray]:
        """Per-box pixel sets: caps with f_sky uniform on [0.05, 0.5]."""
        return [cap_pixels(self.nside, float(f)) for f in batch_fsky(self.batch, self.fsky_seed)]

    def cl(self) -> tuple[np.ndarray, np.ndarray]:
        return cl_family(self.lmax, self.amplitude, self.period, self.damping)


WORKLOADS = {
    # 64^3 box, ~1.2k cap pixels, trilinear: the small parity workload.
    "box64_cap0.1_trilinear": Workload("box64_cap0.1_trilinear", N=64, nside=32, fsky=0.1,
                                       lmax=128, damping=100.0, interp=1),
    # 512^3 box, ~5M cap pixels, tricubic: the single-realization production workload.
    "box512_cap0.4_tricubic": Workload("box512_cap0.4_tricubic", N=512, nside=1024, fsky=0.4,
                                       lmax=768, damping=600.0, interp=3),
    # 64 boxes of 256^3 per step, each with its own cap (f_sky ~ U[0.05, 0.5]
    # of a 12*512^2-point grid, ~55M pixels in all), trilinear.
    "batch64_box256_trilinear": Workload("batch64_box256_trilinear", N=256, nside=512, fsky=0.275,
                                         lmax=128, damping=100.0, interp=1, batch=64),
    # 2048^3 box, ~20M cap pixels, tricubic, P(k) on 512 k nodes from the
    # learned inversion of C_l (l = 2..2048) trained on 100k spectra of the
    # family with amplitude in [1e2, 1e4], period in [15, 30], damping in
    # [800, 2000].
    "box2048_cap0.4_learned": Workload("box2048_cap0.4_learned", N=2048, nside=2048, fsky=0.4,
                                       lmax=2048, damping=1000.0, interp=3, nkbins=512, learned=True),
    # 2-D Fourier method: a 20-degree polar cap (f_sky = (1 - cos 20 deg)/2,
    # ~380k pixels of a 12*1024^2-point grid), N = 512 in x and y with step
    # dp = 0.0034 r (the box spans 1.74 r, about twice the cap), z-period
    # M = 64 and the 22 layers that hold the cap with a tricubic margin;
    # the shape of the paper's Table I row (theta_max = 20 deg, N = 512, M = 64).
    "fourier2d_box512_cap20": Workload("fourier2d_box512_cap20", N=512, nside=1024,
                                       fsky=(1.0 - math.cos(math.radians(20.0))) / 2.0, lmax=768, damping=600.0,
                                       interp=3, method="2d", M=64, theta_max_deg=20.0, dp=0.0034),
    # 1024^3 box, ~20M cap pixels, tricubic; 512 k nodes keep the node
    # spacing of the 512^3 workload's 256.
    "box1024_cap0.4_tricubic": Workload("box1024_cap0.4_tricubic", N=1024, nside=2048, fsky=0.4,
                                        lmax=768, damping=600.0, interp=3, nkbins=512),
}
