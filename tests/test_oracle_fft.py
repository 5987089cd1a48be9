"""Pins of the oracle's draw and inverse transform (Sec. II.D.1 of the paper).

Each check is fixed by mathematics, not by the oracle itself: a brute-force
triple-sum DFT on 8^3 boxes, Parseval's theorem, exact Hermitian symmetry and a
real field, the closed form of a single Fourier mode, and the first and second
moments of the drawn modes (E|T_k|^2 = P_box, Sec. II.D.1).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import cmb3d_oracle as orc


def _pbox_flat(N, value=1.0):
    p = np.full(3 * (N // 2) ** 2 + 1, value)
    return p


def _pbox_ramp(N):
    q = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    return 1.0 / (1.0 + q) ** 1.5


def brute_force_field(half):
    """T(j) = sum over all N^3 modes of T_m exp(+2 pi i m.j/N), written as an
    explicit sum over modes with the conjugate half filled by T_{-m} = conj(T_m)."""
    N = half.shape[0]
    j = np.arange(N)
    out = np.zeros((N, N, N), dtype=np.complex128)
    ez = np.exp(2j * np.pi * np.outer(np.arange(N), j) / N)   # [m, j]
    for mz in range(N):
        for my in range(N):
            for mx in range(N):
                if mx <= N // 2:
                    c = half[mz, my, mx]
                else:
                    c = np.conj(half[(-mz) % N, (-my) % N, N - mx])
                if c == 0:
                    continue
                out += c * (ez[mz][:, None, None] * ez[my][None, :, None] * ez[mx][None, None, :])
    return out


@pytest.mark.parametrize("seed", [0, 5])
def test_inverse_transform_equals_brute_force_dft_8cubed(seed):
    N = 8
    half = orc.draw_half_spectrum(N, _pbox_ramp(N), seed)
    ref = brute_force_field(half)
    rms = np.sqrt(np.mean(ref.real ** 2))
    assert np.max(np.abs(ref.imag)) <= 1e-12 * rms
    got = orc.inverse_transform(half)
    assert np.max(np.abs(got - ref.real)) <= 1e-12 * rms
    full, imax = orc.inverse_transform_full(half)
    assert imax <= 1e-12 * rms
    assert np.max(np.abs(full - ref.real)) <= 1e-12 * rms


@pytest.mark.parametrize("N", [16, 32])
def test_real_and_full_transforms_agree_and_field_is_real(N):
    half = orc.draw_half_spectrum(N, _pbox_ramp(N), 11)
    a = orc.inverse_transform(half)
    b, imax = orc.inverse_transform_full(half)
    rms = np.sqrt(np.mean(a ** 2))
    assert imax <= 1e-12 * rms
    assert np.max(np.abs(a - b)) <= 1e-12 * rms


@pytest.mark.parametrize("N", [8, 32])
def test_parseval(N):
    half = orc.draw_half_spectrum(N, _pbox_ramp(N), 3)
    field = orc.inverse_transform(half)
    full = orc.full_spectrum(half)
    lhs = np.sum(field ** 2)
    rhs = N ** 3 * np.sum(np.abs(full) ** 2)
    assert abs(lhs - rhs) <= 1e-11 * rhs


def test_single_mode_closed_form():
    N = 16
    m = np.array([3, -5, 2])        # (m_x, m_y, m_z) with m_x > 0
    a = 0.7 - 0.4j
    half = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
    half[m[2] % N, m[1] % N, m[0]] = a
    field = orc.inverse_transform(half)
    jz, jy, jx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    phase = 2 * np.pi * (m[0] * jx + m[1] * jy + m[2] * jz) / N
    ref = 2 * abs(a) * np.cos(phase + np.angle(a))
    assert np.max(np.abs(field - ref)) < 1e-13


@pytest.mark.parametrize("N", [8, 16, 64])
def test_draw_hermitian_planes_exact(N):
    half = orc.draw_half_spectrum(N, _pbox_ramp(N), 9)
    neg = (-np.arange(N)) % N
    for mx in (0, N // 2):
        plane = half[:, :, mx]
        partner = plane[neg[:, None], neg[None, :]]
        np.testing.assert_array_equal(plane, np.conj(partner))
        for mz in (0, N // 2):
            for my in (0, N // 2):
                assert plane[mz, my].imag == 0.0
    assert half[0, 0, 0] == 0.0


def test_draw_mode_statistics():
    """Drawn modes are complex normal with E|T|^2 = P_box: real and imaginary
    parts of the interior modes are N(0, P/2) and uncorrelated, self-conjugate
    modes are N(0, P)."""
    N = 64
    pb = _pbox_ramp(N)
    half = orc.draw_half_spectrum(N, pb, 1234)
    q = orc.half_spectrum_q(N)
    inner = half[:, :, 1:N // 2] / np.sqrt(pb[q[:, :, 1:N // 2]] / 2.0)
    re, im = inner.real.ravel(), inner.imag.ravel()
    for g in (re, im):
        assert stats.kstest(g[:200000], "norm").pvalue > 1e-3
        assert abs(np.var(g) - 1.0) < 6 * np.sqrt(2.0 / g.size)
    assert abs(np.mean(re * im)) < 6 / np.sqrt(re.size)


def test_draw_reproducible_and_seed_dependent():
    N = 16
    a = orc.draw_half_spectrum(N, _pbox_ramp(N), 77)
    b = orc.draw_half_spectrum(N, _pbox_ramp(N), 77)
    c = orc.draw_half_spectrum(N, _pbox_ramp(N), 78)
    np.testing.assert_array_equal(a, b)
    assert np.mean(a != c) > 0.99


def test_box_variance_matches_ensemble():
    """The xi(0) check of Sec. III.A: the mean-square of box maps equals the sum
    of P_box over all non-DC modes."""
    N = 16
    pb = _pbox_ramp(N)
    want = orc.box_variance(N, pb)
    ms = np.array([np.mean(orc.realize_field(N, pb, s) ** 2) for s in range(300)])
    z = (ms.mean() - want) / (ms.std(ddof=1) / np.sqrt(ms.size))
    assert abs(z) < 5


def test_box_covariance_matches_ensemble():
    """E[T(x) T(x+d)] = sum_m P_box(q_m) cos(2 pi m.d / N) at a few lags."""
    N = 16
    pb = _pbox_ramp(N)
    cov = orc.box_covariance(N, pb)
    assert abs(cov[0, 0, 0] - orc.box_variance(N, pb)) < 1e-12 * cov[0, 0, 0]
    lags = [(0, 0, 1), (0, 2, 1), (3, 0, 0), (1, 1, 1)]
    prods = {lag: [] for lag in lags}
    for s in range(300):
        f = orc.realize_field(N, pb, 1000 + s)
        for lag in lags:
            prods[lag].append(np.mean(f * np.roll(f, shift=(-lag[0], -lag[1], -lag[2]), axis=(0, 1, 2))))
    for lag in lags:
        v = np.array(prods[lag])
        z = (v.mean() - cov[lag]) / (v.std(ddof=1) / np.sqrt(v.size))
        assert abs(z) < 5, (lag, v.mean(), cov[lag])
