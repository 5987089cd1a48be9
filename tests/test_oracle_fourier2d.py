"""Pins of the 2-D Fourier method oracle (paper Sec. II.D.2).

The method is a linear map from independent standard normals to the layers,
so its exact covariance is A A^T with A built by feeding unit vectors through
the oracle.  It must equal the covariance of the periodic box the method
stands for:
* with z-period M = N, the 3-D oracle's box covariance restricted to the h
  layers (an independent code path: the inverse 3-D FFT of P_box per mode);
* with M != N, a brute-force triple sum of P_box cos(k . d) written here.
A dropped factor (the 1/sqrt 2 of the complex normals, the volume factor of
Eq. 2.11), a wrong sign, a transposed factor or a broken Hermitian rule
changes A A^T and fails.
"""
import numpy as np
import pytest

from oracle import cmb3d_oracle as orc
from oracle import fourier2d as f2

L = 2.2


def smooth(N, nk=64):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 6.0) ** 3)


def covariance_by_linear_map(N, M, h, kn, pn):
    table = f2.sqrt_gamma_table(N, M, h, L, kn, pn)
    shape = (N, N // 2 + 1, h, 2)
    cols = []
    for j in range(int(np.prod(shape))):
        G = np.zeros(int(np.prod(shape)))
        G[j] = 1.0
        cols.append(f2.field_from_hybrid(f2.hybrid_from_normals(N, h, table, G.reshape(shape))).ravel())
    A = np.stack(cols, axis=1)
    return A @ A.T


@pytest.mark.parametrize("h", [8, 3])
def test_exact_covariance_equals_cubic_box_covariance_on_the_layers(h):
    N = M = 8
    kn, pn = smooth(N)
    cov = covariance_by_linear_map(N, M, h, kn, pn)
    c3 = orc.box_covariance(N, orc.p_box_of_q(N, L, kn, pn))          # [dz, dy, dx]
    z, y, x = np.meshgrid(np.arange(h), np.arange(N), np.arange(N), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    ref = c3[(z[None, :] - z[:, None]) % N, (y[None, :] - y[:, None]) % N, (x[None, :] - x[:, None]) % N]
    assert np.max(np.abs(cov - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_exact_covariance_with_a_shorter_z_period_equals_the_triple_sum():
    N, M, h = 8, 4, 3
    kn, pn = smooth(N)
    cov = covariance_by_linear_map(N, M, h, kn, pn)
    dp = L / N
    fx = orc.signed_frequency(np.arange(N), N)
    fz = orc.signed_frequency(np.arange(M), M)
    # brute force: every mode of the N x N x M box, P_box of Eq. 2.11 with M != N
    d = np.zeros((h, N, N))
    for mz in fz:
        for my in fx:
            for mx in fx:
                if mx == my == mz == 0:
                    continue
                k = np.sqrt((2 * np.pi * mx / (N * dp)) ** 2 + (2 * np.pi * my / (N * dp)) ** 2
                            + (2 * np.pi * mz / (M * dp)) ** 2)
                pb = orc.p_inf_at(np.array([k]), kn, pn)[0] * (2 * np.pi / dp) ** 3 / (M * N * N)
                dz, dy, dx = np.meshgrid(np.arange(h), np.arange(N), np.arange(N), indexing="ij")
                d += pb * np.cos(2 * np.pi * (mx * dx / N + my * dy / N + mz * dz / M))
    z, y, x = np.meshgrid(np.arange(h), np.arange(N), np.arange(N), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    ref = d[np.abs(z[None, :] - z[:, None]), (y[None, :] - y[:, None]) % N, (x[None, :] - x[:, None]) % N]
    assert np.max(np.abs(cov - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gamma_is_the_cosine_sum_of_the_column():
    N, M, h = 16, 32, 6
    kn, pn = smooth(N)
    col = f2.pbox_column(N, M, L, kn, pn, 5)
    g = f2.gamma_matrix(col, h)
    d = np.arange(h)
    xi = np.array([np.sum(col * np.cos(2 * np.pi * np.arange(M) * dd / M)) for dd in d])
    assert np.allclose(g, xi[np.abs(d[:, None] - d[None, :])], rtol=1e-13, atol=0)
    assert f2.pbox_column(N, M, L, kn, pn, 0)[0] == 0.0                     # DC removed


def test_symmetric_square_root():
    N, M, h = 16, 16, 7
    kn, pn = smooth(N)
    g = f2.gamma_matrix(f2.pbox_column(N, M, L, kn, pn, 2), h)
    s = f2.sqrt_psd(g)
    assert np.allclose(s, s.T, atol=0)
    assert np.max(np.abs(s @ s - g)) <= 1e-12 * np.max(np.abs(g))
    assert np.min(np.linalg.eigvalsh(s)) >= -1e-12 * np.max(np.abs(s))   # the PSD root


def test_hermitian_rules_and_real_layers():
    N, M, h = 16, 16, 4
    kn, pn = smooth(N)
    table = f2.sqrt_gamma_table(N, M, h, L, kn, pn)
    hyb = f2.hybrid_from_normals(N, h, table, f2.normals_2d(N, h, 3))
    for mx in (0, N // 2):
        for my in range(N):
            assert np.array_equal(hyb[:, my, mx], np.conj(hyb[:, (-my) % N, mx]))
        for my in (0, N // 2):
            assert np.all(hyb[:, my, mx].imag == 0)
    # the full complex inverse transform of the Hermitian completion is real
    full = np.zeros((h, N, N), dtype=np.complex128)
    full[:, :, : N // 2 + 1] = hyb
    for mx in range(N // 2 + 1, N):
        full[:, :, mx] = np.conj(hyb[:, (-np.arange(N)) % N, N - mx])
    layers = np.fft.ifft2(full, axes=(1, 2), norm="forward")
    assert np.max(np.abs(layers.imag)) <= 1e-12 * np.max(np.abs(layers.real))
    assert np.allclose(layers.real, f2.field_from_hybrid(hyb), rtol=0, atol=1e-12 * np.max(np.abs(layers.real)))


def test_normals_use_their_own_philox_counters():
    N, h, seed = 8, 5, 77
    G = f2.normals_2d(N, h, seed)
    k0, k1 = orc.seed_key(seed)
    for (my, mx, i) in [(0, 0, 0), (3, 2, 1), (7, 4, 4), (5, 1, 3)]:
        w = orc.philox4x32_10(mx, my, i // 2, 1, k0, k1)
        wa, wb = (w[0], w[1]) if i % 2 == 0 else (w[2], w[3])
        g1, g2 = orc.box_muller(orc.uniform_from_word(wa), orc.uniform_from_word(wb))
        assert G[my, mx, i, 0] == g1 and G[my, mx, i, 1] == g2


def test_sampling_in_the_layers():
    N, h, z0 = 16, 6, 0.3
    rng = np.random.default_rng(1)
    field = rng.standard_normal((h, N, N))
    dp = L / N
    # points exactly on grid nodes return the node values
    nodes = np.array([[3, 5, 2], [15, 0, 3], [0, 9, 1]])
    pts = np.stack([nodes[:, 0] * dp - L / 2, nodes[:, 1] * dp - L / 2, nodes[:, 2] * dp + z0], axis=1)
    b, t = f2.pixel_cells_2d(pts, N, L, 1.0, z0)
    got = f2.sample_2d(field, b, np.round(t, 12), 3)
    assert np.allclose(got, field[nodes[:, 2], nodes[:, 1], nodes[:, 0]], atol=1e-12)
    with pytest.raises(ValueError):
        f2.sample_2d(field, np.array([[1, 1, 0]]), np.zeros((1, 3)), 3)        # z - 1 < 0


def test_self_conjugate_and_regular_modes_use_the_stated_normals():
    """R5/R6 conventions (a covariance cannot tell g1 from g2): self-conjugate
    modes take S g1, regular modes S (g1 + i g2)/sqrt 2, partners the conjugate."""
    N, M, h = 8, 8, 4
    kn, pn = smooth(N)
    table = f2.sqrt_gamma_table(N, M, h, L, kn, pn)
    G = f2.normals_2d(N, h, 11)
    hyb = f2.hybrid_from_normals(N, h, table, G)
    fy = orc.signed_frequency(np.arange(N), N)
    for mx, my in [(0, 0), (N // 2, 0), (0, N // 2), (N // 2, N // 2)]:
        S = table[mx * mx + int(fy[my]) ** 2]
        assert np.array_equal(hyb[:, my, mx], (S @ G[my, mx, :, 0]).astype(np.complex128))
    S = table[2 * 2 + 3 * 3]
    assert np.array_equal(hyb[:, 3, 2], S @ ((G[3, 2, :, 0] + 1j * G[3, 2, :, 1]) / np.sqrt(2.0)))
    S = table[0 + 3 * 3]
    assert np.array_equal(hyb[:, N - 3, 0], np.conj(S @ ((G[3, 0, :, 0] + 1j * G[3, 0, :, 1]) / np.sqrt(2.0))))
