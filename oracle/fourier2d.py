"""FP64 oracle of the 2-D Fourier method (paper Sec. II.D.2).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package.
Plain numpy, float64; library primitives used: numpy FFTs and
numpy.linalg.eigh.  The random numbers come from the oracle's own Philox
(cmb3d_oracle), so both methods share one generator definition.

The method simulates the box in a hybrid space: Fourier space in x and y,
real space in z, and only on the h layers that hold the cap.  For each
(m_x, m_y) the h values T^(m_x, m_y, z_j) are correlated Gaussians whose
covariance is the z-transform of the box power spectrum along m_z; a 2-D
inverse FFT per layer then gives the real box, which is sampled at the
pixels.

Readings (where the paper is silent or leaves a choice):
 R1. Geometry: N x N points in x and y with spacing dp = L/N, periodic; the
     z direction has period M dp (the N x N x M box of Sec. II.C, never
     built) and only the layers z_j = z0 + j dp, j < h, are simulated.
     Pixel n maps to u_x = (r n_x + L/2)/dp, u_y likewise, and
     u_z = (r n_z - z0)/dp; every interpolation stencil must lie inside the
     h layers (no wrap in z).
 R2. Box spectrum (Eq. 2.11 with M != N): P_box(m) = P_inf(|k|) (2 pi/dp)^3
     / (M N^2) at k = (2 pi m_x/(N dp), 2 pi m_y/(N dp), 2 pi m_z/(M dp)),
     signed frequencies, and P_box(0) = 0 (zero-mean box, as in the 3-D
     method).
 R3. Correlations along z: xi_{m_x m_y}(d dp) = sum_{m_z} P_box(m) e^{+2 pi i
     m_z d / M} (the FFT of the P_box column along z) and Gamma_ij =
     xi(|i - j| dp), h x h.
 R4. Factor: the symmetric square root S = P D^{1/2} P^T of Gamma
     (eigenvalues below zero from rounding set to zero).  The paper uses
     P D^{1/2}; the two differ by an orthogonal rotation of the normals, so
     they give the same distribution, and S is unique where P is not
     (eigenvector signs), which makes it a parity target.
 R5. Normals: Philox4x32-10 with key (seed lo, seed hi) and counter
     (m_x, m_y, i // 2, 1) for layer index i < h; words (0, 1) for even i,
     (2, 3) for odd i; Box-Muller (g1, g2); the complex normal is
     c_i = (g1 + i g2)/sqrt 2 (E|c|^2 = 1), so E[T^ T^H] = Gamma.
 R6. Hermitian symmetry of a real box: on m_x in {0, N/2} the mode with the
     smaller m_y of the pair (m_y, -m_y mod N) draws and its partner takes
     the conjugate; the self-conjugate modes (m_y in {0, N/2}) are real,
     T^ = S g1.
 R7. Field: T(x, y, z_j) = sum T^(m_x, m_y, z_j) e^{+2 pi i (m_x x + m_y y)/N}
     over the full (m_x, m_y) plane (unnormalised inverse DFT, the sign of
     the 3-D method).
"""
from __future__ import annotations

import numpy as np

from oracle.cmb3d_oracle import (box_muller, keys_weights, p_inf_at, philox4x32_10, seed_key,
                                 signed_frequency, trilinear_weights, uniform_from_word)


def pbox_column(N: int, M: int, L: float, knodes, pnodes, q_perp: int) -> np.ndarray:
    """R2: P_box(m_x, m_y, m_z) for m_z = 0 .. M-1 at m_x^2 + m_y^2 = q_perp."""
    dp = L / N
    fz = signed_frequency(np.arange(M), M).astype(np.float64)
    k = np.sqrt((2 * np.pi / (N * dp)) ** 2 * q_perp + (2 * np.pi * fz / (M * dp)) ** 2)
    col = p_inf_at(k, knodes, pnodes) * (2 * np.pi / dp) ** 3 / (M * N * N)
    if q_perp == 0:
        col[0] = 0.0
    return col


def gamma_matrix(col: np.ndarray, h: int) -> np.ndarray:
    """R3: the h x h Toeplitz covariance from the P_box column (length M)."""
    xi = np.fft.ifft(col, norm="forward").real        # sum_mz col[mz] e^{+2 pi i mz d / M}
    d = np.abs(np.arange(h)[:, None] - np.arange(h)[None, :])
    return xi[d % col.size]                           # xi is periodic in d with the z-period M


def sqrt_psd(g: np.ndarray) -> np.ndarray:
    """R4: symmetric square root P D^{1/2} P^T of a symmetric PSD matrix."""
    lam, vec = np.linalg.eigh(g)
    return (vec * np.sqrt(np.clip(lam, 0.0, None))) @ vec.T


def sqrt_gamma_table(N: int, M: int, h: int, L: float, knodes, pnodes) -> dict:
    """S for every q_perp = m_x^2 + m_y^2 of the half plane m_x in [0, N/2]."""
    fy = signed_frequency(np.arange(N), N)
    qs = sorted({int(mx * mx + f * f) for mx in range(N // 2 + 1) for f in fy})
    return {q: sqrt_psd(gamma_matrix(pbox_column(N, M, L, knodes, pnodes, q), h)) for q in qs}


def normals_2d(N: int, h: int, seed: int) -> np.ndarray:
    """R5: real normals G[m_y, m_x, i, (g1, g2)] for m_x in [0, N/2], i < h."""
    k0, k1 = seed_key(seed)
    my, mx, ip = np.meshgrid(np.arange(N), np.arange(N // 2 + 1), np.arange((h + 1) // 2), indexing="ij")
    w = philox4x32_10(mx.ravel(), my.ravel(), ip.ravel(), np.ones(mx.size, dtype=np.int64), k0, k1)
    shape = (N, N // 2 + 1, (h + 1) // 2)
    ga = np.stack(box_muller(uniform_from_word(w[0]), uniform_from_word(w[1])), -1).reshape(shape + (2,))
    gb = np.stack(box_muller(uniform_from_word(w[2]), uniform_from_word(w[3])), -1).reshape(shape + (2,))
    out = np.empty((N, N // 2 + 1, 2 * ((h + 1) // 2), 2))
    out[:, :, 0::2] = ga
    out[:, :, 1::2] = gb
    return out[:, :, :h]


def hybrid_from_normals(N: int, h: int, table: dict, G: np.ndarray) -> np.ndarray:
    """R4-R6: T^[z, m_y, m_x] (complex, m_x in [0, N/2]) from the normals G."""
    fy = signed_frequency(np.arange(N), N)
    out = np.zeros((h, N, N // 2 + 1), dtype=np.complex128)
    for mx in range(N // 2 + 1):
        for my in range(N):
            S = table[int(mx * mx + fy[my] ** 2)]
            if 0 < mx < N // 2:
                out[:, my, mx] = S @ ((G[my, mx, :, 0] + 1j * G[my, mx, :, 1]) / np.sqrt(2.0))
                continue
            py = (-my) % N
            if py == my:
                out[:, my, mx] = S @ G[my, mx, :, 0]
            elif my < py:
                out[:, my, mx] = S @ ((G[my, mx, :, 0] + 1j * G[my, mx, :, 1]) / np.sqrt(2.0))
            else:
                out[:, my, mx] = np.conj(S @ ((G[py, mx, :, 0] + 1j * G[py, mx, :, 1]) / np.sqrt(2.0)))
    return out


def field_from_hybrid(hyb: np.ndarray) -> np.ndarray:
    """R7: the real layers T[z, y, x] from the half-plane hybrid spectrum."""
    N = hyb.shape[1]
    return np.fft.irfft2(hyb, s=(N, N), axes=(1, 2), norm="forward")


def realize_field_2d(N: int, M: int, h: int, L: float, knodes, pnodes, seed: int) -> np.ndarray:
    table = sqrt_gamma_table(N, M, h, L, knodes, pnodes)
    return field_from_hybrid(hybrid_from_normals(N, h, table, normals_2d(N, h, seed)))


def pixel_cells_2d(pix: np.ndarray, N: int, L: float, r: float, z0: float):
    """R1: base cells b (n, 3; x, y, z) and fractions t of the pixels."""
    dp = L / N
    u = np.empty((pix.shape[0], 3))
    u[:, 0] = (r * pix[:, 0] + 0.5 * L) / dp
    u[:, 1] = (r * pix[:, 1] + 0.5 * L) / dp
    u[:, 2] = (r * pix[:, 2] - z0) / dp
    b = np.floor(u)
    return b.astype(np.int64), u - b


def sample_2d(field: np.ndarray, b: np.ndarray, t: np.ndarray, interp: int) -> np.ndarray:
    """Interpolation in the layers (periodic in x and y, none in z)."""
    h, N = field.shape[0], field.shape[1]
    offs, wfun = ((0, 1), trilinear_weights) if interp == 1 else ((-1, 0, 1, 2), keys_weights)
    if (b[:, 2] + offs[0]).min() < 0 or (b[:, 2] + offs[-1]).max() >= h:
        raise ValueError("an interpolation stencil leaves the simulated layers")
    wx, wy, wz = wfun(t[:, 0]), wfun(t[:, 1]), wfun(t[:, 2])
    out = np.zeros(b.shape[0])
    for iz, sz in enumerate(offs):
        for iy, sy in enumerate(offs):
            for ix, sx in enumerate(offs):
                out += wz[iz] * wy[iy] * wx[ix] * field[b[:, 2] + sz, (b[:, 1] + sy) % N, (b[:, 0] + sx) % N]
    return out


def realize_sample_2d(N: int, M: int, h: int, L: float, r: float, z0: float, pix: np.ndarray, knodes, pnodes,
                      seed: int, interp: int) -> np.ndarray:
    """One partial-sky map by the 2-D Fourier method."""
    b, t = pixel_cells_2d(pix, N, L, r, z0)
    return sample_2d(realize_field_2d(N, M, h, L, knodes, pnodes, seed), b, t, interp)
