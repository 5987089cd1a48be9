"""FP64 CPU oracle for the 3-D Fourier method of simulating partial-sky CMB maps.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  The product
path (the C-ABI library and its Python binding) never imports, links or runs
anything under ``oracle/``, and this module imports nothing from the product.

What is computed (paper: Giner Mascarell & Bunn, "Simulating Partial Sky CMB
Maps with 3D Fast Fourier Transforms"):

* Sec. II.C, Eq. (2.8)-(2.11): the box power per Fourier mode,
  P_box = P_inf(k) (2 pi / dp)^3 / (M N^2); for the cubic N^3 box of side L
  this is P_inf(k) (2 pi / L)^3.
* Sec. II.D.1: every mode of the box gets a complex normal number of mean 0 and
  variance P_box(|k|); an inverse FFT gives the field in the box.
* Sec. II.D.1 (sampling): the field is interpolated and evaluated at the
  pixel positions r * n_hat, with the box centred on the sphere.
* Sec. II.A, Eq. (2.1), (2.3), (2.4): xi_sph(theta) from C_l, the chord
  r = 2 sin(theta/2), and xi_inf(r) from P_inf(k).  From the convention
  xi(x) = int d^3k P(k) e^{i k.x} behind Eq. (2.4) and the plane-wave expansion
  follows C_l = 16 pi^2 int k^2 P(k) j_l(k r)^2 dk, which the spectrum
  inversion solves for P >= 0 (non-negative least squares on a hat basis; the
  paper's own linear program of Sec. II.B is an alternative inversion).

Readings where the paper is silent or ambiguous (each one is listed with its
reason in the design notes of the repository):

1. One real map per transform: the spectrum is drawn on the half spectrum
   m_x in [0, N/2] with exact Hermitian symmetry, so the inverse FFT is real.
   (The paper draws a full complex box and uses Re and Im as two maps; the
   distribution of each map is the same.)
2. "Variance P(k)" of a complex normal means E|T_k|^2 = P_box: real and
   imaginary parts each have variance P_box/2; self-conjugate modes (every
   component 0 or N/2) are real with variance P_box.
3. Inverse transform sign: T(j) = sum_m T_m exp(+2 pi i m.j / N), unnormalised
   (the sign of the Fourier series in Sec. I).
4. The DC mode is zero.
5. P_inf between given k nodes is linear in k, constant below the first node
   and zero above the last.
6. Grid points sit at x_j = j dp, periodic; the sphere centre is the box
   centre, so a pixel maps to u = (r n + L/2) / dp in grid units.
7. Interpolation is trilinear, or tricubic with the Keys cubic-convolution
   kernel (a = -1/2), with periodic wrap.
8. Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
   the 64-bit seed (low word, high word).  Mode (m_x, m_y, m_z) (array indices)
   uses counter (m_x, m_y, m_z mod N/2, 0); m_z < N/2 takes output words (0, 1),
   m_z >= N/2 words (2, 3).  A word w becomes the uniform ((w >> 9) + 1/2) 2^-23,
   which is exact in binary32 as well as binary64, and two uniforms become
   two normals by the Box-Muller transform.  On the Hermitian planes
   m_x in {0, N/2} the mode with the smaller index m_z N + m_y of a conjugate
   pair draws; its partner is the conjugate.
"""
from __future__ import annotations

import math

import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85


# --------------------------------------------------------------------------
# Random numbers (reading 8)
# --------------------------------------------------------------------------

def seed_key(seed: int) -> tuple[int, int]:
    """Philox key words of a 64-bit seed: (low 32 bits, high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds (Salmon et al., SC'11), elementwise.

    Counters are arrays (or scalars) of 32-bit values; the key is two 32-bit
    ints.  Each round multiplies words 0 and 2 by the two Philox multipliers,
    XORs the high halves into words 1 and 3 with the round key, and swaps; the
    key is bumped by the two Weyl constants between rounds.  Returns four
    uint64 arrays holding 32-bit output words.
    """
    x0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    x1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    x2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    x3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    ka, kb = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _PHILOX_M0 * x0
        p1 = _PHILOX_M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(ka), lo1,
                          hi0 ^ x3 ^ np.uint64(kb), lo0)
        ka = (ka + _PHILOX_W0) & 0xFFFFFFFF
        kb = (kb + _PHILOX_W1) & 0xFFFFFFFF
    return x0, x1, x2, x3


def uniform_from_word(w) -> np.ndarray:
    """Uniform in (0, 1) from the top 23 bits of a 32-bit word: ((w>>9)+1/2)/2^23.
    Every value is an odd multiple of 2^-24 below 1, so it is exact in binary32."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(u0, u1):
    """Two independent standard normals from two uniforms in (0, 1)."""
    rad = np.sqrt(-2.0 * np.log(u0))
    ang = 2.0 * np.pi * u1
    return rad * np.cos(ang), rad * np.sin(ang)


def unit_normals_half(N: int, seed: int) -> np.ndarray:
    """g1 + i g2 drawn from each mode's own counter, for every mode of the half
    spectrum, shape (N, N, N/2+1) indexed [m_z, m_y, m_x] (no symmetry yet).
    Counter (m_x, m_y, m_z mod N/2, 0) serves the two modes m_z < N/2 (words
    0, 1) and m_z + N/2 (words 2, 3)."""
    k0, k1 = seed_key(seed)
    h = N // 2
    mz, my, mx = np.meshgrid(np.arange(h, dtype=np.uint64), np.arange(N, dtype=np.uint64),
                             np.arange(h + 1, dtype=np.uint64), indexing="ij")
    w0, w1, w2, w3 = philox4x32_10(mx, my, mz, 0, k0, k1)
    del mz, my, mx
    lo1, lo2 = box_muller(uniform_from_word(w0), uniform_from_word(w1))   # m_z < N/2
    hi1, hi2 = box_muller(uniform_from_word(w2), uniform_from_word(w3))   # m_z >= N/2
    del w0, w1, w2, w3
    g = np.empty((N, N, h + 1), dtype=np.complex128)
    g[:h] = lo1 + 1j * lo2
    g[h:] = hi1 + 1j * hi2
    return g


# --------------------------------------------------------------------------
# Spectrum in the box (Sec. II.C)
# --------------------------------------------------------------------------

def signed_frequency(m, N: int):
    """Array index m in [0, N) -> signed frequency in (-N/2, N/2]."""
    m = np.asarray(m, dtype=np.int64)
    return np.where(m <= N // 2, m, m - N)


def half_spectrum_q(N: int) -> np.ndarray:
    """q = m_x^2 + m_y^2 + m_z^2 (signed frequencies) on the half spectrum."""
    f = signed_frequency(np.arange(N), N)
    fx = np.arange(N // 2 + 1, dtype=np.int64)
    return (f[:, None, None] ** 2 + f[None, :, None] ** 2 + fx[None, None, :] ** 2)


def p_inf_at(k, knodes, pnodes) -> np.ndarray:
    """P_inf(k): linear in k between nodes, constant below the first node and
    zero above the last (reading 5)."""
    k = np.asarray(k, dtype=np.float64)
    knodes = np.asarray(knodes, dtype=np.float64)
    pnodes = np.asarray(pnodes, dtype=np.float64)
    out = np.interp(k, knodes, pnodes)
    return np.where(k > knodes[-1], 0.0, out)


def p_box_of_q(N: int, L: float, knodes, pnodes) -> np.ndarray:
    """P_box(q) for q = 0 .. 3 (N/2)^2, Eq. (2.11) for the cubic box:
    P_box = P_inf(k_f sqrt(q)) k_f^3 with k_f = 2 pi / L = 2 pi / (N dp)."""
    kf = 2.0 * np.pi / L
    q = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    return p_inf_at(kf * np.sqrt(q), knodes, pnodes) * kf ** 3


def draw_half_spectrum(N: int, pbox_q: np.ndarray, seed: int) -> np.ndarray:
    """The drawn Fourier coefficients on the half spectrum, shape (N, N, N/2+1)
    indexed [m_z, m_y, m_x], following Sec. II.D.1 with readings 1, 2, 4, 8."""
    pbox_q = np.asarray(pbox_q, dtype=np.float64)
    g = unit_normals_half(N, seed)
    q = half_spectrum_q(N)
    pq = pbox_q[q]
    spec = np.sqrt(pq / 2.0) * g
    idx = np.arange(N)
    lin = idx[:, None] * N + idx[None, :]                 # m_z N + m_y
    pz, py = (-idx) % N, (-idx) % N
    plin = pz[:, None] * N + py[None, :]                  # partner's index
    for mx in (0, N // 2):
        plane = spec[:, :, mx].copy()
        partner = plane[pz[:, None], py[None, :]]
        out = np.where(lin > plin, np.conj(partner), plane)
        selfc = lin == plin
        out[selfc] = np.sqrt(pq[:, :, mx][selfc]) * g[:, :, mx][selfc].real
        spec[:, :, mx] = out
    spec[0, 0, 0] = 0.0
    return spec


def full_spectrum(half: np.ndarray) -> np.ndarray:
    """Extend a Hermitian half spectrum [m_z, m_y, 0..N/2] to all N^3 modes."""
    N = half.shape[0]
    full = np.empty((N, N, N), dtype=np.complex128)
    full[:, :, : N // 2 + 1] = half
    mx = np.arange(N // 2 + 1, N)
    neg = (-np.arange(N)) % N
    full[:, :, mx] = np.conj(half[neg[:, None, None], neg[None, :, None], (N - mx)[None, None, :]])
    return full


def inverse_transform(half: np.ndarray) -> np.ndarray:
    """Real field T[z, y, x] = sum_m T_m exp(+2 pi i m.j / N) (reading 3) of an
    exactly Hermitian half spectrum, by the library real inverse FFT, unnormalised."""
    N = half.shape[0]
    return np.fft.irfftn(half, s=(N, N, N), axes=(0, 1, 2), norm="forward")


def inverse_transform_full(half: np.ndarray) -> np.ndarray:
    """The same sum over the full Hermitian-extended spectrum with the complex
    inverse FFT; returns (real part, max |imaginary part|)."""
    t = np.fft.ifftn(full_spectrum(half), axes=(0, 1, 2), norm="forward")
    return t.real.copy(), float(np.max(np.abs(t.imag)))


# --------------------------------------------------------------------------
# Sampling on the sphere (Sec. II.D.1, readings 6 and 7)
# --------------------------------------------------------------------------

def pixel_cells(pix: np.ndarray, N: int, L: float, r: float):
    """Grid coordinates of r * n_hat: base cell b = floor(u) mod N (int64) and
    fraction t = u - floor(u) (float64), u = (r n + L/2) / dp, dp = L / N,
    evaluated as IEEE double operations in exactly this order."""
    pix = np.asarray(pix, dtype=np.float64)
    dp = L / N
    half_l = 0.5 * L
    u = (r * pix + half_l) / dp
    fl = np.floor(u)
    return fl.astype(np.int64) % N, u - fl


def trilinear_weights(t):
    """Linear interpolation weights for taps 0, 1."""
    t = np.asarray(t, dtype=np.float64)
    return [1.0 - t, t]


def keys_weights(t):
    """Keys cubic-convolution weights (a = -1/2) for taps -1, 0, 1, 2."""
    t = np.asarray(t, dtype=np.float64)
    t2, t3 = t * t, t * t * t
    return [(-t3 + 2.0 * t2 - t) / 2.0,
            (3.0 * t3 - 5.0 * t2 + 2.0) / 2.0,
            (-3.0 * t3 + 4.0 * t2 + t) / 2.0,
            (t3 - t2) / 2.0]


def sample(field: np.ndarray, b: np.ndarray, t: np.ndarray, interp: int) -> np.ndarray:
    """Interpolated field values at grid coordinates b + t with periodic wrap;
    field is indexed [z, y, x], b and t are (n, 3) in (x, y, z) order."""
    N = field.shape[0]
    if interp == 1:
        offs, wfun = (0, 1), trilinear_weights
    elif interp == 3:
        offs, wfun = (-1, 0, 1, 2), keys_weights
    else:
        raise ValueError("interp must be 1 (trilinear) or 3 (tricubic)")
    wx, wy, wz = wfun(t[:, 0]), wfun(t[:, 1]), wfun(t[:, 2])
    out = np.zeros(b.shape[0], dtype=np.float64)
    for iz, sz in enumerate(offs):
        zz = (b[:, 2] + sz) % N
        for iy, sy in enumerate(offs):
            yy = (b[:, 1] + sy) % N
            wyz = wz[iz] * wy[iy]
            for ix, sx in enumerate(offs):
                xx = (b[:, 0] + sx) % N
                out += wyz * wx[ix] * field[zz, yy, xx]
    return out


def realize_field(N: int, pbox_q: np.ndarray, seed: int) -> np.ndarray:
    """Draw and inverse-transform one box realization (float64 [z, y, x])."""
    return inverse_transform(draw_half_spectrum(N, pbox_q, seed))


def realize_sample(N: int, L: float, r: float, pix: np.ndarray, pbox_q: np.ndarray,
                   seed: int, interp: int) -> np.ndarray:
    """One partial-sky map: the realization sampled at the pixels (float64)."""
    field = realize_field(N, pbox_q, seed)
    b, t = pixel_cells(pix, N, L, r)
    return sample(field, b, t, interp)


# --------------------------------------------------------------------------
# Exact second moments of the box (used by the statistical tests)
# --------------------------------------------------------------------------

def box_variance(N: int, pbox_q: np.ndarray) -> float:
    """Var T(x) = sum over all N^3 modes except DC of E|T_m|^2 = P_box(q_m)."""
    f = signed_frequency(np.arange(N), N) ** 2
    q = f[:, None, None] + f[None, :, None] + f[None, None, :]
    tot = float(np.sum(np.asarray(pbox_q)[q]))
    return tot - float(pbox_q[0])


def box_covariance(N: int, pbox_q: np.ndarray) -> np.ndarray:
    """E[T(x) T(x + d)] for every lattice offset d (float64 [dz, dy, dx]):
    the inverse transform of the per-mode power with the DC mode removed."""
    f = signed_frequency(np.arange(N), N) ** 2
    q = f[:, None, None] + f[None, :, None] + f[None, None, :]
    pw = np.asarray(pbox_q, dtype=np.float64)[q]
    pw[0, 0, 0] = 0.0
    return np.fft.ifftn(pw, norm="forward").real


# --------------------------------------------------------------------------
# Angular spectrum <-> 3-D spectrum (Sec. II.A)
# --------------------------------------------------------------------------

def xi_sph(theta, ell, cl) -> np.ndarray:
    """Eq. (2.1): xi(theta) = sum_l (2l+1) C_l P_l(cos theta) / (4 pi)."""
    from scipy.special import eval_legendre
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    x = np.cos(theta)
    ell = np.asarray(ell, dtype=np.int64)
    cl = np.asarray(cl, dtype=np.float64)
    out = np.zeros_like(x)
    for l, c in zip(ell, cl):
        out += (2 * l + 1) * c * eval_legendre(int(l), x)
    return out / (4.0 * np.pi)


def chord(theta):
    """Eq. (2.3): separation of two unit-sphere points an angle theta apart."""
    return 2.0 * np.sin(np.asarray(theta, dtype=np.float64) / 2.0)


def xi_inf(rr, knodes, pnodes, nquad: int = 16) -> np.ndarray:
    """Eq. (2.4): xi(r) = 4 pi int k P(k) sin(kr)/r dk (r > 0), 4 pi int k^2 P dk
    at r = 0, with P linear between nodes (Gauss-Legendre per node interval)."""
    rr = np.atleast_1d(np.asarray(rr, dtype=np.float64))
    xg, wg = np.polynomial.legendre.leggauss(nquad)
    knodes = np.asarray(knodes, dtype=np.float64)
    a, b = knodes[:-1], knodes[1:]
    k = 0.5 * (b - a)[:, None] * xg[None, :] + 0.5 * (b + a)[:, None]
    w = 0.5 * (b - a)[:, None] * wg[None, :]
    p = p_inf_at(k, knodes, pnodes)
    out = np.empty_like(rr)
    for i, r in enumerate(rr):
        kern = k * k if r == 0.0 else k * np.sin(k * r) / r
        out[i] = 4.0 * np.pi * np.sum(w * p * kern)
    return out


def knodes_for_box(N: int, L: float, nk: int) -> np.ndarray:
    """nk uniform k nodes on [0, sqrt(3) pi N / L], the largest |k| of the box."""
    return np.linspace(0.0, math.sqrt(3.0) * math.pi * N / L, nk)


def cl_matrix(ell, knodes, r: float, nquad: int = 16) -> np.ndarray:
    """A[l, j] = 16 pi^2 int k^2 hat_j(k) j_l(k r)^2 dk for the piecewise-linear
    hat basis on the nodes, so that C_l = sum_j A[l, j] P(k_j)."""
    from scipy.special import spherical_jn
    ell = np.asarray(ell, dtype=np.int64)
    knodes = np.asarray(knodes, dtype=np.float64)
    nk = knodes.size
    xg, wg = np.polynomial.legendre.leggauss(nquad)
    A = np.zeros((ell.size, nk))
    for i in range(nk - 1):
        a, b = knodes[i], knodes[i + 1]
        k = 0.5 * (b - a) * xg + 0.5 * (b + a)
        w = 0.5 * (b - a) * wg
        s = (k - a) / (b - a)                   # rising hat of node i+1
        jl2 = spherical_jn(ell[:, None], k[None, :] * r) ** 2
        base = 16.0 * np.pi ** 2 * jl2 * (w * k * k)[None, :]
        A[:, i] += base @ (1.0 - s)
        A[:, i + 1] += base @ s
    return A


def invert_cl(ell, cl, N: int, L: float, r: float, nk: int):
    """P_inf >= 0 on nk k nodes whose forward-projected C_l best match the
    target in relative least squares (scipy NNLS).  Returns (knodes, pnodes,
    max relative C_l error)."""
    from scipy.optimize import nnls
    knodes = knodes_for_box(N, L, nk)
    A = cl_matrix(ell, knodes, r)
    cl = np.asarray(cl, dtype=np.float64)
    Aw = A / cl[:, None]
    x, _ = nnls(Aw, np.ones_like(cl), maxiter=50 * nk)
    err = float(np.max(np.abs(A @ x - cl) / cl))
    return knodes, x, err


# --------------------------------------------------------------------------
# The learned inversion's network, in FP64 (the plain definition of its
# forward pass, loss and gradients; reference for the GPU training kernels)
# --------------------------------------------------------------------------

def mlp_shapes(n_in: int, width: int, depth: int, n_out: int):
    """[(out, in), ...] per layer and the flat offsets of each W and bias."""
    dims, offs, off = [], [], 0
    for l in range(depth + 1):
        di = n_in if l == 0 else width
        do = n_out if l == depth else width
        dims.append((do, di))
        offs.append((off, off + do * di))
        off += do * di + do
    return dims, offs, off


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def bf16_round(x) -> np.ndarray:
    """Each value taken as binary32 and rounded to the nearest bfloat16 (8-bit
    significand, ties to even), returned in float64: the operand precision of
    the network's matrix products (BF16 operands, FP32 accumulation)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_loss_grad(params, n_in, width, depth, n_out, A, mu, sd, logc, operands=None):
    """Loss mean((log(A exp(y)) - log C)^2) of the network with the given flat
    parameters on spectra logc (n x n_in), and its gradient (flat), by the
    chain rule written out layer by layer.

    operands="bf16": both operands of every matrix product (the layers, the
    forward relation and their transposes in the backward pass) are first
    rounded to bfloat16 and the products summed exactly, the definition of the
    mixed-precision network (BF16 operands, FP32 accumulation; the rounding is
    passed through unchanged by the chain rule).  The forward relation is then
    taken shifted by each row's largest y, log(A exp(y)) = ymax + log(A
    exp(y - ymax)), so the rounded operand is exp(y - ymax) <= 1; without
    rounding the shift changes nothing and is not made."""
    rnd = bf16_round if operands == "bf16" else (lambda v: v)
    if operands not in (None, "bf16"):
        raise ValueError("operands must be None or 'bf16'")
    p = np.asarray(params, dtype=np.float64)
    dims, offs, total = mlp_shapes(n_in, width, depth, n_out)
    Ws = [p[o:o + d[0] * d[1]].reshape(d) for d, (o, _) in zip(dims, offs)]
    bs = [p[ob:ob + d[0]] for d, (_, ob) in zip(dims, offs)]
    logc = np.asarray(logc, dtype=np.float64)
    A = np.asarray(A, np.float64)
    x = (logc - np.asarray(mu, np.float64)) / np.asarray(sd, np.float64)
    zs, acts = [], [x]
    for l in range(depth):
        z = rnd(acts[-1]) @ rnd(Ws[l]).T + bs[l]
        zs.append(z)
        acts.append(gelu(z))
    y = rnd(acts[-1]) @ rnd(Ws[depth]).T + bs[depth]
    ymax = y.max(axis=1, keepdims=True) if operands == "bf16" else 0.0
    E = np.exp(y - ymax)
    P = rnd(E) @ rnd(A).T
    d = np.log(P) + ymax - logc
    cnt = d.size
    loss = float(np.sum(d * d) / cnt)
    dP = 2.0 * d / cnt / P
    dY = (rnd(dP) @ rnd(A)) * E
    g = np.zeros(total)
    dcur = dY
    for l in range(depth, -1, -1):
        o, ob = offs[l]
        g[o:o + dims[l][0] * dims[l][1]] = (rnd(dcur).T @ rnd(acts[l])).ravel()
        g[ob:ob + dims[l][0]] = dcur.sum(axis=0)
        if l > 0:
            dcur = (rnd(dcur) @ rnd(Ws[l])) * gelu_grad(zs[l - 1])
    return loss, g
