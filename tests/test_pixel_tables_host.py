"""The plan's host tables without a GPU: the pruned transform's extents (z-planes
of the y pass, (z, y) rows of the x pass, reals the x pass stores in the column
blocks the stencils read) and the gather runs, against the same quantities
derived from the oracle's base cells.  cmb3d_pixel_tables_host runs the code a
plan runs, on the host only."""
import numpy as np
import pytest

from oracle import cmb3d_oracle as orc
from paper_2507_15703_gb300 import cmb3d
from synth import cap_pixels, fibonacci_sphere


def reference_counts(pix, N, L, r, interp, sort=True):
    b, _ = orc.pixel_cells(pix, N, L, r)
    offs = np.array((-1, 0, 1, 2) if interp == 3 else (0, 1))
    z = (b[:, 2][:, None, None, None] + offs[:, None, None]) % N
    y = (b[:, 1][:, None, None, None] + offs[None, :, None]) % N
    x = (b[:, 0][:, None, None, None] + offs[None, None, :]) % N
    row = z * N + y
    rows = np.unique(row)
    planes = np.unique(rows // N)
    blocks = np.unique((row * 32 + x // (N // 32)).ravel())
    cell = (b[:, 2] * N + b[:, 1]) * N + b[:, 0]
    _, per_cell = np.unique(cell, return_counts=True)
    runs = int(np.sum((per_cell + 7) // 8)) if sort else 0
    return len(planes), len(rows), len(blocks) * (N // 32), runs


@pytest.mark.parametrize("N,nside,fsky,interp", [(128, 128, 0.4, 3), (256, 128, 0.1, 1), (256, 256, 0.3, 3),
                                                 (512, 128, 0.05, 3)])
def test_pruned_extents_and_runs_match_the_oracle_cells(N, nside, fsky, interp):
    L, r = 2.2, 1.0
    pix = cap_pixels(nside, fsky)
    got = cmb3d.cmb3d_pixel_tables_host(N, L, r, pix, interp)
    planes, rows, stored, runs = reference_counts(pix, N, L, r, interp)
    assert got == (planes, rows, stored, runs)
    assert rows < N * N and stored < rows * N // 4        # a cap: few rows, and two short windows per row


def test_unsorted_tables_have_no_runs_and_the_same_extents():
    N, L, r = 256, 2.2, 1.0
    pix = cap_pixels(128, 0.2)
    a = cmb3d.cmb3d_pixel_tables_host(N, L, r, pix, 3)
    b = cmb3d.cmb3d_pixel_tables_host(N, L, r, pix, 3, cmb3d.CMB3D_FLAG_NO_SORT)
    assert b[:3] == a[:3] and b[3] == 0 and a[3] > 0


def test_no_pruning_cases():
    L, r = 2.2, 1.0
    pix = cap_pixels(64, 0.2)
    # asked for, below N = 128, and when the stencils reach every row (dense whole sphere, L = 2r)
    assert cmb3d.cmb3d_pixel_tables_host(256, L, r, pix, 3, cmb3d.CMB3D_FLAG_NO_PRUNE)[:3] == (256, 256 ** 2, 256 ** 3)
    assert cmb3d.cmb3d_pixel_tables_host(64, L, r, pix, 3)[:3] == (64, 64 ** 2, 64 ** 3)
    full = fibonacci_sphere(2_000_000)
    got = cmb3d.cmb3d_pixel_tables_host(128, 2.0, 1.0, full, 3, cmb3d.CMB3D_FLAG_ALLOW_WRAP)
    planes, rows, _, _ = reference_counts(full, 128, 2.0, 1.0, 3)
    if rows == 128 * 128:
        assert got[:3] == (128, 128 ** 2, 128 ** 3)
    else:
        assert got[:2] == (planes, rows)


def test_wrapping_stencils_are_counted_modulo_n():
    """L = 2r: stencils of pixels near the box faces wrap in x, y and z."""
    N = 128
    pix = fibonacci_sphere(60000)
    got = cmb3d.cmb3d_pixel_tables_host(N, 2.0, 1.0, pix, 3, cmb3d.CMB3D_FLAG_ALLOW_WRAP)
    planes, rows, stored, runs = reference_counts(pix, N, 2.0, 1.0, 3)
    if rows < N * N:
        assert got == (planes, rows, stored, runs)
    else:
        assert got[:3] == (N, N * N, N ** 3) and got[3] == runs


def test_argument_checks():
    pix = cap_pixels(32, 0.1)
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_pixel_tables_host(100, 2.2, 1.0, pix, 3)            # not a power of two
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_pixel_tables_host(128, 2.0, 1.0, pix, 3)            # L <= 2r without ALLOW_WRAP
    bad = pix.copy()
    bad[0, 0] = np.nan
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_pixel_tables_host(128, 2.2, 1.0, bad, 3)
