"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: Philox words and index work bit-exact; fields and sky maps within
max|T_gpu - T_oracle| / rms(T_oracle) <= 1e-5 (the FP32-path tolerance);
drawn Fourier coefficients within FP32 rounding of the normal numbers.
Sizes span several tiles and ragged pixel counts; the edge cases are the
smallest box, no pixels, pixels on cell boundaries and a sphere that wraps
around the periodic box.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import cap_pixels, cl_family, fibonacci_sphere, WORKLOADS  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()
    torch.cuda.set_device(0)


def smooth_pk(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / np.sqrt(np.mean(ref ** 2)))


def test_philox_bit_exact():
    rng = np.random.default_rng(3)
    n = 5000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [7, 511, 3, 0]
    for seed in (0, 1, 0xDEADBEEFCAFEF00D, 2 ** 64 - 1):
        cdev = torch.tensor(ctr.astype(np.uint32).view(np.int32), device="cuda")
        out = torch.empty_like(cdev)
        cmb3d.cmb3d_philox4x32_10(cdev, seed, out, n)
        got = out.cpu().numpy().view(np.uint32).astype(np.uint64).reshape(n, 4)
        w = orc.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], *orc.seed_key(seed))
        np.testing.assert_array_equal(got, np.stack(w, axis=1))


def packed_reference(half):
    N = half.shape[0]
    p = half[:, :, : N // 2].copy()
    p[:, :, 0] = half[:, :, 0] + 1j * half[:, :, N // 2]
    return p


@pytest.mark.parametrize("N", [8, 16, 64])
def test_draw_matches_oracle(N):
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pb = orc.p_box_of_q(N, L, kn, pk)
    with cmb3d.Plan(N, L, 1.0, np.zeros((0, 3))) as plan:
        plan.set_pk(kn, pk)
        spec = plan.draw_spectrum(123).cpu().numpy().astype(np.float64)
    got = spec[..., 0] + 1j * spec[..., 1]
    ref = packed_reference(orc.draw_half_spectrum(N, pb, 123))
    scale = np.sqrt(pb[orc.half_spectrum_q(N)[:, :, : N // 2]] / 2.0)
    scale[:, :, 0] = np.sqrt(pb[orc.half_spectrum_q(N)[:, :, 0]] + pb[orc.half_spectrum_q(N)[:, :, N // 2]])
    bad = np.abs(got - ref) > 4e-6 * (np.abs(ref) + scale)
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])
    if N >= 64:
        # no mean error: errors of one sign in every normal add up coherently in
        # the inverse FFT (at the origin of the field); over 127k modes the mean
        # of unbiased errors is ~4e-10, a 2 pi rounded to FP32 would give 3.5e-8
        e = (got - ref)[:, :, 1:] / scale[:, :, 1:]
        assert abs(e.real.mean()) < 3e-9 and abs(e.imag.mean()) < 3e-9, (e.real.mean(), e.imag.mean())
    # DC is zero; the packed DC slot holds (T(0,0,0), T(N/2,0,0)) = (0, real)
    assert spec[0, 0, 0, 0] == 0.0


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256])
def test_field_matches_oracle(N):
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pb = orc.p_box_of_q(N, L, kn, pk)
    with cmb3d.Plan(N, L, 1.0, np.zeros((0, 3))) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_field(N + 5).cpu().numpy()
    ref = orc.realize_field(N, pb, N + 5)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("N", [128, 256, 512, 1024])
def test_fused_yx_pass_matches_three_pass_and_oracle(N):
    """The cluster-fused y+x pass (default shape) gives the maps of the
    separate passes of the same radices bit for bit (same device code, no
    implicit contraction) and matches the oracle."""
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(20000, 4999)
    flags = cmb3d.CMB3D_FLAG_STAGE_TIMING | cmb3d.CMB3D_FLAG_NO_PRUNE     # whole-box passes
    with cmb3d.Plan(N, L, 1.0, pix, 3, flags | cmb3d.CMB3D_FLAG_FUSED_YX) as fused, \
            cmb3d.Plan(N, L, 1.0, pix, 3, flags | cmb3d.CMB3D_FLAG_THREE_PASS) as three:
        fused.set_pk(kn, pk)
        three.set_pk(kn, pk)
        assert cmb3d.cmb3d_plan_schedule(fused.handle) == (0, -1, -1, 0)
        a = fused.realize_sample(3).cpu().numpy()
        b = three.realize_sample(3).cpu().numpy()
        np.testing.assert_array_equal(a, b)
        _, cf = cmb3d.cmb3d_stage_times(fused.handle)
        _, ct = cmb3d.cmb3d_stage_times(three.handle)
        assert list(cf) == [1, 0, 0, 1, 1] and list(ct) == [1, 1, 1, 1, 0]
        if N <= 256:
            fa = fused.realize_field(5).cpu().numpy()
            ref = orc.realize_field(N, orc.p_box_of_q(N, L, kn, pk), 5)
            assert rel_err(fa, ref) <= TOL
    if N <= 512:
        ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 3, 3)
        assert rel_err(a, ref) <= TOL


@pytest.mark.parametrize("N", [256, 512])
def test_dsmem_fused_pass_matches_three_pass_and_oracle(N):
    """Fused variant 2: the y+x passes of one z-plane in the distributed shared
    memory of a cluster of N/32 blocks (four-step y transform).  Its
    arithmetic differs from the separate passes (32 x N/32 instead of radix-16
    stages), so both are compared with the oracle and with each other at the
    FP32 tolerance."""
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(20000, 7001)
    pb = orc.p_box_of_q(N, L, kn, pk)
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_STAGE_TIMING | cmb3d.CMB3D_FLAG_NO_PRUNE) as plan:
        plan.set_pk(kn, pk)
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (0, -1, -1, 2))
        a = plan.realize_sample(11).cpu().numpy()
        _, counts = cmb3d.cmb3d_stage_times(plan.handle)
        assert list(counts) == [1, 0, 0, 1, 1]
        field = plan.realize_field(12).cpu().numpy() if N == 256 else None
        cmb3d.cmb3d_plan_set_schedule(plan.handle, (0, 0, 0, -1))
        b = plan.realize_sample(11).cpu().numpy()
    assert rel_err(a, b.astype(np.float64)) <= TOL
    ref = orc.realize_sample(N, L, 1.0, pix, pb, 11, 3)
    assert rel_err(a, ref) <= TOL
    if field is not None:
        assert rel_err(field, orc.realize_field(N, pb, 12)) <= TOL


@pytest.mark.parametrize("N", [256, 512])
def test_every_kernel_variant_matches_oracle(N):
    """Each radix / tile / thread-count variant the autotuner may pick."""
    L = 2.2
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(20000, 6007)
    ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 17, 3)
    ncol = 3 if N >= 2048 else 4                     # draw / y shapes (radix, columns per tile)
    nrow = 4 if N >= 512 else 3                      # x shapes (radix, threads, resident blocks)
    scheds = [(d, 0, 0, -1) for d in range(ncol)] + [(0, y, 0, -1) for y in range(ncol)] + \
             [(0, 0, x, -1) for x in range(nrow)] + [(0, -1, -1, f) for f in range(3)]
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_NO_PRUNE) as plan:
        plan.set_pk(kn, pk)
        for sc in scheds:
            cmb3d.cmb3d_plan_set_schedule(plan.handle, sc)
            assert cmb3d.cmb3d_plan_schedule(plan.handle) == sc
            got = plan.realize_sample(17).cpu().numpy()
            assert rel_err(got, ref) <= TOL, sc
        with pytest.raises(cmb3d.Cmb3dError):
            cmb3d.cmb3d_plan_set_schedule(plan.handle, (ncol, 0, 0, -1))


def test_autotune_picks_valid_schedule():
    N, L = 256, 2.2
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(20000, 3001)
    with cmb3d.Plan(N, L, 1.0, pix, 3, cmb3d.CMB3D_FLAG_AUTOTUNE) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(2).cpu().numpy()
        d, y, x, f = cmb3d.cmb3d_plan_schedule(plan.handle)
        assert 0 <= d < 4 and ((f >= 0 and y == x == -1) or (f == -1 and 0 <= y < 4 and 0 <= x < 3))
    ref = orc.realize_sample(N, L, 1.0, pix, orc.p_box_of_q(N, L, kn, pk), 2, 3)
    assert rel_err(got, ref) <= TOL


def oracle_pk_for(w):
    ell, cl = w.cl()
    kn, pk, _ = orc.invert_cl(ell, cl, w.N, w.L, w.r, w.nkbins)
    return kn, pk


@pytest.mark.parametrize("interp", [1, 3])
@pytest.mark.parametrize("flags", [0, cmb3d.CMB3D_FLAG_NO_SORT])
def test_small_workload_map_matches_oracle(interp, flags):
    w = WORKLOADS["box64_cap0.1_trilinear"]
    kn, pk = oracle_pk_for(w)
    pix = w.pixels()
    assert pix.shape[0] == 1229
    with cmb3d.Plan(w.N, w.L, w.r, pix, interp, flags) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(0).cpu().numpy()
    ref = orc.realize_sample(w.N, w.L, w.r, pix, orc.p_box_of_q(w.N, w.L, kn, pk), 0, interp)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("interp", [1, 3])
def test_cell_run_gather_equals_one_pixel_gather(interp):
    """A sorted table is gathered in runs of up to 8 pixels of one base cell
    (the cell's stencil loaded once); the unsorted table one pixel per thread.
    Dense pixels (about 31 per cell, so runs are cut at 8, ragged ends) over
    the whole sphere with L = 2r, so stencils wrap in x, y and z: the maps
    must be equal bit for bit."""
    N, L, r = 64, 2.0, 1.0
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(400003)
    flags = cmb3d.CMB3D_FLAG_ALLOW_WRAP
    with cmb3d.Plan(N, L, r, pix, interp, flags) as a, \
            cmb3d.Plan(N, L, r, pix, interp, flags | cmb3d.CMB3D_FLAG_NO_SORT) as b:
        a.set_pk(kn, pk)
        b.set_pk(kn, pk)
        for seed in (5, 6):
            np.testing.assert_array_equal(a.realize_sample(seed).cpu().numpy(), b.realize_sample(seed).cpu().numpy())


@pytest.mark.parametrize("N,npix,interp", [(128, 3001, 3), (256, 70001, 1), (8, 257, 3)])
def test_ragged_maps_match_oracle(N, npix, interp):
    L, r = 2.2, 1.0
    kn, pk = smooth_pk(N, L)
    pix = fibonacci_sphere(4 * npix, npix)
    with cmb3d.Plan(N, L, r, pix, interp) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(99).cpu().numpy()
    ref = orc.realize_sample(N, L, r, pix, orc.p_box_of_q(N, L, kn, pk), 99, interp)
    assert rel_err(got, ref) <= TOL


def test_cell_boundaries_and_grid_nodes():
    """Points exactly on grid planes and nodes (t = 0 or just below 1) and the
    box edges: the base cell must agree with the oracle's to the bit."""
    N, L, r = 32, 2.0, 0.5
    dp = L / N
    rng = np.random.default_rng(5)
    j = rng.integers(0, N, size=(600, 3)).astype(np.float64)
    pts = (j * dp - 0.5 * L) / r
    pts[:200] += rng.choice([0.0, 1e-17, -1e-17, 0.5 * dp / r], size=(200, 3))
    pts[200:210] = (np.array([N - 1, 0, N // 2]) * dp - 0.5 * L) / r
    kn, pk = smooth_pk(N, L)
    for interp in (1, 3):
        with cmb3d.Plan(N, L, r, pts, interp) as plan:
            plan.set_pk(kn, pk)
            got = plan.realize_sample(4).cpu().numpy()
        ref = orc.realize_sample(N, L, r, pts, orc.p_box_of_q(N, L, kn, pk), 4, interp)
        assert rel_err(got, ref) <= TOL


def test_sphere_wrapping_the_box():
    N, L, r = 32, 1.5, 1.0                       # L < 2r: the sphere wraps around
    pix = fibonacci_sphere(4000)
    kn, pk = smooth_pk(N, L)
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.Plan(N, L, r, pix)
    with cmb3d.Plan(N, L, r, pix, 3, cmb3d.CMB3D_FLAG_ALLOW_WRAP) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(8).cpu().numpy()
    ref = orc.realize_sample(N, L, r, pix, orc.p_box_of_q(N, L, kn, pk), 8, 3)
    assert rel_err(got, ref) <= TOL


def test_no_pixels_and_errors():
    kn, pk = smooth_pk(16, 2.2)
    with cmb3d.Plan(16, 2.2, 1.0, np.zeros((0, 3))) as plan:
        with pytest.raises(cmb3d.Cmb3dError) as e:
            plan.realize_sample(0)
        assert e.value.status == cmb3d.CMB3D_ENOSPEC
        plan.set_pk(kn, pk)
        out = plan.realize_sample(0)
        assert out.numel() == 0
        torch.cuda.synchronize()
    with cmb3d.Plan(16, 2.2, 1.0, fibonacci_sphere(10)) as plan:
        plan.set_pk(kn, pk)
        with pytest.raises(cmb3d.Cmb3dError) as e:
            cmb3d.cmb3d_realize_sample(plan.handle, 0, 0)
        assert e.value.status == cmb3d.CMB3D_EINVAL
        with cmb3d.Plan(32, 2.2, 1.0, fibonacci_sphere(10)) as other:
            other.set_pk(kn, pk)
            o1 = torch.empty(10, device="cuda")
            with pytest.raises(cmb3d.Cmb3dError):
                cmb3d.cmb3d_realize_sample_batch([plan.handle, other.handle], [0, 1], [o1, o1])


def test_host_batch_and_timing_paths_agree():
    N, L = 64, 2.2
    kn, pk = smooth_pk(N, L)
    pixA = cap_pixels(32, 0.3)
    pixB = cap_pixels(32, 0.05)
    flags = cmb3d.CMB3D_FLAG_STAGE_TIMING
    with cmb3d.Plan(N, L, 1.0, pixA, 3, flags) as a, cmb3d.Plan(N, L, 1.0, pixB, 3) as b:
        a.set_pk(kn, pk)
        b.set_pk(kn, pk)
        da = a.realize_sample(11).cpu().numpy()
        db = b.realize_sample(12).cpu().numpy()
        host = np.empty(pixA.shape[0], dtype=np.float32)
        cmb3d.cmb3d_realize_sample_to_host(a.handle, 11, host)
        np.testing.assert_array_equal(host, da)
        oa = torch.empty(pixA.shape[0], device="cuda")
        ob = torch.empty(pixB.shape[0], device="cuda")
        cmb3d.cmb3d_realize_sample_batch([a.handle, b.handle], [11, 12], [oa, ob])
        np.testing.assert_array_equal(oa.cpu().numpy(), da)
        np.testing.assert_array_equal(ob.cpu().numpy(), db)
        ms, cnt = cmb3d.cmb3d_stage_times(a.handle)
        assert list(cnt) == [3, 3, 3, 3, 0] and np.all(ms[:4] > 0)
        ms2, cnt2 = cmb3d.cmb3d_stage_times(a.handle)
        assert list(cnt2) == [0, 0, 0, 0, 0]


def test_box_variance_over_seeds():
    """Sec. III.A on the GPU path: the mean square of the box equals the sum of
    P_box over all non-DC modes (z-test over 64 seeds)."""
    N, L = 32, 2.2
    kn, pk = smooth_pk(N, L)
    want = orc.box_variance(N, orc.p_box_of_q(N, L, kn, pk))
    with cmb3d.Plan(N, L, 1.0, np.zeros((0, 3))) as plan:
        plan.set_pk(kn, pk)
        ms = np.array([float(torch.mean(plan.realize_field(s).double() ** 2)) for s in range(64)])
    z = (ms.mean() - want) / (ms.std(ddof=1) / np.sqrt(ms.size))
    assert abs(z) < 5


def test_set_spectrum_from_cl_on_plan():
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    with cmb3d.Plan(64, 2.2, 1.0, np.zeros((0, 3))) as plan:
        err = plan.set_cl(ell, cl, 256)
        kn = orc.knodes_for_box(64, 2.2, 256)
        pk = cmb3d.cmb3d_get_pk(plan.handle, kn)
    fwd = orc.cl_matrix(ell, kn, 1.0) @ pk
    assert err < 1e-3 and np.max(np.abs(fwd - cl) / cl) < 1e-3


@pytest.mark.slow
def test_production_workload_full_size():
    """The 512^3 box with ~5M tricubic cap pixels, every pixel against the
    oracle, in the launch configuration the benchmark times."""
    w = WORKLOADS["box512_cap0.4_tricubic"]
    pix = w.pixels()
    kn, pk = smooth_pk(w.N, w.L, 256)
    with cmb3d.Plan(w.N, w.L, w.r, pix, w.interp) as plan:
        plan.set_pk(kn, pk)
        got = plan.realize_sample(0).cpu().numpy()
    ref = orc.realize_sample(w.N, w.L, w.r, pix, orc.p_box_of_q(w.N, w.L, kn, pk), 0, w.interp)
    assert got.shape[0] == 5033165
    assert rel_err(got, ref) <= TOL
