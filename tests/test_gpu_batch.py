"""The batched form: many boxes with their own pixel sets in one persistent
launch replayed from a CUDA graph.

Each map of a batch must equal, bit for bit, the map the single-plan entry
point makes with the same kernel shapes (the same device code, compiled
without implicit contraction, rounds identically in every kernel), and match
the FP64 oracle; a batch
replays with new seeds; an injected withheld producer makes the bounded waits
give up with CMB3D_ETIMEOUT while the context stays usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import batch_fsky, cap_pixels  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
# kernel shapes the batch kernel uses, as (draw, y, x, fused) schedule variants
BATCH_SHAPE = {256: (0, 0, 0, -1), 512: (2, 1, 1, -1)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def close(a, b, tol=0.0):
    """Bit for bit (tol = 0), or max |a - b| <= tol * rms(b) across kernel shapes."""
    if tol == 0.0:
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))
        return
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert np.max(np.abs(a - b)) <= tol * np.sqrt(np.mean(b ** 2))


def smooth_pk(N, L, nk=96):
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, nk)
    return k, 1e-3 / (1.0 + (k / 12.0) ** 3)


def make_plans(N, fskys, nside, interp=3, L=2.2):
    kn, pk = smooth_pk(N, L)
    plans, pixs = [], []
    for i, f in enumerate(fskys):
        pix = cap_pixels(nside, f) if f > 0 else np.zeros((0, 3))
        p = cmb3d.Plan(N, L, 1.0, pix, interp)
        # spectra may differ between boxes: scale each one
        p.set_pk(kn, pk * (1.0 + 0.1 * i))
        plans.append(p)
        pixs.append(pix)
    return plans, pixs, kn, pk


@pytest.mark.parametrize("N,interp", [(256, 3), (256, 1), (512, 3)])
def test_batch_equals_single_plan_maps(N, interp):
    fskys = [0.05, 0.3, 0.0, 0.12] if N == 256 else [0.1, 0.02]
    plans, pixs, kn, pk = make_plans(N, fskys, 64, interp)
    seeds = [11 + 3 * i for i in range(len(plans))]
    outs = [torch.full((max(p.npix, 1),), float("nan"), device="cuda") for p in plans]
    cmb3d.cmb3d_realize_sample_batch([p.handle for p in plans], seeds,
                                     [o if p.npix else None for o, p in zip(outs, plans)])
    for p, o, s in zip(plans, outs, seeds):
        cmb3d.cmb3d_plan_set_schedule(p.handle, BATCH_SHAPE[N])
        if p.npix == 0:
            continue
        ref = p.realize_sample(s).cpu().numpy()
        close(o[: p.npix].cpu().numpy(), ref)
    # oracle parity for the first box
    p0, pix0 = plans[0], pixs[0]
    ref = orc.realize_sample(N, 2.2, 1.0, pix0, orc.p_box_of_q(N, 2.2, kn, pk), seeds[0], interp)
    got = outs[0][: p0.npix].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2)) <= TOL
    for p in plans:
        p.close()


def test_batch_replays_with_new_seeds_and_uneven_pixels():
    N = 256
    fskys = list(batch_fsky(8))
    plans, pixs, kn, pk = make_plans(N, fskys, 64)
    handles = [p.handle for p in plans]
    outs = [torch.empty(p.npix, device="cuda") for p in plans]
    for rep in range(2):
        seeds = [1000 * rep + b for b in range(len(plans))]
        cmb3d.cmb3d_realize_sample_batch(handles, seeds, outs)
        for b in (0, 5):
            cmb3d.cmb3d_plan_set_schedule(plans[b].handle, BATCH_SHAPE[N])
            ref = plans[b].realize_sample(seeds[b]).cpu().numpy()
            close(outs[b].cpu().numpy(), ref)
    for p in plans:
        p.close()


def test_batch_autotune_and_variants_agree():
    N = 256
    plans, pixs, kn, pk = make_plans(N, [0.2, 0.07, 0.3], 64)
    tuned = cmb3d.Plan(N, 2.2, 1.0, pixs[0], 3, cmb3d.CMB3D_FLAG_AUTOTUNE)
    tuned.set_pk(kn, pk)
    handles = [tuned.handle] + [p.handle for p in plans[1:]]
    outs = [torch.empty(p.shape[0], device="cuda") for p in pixs]
    cmb3d.cmb3d_realize_sample_batch(handles, [5, 6, 7], outs)
    ref = [o.cpu().numpy() for o in outs]
    cmb3d.cmb3d_realize_sample_batch([p.handle for p in plans], [5, 6, 7], outs)
    for o, r in zip(outs, ref):
        close(o.cpu().numpy(), r, 1e-6)        # the tuned plan may pick other radices
    tuned.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_forms_agree(form):
    """Persistent kernel (two or one blocks per SM) and the two-stream graph."""
    N = 256
    plans, pixs, kn, pk = make_plans(N, [0.15, 0.0, 0.33, 0.05], 64, interp=1)
    handles = [p.handle for p in plans]
    outs = [torch.empty(max(p.npix, 1), device="cuda") for p in plans]
    seeds = [21, 22, 23, 24]
    try:
        cmb3d.cmb3d_batch_debug(0, False, form)
        cmb3d.cmb3d_realize_sample_batch(handles, seeds, outs)
        cmb3d.cmb3d_realize_sample_batch(handles, [s + 1 for s in seeds], outs)   # replay, new seeds
    finally:
        cmb3d.cmb3d_batch_debug(0, False, -1)
    for p, o, s in zip(plans, outs, seeds):
        if p.npix:
            cmb3d.cmb3d_plan_set_schedule(p.handle, BATCH_SHAPE[N])
            close(o[: p.npix].cpu().numpy(), p.realize_sample(s + 1).cpu().numpy())
    for p in plans:
        p.close()


@pytest.mark.parametrize("form", [0, 2])
def test_batch_mixes_pruned_and_whole_boxes(form):
    """A batch of a whole-box plan (CMB3D_FLAG_NO_PRUNE) and pruned plans: each
    box runs its own extent (planes, rows, stored draw planes) in one launch
    and every map equals the whole-box map of its plan bit for bit."""
    N = 256
    kn, pk = smooth_pk(N, 2.2)
    pixs = [cap_pixels(64, f) for f in (0.2, 0.07, 0.4)]
    flags = [cmb3d.CMB3D_FLAG_NO_PRUNE, 0, 0]
    plans = [cmb3d.Plan(N, 2.2, 1.0, px, 3, fl) for px, fl in zip(pixs, flags)]
    whole = [cmb3d.Plan(N, 2.2, 1.0, px, 3, cmb3d.CMB3D_FLAG_NO_PRUNE) for px in pixs]
    try:
        for p, q in zip(plans, whole):
            p.set_pk(kn, pk)
            q.set_pk(kn, pk)
        assert cmb3d.cmb3d_plan_prune_info(plans[1].handle)[0] < N      # pruned: fewer planes
        outs = [torch.empty(px.shape[0], device="cuda") for px in pixs]
        seeds = [31, 32, 33]
        cmb3d.cmb3d_batch_debug(0, False, form)
        try:
            cmb3d.cmb3d_realize_sample_batch([p.handle for p in plans], seeds, outs)
        finally:
            cmb3d.cmb3d_batch_debug(0, False, -1)
        for q, o, s in zip(whole, outs, seeds):
            cmb3d.cmb3d_plan_set_schedule(q.handle, BATCH_SHAPE[N])
            close(o.cpu().numpy(), q.realize_sample(s).cpu().numpy())
    finally:
        for p in plans + whole:
            p.close()


def test_batch_bounded_wait_times_out_and_recovers():
    N = 256
    plans, pixs, kn, pk = make_plans(N, [0.05, 0.05], 32)
    handles = [p.handle for p in plans]
    outs = [torch.empty(p.npix, device="cuda") for p in plans]
    try:
        cmb3d.cmb3d_batch_debug(2000, True, 0)   # draw items never report: waits must give up
        with pytest.raises(cmb3d.Cmb3dError) as e:
            cmb3d.cmb3d_realize_sample_batch(handles, [1, 2], outs)
        assert e.value.status == cmb3d.CMB3D_ETIMEOUT
    finally:
        cmb3d.cmb3d_batch_debug(0, False, -1)
    torch.cuda.synchronize()                     # the context is still usable
    cmb3d.cmb3d_realize_sample_batch(handles, [1, 2], outs)
    cmb3d.cmb3d_plan_set_schedule(plans[1].handle, BATCH_SHAPE[N])
    close(outs[1].cpu().numpy(), plans[1].realize_sample(2).cpu().numpy())
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_realize_sample_batch([handles[0], handles[0]], [1, 2], [outs[0], outs[0]])
    for p in plans:
        p.close()
