"""The learned inversion's GPU training kernels against the FP64 oracle.

Gradients of every layer (tcgen05 BF16 GEMMs, FP32 accumulation) must match
the oracle's to BF16 accuracy; training must lower the loss of the forward
relation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import random_cl_family  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cmb3d.load()


def problem(lmax, nk, n, seed):
    ell = np.arange(2, lmax + 1, dtype=np.float64)
    _, cl = random_cl_family(np.random.default_rng(seed), n, lmax, damping_range=(0.4 * lmax, lmax))
    kn = np.linspace(0.0, 1.12 * lmax, nk)
    A = cmb3d.cmb3d_cl_matrix(ell, kn, 1.0)
    logc = np.log(cl)
    return ell, kn, A, logc


@pytest.mark.parametrize("n_in_lmax,width,depth,n_out,batch", [(301, 64, 3, 96, 37), (130, 256, 2, 160, 130)])
def test_gradients_match_oracle(n_in_lmax, width, depth, n_out, batch):
    ell, kn, A, logc = problem(n_in_lmax, n_out, batch, 5)
    n_in = ell.size
    mu, sd = logc.mean(0), logc.std(0) + 1e-3
    out_bias = np.full(n_out, np.log(np.mean(np.exp(logc)) / np.mean(A.sum(1))))
    mlp = cmb3d.cmb3d_mlp_create(n_in, width, depth, n_out, A, mu, sd, out_bias, batch_cap=256, seed=11)
    try:
        x = torch.tensor(logc, dtype=torch.float32, device="cuda")
        _, _, total = orc.mlp_shapes(n_in, width, depth, n_out)
        g = torch.empty(total, dtype=torch.float32, device="cuda")
        loss = cmb3d.cmb3d_mlp_loss_grad(mlp, x, batch, g)
        params = cmb3d.cmb3d_mlp_params(mlp).astype(np.float64)
        # the oracle sees the FP32-rounded inputs the GPU sees
        ref_loss, ref_g = orc.mlp_loss_grad(params, n_in, width, depth, n_out, A.astype(np.float32),
                                            mu.astype(np.float32), sd.astype(np.float32),
                                            logc.astype(np.float32))
        assert abs(loss - ref_loss) <= 2e-2 * ref_loss
        gg = g.cpu().numpy().astype(np.float64)
        dims, offs, _ = orc.mlp_shapes(n_in, width, depth, n_out)
        for l, (d, (o, ob)) in enumerate(zip(dims, offs)):
            for lo, hi in ((o, o + d[0] * d[1]), (ob, ob + d[0])):
                a, b = gg[lo:hi], ref_g[lo:hi]
                rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
                cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
                assert rel < 5e-2 and cos > 0.998, (l, lo, rel, cos)
    finally:
        cmb3d.cmb3d_mlp_destroy(mlp)


def test_training_lowers_the_forward_loss():
    ell, kn, A, logc = problem(400, 128, 3000, 9)
    n_in, n_out = ell.size, kn.size
    mu, sd = logc.mean(0), logc.std(0) + 1e-3
    out_bias = np.full(n_out, np.log(np.mean(np.exp(logc)) / np.mean(A.sum(1))))
    mlp = cmb3d.cmb3d_mlp_create(n_in, 128, 3, n_out, A, mu, sd, out_bias, batch_cap=256, seed=1)
    try:
        x = torch.tensor(logc, dtype=torch.float32, device="cuda")
        l0 = cmb3d.cmb3d_mlp_loss_grad(mlp, x[:256], 256)
        losses = cmb3d.cmb3d_mlp_train(mlp, x, 3000, 15, 200, 2e-3, seed=3)
        l1 = cmb3d.cmb3d_mlp_loss_grad(mlp, x[:256], 256)
        assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
        assert l1 < 0.5 * l0, (l0, l1, losses)
        out = torch.empty((3000, n_out), dtype=torch.float32, device="cuda")
        cmb3d.cmb3d_mlp_predict(mlp, x, 3000, out)
        y = out[:256].cpu().numpy().astype(np.float64)
        pred = np.log(np.exp(y) @ A.T)
        assert abs(np.mean((pred - logc[:256]) ** 2) - l1) < 0.05 * l1 + 1e-6
    finally:
        cmb3d.cmb3d_mlp_destroy(mlp)
