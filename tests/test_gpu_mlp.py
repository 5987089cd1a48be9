"""The learned inversion's GPU training kernels against the FP64 oracle.

The network's tcgen05 matrix-product kernel (BF16 operands, FP32 accumulation)
must equal the exact sums of the same BF16-rounded operands element by element,
within the FP32-accumulation bound 2 K 2^-24 sum_k |a_k b_k|.  The loss and
every gradient element must match the oracle's network evaluated with the same
operand rounding (operands="bf16", exact sums); training must lower the loss of
the forward relation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cmb3d_oracle as orc  # noqa: E402
from paper_2507_15703_gb300 import cmb3d  # noqa: E402
from synth import random_cl_family  # noqa: E402

pytestmark = pytest.mark.gpu
GRAD_RTOL, GRAD_ATOL = 2e-3, 2e-4


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


def _bf16(x):
    return orc.bf16_round(x)


@pytest.mark.parametrize("M,N,K,ta,tb,gelu", [(300, 200, 1000, False, False, False), (37, 2047, 512, True, False, False),
                                              (256, 129, 2047, False, True, True), (130, 96, 40, True, True, True)])
def test_gemm_matches_exact_sums_of_bf16_operands(M, N, K, ta, tb, gelu):
    rng = np.random.default_rng(M * 7 + K)
    a = rng.standard_normal((M, K)) * rng.uniform(0.1, 10.0, (M, 1))
    b = rng.standard_normal((N, K)) * rng.uniform(0.1, 10.0, (N, 1))
    bias = rng.standard_normal(N)
    alpha = 0.37
    # strided operands: a transposed operand is stored (K, M) and read with strides (1, M)
    a_dev = torch.tensor(a.T.copy() if ta else a, dtype=torch.float32, device="cuda")
    b_dev = torch.tensor(b.T.copy() if tb else b, dtype=torch.float32, device="cuda")
    bias_dev = torch.tensor(bias, dtype=torch.float32, device="cuda")
    out = torch.empty((M, N), dtype=torch.float32, device="cuda")
    cmb3d.cmb3d_mlp_gemm(M, N, K, a_dev, (1, M) if ta else (K, 1), b_dev, (1, N) if tb else (K, 1), out, (N, 1),
                         alpha, bias_dev, gelu)
    got = out.cpu().numpy().astype(np.float64)
    a32, b32, bias32 = (np.asarray(v, np.float32).astype(np.float64) for v in (a, b, bias))
    ab, bb = _bf16(a32), _bf16(b32)
    acc = ab @ bb.T
    bound_acc = 2.0 * K * 2.0 ** -24 * (np.abs(ab) @ np.abs(bb).T) + 1e-30
    z = np.float32(alpha) * acc + bias32
    bound = abs(float(np.float32(alpha))) * bound_acc + 4.0 * 2.0 ** -24 * (np.abs(z) + np.abs(bias32))
    if gelu:
        ref = orc.gelu(z)
        bound = 1.2 * bound + 4.0 * 2.0 ** -24 * np.abs(ref) + 1e-12
    else:
        ref = z
    err = np.abs(got - ref)
    assert np.all(err <= bound), (np.max(err / bound), np.unravel_index(np.argmax(err / bound), err.shape))


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
        # the oracle sees the FP32-rounded inputs the GPU sees, and rounds the
        # operands of every matrix product to BF16 as the GPU does
        ref_loss, ref_g = orc.mlp_loss_grad(params, n_in, width, depth, n_out, A.astype(np.float32),
                                            mu.astype(np.float32), sd.astype(np.float32),
                                            logc.astype(np.float32), operands="bf16")
        assert abs(loss - ref_loss) <= 1e-4 * ref_loss
        gg = g.cpu().numpy().astype(np.float64)
        dims, offs, _ = orc.mlp_shapes(n_in, width, depth, n_out)
        for l, (d, (o, ob)) in enumerate(zip(dims, offs)):
            for lo, hi in ((o, o + d[0] * d[1]), (ob, ob + d[0])):
                a, b = gg[lo:hi], ref_g[lo:hi]
                # FP32 accumulation over up to 2047 terms plus the rare operand
                # whose FP32 and FP64 values round to different BF16 neighbours
                tol = GRAD_RTOL * np.abs(b) + GRAD_ATOL * np.max(np.abs(b))
                bad = np.abs(a - b) > tol
                assert not np.any(bad), (l, lo, int(bad.sum()), float(np.max(np.abs(a - b) / (np.abs(b) + 1e-30))))
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
