"""Pin of the oracle's learned-inversion network: its analytic gradient equals
central finite differences of its loss in FP64 (a dropped term, a wrong sign
or a transposed factor in any layer would fail), and the loss is the mean
squared log error of the forward relation."""
import numpy as np
import pytest

from oracle import cmb3d_oracle as orc


def tiny_problem(seed=0, n=5, n_in=7, width=6, depth=2, n_out=4):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.1, 1.0, size=(n_in, n_out))
    logc = rng.normal(0.0, 0.5, size=(n, n_in))
    mu, sd = rng.normal(size=n_in) * 0.1, rng.uniform(0.5, 2.0, size=n_in)
    _, _, total = orc.mlp_shapes(n_in, width, depth, n_out)
    params = rng.normal(0.0, 0.4, size=total)
    return params, (n_in, width, depth, n_out, A, mu, sd, logc)


def test_mlp_gradient_equals_finite_differences():
    params, args = tiny_problem()
    loss, g = orc.mlp_loss_grad(params, *args)
    h = 1e-6
    num = np.zeros_like(g)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = h
        num[i] = (orc.mlp_loss_grad(params + e, *args)[0] - orc.mlp_loss_grad(params - e, *args)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-9)


def test_mlp_loss_definition_without_hidden_layers():
    # depth 0: y = W x + b, loss = mean (log(A exp y) - log C)^2 written out directly
    rng = np.random.default_rng(3)
    n_in, n_out = 5, 3
    A = rng.uniform(0.2, 1.0, size=(n_in, n_out))
    logc = rng.normal(size=(4, n_in))
    W, b = rng.normal(size=(n_out, n_in)), rng.normal(size=n_out)
    params = np.concatenate([W.ravel(), b])
    loss, _ = orc.mlp_loss_grad(params, n_in, 1, 0, n_out, A, np.zeros(n_in), np.ones(n_in), logc)
    want = 0.0
    for r in range(4):
        y = W @ logc[r] + b
        pred = np.log(A @ np.exp(y))
        want += np.sum((pred - logc[r]) ** 2)
    assert abs(loss - want / logc.size) < 1e-12


def test_gelu_values():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    from scipy.stats import norm
    np.testing.assert_allclose(orc.gelu(x), x * norm.cdf(x), rtol=1e-14)
    np.testing.assert_allclose(orc.gelu_grad(x), norm.cdf(x) + x * norm.pdf(x), rtol=1e-13)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.uniform(-30, 30, 5000),
                        1.0 + np.arange(-600, 600) * 2.0 ** -16])           # ties and near-ties around 1
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(orc.bf16_round(x), ref)


def test_bf16_operand_network_matches_torch_autograd():
    """With operands="bf16" the loss and gradient equal an independent
    autograd evaluation of the same network whose every matrix product takes
    BF16-rounded operands (the rounding passed through unchanged)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    n_in, width, depth, n_out, n = 9, 7, 2, 5, 6
    dims, offs, total = orc.mlp_shapes(n_in, width, depth, n_out)
    params = rng.standard_normal(total) * 0.5
    A = rng.uniform(0.1, 1.0, (n_in, n_out))
    mu, sd = rng.standard_normal(n_in) * 0.1, rng.uniform(0.5, 2.0, n_in)
    logc = rng.standard_normal((n, n_in))
    loss, g = orc.mlp_loss_grad(params, n_in, width, depth, n_out, A, mu, sd, logc, operands="bf16")

    def bf(t):   # binary32, then bfloat16
        return t.float().to(torch.bfloat16).double()

    class BfMatmul(torch.autograd.Function):
        """a @ b.T with both operands rounded; the backward products round
        theirs too (the incoming gradient and the saved operand)."""
        @staticmethod
        def forward(ctx, a, b):
            ctx.save_for_backward(a, b)
            return bf(a) @ bf(b).T

        @staticmethod
        def backward(ctx, gz):
            a, b = ctx.saved_tensors
            return bf(gz) @ bf(b), bf(gz).T @ bf(a)

    p = torch.tensor(params, requires_grad=True)
    At = torch.tensor(A)
    x = (torch.tensor(logc) - torch.tensor(mu)) / torch.tensor(sd)
    h = x
    for l in range(depth + 1):
        (o, ob), d = offs[l], dims[l]
        W, b = p[o:o + d[0] * d[1]].reshape(d), p[ob:ob + d[0]]
        z = BfMatmul.apply(h, W) + b
        h = torch.nn.functional.gelu(z) if l < depth else z
    ymax = h.detach().max(dim=1, keepdim=True).values
    P = BfMatmul.apply(torch.exp(h - ymax), At)
    lt = torch.mean((torch.log(P) + ymax - torch.tensor(logc)) ** 2)
    lt.backward()
    assert abs(lt.item() - loss) <= 1e-12 * loss
    assert np.allclose(p.grad.numpy(), g, rtol=1e-9, atol=1e-12 * np.max(np.abs(g)))
