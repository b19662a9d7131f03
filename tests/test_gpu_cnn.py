"""The guess network's CUDA kernels (BF16 tensor-core convolutions, FP32
gradients, Adam) against the FP64 CPU reference with the same bfloat16
rounding points."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build
    build.build()
    from paper_2410_17446_gb300 import guess
    return guess


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("chans", [[16, 32, 32, 16], [32, 16, 32]])
def test_forward_and_gradients_match_oracle(G, chans):
    import torch
    from oracle import cnn
    rng = np.random.default_rng(4)
    N, H, W = 2, 16, 64
    net = G.GuessNet(chans, seed=5)
    for b in net.b32:
        b.copy_(torch.tensor(rng.standard_normal(b.shape).astype(np.float32) * 0.1))
    Ws = [w.cpu().numpy().astype(np.float64) for w in net.w32]
    bs = [b.cpu().numpy().astype(np.float64) for b in net.b32]
    x = cnn.bf16_round(rng.standard_normal((N, H, W, chans[0])))
    tgt = rng.standard_normal((N, H, W, chans[-1]))
    xd = torch.tensor(x, dtype=torch.bfloat16, device="cuda")
    out, acts = net.forward(xd, keep=True)
    a_ref, y_ref = cnn.forward(x, Ws, bs, bf16=True)
    assert rel(out.cpu().numpy(), a_ref[-1]) < 1e-2
    valid = chans[-1] - 3
    loss, grad = net.mse(out, torch.tensor(tgt, dtype=torch.float32, device="cuda"), valid)
    dws, dbs = net.backward(acts, grad)
    npix = N * H * W
    d = a_ref[-1] - tgt
    d[..., valid:] = 0.0
    assert abs(loss.item() - 0.5 * np.sum(d ** 2) / npix) < 1e-3 * abs(loss.item())
    gW, gb, _ = cnn.backward(a_ref, y_ref, Ws, d / npix, bf16=True)
    for l in range(len(Ws)):
        assert rel(dws[l].cpu().numpy(), gW[l]) < 2e-2, l
        assert rel(dbs[l].cpu().numpy(), gb[l]) < 2e-2, l


def test_training_reduces_loss(G):
    """A few Adam steps of the GPU kernels on a fixed regression target."""
    import torch
    rng = np.random.default_rng(0)
    net = G.GuessNet([16, 32, 16], seed=1)
    x = torch.tensor(rng.standard_normal((2, 16, 64, 16)), dtype=torch.bfloat16, device="cuda")
    teacher = G.GuessNet([16, 32, 16], seed=9)
    tgt = teacher.forward(x)
    losses = []
    for _ in range(60):
        out, acts = net.forward(x, keep=True)
        loss, grad = net.mse(out, tgt, 16)
        dws, dbs = net.backward(acts, grad)
        net.adam(dws, dbs, lr=3e-3)
        losses.append(loss.item())
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
