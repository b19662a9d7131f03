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


@pytest.mark.parametrize("H,W", [(32, 128), (6, 256), (37, 256), (120, 1024), (8, 64)])
@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 16), (32, 32)])
def test_tensor_core_paths_agree(G, cin, cout, H, W):
    """The tcgen05 convolutions (strips of 128-pixel row tiles for W a multiple
    of 128, one row chunk per CTA, down to chunks of one row; else 128-pixel
    tiles; accumulators in tensor memory) and the
    warp-level mma.sync one give the same layer, in all three output modes, and
    an inactive image is left untouched; the bounded wait never gave up."""
    import ctypes as ct
    import torch
    from oracle import cnn
    from paper_2410_17446_gb300 import prop as P
    L = P.lib()
    rng = np.random.default_rng(cin + cout)
    N = 3
    x = torch.tensor(rng.standard_normal((N, H, W, cin)), dtype=torch.bfloat16, device="cuda")
    w = torch.tensor(rng.standard_normal((9, cout, cin)) / np.sqrt(9 * cin), dtype=torch.bfloat16, device="cuda")
    b = torch.tensor(rng.standard_normal(cout) * 0.1, dtype=torch.float32, device="cuda")
    active = torch.tensor([1, 0, 1], dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    outs = {}
    try:
        for path in (0, 1):   # PROP_CNN_PATH_AUTO (tcgen05 here), PROP_CNN_PATH_MMA_SYNC
            assert L.prop_cnn_set_path(path) == 0
            for mode, dt in ((0, torch.bfloat16), (1, torch.bfloat16), (2, torch.float32)):
                o = torch.full((N, H, W, cout), 7.0, dtype=dt, device="cuda")
                assert L.prop_cnn_conv(cin, cout, mode, x.data_ptr(), w.data_ptr(), b.data_ptr(), o.data_ptr(), N, H,
                                       W, active.data_ptr(), 1, 1, ct.c_void_p(st)) == 0
                outs[path, mode] = o.float().cpu().numpy()
        assert L.prop_cnn_check(ct.c_void_p(st)) == 0
    finally:
        L.prop_cnn_set_path(0)
    ref = cnn.forward(x.float().cpu().numpy().astype(np.float64), [w.float().cpu().numpy().astype(np.float64)],
                      [b.cpu().numpy().astype(np.float64)], bf16=False)[1][0]
    for mode in (0, 1, 2):
        tc, ms = outs[0, mode], outs[1, mode]
        assert np.all(tc[1] == 7.0) and np.all(ms[1] == 7.0)   # the inactive image
        tol = 1e-5 if mode == 2 else 1e-2
        assert rel(tc[[0, 2]], ms[[0, 2]]) < tol, mode
        r = np.maximum(ref, 0.0) if mode == 0 else ref
        assert rel(tc[[0, 2]], r[[0, 2]]) < tol, mode
