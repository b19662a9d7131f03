"""The learned initial guess end to end on the GPU: training pairs from the
plain path, a short training run with the library's kernels, and the learned
path reaching the same field as x0 = 0 (GMRES runs to the same tolerance).
Arnoldi-step counts of both are printed; the gain is measured in bench.py."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def GT():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build
    build.build()
    from paper_2410_17446_gb300 import guess_train
    return guess_train


def test_learned_guess_trains_and_keeps_the_answer(GT):
    from paper_2410_17446_gb300 import guess as G
    X, Y = GT.generate("scalar", 64, seeds=range(100, 106), steps=2)
    assert X.shape == (6 * 2 * 12, 64, 64, 16)
    net = G.GuessNet(GT.CHANNELS, seed=0)
    losses = GT.train(net, X, Y, valid=2, steps=300, batch=8, lr=1e-3)
    assert np.mean(losses[-20:]) < 0.6 * np.mean(losses[:20])
    st = net.state()
    tab = GT.table("uneven_batch")
    for seed in (300, 301):
        r = GT.run_pair(GT.scalar_family(64, seed), tab, 2, st)
        d = np.linalg.norm(r["learned"][0] - r["plain"][0]) / np.linalg.norm(r["plain"][0])
        print(f"medium {seed}: Arnoldi steps plain {r['plain'][1]}, learned {r['learned'][1]}, rel diff {d:.2e}")
        assert d < 1e-5


def test_learned_guess_needs_a_network(GT):
    from paper_2410_17446_gb300 import prop as P
    W = GT.scalar_family(64, 5)
    pr = GT.make_propagator(W, GT.table("uneven_batch"), P.PROP_GUESS_LEARNED)
    with pytest.raises(P.PropError):
        pr.set_guess_net([16, 32], [np.zeros((9, 32, 16))], [np.zeros(32)])   # last width must be 16
    # without a network the learned mode falls back to x0 = 0
    pr.set_field(0, W.beams[0].w0)
    pr.set_medium(0, W.beams[0].medium(0))
    pr.step()
    assert pr.iterations().sum() > 0
