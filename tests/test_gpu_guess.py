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


def _oracle_run(W, tab_name, steps):
    from oracle import aaa_lawson as al
    from oracle import propagator as orp
    import json
    import os
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    T = al.PoleTable.from_json(json.load(open(os.path.join(here, "paper_2410_17446_gb300", "tables",
                                                           tab_name + ".json"))))
    b = W.beams[0]
    return orp.run(b, W.k0, W.n0, T, W.ncomp, steps, tol=1e-12)


@pytest.mark.parametrize("family,n,steps", [("vector", 64, 3), ("vector", 128, 2), ("scalar", 128, 3)])
def test_learned_path_matches_the_oracle(GT, family, n, steps):
    """The learned initial guess with the committed network, against the
    complex128 oracle (not against the plain GPU path), on media of the
    benchmark families the network never saw (seeds 300+): relative L2 field
    error within the FP32 bar of 1e-5.  Vector: the 512^2 workload's recipe
    (random n^2, lambda/6, border) reduced; scalar: the 1024^2 workload's."""
    import os
    from paper_2410_17446_gb300 import prop as P
    from paper_2410_17446_gb300 import workloads as wl
    net = GT.load(os.path.join(os.path.dirname(GT.__file__), "nets", f"guess_{family}.npz"))
    if family == "vector":
        W = wl.vector_random_512(steps, n=n, seed=300 + n)
        tab_name = "vector_random_512"
    else:
        W = wl.batched_scalar_1024(steps, n=n)
        tab_name = "batched_scalar_1024"
    pr = GT.make_propagator(W, GT.table(tab_name), P.PROP_GUESS_LEARNED)
    pr.set_guess_net(net["channels"], net["weights"], net["biases"])
    b = W.beams[0]
    pr.set_field(0, np.ascontiguousarray(b.w0))
    for s in range(steps):
        if s == 0 or b.medium_changes(s):
            pr.set_medium(0, np.ascontiguousarray(b.medium(s)))
        pr.step()
    got = pr.get_field(0)
    ref = _oracle_run(W, tab_name, steps)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"{family} {n}^2 x {steps}: learned path vs oracle {err:.2e}")
    assert err < 1e-5


def test_learned_guess_gain_on_held_out_vector_media(GT):
    """What the trained vector network gains: on held-out media of the vector
    family (seeds 200-203, never used in training) the learned guess takes
    fewer Arnoldi steps in total than x0 = 0, and both reach the same field."""
    import os
    net = GT.load(os.path.join(os.path.dirname(GT.__file__), "nets", "guess_vector.npz"))
    tab = GT.table("vector_random_512")
    plain = learned = 0
    for seed in range(200, 204):
        r = GT.run_pair(GT.vector_family(128, seed), tab, 3, net)
        plain += sum(r["plain"][1])
        learned += sum(r["learned"][1])
        d = np.linalg.norm(r["learned"][0] - r["plain"][0]) / np.linalg.norm(r["plain"][0])
        assert d < 1e-5
    print(f"held-out vector media: Arnoldi steps plain {plain}, learned {learned}")
    assert learned < plain
