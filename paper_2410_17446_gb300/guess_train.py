"""Training of the learned GMRES initial guess on data from the plain GPU path.

The training pairs are (R0_k / rms, 10 delta, p_k) -> e_k / rms of steps run
with x0 = 0 (prop_get_net_io); the network (guess.GuessNet) is trained with
the library's own forward, backward and Adam kernels.  Media are drawn from
the same families as the workloads but with other seeds, so that evaluation
media are never seen in training.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, List, Sequence

import numpy as np

from . import guess as Gmod
from . import prop as P
from . import workloads as wl

CHANNELS = [16, 32, 32, 32, 32, 32, 16]     # six 3x3 layers, 32 hidden channels
HERE = os.path.dirname(os.path.abspath(__file__))


def scalar_family(n: int, seed: int):
    """A sine-product medium with random eps, period and waist (the uneven-batch family), dx = lambda/4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = float(rng.uniform(0.02, 0.1))
    period = float(rng.uniform(1.0, 3.0))
    waist = float(rng.uniform(2.0, 8.0))
    g = wl.Grid(n, n, 0.25, 0.25)
    width = max(8, n // 16)
    dz = 0.5
    beam = wl.Beam(g, wl.gaussian_beam(g, waist)[None],
                   lambda s: wl.sine_product_n2(g, eps, period, (s + 0.5) * dz, width, 0.2), lambda s: True, width, 0.2)
    return wl.Workload(f"scalar_family_{seed}", wl.K0, 1.0, dz, 0, 12, 1, "fp32", 20, 1e-7, [beam])


def vector_family(n: int, seed: int):
    """A Gaussian random medium (l = lambda) with an x-polarised beam, dx = lambda/6."""
    return wl.vector_random_512(16, n=n, seed=seed)


FAMILIES: Dict[str, tuple] = {
    "scalar": (scalar_family, "uneven_batch", 1),
    "vector": (vector_family, "vector_random_512", 2),
}


def table(name: str) -> dict:
    with open(os.path.join(HERE, "tables", name + ".json")) as f:
        return json.load(f)


def make_propagator(W, tab, guess: int = P.PROP_GUESS_ZERO):
    grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in W.beams]
    return P.Propagator.from_table(grids, W.k0, W.n0, W.dz, tab, ncomp=W.ncomp, precision=P.PROP_FP32, guess=guess)


def generate(family: str, n: int, seeds: Sequence[int], steps: int):
    """Training pairs from plain runs: X bf16 [S, n, n, 16], Y float32 [S, n, n, 16]."""
    import torch
    maker, tname, ncomp = FAMILIES[family]
    tab = table(tname)
    X, Y = [], []
    for seed in seeds:
        W = maker(n, seed)
        pr = make_propagator(W, tab)
        b = W.beams[0]
        pr.set_field(0, np.ascontiguousarray(b.w0))
        for s in range(steps):
            if s == 0 or b.medium_changes(s):
                pr.set_medium(0, np.ascontiguousarray(b.medium(s)))
            pr.step()
            for k in range(pr.npoles):
                x = torch.empty((n, n, 16), dtype=torch.bfloat16, device="cuda")
                y = torch.empty((n, n, 16), dtype=torch.float32, device="cuda")
                pr.get_net_io(0, k, x, y)
                X.append(x)
                Y.append(y)
        pr.close()
    return torch.stack(X), torch.stack(Y)


def normalise_targets(Y, valid: int):
    """Each target divided by its own RMS: the network learns the shape of e_k;
    the minimal-residual scaling in the step supplies magnitude and phase."""
    import torch
    rms = torch.sqrt((Y[..., :valid] ** 2).mean(dim=(1, 2, 3), keepdim=True)).clamp_min(1e-30)
    return Y / rms


def train(net: Gmod.GuessNet, X, Y, valid: int, steps: int = 300, batch: int = 8, lr: float = 2e-3,
          seed: int = 0) -> List[float]:
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    S = X.shape[0]
    Y = normalise_targets(Y, valid)
    for it in range(steps):
        idx = torch.randint(0, S, (min(batch, S),), generator=g).to(X.device)
        xb, yb = X[idx].contiguous(), Y[idx].contiguous()
        out, acts = net.forward(xb, keep=True)
        loss, grad = net.mse(out, yb, valid)
        dws, dbs = net.backward(acts, grad)
        cur = lr * 0.5 * (1 + math.cos(math.pi * it / steps))
        net.adam(dws, dbs, lr=cur)
        losses.append(float(loss.item()))
    return losses


def run_pair(W, tab, steps: int, net_state=None):
    """Run W with x0 = 0 and (if net_state) with the learned guess; returns fields and
    per-step Arnoldi-step totals of each run."""
    out = {}
    for mode in ("plain", "learned"):
        if mode == "learned" and net_state is None:
            continue
        pr = make_propagator(W, tab, P.PROP_GUESS_LEARNED if mode == "learned" else P.PROP_GUESS_ZERO)
        if mode == "learned":
            pr.set_guess_net(net_state["channels"], net_state["weights"], net_state["biases"])
        b = W.beams[0]
        pr.set_field(0, np.ascontiguousarray(b.w0))
        its = []
        for s in range(steps):
            if s == 0 or b.medium_changes(s):
                pr.set_medium(0, np.ascontiguousarray(b.medium(s)))
            pr.step()
            its.append(int(pr.iterations().sum()))
        out[mode] = (pr.get_field(0), its)
        pr.close()
    return out


def save(net: Gmod.GuessNet, path: str, meta: dict) -> None:
    st = net.state()
    arrays = {f"w{l}": w for l, w in enumerate(st["weights"])}
    arrays.update({f"b{l}": b for l, b in enumerate(st["biases"])})
    np.savez(path, channels=np.array(st["channels"]), meta=json.dumps(meta), **arrays)


def load(path: str) -> dict:
    z = np.load(path)
    L = len(z["channels"]) - 1
    return {"channels": [int(c) for c in z["channels"]], "weights": [z[f"w{l}"] for l in range(L)],
            "biases": [z[f"b{l}"] for l in range(L)], "meta": json.loads(str(z["meta"]))}


def main(argv=None) -> int:
    """python -m paper_2410_17446_gb300.guess_train FAMILY N OUT.npz [--media M] [--steps S] [--iters I]"""
    import argparse
    import time
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("family", choices=sorted(FAMILIES))
    ap.add_argument("n", type=int)
    ap.add_argument("out")
    ap.add_argument("--media", type=int, default=20)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--eval-media", type=int, default=4)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    maker, tname, ncomp = FAMILIES[a.family]
    t0 = time.time()
    X, Y = generate(a.family, a.n, range(100, 100 + a.media), a.steps)
    torch.cuda.synchronize()
    t1 = time.time()
    net = Gmod.GuessNet(CHANNELS, seed=0)
    losses = train(net, X, Y, valid=2 * ncomp, steps=a.iters, batch=8, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.time()
    st = net.state()
    tab = table(tname)
    ev = {"plain": 0, "learned": 0, "max_rel_diff": 0.0}
    for seed in range(200, 200 + a.eval_media):
        r = run_pair(maker(a.n, seed), tab, 3, st)
        ev["plain"] += sum(r["plain"][1])
        ev["learned"] += sum(r["learned"][1])
        d = float(np.linalg.norm(r["learned"][0] - r["plain"][0]) / np.linalg.norm(r["plain"][0]))
        ev["max_rel_diff"] = max(ev["max_rel_diff"], d)
    meta = {"family": a.family, "n": a.n, "train_media_seeds": [100, 100 + a.media], "steps_per_medium": a.steps,
            "solves": int(X.shape[0]), "adam_iterations": a.iters, "loss_first10": float(np.mean(losses[:10])),
            "loss_last10": float(np.mean(losses[-10:])), "generate_s": t1 - t0, "train_s": t2 - t1,
            "eval_media_seeds": [200, 200 + a.eval_media], "eval_arnoldi_steps": ev}
    save(net, a.out, meta)
    print(json.dumps(meta))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
