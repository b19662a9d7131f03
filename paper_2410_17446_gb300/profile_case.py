"""A small, self-contained case of a benchmark workload for profiler captures.

``python -m paper_2410_17446_gb300.profile_case --workload batched_scalar_1024 --poles 4 --steps 2``
runs the first ``--poles`` poles of the workload's table for ``--steps`` z-steps
on the first ``--beams`` beams (all by default), synchronises and prints the
Arnoldi steps taken.  Small enough for an ``ncu --set full`` capture of one or
a few launches, large enough (one 1024² basis of a few systems) that the sweeps'
inputs exceed the L2 cache.
"""
from __future__ import annotations

import argparse
import json
import os

from . import build, prop as P, tables, workloads as wl

BUILDERS = {
    "batched_scalar_1024": lambda steps: wl.batched_scalar_1024(steps),
    "vector_random_512": lambda steps: wl.vector_random_512(steps),
    "uneven_batch": lambda steps: wl.uneven_batch(nsteps=steps),
    "homogeneous_aperture_1024": lambda steps: wl.homogeneous_aperture_1024(steps),
}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="batched_scalar_1024", choices=sorted(BUILDERS))
    ap.add_argument("--poles", type=int, default=4)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--beams", type=int, default=0, help="first N beams (0: all)")
    ap.add_argument("--multigroup", default="on", choices=["on", "off"])
    ap.add_argument("--learned", action="store_true", help="the learned initial guess (committed network)")
    args = ap.parse_args(argv)
    import torch
    build.build()
    W = BUILDERS[args.workload](args.steps)
    beams = W.beams[:args.beams] if args.beams else W.beams
    tab = dict(tables.load(args.workload))
    tab["poles"] = tab["poles"][:args.poles]
    tab["residues"] = tab["residues"][:args.poles]
    grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in beams]
    pr = P.Propagator.from_table(grids, W.k0, W.n0, W.dz, tab, ncomp=W.ncomp, precision=P.PROP_FP32,
                                 multigroup=args.multigroup == "on",
                                 guess=P.PROP_GUESS_LEARNED if args.learned else P.PROP_GUESS_ZERO)
    if args.learned:
        from . import guess_train
        fam = "vector" if W.ncomp == 2 else "scalar"
        net = guess_train.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "nets", f"guess_{fam}.npz"))
        pr.set_guess_net(net["channels"], net["weights"], net["biases"])
    for i, b in enumerate(beams):
        pr.set_field(i, b.w0)
    for s in range(args.steps):
        for i, b in enumerate(beams):
            if s == 0 or b.medium_changes(s):
                pr.set_medium(i, b.medium(s))
        pr.step()
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "beams": len(beams), "poles": args.poles, "steps": args.steps,
                      "arnoldi_steps": int(pr.stats().total_iters), "workspace_gb": pr.ws_bytes / 1e9,
                      "pid": os.getpid()}))


if __name__ == "__main__":
    main()
