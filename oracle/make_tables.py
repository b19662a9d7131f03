"""Write the pole tables the propagator consumes (oracle, test infrastructure).

Run ``python -m oracle.make_tables`` from the repository root.  For each
workload it fits g(zeta) = exp(iK(-1+sqrt(1+zeta))) with the AAA-Lawson
oracle (Sec. 3.1) on the range the grid's spectrum needs: Re zeta from
min(-4, zeta_min + min Re delta - 0.5) to 2 (the paper's default upper end,
Sec. 3), plus the strip Im zeta in {sigma, 2 sigma} that the absorbing border
moves the spectrum into.  Samples are uniform (no clustering at the branch
point), which keeps the poles off the real axis.  The result -- the paper's
"lookup table" of expansion coefficients for one K (Sec. 3.1) -- is written as
JSON next to the package that reads it.  Only this script writes those files,
and it calls nothing outside ``oracle/`` and the input generators.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

from . import aaa_lawson as al
from . import operators as ops

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_DIR = os.path.join(os.path.dirname(HERE), "paper_2410_17446_gb300", "tables")


def table_for(workload, probe_steps=(0,)) -> al.PoleTable:
    lo = 0.0
    sig = 0.0
    for b in workload.beams:
        g = b.grid
        dmin = min(float(ops.delta_of(b.medium(s), workload.n0).real.min()) for s in probe_steps)
        lo = min(lo, al.fit_domain(g.nx, g.ny, g.dx, g.dy, workload.k0 * workload.n0, dmin))
        sig = max(sig, b.sigma_max if b.border > 0 else 0.0)
    # the medium amplitudes are bounded by the generator's eps, so widen by its bound
    lo = float(np.floor(lo * 10) / 10)
    shifts = (sig, 2 * sig) if sig > 0 else ()
    return al.fit(workload.K, workload.npoles, lo, 2.0, im_shifts=shifts)


def main(argv=None) -> int:
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2410_17446_gb300 import workloads as wl
    os.makedirs(TABLE_DIR, exist_ok=True)
    makers = {
        "plain_scalar_64": lambda: wl.plain_scalar_64(1),
        "homogeneous_aperture_1024": lambda: wl.homogeneous_aperture_1024(1),
        "batched_scalar_1024": lambda: wl.batched_scalar_1024(1, n=256),
        "vector_random_512": lambda: wl.vector_random_512(1, n=128),
        "uneven_batch": lambda: wl.uneven_batch(nbeams=48, nsteps=1, sizes=(128,)),
    }
    names = argv or list(makers)
    for name in names:
        W = makers[name]()
        T = table_for(W)
        d = T.to_json()
        d["workload"] = name
        d["source"] = "oracle.make_tables (AAA-Lawson oracle, uniform samples + absorbing strip)"
        with open(os.path.join(TABLE_DIR, name + ".json"), "w") as f:
            json.dump(d, f, indent=1)
        print(f"{name}: K={T.K:.6f} P={T.npoles} domain=[{T.lo}, {T.hi}] shifts={T.im_shifts} "
              f"fit max err={T.fit_max_err:.3e} min|Im p|={np.abs(T.poles.imag).min():.2e}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main(sys.argv[1:]))
