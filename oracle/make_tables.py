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


def pf_max_err(T: al.PoleTable, lo: float, hi: float, shifts=()) -> float:
    """Largest |r - g| of the partial-fraction form on a uniform sampling of the fit range."""
    z = np.linspace(lo, hi, 4001).astype(np.complex128)
    z = np.concatenate([z] + [z + 1j * s for s in shifts])
    return float(np.max(np.abs(T(z) - al.target(z, T.K))))


def pade_table(workload) -> dict:
    """The shifted and rotated (10,10) Padé approximant (Sec. 3.1) for the workload's K."""
    from . import pade
    T = pade.rotated_pade_table(workload.K, 10)
    d = T.to_json()
    d["fit_max_err"] = pf_max_err(T, -1.0, 2.0)
    d["kind"] = "pade_rotated"
    d["alpha"] = float(np.pi / 8)
    return d


# The paper's lookup table for air (Sec. 3.1): one n0 = 1.00030, a set of k0 dz,
# AAA-Lawson on its default range Re zeta in [-4, 2].
LOOKUP_N0 = 1.0003
LOOKUP_DZ = (0.25, 0.5, 1.0, 2.0, 5.0)
LOOKUP_POLES = {5.0: 28}


def lookup_table() -> dict:
    entries = []
    for dz in LOOKUP_DZ:
        K = 2 * np.pi * LOOKUP_N0 * dz
        T = al.fit(K, LOOKUP_POLES.get(dz, 25), -4.0, 2.0)
        e = T.to_json()
        e["k0dz"] = 2 * np.pi * dz
        e["pf_max_err"] = pf_max_err(T, -4.0, 2.0)
        entries.append(e)
    return {"n0": LOOKUP_N0, "domain": [-4.0, 2.0], "entries": entries,
            "source": "oracle.make_tables (AAA-Lawson oracle, uniform samples on [-4, 2])"}


def cauchy_table() -> dict:
    """The Cauchy-integral square root of Sec. 3.2 (N = 25, alpha = 1), the table
    of the pseudo-differential form (S(zeta) ~ sqrt(1 + zeta); K is not used)."""
    from . import cauchy
    T = cauchy.cauchy_sqrt_table(25, 1.0)
    d = T.to_json()
    z = np.linspace(-4, 2, 6001)
    far = np.abs(z + 1) > 0.2
    d["fit_max_err"] = float(np.max(np.abs(T(z[far]) - np.sqrt(1 + z[far] + 0j))))
    d["kind"] = "cauchy_sqrt"
    d["alpha"] = 1.0
    return d


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
        "multiwave_scalar_64": lambda: wl.multiwave_scalar_64(1),
        "sineprod_q2": lambda: wl.sineprod_helmholtz(2.0, 1, 64),
        "sineprod_q1": lambda: wl.sineprod_helmholtz(1.0, 1, 64),
        "sineprod_q05": lambda: wl.sineprod_helmholtz(0.5, 1, 64),
    }
    extra = {"pade_scalar_64": lambda: pade_table(wl.plain_scalar_64(1)),
             "lookup_n0_1.0003": lookup_table,
             "cauchy_sqrt_25": cauchy_table}
    names = argv or (list(makers) + list(extra))
    for name in names:
        if name in extra:
            d = extra[name]()
            d["workload"] = name
            with open(os.path.join(TABLE_DIR, name + ".json"), "w") as f:
                json.dump(d, f, indent=1)
            print(f"{name}: written")
            continue
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
