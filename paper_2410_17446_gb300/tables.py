"""Pole tables the propagator consumes (host set-up data, not hot path).

Each table gives r(zeta) = r0 + sum_k r_k/(zeta - p_k) for one K = k0 n0 dz,
as JSON written by the table script next to the oracle: one file per
workload, the shifted/rotated Padé approximant of Sec. 3.1, and the paper's
lookup table of expansion coefficients for a fixed n0 and a set of k0 dz
(Sec. 3.1: for propagation in air one table with n0 = 1.00030 serves).
This module only reads those files.
"""
from __future__ import annotations

import json
import math
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables")


def load(name: str) -> dict:
    """The table file ``tables/<name>.json``."""
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


def lookup(n0: float, k0dz: float, rel: float = 1e-9) -> dict:
    """The entry of the lookup table for reference index n0 whose k0 dz matches
    (relative tolerance ``rel``); KeyError if the table has no such entry."""
    name = f"lookup_n0_{n0:.4f}".rstrip("0").rstrip(".")
    path = os.path.join(HERE, name + ".json")
    if not os.path.exists(path):
        raise KeyError(f"no lookup table for n0 = {n0}")
    with open(path) as f:
        tab = json.load(f)
    for e in tab["entries"]:
        if math.isclose(e["k0dz"], k0dz, rel_tol=rel):
            return e
    raise KeyError(f"no entry for k0 dz = {k0dz} in {name} (have {[e['k0dz'] for e in tab['entries']]})")
