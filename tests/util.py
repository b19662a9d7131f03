"""Shared helpers for the tests: loading tables, running the GPU path, errors."""
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_2410_17446_gb300", "tables")


def table_json(name):
    return json.load(open(os.path.join(TABLES, name + ".json")))


def oracle_table(name):
    from oracle import aaa_lawson as al
    return al.PoleTable.from_json(table_json(name))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def gpu_propagator(workload, table_name, precision, **kw):
    """A Propagator for every beam of a workload, fields and step-0 media set."""
    from paper_2410_17446_gb300 import prop as P
    grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in workload.beams]
    pr = P.Propagator.from_table(grids, workload.k0, workload.n0, workload.dz, table_json(table_name),
                                 ncomp=workload.ncomp, precision=precision, **kw)
    for i, b in enumerate(workload.beams):
        pr.set_field(i, np.ascontiguousarray(b.w0))
    return pr


def gpu_run(pr, workload, nsteps, first_step=0):
    for s in range(first_step, first_step + nsteps):
        for i, b in enumerate(workload.beams):
            if s == first_step or b.medium_changes(s):
                pr.set_medium(i, np.ascontiguousarray(b.medium(s)))
        pr.step()
    return [pr.get_field(i) for i in range(len(workload.beams))]
