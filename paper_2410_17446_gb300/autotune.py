"""FFT plan autotuner: times the variants of the row and column passes on this
GPU (prop_fft_autotune) and installs the fastest (prop_set_fft_plan).

Results are cached as JSON keyed by the GPU's name: ``load_or_tune`` installs a
cached plan when one exists for this GPU and size, and otherwise tunes, installs
and records it.  The package ships the plans measured on GB300 in
``tune/fft_plans.json``.  The tuning data are ``batch`` n x n complex arrays of
at least 256 MiB in all, more than the L2 cache, so that each timing reads HBM.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional

from . import prop as P

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tune", "fft_plans.json")
ROWS = {P.PROP_ROWS_BLOCK: "block", P.PROP_ROWS_WARP: "warp"}
COLS = {P.PROP_COLS_TMA: "tma", P.PROP_COLS_PLAIN: "plain", P.PROP_COLS_WARP: "warp"}
PREC = {P.PROP_FP32: "fp32", P.PROP_FP64: "fp64"}


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _time(n: int, precision: int, batch: int, reps: int, l2cold: int):
    import torch
    nb = P.prop_fft_autotune_workspace_size(n, precision, batch)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    best, ms = P.prop_fft_autotune(n, precision, batch, reps, work, nb, stream, l2cold)
    del work
    return best, {f"{ROWS[v // 3]}+{COLS[v % 3]}": ms[v] for v in range(6) if ms[v] >= 0}


def tune(n: int, precision: int, reps: int = 5, batch: int = 16) -> dict:
    """Time every (rows, cols) combination for size n at two launch sizes: `batch`
    arrays (the large class: the early Arnoldi steps, all poles iterating) and a
    single array (the small class: the late steps), the data left in L2 between
    runs as they pass from one pass to the next in the Arnoldi step; returns the
    record."""
    batch = max(1 + P.PROP_FFT_SMALL_ITEMS, batch)
    big, ms_big = _time(n, precision, batch, reps, 0)
    small, ms_small = _time(n, precision, 1, reps, 0)
    return {"n": n, "precision": PREC[precision], "batch": batch, "reps": reps,
            "round_trip_ms": ms_big, "round_trip_ms_small": ms_small,
            "rows": ROWS[big.rows], "cols": COLS[big.cols],
            "rows_small": ROWS[small.rows], "cols_small": COLS[small.cols]}


def install(rec: dict) -> None:
    prec = {v: k for k, v in PREC.items()}[rec["precision"]]
    R = {v: k for k, v in ROWS.items()}
    Cc = {v: k for k, v in COLS.items()}
    P.prop_set_fft_plan(rec["n"], prec, R[rec["rows"]], Cc[rec["cols"]], R[rec["rows_small"]], Cc[rec["cols_small"]])


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def load_or_tune(sizes: Iterable[int], precision: int = P.PROP_FP32, path: Optional[str] = None,
                 write: bool = True, retune: bool = False) -> Dict[int, dict]:
    """Install a plan for each size: from the cache for this GPU, else by tuning
    (then recorded in the cache when `write`).  Returns the records used."""
    path = path or CACHE
    data = _read(path)
    name = gpu_name()
    entry = data.setdefault(name, {})
    used, changed = {}, False
    for n in sorted(set(int(x) for x in sizes)):
        key = f"{PREC[precision]}:{n}"
        rec = None if retune else entry.get(key)
        if rec is not None and "round_trip_ms" not in rec:
            rec = None                      # a record of an earlier tuner
        source = "cache"
        if rec is None:
            rec = tune(n, precision)
            entry[key] = rec
            changed, source = True, "tuned now"
        install(rec)
        used[n] = dict(rec, source=source, gpu=name)
    if changed and write:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return used


def main(argv=None) -> int:
    """python -m paper_2410_17446_gb300.autotune [--out PATH] [--fp64] N [N ...]: tune and record."""
    import argparse
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("sizes", type=int, nargs="+")
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--fp64", action="store_true")
    a = ap.parse_args(argv)
    build.build()
    used = load_or_tune(a.sizes, P.PROP_FP64 if a.fp64 else P.PROP_FP32, a.out, retune=True)
    print(json.dumps(used, indent=1))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
