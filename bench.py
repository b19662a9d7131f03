"""Benchmark of the GB300 propagator: Mpoint*steps/s on one workload.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one z-step of the exponential propagator (Eq. approx_prop) for
every beam of the workload: medium refresh (when the workload's n^2 changes),
the free-space part, the shifted GMRES solves and the residue sum.  Each rank
runs its own replica of the workload (the path has no exchange step), so
``value`` is the total over ranks (weak scaling).  Time is taken with CUDA
events on the library's stream around each step; an L2 flush (a 256 MiB
write) runs between steps outside the timed intervals.  ``--impl reference``
times the CPU oracle (complex128 NumPy) on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpoint·steps/s at 1024² scalar & 512² vector, learned vs plain, at 1e-5 L2 err"
UNIT = "Mpoint·steps/s"
DEFAULT_WORKLOAD = "homogeneous_aperture_1024"
CONFIG_STEPS = {"homogeneous_aperture_1024": 100, "batched_scalar_1024": 200, "plain_scalar_64": 16,
                "vector_random_512": 150, "uneven_batch": 64}
GATE_CYCLES = 400_000      # ~0.2 ms of GPU sleep before each timed step (outside the interval)
TABLE_OF = {"homogeneous_aperture_1024": "homogeneous_aperture_1024", "batched_scalar_1024": "batched_scalar_1024",
            "plain_scalar_64": "plain_scalar_64", "vector_random_512": "vector_random_512",
            "uneven_batch": "uneven_batch"}


def make_workload(name: str, nsteps: int, n: int = 0):
    """The named workload; n > 0 shrinks a single-grid workload to n x n (profiling only)."""
    from paper_2410_17446_gb300 import workloads as wl
    if name == "homogeneous_aperture_1024":
        return wl.homogeneous_aperture_1024(nsteps, **({"n": n} if n else {}))
    if name == "batched_scalar_1024":
        return wl.batched_scalar_1024(nsteps, **({"n": n} if n else {}))
    if name == "plain_scalar_64":
        return wl.plain_scalar_64(nsteps)
    if name == "vector_random_512":
        return wl.vector_random_512(nsteps)
    if name == "uneven_batch":
        return wl.uneven_batch(nsteps=nsteps)
    raise SystemExit(f"unknown workload {name}")


def load_table(name: str) -> dict:
    with open(os.path.join(ROOT, "paper_2410_17446_gb300", "tables", TABLE_OF[name] + ".json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if t < t0 or t > t1 + 0.25:
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on the host cores
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time, os
sys.path.insert(0, {root!r})
import numpy as np
from oracle import aaa_lawson as al, propagator as pr, operators as ops
from paper_2410_17446_gb300 import workloads as wl
import bench
W = bench.make_workload({name!r}, 64)
T = al.PoleTable.from_json(bench.load_table({name!r}))
budget = {budget}
t0 = time.perf_counter(); steps = 0; pts = 0
beams = W.beams
w = [b.w0.copy() for b in beams]
med = [None] * len(beams)
its = []
while True:
    for i, b in enumerate(beams):
        if med[i] is None or b.medium_changes(steps):
            med[i] = ops.Medium(b.medium(steps), b.grid.dx, b.grid.dy, W.k0, W.n0, W.ncomp)
        w[i], st = pr.step(med[i], w[i], T, tol=1e-12)
        its += st.iterations
        pts += b.grid.nx * b.grid.ny
        if time.perf_counter() - t0 > budget and i + 1 < len(beams):
            break
    steps += 1
    el = time.perf_counter() - t0
    if el > budget or steps >= {max_steps}:
        break
print(json.dumps({{"seconds": el, "steps": steps, "point_steps": pts, "mean_iters": float(np.mean(its))}}))
"""


def run_oracle_sample(name: str, budget_s: float, max_steps: int) -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, budget=budget_s, max_steps=max_steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=max(600, 20 * budget_s))
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["value"] = d["point_steps"] / d["seconds"] / 1e6
    d["cores"] = 1
    d["sample"] = (f"{d['steps']} step(s) of {name} by the complex128 oracle (GMRES tol 1e-12, "
                   f"numpy.fft single-threaded, BLAS threads = 1), {d['seconds']:.1f} s")
    return d


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over the ranks (the job's time is its slowest replica's)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws: int, points: int, steps: int, seconds: float) -> float:
    """Mpoint·steps/s of ws replicas that each advance `points` points by `steps` steps in `seconds`."""
    return ws * points * steps / seconds / 1e6


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args) -> None:
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    budget = 20.0
    d = run_oracle_sample(args.workload, budget, 10 ** 6)
    W = make_workload(args.workload, 1)
    line = {"impl": "reference", "metric": METRIC, "value": d["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": d["steps"], "warmup": 0, "ms_per_step": 1e3 * d["seconds"] / max(1, d["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "points_per_step": W.points,
                                            "poles": W.npoles},
            "cpu_baseline": {"value": d["value"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
                             "sample": d["sample"]},
            "e2e": {"value": d["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def ours(args) -> None:
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2410_17446_gb300 import build as B
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2410_17446_gb300 import prop as P

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = run_oracle_sample(args.workload, args.cpu_seconds, 10 ** 6)

    total = args.warmup + args.steps
    W = make_workload(args.workload, max(total, 1), args.n)
    tab = load_table(args.workload)
    grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in W.beams]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        pr = P.Propagator.from_table(grids, W.k0, W.n0, W.dz, tab, ncomp=W.ncomp, precision=P.PROP_FP32,
                                     restart=W.restart, stream=stream)
    for i, b in enumerate(W.beams):
        pr.set_field(i, np.ascontiguousarray(b.w0))
    # media for every step, resident on the device before timing
    media = {}
    for s in range(total):
        for i, b in enumerate(W.beams):
            if s == 0 or b.medium_changes(s):
                media[(s, i)] = torch.tensor(b.medium(s), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(prx, clocks_on=True):
        """W warm-up steps, then K steps each timed by events on the library stream."""
        def step_of(s):
            for i in range(len(W.beams)):
                m = media.get((s, i))
                if m is not None:
                    prx.set_medium(i, m)
            prx.step()
        with torch.cuda.stream(stream):
            for s in range(args.warmup):
                step_of(s)
            torch.cuda.synchronize(dev)
            l0 = prx.stats().kernel_launches
            prx.set_profiling(True)
            st_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            en_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            clocks = ClockSampler(local) if clocks_on else None
            if ws > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            if clocks:
                clocks.start()
                time.sleep(0.3)
            t0 = time.perf_counter()
            its_total = 0
            for k in range(args.steps):
                flush.zero_()
                # keep the GPU busy while the host enqueues the step, so that the
                # timed interval holds device work, not host launch latency
                torch.cuda._sleep(GATE_CYCLES)
                st_ev[k].record(stream)
                step_of(args.warmup + k)
                en_ev[k].record(stream)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            clk = None
            if clocks:
                time.sleep(0.3)
                clk = clocks.stop(t0, t1)
            if ws > 1:
                torch.distributed.barrier()
            dms = sum(a.elapsed_time(b) for a, b in zip(st_ev, en_ev))
            prof = prx.profile()
            prx.set_profiling(False)
            stx = prx.stats()
            return {"dev_ms": dms, "wall": t1 - t0, "clk": clk, "prof": prof,
                    "launches": stx.kernel_launches - l0, "st": stx, "iters": prx.iterations()}

    res = timed(pr)
    dev_ms, wall, clk, prof = res["dev_ms"], res["wall"], res["clk"], res["prof"]
    launches, st, iters = res["launches"], res["st"], res["iters"]

    learned = None
    if args.guess == "both":
        from paper_2410_17446_gb300 import guess_train as GT
        fam = "vector" if W.ncomp == 2 else "scalar"
        net = GT.load(os.path.join(ROOT, "paper_2410_17446_gb300", "nets", f"guess_{fam}.npz"))
        with torch.cuda.stream(stream):
            prl = P.Propagator.from_table(grids, W.k0, W.n0, W.dz, tab, ncomp=W.ncomp, precision=P.PROP_FP32,
                                          restart=W.restart, stream=stream, guess=P.PROP_GUESS_LEARNED)
            prl.set_guess_net(net["channels"], net["weights"], net["biases"])
            for i, b in enumerate(W.beams):
                prl.set_field(i, np.ascontiguousarray(b.w0))
        rl = timed(prl, clocks_on=False)
        ml = max_over_ranks(rl["dev_ms"], ws, dev)
        learned = {"value": whole_job_value(ws, W.points, args.steps, ml / 1e3), "ms_per_step": ml / args.steps,
                   "arnoldi_steps_total": int(rl["st"].total_iters), "net": net["meta"],
                   "guess_net_ms": round(rl["prof"]["guess_net"]["total_ms"], 3)}
        prl.close()

    ms = max_over_ranks(dev_ms, ws, dev)
    pts = W.points
    value = whole_job_value(ws, pts, args.steps, ms / 1e3)

    # accuracy over the configuration's own run length, where a closed form exists
    acc = None
    if args.workload == "homogeneous_aperture_1024" and rank == 0:
        b = W.beams[0]
        total = CONFIG_STEPS[args.workload]          # the medium is constant: n^2 = 1
        with torch.cuda.stream(stream):
            pr.set_field(0, np.ascontiguousarray(b.w0))
            for s in range(total):
                pr.step()
            w = pr.get_field(0)[0]
        z = -(np.fft.fftfreq(b.grid.nx, b.grid.dx)[None, :] ** 2 + np.fft.fftfreq(b.grid.ny, b.grid.dy)[:, None] ** 2) \
            * (2 * math.pi) ** 2 / (W.k0 * W.n0) ** 2
        poles = np.array([complex(*p) for p in tab["poles"]])
        res = np.array([complex(*r) for r in tab["residues"]])
        R = complex(*tab["r0"]) + sum(r / (z - p) for p, r in zip(poles, res))
        ref = np.fft.ifft2(R ** total * np.fft.fft2(b.w0[0]))
        acc = float(np.linalg.norm(w - ref) / np.linalg.norm(ref))

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host_out = [torch.empty(pr.shape(i), dtype=torch.complex128).pin_memory() for i in range(len(W.beams))]
        host_media = {key: m.cpu().pin_memory() for key, m in media.items() if key[0] >= args.warmup}
        h2d = d2h = 0
        with torch.cuda.stream(stream):
            for i, b in enumerate(W.beams):
                pr.set_field(i, torch.tensor(b.w0).pin_memory())
            torch.cuda.synchronize(dev)
            if ws > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            for k in range(args.steps):
                s = args.warmup + k
                for i in range(len(W.beams)):
                    m = host_media.get((s, i))
                    if m is not None:
                        pr.set_medium(i, m)
                        h2d += m.numel() * 16
                pr.step()
                for i in range(len(W.beams)):
                    pr.get_field(i, host_out[i])
                    d2h += host_out[i].numel() * 16
            torch.cuda.synchronize(dev)
            e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, ws, dev)
        e2e = {"value": whole_job_value(ws, pts, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    # roofline of the dominant kernel (largest device time in the timed region)
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"])
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = dom[1]["alg_bytes"] / (dom[1]["total_ms"] / 1e3) / 1e9 if dom[1]["total_ms"] > 0 else 0.0
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{args.workload}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        traffic = tj.get(dom[0])
    roof = {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
            "alg_bytes_per_launch": dom[1]["alg_bytes"] / max(1, dom[1]["launches"]),
            "launches": dom[1]["launches"], "share_of_step": dom[1]["total_ms"] / ms if ms else None}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "points_per_step": pts, "beams": len(W.beams),
                           "grid": f"{W.beams[0].grid.nx}x{W.beams[0].grid.ny}", "poles": W.npoles,
                           "ncomp": W.ncomp, "restart": W.restart, "tol": pr.opts.tol,
                           "l2": "flushed (256 MiB write) between timed steps",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roof, "gpu_launches": launches, "clocks": clk,
                "wall_s": wall,
                "gmres": {"iters_sum_last_step": int(iters.sum()), "iters_max_last_step": int(iters.max()),
                          "total_iters": int(st.total_iters)},
                "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                                "GBps": (v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9) if v["total_ms"] > 0 else None}
                            for k, v in prof.items() if v["launches"]},
                "rel_err_vs_closed_form": acc,
                "learned_guess": learned,
                "plain_arnoldi_steps_total": int(st.total_iters),
                "rel_err_steps": CONFIG_STEPS[args.workload] if acc is not None else None, "e2e": e2e}
        if cpu is not None:
            line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                                    "sample": cpu["sample"]}
        print(json.dumps(line), flush=True)
    pr.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: enough for a timed region of a few seconds)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(TABLE_OF))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--n", type=int, default=0, help="shrink the grid (profiling runs only; not a bench line)")
    ap.add_argument("--guess", default="plain", choices=["plain", "both"],
                    help="both: also time the learned initial guess (GMRES to the same tolerance)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"homogeneous_aperture_1024": 20000, "plain_scalar_64": 2000}.get(args.workload, 100)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
