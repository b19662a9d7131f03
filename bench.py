"""Benchmark of the GB300 propagator: Mpoint*steps/s, learned vs plain.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--extra NAMES]
                [--guess plain|both] [--impl ours|reference]

A step is one z-step of the exponential propagator (Eq. approx_prop) for every
beam of the workload: medium refresh (when the workload's n^2 changes), the
free-space part, the shifted GMRES solves and the residue sum.  The default
workload is the 1024^2 batched scalar one (16 poles, z-varying sine-product
n^2, absorbing border); the 512^2 vector workload (14 poles, random n^2,
cross-polarisation) is measured beside it, each with x0 = 0 (plain) and with
the learned initial guess.  Each rank runs its own replica (the path has no
exchange step), so ``value`` is the total over ranks (weak scaling).  Time is
taken with CUDA events on the library's stream around each step; an L2 flush
(a 256 MiB write) runs between steps outside the timed intervals.

The CPU baseline (rank 0, one GPU only) times the complex128 oracle on all host
cores on a bounded sample of each workload: the same recipe (spacing, border
fraction, medium, beam, pole table) on a reduced grid, one z-step.  The GPU
then runs the same sample from the same inputs, and the relative L2 difference
of the two fields is reported with each leg.  ``--impl reference`` times the
oracle alone on such samples.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpoint·steps/s at 1024² scalar & 512² vector, learned vs plain, at 1e-5 L2 err"
UNIT = "Mpoint·steps/s"
DEFAULT_WORKLOAD = "batched_scalar_1024"
DEFAULT_EXTRA = "vector_random_512"
CONFIG_STEPS = {"homogeneous_aperture_1024": 100, "batched_scalar_1024": 200, "plain_scalar_64": 16,
                "vector_random_512": 150, "uneven_batch": 64}
DEFAULT_STEPS = {"homogeneous_aperture_1024": 20000, "plain_scalar_64": 2000, "uneven_batch": 6}
GATE_CYCLES = 400_000      # ~0.2 ms of GPU sleep before each timed step (outside the interval)
TABLE_OF = {"homogeneous_aperture_1024": "homogeneous_aperture_1024", "batched_scalar_1024": "batched_scalar_1024",
            "plain_scalar_64": "plain_scalar_64", "vector_random_512": "vector_random_512",
            "uneven_batch": "uneven_batch"}
# grid of the CPU sample of each workload (same recipe, reduced grid; None: the workload itself)
SAMPLE_N = {"batched_scalar_1024": 256, "vector_random_512": 128, "homogeneous_aperture_1024": 256,
            "plain_scalar_64": None, "uneven_batch": 128}
FP32_BAR = 1e-5


def make_workload(name: str, nsteps: int, n: int = 0):
    """The named workload; n > 0 shrinks a single-grid workload to n x n (same spacing, border fraction)."""
    from paper_2410_17446_gb300 import workloads as wl
    if name == "homogeneous_aperture_1024":
        return wl.homogeneous_aperture_1024(nsteps, **({"n": n} if n else {}))
    if name == "batched_scalar_1024":
        return wl.batched_scalar_1024(nsteps, **({"n": n} if n else {}))
    if name == "plain_scalar_64":
        return wl.plain_scalar_64(nsteps)
    if name == "vector_random_512":
        return wl.vector_random_512(nsteps, **({"n": n} if n else {}))
    if name == "uneven_batch":
        return wl.uneven_batch(nsteps=nsteps) if not n else wl.uneven_batch(nbeams=4, nsteps=nsteps, sizes=(n,))
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
# CPU baseline / reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time, os
sys.path.insert(0, {root!r})
import numpy as np
from oracle import aaa_lawson as al, propagator as pr, operators as ops
ops.FFT_WORKERS = {workers}
import bench
W = bench.make_workload({name!r}, {nsteps}, {n})
T = al.PoleTable.from_json(bench.load_table({name!r}))
fields = []
t0 = time.perf_counter(); pts = 0; its = []
for i, b in enumerate(W.beams):
    med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, W.ncomp)
    w = b.w0.copy()
    for s in range({nsteps}):
        if s > 0 and b.medium_changes(s):
            med = ops.Medium(b.medium(s), b.grid.dx, b.grid.dy, W.k0, W.n0, W.ncomp)
        w, st = pr.step(med, w, T, tol=1e-12)
        its += st.iterations
        pts += b.grid.nx * b.grid.ny
    fields.append(w)
el = time.perf_counter() - t0
if {out!r}:
    np.savez({out!r}, *fields)
print(json.dumps({{"seconds": el, "point_steps": pts, "mean_iters": float(np.mean(its))}}))
"""


def cpu_info() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "CPU part", "Hardware"):
            for ln in txt.splitlines():
                if ln.lower().startswith(key.lower()):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_oracle_sample(name: str, nsteps: int = 1, out: str = "") -> dict:
    """The oracle (complex128) on the CPU sample of `name`: its recipe on the SAMPLE_N grid,
    `nsteps` z-steps from the initial field, all host cores (scipy.fft workers and BLAS threads)."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    n = SAMPLE_N.get(name) or 0
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, nsteps=nsteps, n=n, workers=cores, out=out)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["value"] = d["point_steps"] / d["seconds"] / 1e6
    d["cores"] = cores
    W = make_workload(name, 1, n)
    grid = f"{W.beams[0].grid.nx}x{W.beams[0].grid.ny}"
    d["grid"] = grid
    d["sample"] = (f"{nsteps} z-step(s) of {name}'s recipe on a {grid} grid ({len(W.beams)} beam(s), "
                   f"{W.npoles} poles sequential, GMRES tol 1e-12, mean {d['mean_iters']:.1f} Arnoldi steps per "
                   f"pole) by the complex128 oracle, scipy.fft workers = BLAS threads = {cores} on "
                   f"{cpu_info()}, {d['seconds']:.1f} s")
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
    """The oracle, as it stands, on the host cores: K samples (one z-step of the
    workload's recipe on its reduced grid each), rank 0 only."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    steps = max(1, int(getattr(args, "steps", 1) or 1))
    warmup = max(0, int(getattr(args, "warmup", 0) or 0))
    for _ in range(warmup):   # untimed samples first, as for the GPU arm
        run_oracle_sample(args.workload, 1)
    secs, pts, its, d = 0.0, 0, [], None
    for _ in range(steps):
        d = run_oracle_sample(args.workload, 1)
        secs += d["seconds"]
        pts += d["point_steps"]
        its.append(d["mean_iters"])
    value = pts / secs / 1e6
    W = make_workload(args.workload, 1)
    sample = f"{steps} x [{d['sample']}]"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * secs / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "points_per_step": W.points,
                                            "poles": W.npoles, "sample_grid": d["grid"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": d["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f).get("hbm_gbs")
    except OSError:
        pk = None
    return (pk, "measured") if pk else (6800.0, "fallback")


def _tensor_peak():
    """Sustained dense BF16 tensor throughput of this GPU (TFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f).get("bf16_tflops_sustained")
    except OSError:
        pk = None
    return (pk, "measured (sustained)") if pk else (1700.0, "fallback (sustained)")


def roofline_of(name: str, prof: dict) -> dict:
    """HBM roofline of the kernel kind with the largest device time in the timed region:
    summed algorithmic bytes / summed CUDA-event durations of its launches."""
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"])
    peak, src = _peak()
    achieved = dom[1]["alg_bytes"] / (dom[1]["total_ms"] / 1e3) / 1e9 if dom[1]["total_ms"] > 0 else 0.0
    # DRAM bytes per launch from an ncu capture of the current kernel: stored as measured
    # DRAM bytes per algorithmic byte (a smaller capture, scaled to this launch's units)
    traffic = None
    alg_launch = dom[1]["alg_bytes"] / max(1, dom[1]["launches"])
    tpath = os.path.join(ROOT, "profiles", f"traffic_{name}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            t = json.load(f).get(dom[0])
        if isinstance(t, dict) and t.get("dram_per_alg_byte"):
            traffic = t["dram_per_alg_byte"] * alg_launch
    return {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": src,
            "alg_bytes_per_launch": alg_launch,
            "launches": dom[1]["launches"],
            "share_of_kernel_time": dom[1]["total_ms"] / max(1e-12, sum(v["total_ms"] for v in prof.values()))}


class Runner:
    """One workload on this rank's GPU: media resident on the device, timed legs."""

    def __init__(self, args, name, P, torch, dev, stream, ws, local):
        self.args, self.name, self.P, self.torch, self.dev, self.stream = args, name, P, torch, dev, stream
        self.ws, self.local = ws, local
        total = args.warmup + args.steps
        self.W = make_workload(name, max(total, 1), args.n)
        self.tab = load_table(name)
        self.grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in self.W.beams]
        self.media = {}
        for s in range(total):
            for i, b in enumerate(self.W.beams):
                if s == 0 or b.medium_changes(s):
                    self.media[(s, i)] = torch.tensor(b.medium(s), dtype=torch.complex128, device=dev)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.net = None

    def propagator(self, guess: str, W=None):
        P = self.P
        W = W or self.W
        grids = [(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in W.beams]
        with self.torch.cuda.stream(self.stream):
            pr = P.Propagator.from_table(grids, W.k0, W.n0, W.dz, self.tab, ncomp=W.ncomp, precision=P.PROP_FP32,
                                         restart=self.args.restart or W.restart, stream=self.stream,
                                         guess=P.PROP_GUESS_LEARNED if guess == "learned" else P.PROP_GUESS_ZERO,
                                         multigroup=self.args.multigroup == "on")
            if guess == "learned":
                net = self.load_net()
                pr.set_guess_net(net["channels"], net["weights"], net["biases"])
            for i, b in enumerate(W.beams):
                pr.set_field(i, np.ascontiguousarray(b.w0))
        return pr

    def load_net(self):
        if self.net is None:
            from paper_2410_17446_gb300 import guess_train as GT
            fam = "vector" if self.W.ncomp == 2 else "scalar"
            self.net = GT.load(os.path.join(ROOT, "paper_2410_17446_gb300", "nets", f"guess_{fam}.npz"))
        return self.net

    def timed(self, prx, clocks_on: bool) -> dict:
        """W warm-up steps; K steps timed by events on the library stream (the
        value); then the same K steps' media again with an event pair around every
        kernel launch (the per-kernel durations of the roofline).  The per-launch
        events are kept out of the value's pass: on the batched-scalar step they
        cost 13 % of the step time."""
        torch, args, stream, dev = self.torch, self.args, self.stream, self.dev

        def step_of(s):
            for i in range(len(self.W.beams)):
                m = self.media.get((s, i))
                if m is not None:
                    prx.set_medium(i, m)
            prx.step()

        def run_pass(reset_media):
            st_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            en_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            for k in range(args.steps):
                self.flush.zero_()
                # keep the GPU busy while the host enqueues the step, so that the
                # timed interval holds device work, not host launch latency
                torch.cuda._sleep(GATE_CYCLES)
                st_ev[k].record(stream)
                s = args.warmup + k
                if k == 0 and reset_media:   # the replay starts from the step's own media
                    for i, b in enumerate(self.W.beams):
                        prx.set_medium(i, self.media.get((s, i), self.last_medium(s, i)))
                    prx.step()
                else:
                    step_of(s)
                en_ev[k].record(stream)
            torch.cuda.synchronize(dev)
            return sum(a.elapsed_time(b) for a, b in zip(st_ev, en_ev))

        with torch.cuda.stream(stream):
            for s in range(args.warmup):
                step_of(s)
            torch.cuda.synchronize(dev)
            # the state the timed steps start from (the end-to-end pass replays them from it)
            start_fields = [prx.get_field(i) for i in range(len(self.W.beams))]
            l0 = prx.stats().kernel_launches
            it0 = prx.stats().total_iters
            clocks = ClockSampler(self.local) if clocks_on else None
            if self.ws > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            if clocks:
                clocks.start()
                time.sleep(0.3)
            t0 = time.perf_counter()
            dms = run_pass(False)
            t1 = time.perf_counter()
            clk = None
            if clocks:
                time.sleep(0.3)
                clk = clocks.stop(t0, t1)
            if self.ws > 1:
                torch.distributed.barrier()
            stx = prx.stats()
            iters = prx.iterations()
            # kernel pass
            prx.set_profiling(True)
            dms_k = run_pass(True)
            prof = prx.profile()
            prx.set_profiling(False)
        ms = max_over_ranks(dms, self.ws, dev)
        return {"dev_ms": ms, "kernel_pass_ms": dms_k, "wall": t1 - t0, "clk": clk, "prof": prof,
                "start_fields": start_fields,
                "launches": stx.kernel_launches - l0, "arnoldi": int(stx.total_iters - it0), "iters": iters}

    def last_medium(self, s, i):
        """The medium beam i holds at step s (its last change at or before s)."""
        for t in range(s, -1, -1):
            m = self.media.get((t, i))
            if m is not None:
                return m
        raise KeyError((s, i))

    def leg(self, guess: str, clocks_on: bool = False) -> dict:
        pr = self.propagator(guess)
        r = self.timed(pr, clocks_on)
        ms = r["dev_ms"]
        prof = r["prof"]
        d = {"value": whole_job_value(self.ws, self.W.points, self.args.steps, ms / 1e3),
             "ms_per_step": ms / self.args.steps,
             "roofline": dict(roofline_of(self.name, prof),
                              measured_in="kernel pass: the timed steps' media replayed with a CUDA-event pair "
                                          "around every launch on the library stream (a device spin heads each "
                                          "run of launches the host enqueues after a wait, so that the events "
                                          "time kernels, not submission)"),
             "arnoldi_steps_total": r["arnoldi"],
             "arnoldi_steps_per_solve": r["arnoldi"] / (self.args.steps * len(self.W.beams) * self.W.npoles),
             "gmres_last_step": {"sum": int(r["iters"].sum()), "max": int(r["iters"].max())},
             "gpu_launches": r["launches"],
             "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                             "GBps": (v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9) if v["total_ms"] > 0 else None}
                         for k, v in prof.items() if v["launches"]}}
        if guess == "learned":
            d["guess_net_ms"] = round(prof["guess_net"]["total_ms"], 3)
            # tensor-pipe view of the network: its 3x3 convolutions' FLOPs (the stored,
            # 16-padded channel counts the kernels compute) over every system's points,
            # against the sustained BF16 peak (the network runs inside a long step)
            ch = [int(c) for c in self.load_net()["channels"]]
            flop = 2 * 9 * sum(a * b for a, b in zip(ch[:-1], ch[1:])) * self.W.points * self.W.npoles * self.args.steps
            tf = flop / (prof["guess_net"]["total_ms"] / 1e3) / 1e12 if prof["guess_net"]["total_ms"] > 0 else 0.0
            tpk, tsrc = _tensor_peak()
            d["guess_net_tensor"] = {"bound": "tensor", "achieved": tf, "peak": tpk, "unit": "TFLOP/s",
                                     "frac": tf / tpk, "peak_source": tsrc, "flop_per_step": flop / self.args.steps}
            d["net"] = {k: v for k, v in self.load_net()["meta"].items()
                        if k in ("family", "n", "train_media_seeds", "solves", "adam_iterations")}
        self._last = (pr, r)
        return d

    def sample_error(self, guess: str, oracle_npz: str, nsteps: int = 1) -> dict:
        """GPU run of the CPU sample (reduced grid, same inputs) against the oracle's fields."""
        n = SAMPLE_N.get(self.name) or 0
        W = make_workload(self.name, nsteps, n)
        pr = self.propagator(guess, W)
        with self.torch.cuda.stream(self.stream):
            for s in range(nsteps):
                for i, b in enumerate(W.beams):
                    if s == 0 or b.medium_changes(s):
                        pr.set_medium(i, np.ascontiguousarray(b.medium(s)))
                pr.step()
            got = [pr.get_field(i) for i in range(len(W.beams))]
        pr.close()
        z = np.load(oracle_npz)
        ref = [z[f"arr_{i}"] for i in range(len(W.beams))]
        errs = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(got, ref)]
        return {"value": max(errs), "bar": FP32_BAR, "grid": f"{W.beams[0].grid.nx}x{W.beams[0].grid.ny}",
                "steps": nsteps, "against": "complex128 oracle (the cpu_baseline sample: same recipe, reduced grid)"}


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

    names = [args.workload] + [x for x in args.extra.split(",") if x and x != "none" and x != args.workload]
    guesses = ["plain", "learned"] if args.guess == "both" else ["plain"]

    # CPU samples first (all host cores; nothing on the GPU runs meanwhile)
    tmpdir = tempfile.mkdtemp(prefix="bench_oracle_")
    cpu = {}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        for nm in names:
            cpu[nm] = run_oracle_sample(nm, 1, os.path.join(tmpdir, nm + ".npz"))

    # FFT pass variants for the grid sizes in use: the committed plans measured on this
    # GPU model, else tuned here (prop_fft_autotune) before anything is timed
    from paper_2410_17446_gb300 import autotune as AT
    sizes = set()
    for nm in names:
        for b in make_workload(nm, 1, args.n).beams:
            sizes |= {b.grid.nx, b.grid.ny}
    plans = AT.load_or_tune(sizes, P.PROP_FP32, write=False, retune=args.retune)

    stream = torch.cuda.Stream(device=dev)
    legs = {}
    main = None
    for nm in names:
        R = Runner(args, nm, P, torch, dev, stream, ws, local)
        legs[nm] = {}
        for gi, guess in enumerate(guesses):
            d = R.leg(guess, clocks_on=(nm == args.workload and guess == "plain"))
            if nm in cpu:
                d["rel_l2_vs_oracle"] = R.sample_error(guess, os.path.join(tmpdir, nm + ".npz"))
            if nm == args.workload and guess == "plain":
                main = (R, d, R._last)
            else:
                R._last[0].close()
            legs[nm][guess] = d
        if nm != args.workload:
            del R
    R, d0, (pr, r0) = main
    W = R.W

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
        poles = np.array([complex(*p) for p in R.tab["poles"]])
        res = np.array([complex(*r) for r in R.tab["residues"]])
        Rz = complex(*R.tab["r0"]) + sum(r / (z - p) for p, r in zip(poles, res))
        ref = np.fft.ifft2(Rz ** total * np.fft.fft2(b.w0[0]))
        acc = float(np.linalg.norm(w - ref) / np.linalg.norm(ref))

    # end to end through the public API with host buffers (pinned): each step's medium
    # copied in and the field read back inside the timed region
    e2e = None
    if not args.no_e2e:
        host_out = [torch.empty(pr.shape(i), dtype=torch.complex128).pin_memory() for i in range(len(W.beams))]
        host_media = {key: m.cpu().pin_memory() for key, m in R.media.items() if key[0] >= args.warmup}
        h2d = d2h = 0
        with torch.cuda.stream(stream):
            # the same steps as the timed pass, from the same field
            for i in range(len(W.beams)):
                pr.set_field(i, torch.tensor(r0["start_fields"][i]).pin_memory())
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
        e2e = {"value": whole_job_value(ws, W.points, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    if rank == 0:
        line = {"metric": METRIC, "value": d0["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": d0["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "points_per_step": W.points, "beams": len(W.beams),
                           "grid": f"{W.beams[0].grid.nx}x{W.beams[0].grid.ny}", "poles": W.npoles,
                           "ncomp": W.ncomp, "restart": pr.opts.restart, "tol": pr.opts.tol,
                           "precond": "mean n^2" if pr.opts.precond == P.PROP_PRECOND_MEAN else "free space",
                           "l2": "flushed (256 MiB write) between timed steps",
                           "grids": len({(b.grid.nx, b.grid.ny, b.grid.dx, b.grid.dy) for b in W.beams}),
                           "multigroup": args.multigroup,
                           "parallelism": f"replicas x{ws}"},
                "roofline": d0["roofline"], "gpu_launches": d0["gpu_launches"], "clocks": r0["clk"],
                "wall_s": r0["wall"],
                "arnoldi_steps_total": d0["arnoldi_steps_total"],
                "rel_l2_vs_oracle": d0.get("rel_l2_vs_oracle"),
                "rel_err_vs_closed_form": acc,
                "rel_err_steps": CONFIG_STEPS[args.workload] if acc is not None else None,
                "legs": legs, "e2e": e2e,
                "fft_plans": {str(n): {k: r.get(k) for k in ("rows", "cols", "rows_small", "cols_small",
                                                              "round_trip_ms", "round_trip_ms_small", "source")}
                              for n, r in plans.items()}}
        if args.workload in cpu:
            c = cpu[args.workload]
            line["cpu_baseline"] = {"value": c["value"], "unit": UNIT, "cores": c["cores"], "kind": "oracle",
                                    "sample": c["sample"]}
            line["cpu_baseline_extra"] = {nm: {"value": c2["value"], "sample": c2["sample"]}
                                          for nm, c2 in cpu.items() if nm != args.workload}
        print(json.dumps(line), flush=True)
    pr.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20, enough for a timed region of a few seconds)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(TABLE_OF))
    ap.add_argument("--extra", default=DEFAULT_EXTRA,
                    help="comma-separated workloads measured beside the main one ('none' for none)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="shrink the grid (profiling runs only; not a bench line)")
    ap.add_argument("--restart", type=int, default=0, help="GMRES restart length (default: the workload's)")
    ap.add_argument("--retune", action="store_true", help="time the FFT variants here even if plans are cached")
    ap.add_argument("--multigroup", default="on", choices=["on", "off"],
                    help="on: grids of different sizes advance in lockstep, one launch per Arnoldi pass")
    ap.add_argument("--guess", default="both", choices=["plain", "both"],
                    help="both: also time the learned initial guess (GMRES to the same tolerance)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 20)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
