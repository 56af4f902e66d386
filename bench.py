"""Benchmark of the S-DUGKS D2Q9 step on one GB300 (or N replicas, one per GPU).

Workload (default): the lid-driven cavity of 256 x 256 unit cells, Re 1000, lid
U = 0.1, CFL 0.5, f stored in FP32, started from rest (the configuration the metric is
quoted on).  One benchmark step is five residual intervals: 5 x (1000 fused S-DUGKS
time steps, steps 1-11 of Sec. II, each one kernel launch, replayed from captured CUDA
graphs, then the FP64 residual and mass reduction of Sec. IV).  The launch
configuration (block shape, staging, graph length) is the autotuner's choice.

Metric: MLUPS = cells x 9 velocities x time steps / s / 1e6 ("cell-Q updates").
The device-timed region starts with f, W resident in HBM; L2 is flushed (a 256 MB
buffer is rewritten) before every timed step, outside its events.  The state of
this case is 7.9 MB, so inside a step the launches run from L2 (the roofline object
says so: "l2_resident").

The same line carries the other single-GPU configurations, each timed the same way
and with its own roofline ("configs"): the 512 x 256 cylinder O-mesh (bf16-deviation
storage, unstructured tiled kernel) and the batch of 256 cavities (11.7 M cells,
1.4 GB of state: HBM-resident).

e2e: the same metric through the C-ABI from pinned host buffers: each step uploads
the full state (f, W in FP64), advances the time steps, runs the residual and reads
rho and u back.

--impl reference: the FP64 C oracle, as it stands, on the host cores, on bounded
samples of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_07347_gb300 import meshes as M  # noqa: E402

INTERVAL = 1000            # time steps per residual check (Sec. IV)
INTERVALS_PER_STEP = 5     # residual intervals per benchmark step
STATE_BYTES = {"fp64": 192, "fp32": 120, "bf16dev": 84, "fp16dev": 84}    # f and W (FP64) each read and written once
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=17)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "bf16dev", "fp16dev"],
                    help="storage of f (default: fp32; bf16dev for the cylinder)")
    ap.add_argument("--n", type=int, default=256, help="cavity cells per side")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="cavity",
                    choices=["cavity", "cylinder", "batch", "batch-solve", "serve", "rarefied"],
                    help="cavity: the headline single solve; cylinder: the 512 x 256 O-mesh (shuffled, "
                         "unstructured kernel); batch: 256 cavities in one batch against the plain "
                         "one-at-a-time path; serve: the continuous-batching request loop; rarefied: the "
                         "40x40 micro cavity on a 100x100 velocity grid (Kn 1)")
    ap.add_argument("--tile-cells", type=int, default=0,
                    help="block / tile size of the solver (0: the solver's own choice)")
    ap.add_argument("--staging", default=None, choices=["loads", "tma"],
                    help="cavity: how the Cartesian kernel stages its interior blocks (per-thread loads or "
                         "TMA tensor copies; default: the autotuner's choice)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="the solver's own launch configuration instead of the autotuner's")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other single-GPU configurations (cylinder, batch) in the default line")
    ap.add_argument("--target", type=float, default=1e-6, help="batch-solve / serve: residual target")
    ap.add_argument("--cap-steps", type=int, default=400000, help="batch-solve: steps before an instance is capped")
    ap.add_argument("--stall-checks", type=int, default=50,
                    help="batch-solve: residual checks without a 1 %% lower minimum before an instance is "
                         "retired as stalled at its floor")
    ap.add_argument("--plain-sample", type=int, default=16,
                    help="batch-solve: converged instances solved again one at a time (plain path) and as "
                         "their own batch, for the solves/s comparison; serve: requests solved one at a time "
                         "(0: every request)")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--step-cap", type=int, default=400000, help="serve: steps before a request is reported capped")
    ap.add_argument("--serve-sizes", default="config", choices=["config", "small"],
                    help="serve: the configuration's size ranges, or smaller ones the box finishes in minutes")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "bf16dev" if args.workload == "cylinder" else "fp32"
    return args


def workload(args):
    if args.workload == "cylinder":
        return M.cylinder(512, 256)
    return M.cavity(args.n, U=0.1, Re=1000.0, cfl=0.5)


def workload_name(args):
    if args.workload == "cylinder":
        return ("cylinder O-mesh 512x256 (r 0.5-50, first cell 0.005), Re 40, U 0.1, far field + no-slip wall, "
                "cell ids shuffled (seed 0), from uniform flow")
    return f"lid-driven cavity {args.n}x{args.n}, Re 1000, lid 0.1, CFL 0.5, from rest"


def workload_tag(args):
    return "cylinder512x256" if args.workload == "cylinder" else f"cavity{args.n}"


def initial_u(case):
    """Uniform initial velocity of the case (None: at rest)."""
    if tuple(case.u0) == (0.0, 0.0):
        return None
    return np.tile(np.asarray(case.u0, dtype=np.float64), (case.mesh.n_cells, 1))


def config(args, case):
    state_mb = STATE_BYTES[args.precision] * case.mesh.n_cells / 1e6
    return {"workload": workload_name(args),
            "cells": case.mesh.n_cells, "velocities": 9, "time_steps_per_step": INTERVAL * INTERVALS_PER_STEP,
            "storage": args.precision, "tau": case.tau, "dt": case.dt,
            "l2": f"flushed (256 MB rewrite) before each timed step; the {state_mb:.1f} MB state is L2-resident "
                  f"within a step",
            "parallelism": f"replicas x{args.gpus}"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers

def max_over_ranks(value: float, world: int) -> float:
    """The largest value over all ranks (each rank's timed-region duration); the
    process group must be initialised when world > 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STEP_SOURCES = {
    "k_step_cart": ["d2q9.cuh", "sdugks_internal.h", "step_cart.cuh", "k_cart.cu"],
    "k_step_tiled": ["d2q9.cuh", "sdugks_internal.h", "step_tiled.cuh", "k_step_fp32.cu"],
    "k_step_batch": ["d2q9.cuh", "sdugks_internal.h", "step_cart.cuh", "k_batch.cu"],
}


def kernel_source_hash(kernel: str = "k_step_cart"):
    """Hash of the sources a step kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_07347_gb300", "csrc")
    for name in STEP_SOURCES[kernel]:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_key)
        kernel = next(k for k in STEP_SOURCES if kernel_key.startswith(k))
        if e and e.get("source_hash") == kernel_source_hash(kernel):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def cpu_baseline(case, seconds: float):
    """The FP64 oracle as it stands on this host's cores, on a bounded sample: as many
    10-step chunks of the workload as fit in about `seconds`."""
    import oracle as O
    threads = O.set_threads(0)
    st = O.init(case.mesh.n_cells, u=initial_u(case))
    O.run(case, st, 1)                       # geometry warm-up, untimed
    steps, t0 = 0, time.perf_counter()
    while True:
        O.run(case, st, 10)
        steps += 10
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    mlups = case.mesh.n_cells * 9 * steps / el / 1e6
    # the same oracle on one thread, a short sample
    O.set_threads(1)
    t0 = time.perf_counter()
    O.run(case, st, 2)
    el1 = time.perf_counter() - t0
    O.set_threads(threads)
    return {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{steps} time steps of the same {case.mesh.n_cells}-cell workload "
                      f"({el:.1f} s, {threads} OpenMP threads, FP64)",
            "single_thread_value": case.mesh.n_cells * 9 * 2 / el1 / 1e6}


# ----------------------------------------------------------------------------- arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    case = workload(args)
    threads = O.set_threads(0)
    st = O.init(case.mesh.n_cells, u=initial_u(case))
    sample = 10                              # time steps per benchmark step
    for _ in range(args.warmup):
        O.run(case, st, sample)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.run(case, st, sample)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    mlups = case.mesh.n_cells * 9 * sample * args.steps / tot / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config(args, case), time_steps_per_step=sample,
                                                l2="n/a (CPU)", parallelism="host cores"),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"{sample} time steps per benchmark step, {threads} OpenMP threads"},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def make_solver(S, case, args, precision, stream, cartesian_options=True):
    """The solver of a workload: the autotuner's launch configuration, unless one was
    given on the command line (or --no-autotune)."""
    if args.no_autotune or args.tile_cells or (args.staging and cartesian_options):
        kw = {"tile_cells": args.tile_cells}
        if cartesian_options and args.staging:
            kw["staging"] = args.staging
        return S.Solver.from_case(case, precision, stream=stream, **kw), None
    s = S.Solver.tuned(case, precision, stream=stream)
    return s, s.tune


def time_steps(s, steps, warmup, stream, flush, clk=None):
    """Benchmark steps of INTERVALS_PER_STEP x (INTERVAL time steps + residual), L2
    flushed before each: per-step ms, mean ms per step launch, last (eps, mass)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            for _ in range(INTERVALS_PER_STEP):
                s.step(INTERVAL)
                s.residual()
        torch.cuda.synchronize()
        E = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
        ev = [(E(), E(), [(E(), E()) for _ in range(INTERVALS_PER_STEP)]) for _ in range(steps)]
        last = None
        if clk:
            clk.__enter__()
        try:
            for k in range(steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                for a, b in ev[k][2]:
                    a.record(stream)
                    s.step(INTERVAL)
                    b.record(stream)
                    last = s.residual()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        finally:
            if clk:
                clk.__exit__(None, None, None)
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    launch_ms = float(np.mean([a.elapsed_time(b) / INTERVAL for e in ev for a, b in e[2]]))
    return step_ms, launch_ms, last


def roofline_of(info, precision, n, launch_ms, key):
    """Roofline of the step kernel: algorithmic bytes (state read and written once, plus
    the mesh data an unstructured step must read) over the mean launch time."""
    peak, peak_kind = measured_peaks()
    mesh_b = info["mesh_bytes_per_cell_step"] if info["kernel"] == 1 else 0.0
    alg_bytes = (STATE_BYTES[precision] + mesh_b) * n
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    kname = {1: "k_step_tiled", 2: "k_step_cart"}[info["kernel"]]
    resident = (STATE_BYTES[precision] + mesh_b) * n < 0.8 * L2_BYTES
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profiled_traffic(key), "kernel": kname, "algorithmic_bytes_per_launch": alg_bytes,
            "state_bytes_per_cell_step": STATE_BYTES[precision], "mesh_bytes_per_cell_step": mesh_b,
            "avg_launch_us": launch_ms * 1e3, "peak_kind": f"{peak_kind} (hbm_gbs)",
            "l2_resident": resident,
            "note": ("state and mesh fit in L2 (129 MB) and stay there within a benchmark step: achieved counts "
                     "algorithmic bytes, DRAM moves less (traffic)") if resident else
                    "state larger than L2: every launch streams it from HBM"}


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2007_07347_gb300 import sdugks as S
    S.lib()
    case = workload(args)
    n = case.mesh.n_cells
    stream = torch.cuda.Stream()
    s, tune = make_solver(S, case, args, args.precision, stream, cartesian_options=args.workload == "cavity")
    s.init(None, initial_u(case))
    info = s.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    barrier()
    clk = ClockSampler(torch.cuda.current_device())
    step_ms, launch_ms, last = time_steps(s, args.steps, args.warmup, stream, flush, clk)
    barrier()
    total_ms = max_over_ranks(sum(step_ms), world)
    tsteps = INTERVAL * INTERVALS_PER_STEP
    value = n * 9 * tsteps * args.steps * world / (total_ms / 1e3) / 1e6

    # ---- e2e through the C-ABI with pinned host buffers
    f_h = torch.empty((n, 9), dtype=torch.float64).pin_memory().numpy()
    W_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    rho_h = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    u_h = torch.empty((n, 2), dtype=torch.float64).pin_memory().numpy()
    s.get_state_into(f_h, W_h)
    e2e_steps = max(3, min(args.steps, 10))
    import ctypes as C
    L = S.lib()
    P = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S._ck(L.sdugks_set_state(s._h, P(f_h), P(W_h)), "set_state")
        for _ in range(INTERVALS_PER_STEP):
            S._ck(L.sdugks_step(s._h, INTERVAL), "step")
            s.residual()
        S._ck(L.sdugks_get_macros(s._h, P(rho_h), P(u_h)), "get_macros")
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_val = n * 9 * tsteps * e2e_steps * world / e2e_s / 1e6

    configs = {}
    if args.workload == "cavity" and not args.no_configs and args.n == 256 and args.precision == "fp32":
        configs = other_configs(args, S, stream, flush)
    if rank != 0:
        return
    key = f"{ {1: 'k_step_tiled', 2: 'k_step_cart'}[info['kernel']] }_{args.precision}_{workload_tag(args)}"
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16dev": "f32 (bf16 storage)", "fp16dev": "f32 (fp16 storage)"}[args.precision],
        "data": "synthetic", "config": config(args, case),
        "roofline": roofline_of(info, args.precision, n, launch_ms, key),
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": n * 12 * 8,
                "d2h_bytes_per_step": n * 3 * 8 + 32 * INTERVALS_PER_STEP, "steps": e2e_steps},
        "gpu_launches": args.steps * INTERVALS_PER_STEP * (INTERVAL + 2),
        "residual_last": last[0], "mass_last": last[1],
        "solver": {k: info[k] for k in ("n_tiles", "halo_cells", "mesh_bytes_per_cell_step", "kernel", "tile_cells",
                                        "staging", "one_code_path")},
        "autotune": tune,
        "mcell_steps_per_s": value / 9,
    }
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if configs:
        line["configs"] = configs
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(case, args.cpu_seconds)
    print(json.dumps(line))


def other_configs(args, S, stream, flush):
    """The other single-GPU configurations, each timed like the headline (CUDA events on
    the launching stream, L2 flushed before each timed step): the cylinder O-mesh in
    bf16-deviation storage on the unstructured kernel, and the batch of 256 cavities."""
    import torch
    out = {}
    # -- cylinder: 512 x 256 O-mesh, Re 40, far field at 50 D, ids shuffled, from the free stream
    case = M.cylinder(512, 256)
    n = case.mesh.n_cells
    s, tune = make_solver(S, case, args, "bf16dev", stream, cartesian_options=False)
    s.init(None, initial_u(case))
    info = s.info()
    steps = max(3, min(args.steps, 10))
    clk = ClockSampler(torch.cuda.current_device())
    step_ms, launch_ms, last = time_steps(s, steps, 2, stream, flush, clk)
    tsteps = INTERVAL * INTERVALS_PER_STEP
    out["cylinder_512x256_bf16dev"] = {
        "workload": "cylinder O-mesh 512x256 (r 0.5-50, first cell 0.005), Re 40, U 0.1, far field + no-slip wall, "
                    "cell ids shuffled (seed 0), from uniform flow; f as bf16 deviation, FP32 compute",
        "value": n * 9 * tsteps * steps / (sum(step_ms) / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
        "time_steps_per_step": tsteps, "ms_per_step": sum(step_ms) / steps, "cells": n,
        "roofline": roofline_of(info, "bf16dev", n, launch_ms, f"k_step_tiled_bf16dev_cylinder512x256"),
        "autotune": tune, "residual_last": last[0], "clocks": clk.summary(),
        "gpu_launches": steps * INTERVALS_PER_STEP * (INTERVAL + 2)}
    s.close()
    # -- batch: 256 cavities, N ~ logU[32, 512], Re ~ logU[100, 5000] (seed 1), FP32, 11.7 M cells
    specs = M.batch_cavities(256, seed=1)
    cases = [M.cavity(nn, Re=re) for nn, re in specs]
    cells = sum(c.mesh.n_cells for c in cases)
    probe = S.Batch(1 << 20, "fp32", 4)
    meshes = [S.Mesh(c.mesh, c.bcs) for c in cases]
    need = sum(probe.footprint(m) for m in meshes)
    probe.close()
    b = S.Batch(need + (64 << 20), "fp32", 512, stream=stream)
    for c, m in zip(cases, meshes):
        b.add(m, c.tau, c.dt)
    b.autotune(2)
    interval, bsteps = 100, 5
    with torch.cuda.stream(stream):
        b.step(2 * interval)
        b.residual()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(torch.cuda.current_device())
        with clk:
            e0.record(stream)
            for _ in range(bsteps):
                b.step(interval)
                b.residual()
            e1.record(stream)
            torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    peak, peak_kind = measured_peaks()
    alg = 120.0 * cells
    launch_s = t / (interval * bsteps)               # the residual reductions are included
    out["batch_256_cavities_fp32"] = {
        "workload": "batch of 256 lid-driven cavities, N~logU[32,512], Re~logU[100,5000], seed 1, lid 0.1, CFL 0.5, "
                    "FP32, one batched launch per step over the (instance, 16x8 block) work list",
        "value": cells * 9 * interval * bsteps / t / 1e6, "unit": "MLUPS", "steps": bsteps,
        "time_steps_per_step": interval, "ms_per_step": 1e3 * t / bsteps, "cells": cells,
        "roofline": {"bound": "hbm", "achieved": alg / launch_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / launch_s / 1e9 / peak, "traffic": profiled_traffic("k_step_batch_fp32_batch256"),
                     "kernel": "k_step_batch",
                     "algorithmic_bytes_per_launch": alg, "avg_launch_us": launch_s * 1e6,
                     "peak_kind": f"{peak_kind} (hbm_gbs)", "l2_resident": False,
                     "note": "1.4 GB of state: every launch streams it from HBM; the launch time includes the share "
                             "of the per-instance residual reductions (one per 100 steps)"},
        "batch": b.info(), "clocks": clk.summary(),
        "gpu_launches": bsteps * (interval + 2)}
    b.close()
    return out


def run_batch(args):
    """256 lid-driven cavities (N ~ logU[32, 512], Re ~ logU[100, 5000], seed 1, lid 0.1,
    CFL 0.5, FP32) advanced together, against the plain path (each solved alone)."""
    import torch
    from paper_2007_07347_gb300 import sdugks as S
    torch.cuda.set_device(0)
    specs = M.batch_cavities(256, seed=1)
    cases = [M.cavity(n, Re=re) for n, re in specs]
    cells = sum(c.mesh.n_cells for c in cases)
    stream = torch.cuda.Stream()
    probe = S.Batch(1 << 20, args.precision, 4)
    need = sum(probe.footprint(S.Mesh(c.mesh, c.bcs)) for c in cases)
    b = S.Batch(need + (64 << 20), args.precision, 512, stream=stream)
    for c in cases:
        b.add_case(c)
    b.autotune(2)
    interval = 100
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step(interval)
            b.residual()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            b.step(interval)
            b.residual()
        e1.record(stream)
        torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    batch_mlups = cells * 9 * interval * args.steps / t_batch / 1e6
    # plain path: each instance alone (same kernel family, one solver per case), 2 x 64 steps each
    plain_steps = 128
    t_plain = 0.0
    with torch.cuda.stream(stream):
        for c in cases:
            s = S.Solver.from_case(c, args.precision, stream=stream).init()
            s.step(64)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(plain_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            t_plain += e0.elapsed_time(e1) / 1e3
            s.close()
    plain_mlups = cells * 9 * plain_steps / t_plain / 1e6
    info = b.info()
    print(json.dumps({"metric": "MLUPS", "value": batch_mlups, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps, "higher_is_better": True,
                      "dtype": args.precision, "data": "synthetic",
                      "config": {"workload": "batch of 256 lid-driven cavities, N~logU[32,512], Re~logU[100,5000], "
                                             "seed 1, FP32", "cells": cells, "time_steps_per_step": interval},
                      "plain_path_mlups": plain_mlups, "batched_over_plain": batch_mlups / plain_mlups,
                      "batch": info}))


class Retire:
    """Stopping rule of a batched or plain solve, checked every INTERVAL steps (Sec. IV
    residual): converged below the target; stalled when `stall` checks in a row bring no
    new minimum 1 % below the previous one (the FP32 state has reached the floor of its
    rounding noise); capped at `cap` steps."""

    def __init__(self, target, cap, stall):
        self.target, self.cap, self.stall = target, cap, stall
        self.best, self.since = math.inf, 0

    def __call__(self, eps, steps):
        if eps < self.target:
            return "converged"
        if not (eps == math.inf or eps == eps):        # NaN
            return "diverged"
        if eps < 0.99 * self.best:
            self.best, self.since = eps, 0
        else:
            self.since += 1
        if self.since >= self.stall:
            return "stalled"
        if steps >= self.cap:
            return "capped"
        return None


def batch_to_target(S, cases, args, stream, label=""):
    """Advance the cases as one batch until each retires (Retire); per instance: status,
    steps, wall time at retirement, last and lowest residual."""
    import torch
    probe = S.Batch(1 << 20, "fp32", 4)
    meshes = [S.Mesh(c.mesh, c.bcs) for c in cases]
    need = sum(probe.footprint(m) for m in meshes)
    probe.close()
    b = S.Batch(need + (64 << 20), "fp32", max(512, len(cases)), stream=stream)
    ids = {b.add(m, c.tau, c.dt): k for k, (c, m) in enumerate(zip(cases, meshes))}
    b.autotune(2)
    rules = {k: Retire(args.target, args.cap_steps, args.stall_checks) for k in range(len(cases))}
    out = [None] * len(cases)
    cell_steps = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        while ids:
            cell_steps += INTERVAL * sum(cases[k].mesh.n_cells for k in ids.values())
            b.step(INTERVAL)
            res = b.residual()
            for i, (eps, _, st) in res.items():
                k = ids[i]
                why = rules[k](eps, st)
                if why:
                    out[k] = {"status": why, "steps": st, "wall_s": time.perf_counter() - t0, "eps": eps,
                              "eps_min": min(rules[k].best, eps)}
                    b.remove(i)
                    del ids[i]
    wall = time.perf_counter() - t0
    b.close()
    return out, wall, cell_steps


def plain_to_target(S, case, args, stream):
    """One instance alone on the plain FP32 path (its own solver, default launch
    configuration), with the same stopping rule."""
    import torch
    s = S.Solver.from_case(case, "fp32", stream=stream).init(None, initial_u(case))
    rule = Retire(args.target, args.cap_steps, args.stall_checks)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    while True:
        s.step(INTERVAL)
        steps += INTERVAL
        eps, _ = s.residual()
        why = rule(eps, steps)
        if why:
            break
    wall = time.perf_counter() - t0
    s.close()
    return {"status": why, "steps": steps, "wall_s": wall, "eps": eps}


def run_batch_solve(args):
    """The batch of 256 lid-driven cavities (N ~ logU[32, 512], Re ~ logU[100, 5000], seed 1,
    FP32) run to the per-instance residual target with retirement, and, on a seeded sample
    of the instances that converged, the same solves one at a time on the plain path and
    as their own batch: solves/s at equal accuracy (the same stopping rule)."""
    import torch
    from paper_2007_07347_gb300 import sdugks as S
    torch.cuda.set_device(0)
    specs = M.batch_cavities(256, seed=1)
    cases = [M.cavity(nn, Re=re) for nn, re in specs]
    stream = torch.cuda.Stream()
    res, wall, cell_steps = batch_to_target(S, cases, args, stream)
    conv = [k for k, r in enumerate(res) if r["status"] == "converged"]
    stalled = [k for k, r in enumerate(res) if r["status"] == "stalled"]
    tts = np.array([res[k]["wall_s"] for k in conv])
    full = {"instances": len(cases), "cells": sum(c.mesh.n_cells for c in cases), "wall_s": wall,
            "converged": len(conv), "stalled": len(stalled),
            "capped": sum(r["status"] == "capped" for r in res), "diverged": sum(r["status"] == "diverged" for r in res),
            "solves_per_s": len(conv) / wall,
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if len(tts) else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if len(tts) else None,
            "mlups": 9 * cell_steps / wall / 1e6,
            "stalled_floor": ({"eps_min_lo": min(res[k]["eps_min"] for k in stalled),
                               "eps_min_hi": max(res[k]["eps_min"] for k in stalled)} if stalled else None),
            "per_instance": [{"N": specs[k][0], "Re": round(specs[k][1], 1), **{kk: (round(v, 4) if isinstance(v, float)
                              else v) for kk, v in res[k].items()}} for k in range(len(cases))]}
    # equal-accuracy comparison on a seeded sample of the converged instances
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(conv, size=min(args.plain_sample, len(conv)), replace=False).tolist()) if conv else []
    cmp = None
    if sample:
        sub = [cases[k] for k in sample]
        bres, bwall, _ = batch_to_target(S, sub, args, stream)
        pres = [plain_to_target(S, c, args, stream) for c in sub]
        pwall = sum(r["wall_s"] for r in pres)
        cmp = {"sample": [{"N": specs[k][0], "Re": round(specs[k][1], 1)} for k in sample],
               "batched": {"wall_s": bwall, "converged": sum(r["status"] == "converged" for r in bres),
                           "solves_per_s": sum(r["status"] == "converged" for r in bres) / bwall},
               "plain": {"wall_s": pwall, "converged": sum(r["status"] == "converged" for r in pres),
                         "solves_per_s": sum(r["status"] == "converged" for r in pres) / pwall},
               "steps_batched": [r["steps"] for r in bres], "steps_plain": [r["steps"] for r in pres]}
        cmp["batched_over_plain"] = cmp["batched"]["solves_per_s"] / max(cmp["plain"]["solves_per_s"], 1e-30)
    print(json.dumps({"metric": "solves/s", "value": full["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
                      "higher_is_better": True, "data": "synthetic", "dtype": "f32",
                      "config": {"workload": "batch of 256 lid-driven cavities, N~logU[32,512], Re~logU[100,5000], "
                                             "seed 1, lid 0.1, CFL 0.5, FP32, to eps < target (check every 1000 steps)",
                                 "target": args.target, "cap_steps": args.cap_steps,
                                 "stall_checks": args.stall_checks},
                      "batch": full, "equal_accuracy": cmp}))


def run_serve(args):
    """Continuous-batching request loop on the config-shaped request mix (seed 2): Poisson
    arrivals at 200/s of 60/30/10 cavities / Couette channels / cylinder O-meshes, each run
    to the residual target (stopping rule of Retire: converged, stalled, capped).  With
    --serve-sizes small the size ranges are those the box finishes in minutes (cavities
    32^2-128^2, Couette 4x32-4x256, cylinders 128x64; Re ranges unchanged).  A seeded
    sample of the requests is then solved one at a time on the plain FP32 path with the
    same stopping rule (solves/s at equal accuracy)."""
    import torch
    from paper_2007_07347_gb300 import serve as V
    from paper_2007_07347_gb300 import sdugks as S
    torch.cuda.set_device(0)
    if args.serve_sizes == "small":
        wl = V.Workload(n_requests=args.requests, cavity_n=(32, 128), couette_ny=(32, 256),
                        cylinder=((128, 64), (128, 64)))
        sizes = "cavities 32^2-128^2 Re 100-5000 / Couette 4x32-4x256 Re 10 / cylinders 128x64 Re 10-100"
    else:
        wl = V.Workload(n_requests=args.requests)
        sizes = "cavities 64^2-1024^2 Re 100-5000 / Couette 4x64-4x1024 Re 10 / cylinders 128x64-512x256 Re 10-100"
    reqs = wl.requests()
    srv = V.Server(pool_bytes=16 << 30, precision=args.precision, target=args.target, check_every=INTERVAL,
                   step_cap=args.step_cap, stall_checks=args.stall_checks)
    sb = torch.cuda.Stream()
    ss = [torch.cuda.Stream() for _ in range(8)]          # single (tiled) solvers take these in turn
    out = srv.run(reqs, stream_batch=sb, stream_solvers=ss)
    out["cell_steps_per_s"] = out["cell_steps"] / out["wall_s"]
    out["mlups"] = 9 * out["cell_steps_per_s"] / 1e6
    out["by_kind"] = {k: {st: sum(r.kind == k and r.status == st for r in reqs)
                          for st in ("converged", "stalled", "capped", "diverged")}
                      for k in ("cavity", "couette", "cylinder")}
    # equal accuracy: the same requests solved one at a time on the plain FP32 path with the
    # same stopping rule (every request, or a seeded sample with --plain-sample > 0)
    rng = np.random.default_rng(11)
    pick = (list(range(len(reqs))) if args.plain_sample <= 0 else
            sorted(rng.choice(len(reqs), size=min(args.plain_sample, len(reqs)), replace=False).tolist()))
    stream = torch.cuda.Stream()
    plain = [plain_to_target(S, reqs[i].build(), args, stream) for i in pick]
    p_wall = sum(p["wall_s"] for p in plain)
    n_ok = sum(p["status"] == "converged" for p in plain)
    same = sum(p["status"] == reqs[i].status for p, i in zip(plain, pick))
    out["equal_accuracy"] = {
        "requests": len(pick), "same_outcome": same,
        "plain": {"wall_s": p_wall, "converged": n_ok, "solves_per_s": n_ok / p_wall if p_wall > 0 else 0.0},
        "served_over_plain_solves_per_s": (out["solves_per_s"] / (n_ok / p_wall)) if n_ok else None,
        "steps_differ": sum(p["steps"] != reqs[i].steps for p, i in zip(plain, pick))}
    out["config"] = {"workload": f"{args.requests} Poisson requests (200/s, seed 2), 60/30/10 {sizes}, target "
                                 f"{args.target}, residual checked every {INTERVAL} steps, cap {args.step_cap} steps, "
                                 f"stalled after {args.stall_checks} checks without a 1 % lower minimum",
                     "precision": args.precision}
    print(json.dumps(out))


def run_rarefied(args):
    """Micro cavity of Sec. IV: 40 x 40 cells, 100 x 100 velocities on [-2, 2]^2, Kn = 1,
    diffuse walls, lid 0.1, FP32 f.  One benchmark step = 200 time steps (2 launches
    each, face and cell kernels, graphs of 32 steps; the cell kernel leaves the next
    step's fbar+).  MLUPS counts cell-velocity updates (Q = 10^4)."""
    import torch
    from paper_2007_07347_gb300 import sdugks as S
    torch.cuda.set_device(0)
    case = M.micro_cavity(40, Kn=1.0)
    prec = "fp32" if args.precision == "bf16dev" else args.precision
    stream = torch.cuda.Stream()
    d = S.Dvm.from_case(case, prec, stream=stream).init()
    sz = d.sizes()
    n, Q, nf = sz["n_cells"], sz["Q"], sz["n_faces"]
    interval = 200
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            d.step(interval)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        with ClockSampler(torch.cuda.current_device()) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                d.step(interval)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
    ms = [e[0].elapsed_time(e[1]) for e in ev]
    tot_s = sum(ms) / 1e3
    value = n * Q * interval * args.steps / tot_s / 1e6
    step_s = tot_s / (interval * args.steps)
    rs = 8 if prec == "fp64" else 4
    alg = n * Q * 2 * rs + n * 4 * 8 * 2              # f read and written once, W read and written
    scratch = (n * Q * 2 + nf * Q * 3) * rs            # fbar+ (write, read) and face fluxes (write, read twice)
    peak, peak_kind = measured_peaks()
    # e2e: through the C-ABI, the macroscopic state read back to the host every benchmark step
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 4))
    for _ in range(e2e_steps):
        d.step(interval)
        d.macros()
    e2e_s = time.perf_counter() - t0
    rho, u, RT = d.macros()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        threads = O.set_threads(0)
        mt = case.meta
        xi, wq = O.dvm_grid(mt["nv"], mt["vmax"])
        st = O.dvm_init(n, xi, wq, RT0=mt["RT0"])
        O.dvm_run(case.mesh, case.bcs, st, xi, wq, mt["RT0"], case.tau, case.dt, 1)     # warm-up, untimed
        steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
            O.dvm_run(case.mesh, case.bcs, st, xi, wq, mt["RT0"], case.tau, case.dt, 1)
            steps += 1
        el = time.perf_counter() - t0
        cpu = {"value": n * Q * steps / el / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{steps} time steps of the same micro cavity ({el:.1f} s, {threads} OpenMP threads, FP64)"}
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS (cell-velocity updates, Q = 10^4)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "rarefied micro cavity 40x40, 100x100 velocities on [-2,2]^2, Kn 1, lid 0.1, "
                                   "diffuse walls", "cells": n, "velocities": Q, "time_steps_per_step": interval,
                       "storage": prec, "tau": case.tau, "dt": case.dt,
                       "l2": "flushed (256 MB rewrite) before each timed step; f, fbar+ and the face fluxes "
                             f"({(2 * n + nf) * Q * rs / 1e6:.0f} MB) exceed L2"},
            "roofline": {"bound": "hbm", "achieved": alg / step_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / step_s / 1e9 / peak, "traffic": None,
                         "kernel": "one time step (k_dvm_face + k_dvm_cell)",
                         "algorithmic_bytes_per_launch": alg, "scratch_bytes_per_step": scratch,
                         "avg_step_us": step_s * 1e6, "peak_kind": f"{peak_kind} (hbm_gbs)"},
            "e2e": {"value": n * Q * interval * e2e_steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": n * 4 * 8},
            "gpu_launches": 2 * interval * args.steps,
            "max_u_over_lid": float(np.abs(u).max() / 0.1), "mass": float(rho.sum())}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch-solve":
        run_batch_solve(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "rarefied":
        run_rarefied(args)
    else:
        run_ours(args)           # cavity or cylinder


if __name__ == "__main__":
    main()
