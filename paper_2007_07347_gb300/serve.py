"""Continuous-batching request loop over the batched S-DUGKS solver.

Requests (seeded Poisson arrivals of a mix of lid-driven cavities, Couette channels
and cylinder O-meshes) are admitted while their device-memory footprint fits: uniform
grids join one `Batch` (one kernel launch per step over every admitted instance) and
cylinder O-meshes run as tiled single solvers on a second CUDA stream, so their work
overlaps on the GPU.  Every `check_every` steps the residual of each running solve is
read; solves whose residual is below `target` retire as converged, and so do, as not
converged, solves that reached `step_cap`, whose residual stopped falling (no new minimum
1 % below the last one for `stall_checks` checks: the floor of the FP32 state's rounding
noise, or an unsteady flow) or that diverged; each frees its memory for queued requests.
Latency is retire time minus arrival time.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import meshes as M
from . import sdugks as S


@dataclass
class Request:
    rid: int
    kind: str            # "cavity" | "couette" | "cylinder"
    size: tuple
    re: float
    arrival: float
    case: M.Case = None
    admitted: float = math.nan
    done: float = math.nan
    steps: int = 0
    eps: float = math.inf
    status: str = "queued"   # queued | running | converged | capped | stalled | diverged
    eps_best: float = math.inf
    stall: int = 0
    handle: object = None
    result: tuple = None
    mesh: object = None      # the library mesh (built once, while the GPU steps)

    def build(self):
        if self.case is None:
            if self.kind == "cavity":
                self.case = M.cavity(self.size[0], Re=self.re)
            elif self.kind == "couette":
                self.case = M.couette(self.size[1], nx=self.size[0], Re=self.re)
            else:
                self.case = M.cylinder(self.size[0], self.size[1], Re=self.re, first=0.005,
                                       r_far=50.0, shuffle_seed=None)
        return self.case


@dataclass
class Workload:
    """Request generator: arrival rate, mix and size/Re ranges (seeded)."""
    n_requests: int = 1000
    rate: float = 200.0
    mix: tuple = (0.6, 0.3, 0.1)
    cavity_n: tuple = (64, 1024)
    cavity_re: tuple = (100.0, 5000.0)
    couette_ny: tuple = (64, 1024)
    couette_re: float = 10.0
    cylinder: tuple = ((128, 64), (512, 256))
    cylinder_re: tuple = (10.0, 100.0)
    seed: int = 2

    def requests(self) -> list:
        rng = np.random.default_rng(self.seed)
        t = 0.0
        out = []

        def logu(lo, hi):
            return math.exp(rng.uniform(math.log(lo), math.log(hi)))

        for i in range(self.n_requests):
            t += rng.exponential(1.0 / self.rate)
            k = rng.choice(3, p=np.asarray(self.mix) / sum(self.mix))
            if k == 0:
                n = int(round(logu(*self.cavity_n)))
                out.append(Request(i, "cavity", (n, n), logu(*self.cavity_re), t))
            elif k == 1:
                ny = int(round(logu(*self.couette_ny)))
                out.append(Request(i, "couette", (4, ny), self.couette_re, t))
            else:
                a = logu(self.cylinder[0][0], self.cylinder[1][0])
                nt = int(round(a / 16)) * 16
                nr = max(16, nt // 2)
                out.append(Request(i, "cylinder", (nt, nr), logu(*self.cylinder_re), t))
        return out


@dataclass
class Server:
    pool_bytes: int = 8 << 30
    precision: str = "fp32"
    max_instances: int = 4096
    target: float = 1e-6
    check_every: int = 1000
    step_cap: int = 200000
    stall_checks: int = 0    # 0: no stall rule
    prep_threads: int = 4    # host threads that build the arrivals' meshes (0: in the loop)
    solver_pool_bytes: int = 4 << 30
    keep_results: bool = False
    log: list = field(default_factory=list)

    def run(self, requests: list, stream_batch=None, stream_solvers=None) -> dict:
        """stream_solvers: one stream, or a list of streams that the single (tiled) solvers
        take in turn, so that the steps of several small solves run at the same time."""
        import torch
        from concurrent.futures import ThreadPoolExecutor
        batch = S.Batch(self.pool_bytes, self.precision, self.max_instances, stream=stream_batch)
        solver_bytes = 0
        # mesh building of the arrivals (the case's arrays, then sdugks_mesh_create, which
        # runs without the interpreter lock) on worker threads, off the loop's path
        workers = ThreadPoolExecutor(self.prep_threads) if self.prep_threads > 0 else None
        prep = {}

        def prepare(r):
            case = r.build()
            if r.mesh is None:
                r.mesh = S.Mesh(case.mesh, case.bcs)
            return r
        queue = sorted(requests, key=lambda r: r.arrival)
        pending = list(queue)
        running = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        idle_waits = 0
        while pending or running:
            # advance everything running by one residual interval (asynchronous; the two
            # streams overlap), then prepare and admit arrivals while the GPU works
            stepped = list(running)
            for r in stepped:
                if r.handle[0] == "solver":
                    r.handle[1].step(self.check_every)
            if stepped:
                batch.step(self.check_every)
            arrived = [r for r in pending if r.arrival <= now()]
            for r in arrived:                    # host-side mesh work, overlapping the steps
                if workers is None:
                    prepare(r)
                elif r.rid not in prep:
                    prep[r.rid] = workers.submit(prepare, r)
            # admit every arrived request that is prepared and whose footprint fits (FIFO,
            # skipping ahead); adding to the batch waits for the interval in flight on its stream
            for r in arrived:
                if workers is not None:
                    fu = prep[r.rid]
                    if not fu.done():
                        continue
                    fu.result()                  # re-raises a failure of the mesh set-up
                case, m = r.case, r.mesh
                if r.kind == "cylinder":
                    need = 400 * case.mesh.n_cells          # state + mesh data, tiled FP32 path
                    if solver_bytes + need > self.solver_pool_bytes:
                        continue
                    pool = stream_solvers if isinstance(stream_solvers, (list, tuple)) else [stream_solvers]
                    s = S.Solver(m, case.tau, case.dt, self.precision, stream=pool[r.rid % len(pool)])
                    s._mesh = m
                    s.init(None, np.tile(case.u0, (case.mesh.n_cells, 1)))
                    r.handle = ("solver", s, need)
                    solver_bytes += need
                else:
                    try:
                        ident = batch.add(m, case.tau, case.dt)
                    except S.SdugksError as e:
                        if e.name == "FULL":
                            continue
                        raise
                    r.handle = ("batch", ident)
                r.admitted = now()
                r.status = "running"
                pending.remove(r)
                running.append(r)
            if not stepped:
                if not running:
                    nxt = min(r.arrival for r in pending)
                    time.sleep(max(0.0, min(0.01, nxt - now())) if nxt > now() else 0.001)
                    idle_waits += 1
                continue
            res = batch.residual()
            for r in stepped:
                if r.handle[0] == "solver":
                    try:
                        eps, _ = r.handle[1].residual()
                    except S.SdugksError as e:
                        if e.name != "DIVERGED":
                            raise
                        eps = math.nan
                    r.steps += self.check_every
                else:
                    eps, _, r.steps = res[r.handle[1]]
                r.eps = eps
                diverged = math.isnan(eps)
                if eps < 0.99 * r.eps_best:
                    r.eps_best, r.stall = eps, 0
                else:
                    r.stall += 1
                stalled = self.stall_checks > 0 and r.stall >= self.stall_checks
                if eps < self.target or r.steps >= self.step_cap or diverged or stalled:
                    r.status = ("converged" if eps < self.target else "diverged" if diverged
                                else "stalled" if stalled else "capped")
                    if self.keep_results:
                        r.result = (r.handle[1].macros() if r.handle[0] == "solver" else batch.macros(r.handle[1]))
                    if r.handle[0] == "solver":
                        solver_bytes -= r.handle[2]
                        r.handle[1].close()
                    else:
                        batch.remove(r.handle[1])
                    r.handle = None
                    r.mesh = None
                    r.done = now()
                    running.remove(r)
        wall = now()
        torch.cuda.synchronize()
        if workers is not None:
            workers.shutdown()
        return {**serve_stats(requests, wall), "batch": batch.info()}


def serve_stats(requests: list, wall: float) -> dict:
    """Throughput and latency of a finished run.  Only requests that reached the residual
    target count as solves: solves/s and the p50/p99 latencies are taken over the
    converged requests; requests stopped at the step cap (or diverged) are counted
    beside them, and ``met_target`` is False when any request did not converge."""
    conv = [r for r in requests if r.status == "converged"]
    lat = np.array([r.done - r.arrival for r in conv])
    out = {"requests": len(requests), "converged": len(conv),
           "capped": sum(r.status == "capped" for r in requests),
           "stalled": sum(r.status == "stalled" for r in requests),
           "diverged": sum(r.status == "diverged" for r in requests),
           "met_target": len(conv) == len(requests),
           "wall_s": wall, "solves_per_s": len(conv) / wall if wall > 0 else 0.0,
           "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
           "cell_steps": int(sum(r.steps * r.case.mesh.n_cells for r in requests))}
    return out
