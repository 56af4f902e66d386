"""CPU checks of the serving loop's host logic (serve.Server.run) with the library
objects replaced by fakes: every request finishes; the batch admits by footprint and
a request that does not fit waits (FULL) and is admitted once memory returns;
retirement at the residual target or the step cap; the reported counts and latencies."""
import math

import pytest

from paper_2007_07347_gb300 import serve as V
from paper_2007_07347_gb300 import sdugks as S

FULL = next(code for code, name in S.ERRORS.items() if name == "FULL")


class FakeMesh:
    threads = set()

    def __init__(self, mesh, bcs):
        import threading
        self.n_cells = mesh.n_cells
        FakeMesh.threads.add(threading.get_ident())


class FakeBatch:
    """Capacity in cells; eps of an instance = 1 / (1 + steps / 1000)."""
    log = []

    def __init__(self, pool_bytes, precision, max_instances, stream=None):
        self.cap, self.used, self.items, self.next = pool_bytes, 0, {}, 0
        FakeBatch.log = []

    def add(self, mesh, tau, dt):
        if self.used + mesh.n_cells > self.cap:
            raise S.SdugksError(FULL, "sdugks_batch_add", "pool full")
        self.used += mesh.n_cells
        self.next += 1
        self.items[self.next] = [mesh.n_cells, 0]
        FakeBatch.log.append(("add", self.next, self.used))
        return self.next

    def step(self, n):
        for it in self.items.values():
            it[1] += n

    def residual(self):
        return {i: (1.0 / (1.0 + it[1] / 1000.0), 1.0, it[1]) for i, it in self.items.items()}

    def remove(self, ident):
        self.used -= self.items.pop(ident)[0]
        FakeBatch.log.append(("remove", ident, self.used))

    def macros(self, ident):
        return None

    def info(self):
        return {"instances": len(self.items), "cells": self.used}


class FakeSolver:
    def __init__(self, mesh, tau, dt, precision, stream=None):
        self.steps, self.closed = 0, False

    def init(self, rho, u):
        return self

    def step(self, n):
        self.steps += n

    def residual(self):
        return 1.0 / (1.0 + self.steps / 1000.0), 1.0

    def close(self):
        self.closed = True


@pytest.fixture
def fakes(monkeypatch):
    import torch
    monkeypatch.setattr(S, "Mesh", FakeMesh)
    monkeypatch.setattr(S, "Batch", FakeBatch)
    monkeypatch.setattr(S, "Solver", FakeSolver)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def _requests(n):
    reqs = V.Workload(n_requests=n, rate=1e6, cavity_n=(16, 48), couette_ny=(16, 48),
                      cylinder=((32, 16), (64, 32))).requests()
    return reqs


def test_every_request_finishes_and_the_pool_is_respected(fakes):
    reqs = _requests(40)
    cap = 6000                                     # cells: far fewer than the 40 requests need at once
    srv = V.Server(pool_bytes=cap, check_every=500, step_cap=3000, target=1e-9, solver_pool_bytes=1 << 40)
    out = srv.run(reqs)
    assert out["requests"] == 40 and out["converged"] == 0 and out["capped"] == 40
    assert all(r.status == "capped" and r.steps == 3000 for r in reqs)
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)
    assert max(used for _, _, used in FakeBatch.log) <= cap
    adds = [e for e in FakeBatch.log if e[0] == "add"]
    assert len(adds) == sum(r.kind != "cylinder" for r in reqs)
    first_remove = next(k for k, e in enumerate(FakeBatch.log) if e[0] == "remove")
    assert any(e[0] == "add" for e in FakeBatch.log[first_remove:])      # admitted once memory returned
    assert out["cell_steps"] == sum(3000 * r.case.mesh.n_cells for r in reqs)
    # capped requests are not solves: no throughput, no latency, the target not met
    assert out["solves_per_s"] == 0.0 and out["p50_latency_s"] is None and out["met_target"] is False


def test_retirement_at_the_residual_target(fakes):
    reqs = _requests(12)
    srv = V.Server(pool_bytes=1 << 40, check_every=500, step_cap=10 ** 6, target=0.5, solver_pool_bytes=1 << 40)
    out = srv.run(reqs)
    # eps = 1 / (1 + steps / 1000) falls below 0.5 after 1500 steps (three intervals)
    assert out["converged"] == 12 and out["met_target"] is True
    assert all(r.status == "converged" and r.steps == 1500 and r.eps < 0.5 for r in reqs)
    assert all(math.isfinite(r.done) for r in reqs)
    assert out["solves_per_s"] == pytest.approx(12 / out["wall_s"])
    assert 0 <= out["p50_latency_s"] <= out["p99_latency_s"]


def test_stats_count_converged_requests_only(fakes):
    """Mixed outcome: solves/s and the latency percentiles come from the converged
    requests alone; the capped ones are counted beside them."""
    reqs = _requests(10)
    for k, r in enumerate(reqs):
        r.build()
        r.status = "converged" if k < 6 else "capped"
        r.arrival, r.done = 0.0, 1.0 + k
    out = V.serve_stats(reqs, wall=4.0)
    assert out["converged"] == 6 and out["capped"] == 4 and out["met_target"] is False
    assert out["solves_per_s"] == pytest.approx(1.5)
    assert out["p99_latency_s"] <= 6.0 + 1e-12          # the capped requests' latencies (7-10 s) are left out


def test_a_residual_that_stops_falling_retires_as_stalled(fakes, monkeypatch):
    """A residual floor (eps constant at 0.5 after the first check) retires the request as
    stalled once `stall_checks` checks in a row bring no new minimum; it is not a solve."""
    monkeypatch.setattr(FakeBatch, "residual",
                        lambda self: {i: (0.5, 1.0, it[1]) for i, it in self.items.items()})
    monkeypatch.setattr(FakeSolver, "residual", lambda self: (0.5, 1.0))
    reqs = _requests(6)
    srv = V.Server(pool_bytes=1 << 40, check_every=500, step_cap=10 ** 6, target=1e-9, stall_checks=3,
                   solver_pool_bytes=1 << 40)
    out = srv.run(reqs)
    assert out["stalled"] == 6 and out["converged"] == 0 and out["met_target"] is False
    assert all(r.status == "stalled" and r.steps == 4 * 500 for r in reqs)   # the first check sets the minimum
    assert out["solves_per_s"] == 0.0


def test_meshes_are_built_off_the_loop_thread(fakes):
    """The arrivals' meshes are built on the worker threads (prep_threads > 0), and in the
    loop itself with prep_threads = 0; every request finishes either way."""
    import threading
    for workers in (4, 0):
        FakeMesh.threads = set()
        reqs = _requests(10)
        out = V.Server(pool_bytes=1 << 40, check_every=500, step_cap=3000, target=1e-9, prep_threads=workers,
                       solver_pool_bytes=1 << 40).run(reqs)
        assert out["capped"] == 10
        main = threading.get_ident() in FakeMesh.threads
        assert (not main) if workers else (FakeMesh.threads == {threading.get_ident()})

