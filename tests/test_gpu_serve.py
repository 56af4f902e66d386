"""Continuous batching: requests that arrive while others run are admitted as memory
frees up, their work overlaps on the device (batched uniform grids on one stream,
tiled cylinder solvers on another), and each result is the same as the same request
run alone for the same number of steps (bit for bit: within one kernel an instance's
arithmetic does not depend on the rest of the mix)."""
import numpy as np
import pytest

from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_runs():
    import torch
    from paper_2007_07347_gb300 import sdugks as S
    from paper_2007_07347_gb300 import serve as V
    torch.cuda.set_device(0)
    wl = V.Workload(n_requests=10, rate=400.0, cavity_n=(24, 48), cavity_re=(50.0, 200.0), couette_ny=(16, 32),
                    cylinder=((32, 16), (48, 24)), cylinder_re=(10.0, 20.0), seed=7)
    reqs = wl.requests()
    assert {r.kind for r in reqs} >= {"cavity", "couette"}
    # a pool that holds only a few instances at a time: later requests wait for memory
    probe = S.Batch(1 << 20, "fp32", 4)
    fp = max(probe.footprint(S.Mesh(r.build().mesh, r.case.bcs)) for r in reqs if r.kind != "cylinder")
    srv = V.Server(pool_bytes=3 * fp, precision="fp32", max_instances=16, target=1e-4, check_every=200,
                   step_cap=1200, keep_results=True)
    sb, ss = torch.cuda.Stream(), torch.cuda.Stream()
    out = srv.run(reqs, stream_batch=sb, stream_solvers=ss)
    assert out["requests"] == 10 and out["converged"] + out["capped"] == 10
    assert max(r.admitted for r in reqs) > min(r.done for r in reqs)     # admissions after retirements
    for r in reqs:
        case = r.case
        if r.kind == "cylinder":
            s = S.Solver.from_case(case, "fp32")
            s.init(None, np.tile(case.u0, (case.mesh.n_cells, 1)))
            s.step(r.steps)
            rho, u = s.macros()
        else:
            b = S.Batch(fp + (1 << 20), "fp32", 2)
            i = b.add_case(case)
            b.step(r.steps)
            rho, u = b.macros(i)
        np.testing.assert_array_equal(rho, r.result[0])
        np.testing.assert_array_equal(u, r.result[1])
