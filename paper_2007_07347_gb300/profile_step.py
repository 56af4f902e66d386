"""Profiling driver: N separate step launches (no graph) of one case.

    python -m paper_2007_07347_gb300.profile_step CASE [PRECISION] [STEPS] [TILE] [STAGING]

CASE is one of cavity128, cavity256, cavity1024, cylinder (512 x 256 O-mesh),
microcavity (the rarefied solver: 40 x 40 cells, 100 x 100 velocities, Kn 1), batch
(the 256 cavities of the batched configuration, N ~ logU[32, 512], seed 1) or batchK
(the first K of those 256, e.g. batch32 for a capture that holds less device memory).  Used
under ncu with ``-k regex:k_step`` (``regex:k_dvm`` for the rarefied kernels) to
capture single step launches.  STAGING (Cartesian kernel): loads (default) or tma.
"""
import sys

import numpy as np
import torch

from . import meshes as M
from . import sdugks as S

CASES = {
    "cavity128": lambda: M.cavity(128),
    "cavity256": lambda: M.cavity(256),
    "cavity1024": lambda: M.cavity(1024),
    "cylinder": lambda: M.cylinder(512, 256),
}


def main(argv):
    name = argv[1] if len(argv) > 1 else "cavity256"
    prec = argv[2] if len(argv) > 2 else "fp32"
    nsteps = int(argv[3]) if len(argv) > 3 else 10
    tile = int(argv[4]) if len(argv) > 4 else 0
    staging = argv[5] if len(argv) > 5 else "loads"
    torch.cuda.set_device(0)
    if name.startswith("batch"):
        count = int(name[5:]) if len(name) > 5 else 256
        cases = [M.cavity(n, Re=re) for n, re in M.batch_cavities(256, seed=1)[:count]]
        meshes = [S.Mesh(c.mesh, c.bcs) for c in cases]
        probe = S.Batch(1 << 20, prec, 4)
        need = sum(probe.footprint(m) for m in meshes)
        probe.close()
        b = S.Batch(need + (64 << 20), prec, 512)
        for c, m in zip(cases, meshes):
            b.add(m, c.tau, c.dt)
        b.step(nsteps)
        torch.cuda.synchronize()
        print("batch", b.info())
        return
    if name == "microcavity":
        d = S.Dvm.from_case(M.micro_cavity(40, Kn=1.0), "fp64" if prec == "fp64" else "fp32", graph_steps=-1).init()
        d.step(nsteps)
        torch.cuda.synchronize()
        print("sizes", d.sizes())
        return
    case = CASES[name]()
    s = S.Solver.from_case(case, prec, graph_steps=-1, tile_cells=tile, staging=staging)
    u = None if case.u0 == (0.0, 0.0) else np.tile(case.u0, (case.mesh.n_cells, 1))
    s.init(None, u)
    s.step(nsteps)
    torch.cuda.synchronize()
    print("info", s.info())


if __name__ == "__main__":
    main(sys.argv)
