"""Full-length validation runs of the configurations, with the tolerances of the
scope stated beside each measured number.

    python -m paper_2007_07347_gb300.validate cavity   # 256^2 Re 1000, 20k FP32 steps vs the FP64 oracle
    python -m paper_2007_07347_gb300.validate cylinder # 512x256 O-mesh Re 40 to steady state, FP64/FP32/bf16

Writes one JSON line per case to stdout.  The oracle (test infrastructure) is used
only as the reference of the cavity comparison.
"""
import json
import math
import sys
import time

import numpy as np


def cavity(steps=20000):
    import torch
    import oracle as O
    from . import meshes as M
    from . import sdugks as S
    torch.cuda.set_device(0)
    case = M.cavity(256)
    s = S.Solver.from_case(case, "fp32").init()
    _, m0 = s.residual()
    t0 = time.perf_counter()
    s.step(steps)
    rho, u = s.macros()
    t_gpu = time.perf_counter() - t0
    _, m1 = s.residual()
    st = O.init(case.mesh.n_cells)
    vol = O.geometry(case.mesh, case.bcs)["vol"]
    mo0 = float(vol @ st.W[:, 0])
    t0 = time.perf_counter()
    O.run(case, st, steps)
    t_cpu = time.perf_counter() - t0
    mo1 = float(vol @ st.W[:, 0])
    U = case.meta["U"]
    n = 256
    ug, uo = u.reshape(n, n, 2), st.u.reshape(n, n, 2)
    # vertical centreline u(y) at x = L/2 and horizontal centreline v(x) at y = L/2
    # (mean of the two cell columns/rows either side of the centre line)
    cu_g = 0.5 * (ug[:, n // 2 - 1, 0] + ug[:, n // 2, 0])
    cu_o = 0.5 * (uo[:, n // 2 - 1, 0] + uo[:, n // 2, 0])
    cv_g = 0.5 * (ug[n // 2 - 1, :, 1] + ug[n // 2, :, 1])
    cv_o = 0.5 * (uo[n // 2 - 1, :, 1] + uo[n // 2, :, 1])
    out = {"case": "cavity 256x256 Re 1000 lid 0.1, FP32 vs FP64 oracle", "steps": steps,
           "rel_l2_u": float(np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2))), "tol_rel_l2_u": 1e-4,
           "centreline_max_err_over_U": float(max(np.abs(cu_g - cu_o).max(), np.abs(cv_g - cv_o).max()) / U),
           "tol_centreline_over_U": 1e-4,
           "mass_drift_gpu": (m1 - m0) / m0, "mass_drift_oracle": (mo1 - mo0) / mo0,
           "max_rho_diff": float(np.abs(rho - st.W[:, 0]).max()),
           "gpu_s": t_gpu, "oracle_s": t_cpu, "oracle_threads": O.set_threads(0)}
    print(json.dumps(out), flush=True)


def cylinder(max_steps=600000, interval=5000, target=1e-7, precisions=("fp64", "fp32", "bf16dev")):
    import torch
    from . import meshes as M
    from . import sdugks as S
    torch.cuda.set_device(0)
    case = M.cylinder(512, 256)
    U, D, R = case.meta["U"], 1.0, 0.5
    meta = case.mesh.meta
    res = {}
    for prec in precisions:
        u0 = np.tile(case.u0, (case.mesh.n_cells, 1))
        s = S.Solver.from_case(case, prec).init(None, u0)
        t0 = time.perf_counter()
        steps, eps = 0, math.inf
        hist = []
        while steps < max_steps:
            s.step(interval - 1)
            F = s.step_forces()
            steps += interval
            eps, _ = s.residual()
            hist.append((steps, eps, F[0, 0] / (0.5 * U * U * D), F[0, 1] / (0.5 * U * U * D)))
            if eps < target:
                break
        wall = time.perf_counter() - t0
        rho, u = s.macros()
        # recirculation length on the wake axis (theta = 0): mean of the cells either side
        nt = meta["n_theta"]
        radii = meta["radii"]
        rc = 0.5 * (radii[:-1] + radii[1:])
        ax = np.zeros(len(rc))
        for i_side in (0, nt - 1):
            sel = meta["cell_i"] == i_side
            order = np.argsort(meta["cell_k"][sel])
            ax += 0.5 * u[sel][order][:, 0]
        neg = np.where(ax < 0)[0]
        lr = math.nan
        if len(neg):
            k = neg[-1]
            if k + 1 < len(ax):
                r0 = rc[k] + (rc[k + 1] - rc[k]) * (-ax[k]) / (ax[k + 1] - ax[k])
                lr = (r0 - R) / R
        cd, cl = hist[-1][2], hist[-1][3]
        res[prec] = {"steps": steps, "eps": eps, "Cd": cd, "Cl": cl, "L_over_R": lr, "wall_s": wall,
                     "cell_steps_per_s": case.mesh.n_cells * steps / wall}
        print(json.dumps({"case": "cylinder 512x256 O-mesh Re 40", "precision": prec, **res[prec],
                          "paper_Cd": 1.557, "paper_L_over_R": 4.490}), flush=True)
    if "fp64" in res:
        for prec in res:
            if prec != "fp64":
                print(json.dumps({"precision": prec, "Cd_rel_diff_vs_fp64": res[prec]["Cd"] / res["fp64"]["Cd"] - 1,
                                  "tol_bf16_Cd": 0.01}), flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "cavity"
    {"cavity": cavity, "cylinder": cylinder}[what]()
