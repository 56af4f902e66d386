"""Full-length validation runs of the configurations, with the tolerances of the
scope stated beside each measured number.

    python -m paper_2007_07347_gb300.validate cylinder # 512x256 O-mesh Re 40 to steady state, FP64/FP32/bf16
    python -m paper_2007_07347_gb300.validate cylinder fp16dev   # the same for the listed storages only
    python -m paper_2007_07347_gb300.validate cylinder fp32 --max-steps 3000000   # a longer cap (default 600,000)
    python -m paper_2007_07347_gb300.validate shedding # 512x256 O-mesh Re 60/80/100: St and mean Cd
    python -m paper_2007_07347_gb300.validate plate    # laminar flat plate Re_L 1e5: Cd against Blasius

Writes one JSON line per case to stdout.  The comparison of the 256^2 cavity with the
FP64 oracle is test infrastructure and lives with the tests (tests/validate_cavity.py).
"""
import json
import math
import sys
import time

import numpy as np


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


def shedding_analysis(t, cd, cl, D=1.0, U=0.1, t_from=None):
    """Strouhal number and mean drag from a lift/drag history: upward zero crossings
    of Cl - mean(Cl) (linear interpolation) after t_from; St = D / (U T) with T the
    mean period; mean Cd and the Cl amplitude over the whole periods between the
    first and the last crossing."""
    t, cd, cl = map(np.asarray, (t, cd, cl))
    sel = t >= (t_from if t_from is not None else t[0])
    t, cd, cl = t[sel], cd[sel], cl[sel]
    c = cl - cl.mean()
    up = np.where((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(up) < 3:
        return {"St": math.nan, "Cd_mean": float(cd.mean()), "Cl_amp": 0.5 * float(cl.max() - cl.min()),
                "periods": max(len(up) - 1, 0)}
    tz = t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])
    T = (tz[-1] - tz[0]) / (len(tz) - 1)
    w = (t >= tz[0]) & (t <= tz[-1])
    return {"St": D / (U * T), "Cd_mean": float(cd[w].mean()), "Cl_amp": 0.5 * float(cl[w].max() - cl[w].min()),
            "periods": len(tz) - 1, "period_spread": float(np.std(np.diff(tz)) / T)}


def cylinder_unsteady(Re=100.0, n_theta=512, n_r=256, first=0.005, r_far=50.0, t_end=1000.0, t_from=600.0,
                      sample_dt=0.25, precision="fp32"):
    """Vortex shedding behind the cylinder: start from the free stream plus a small
    deterministic asymmetric kick in the near wake, record Cd, Cl from the wall
    momentum flux every sample_dt, and analyse the periodic state after t_from."""
    import torch
    from . import meshes as M
    from . import sdugks as S
    torch.cuda.set_device(0)
    case = M.cylinder(n_theta, n_r, Re=Re, first=first, r_far=r_far)
    U, D = case.meta["U"], 1.0
    meta = case.mesh.meta
    radii = meta["radii"]
    rc = 0.5 * (radii[:-1] + radii[1:])
    th = 2.0 * math.pi * (meta["cell_i"] + 0.5) / meta["n_theta"]
    r = rc[meta["cell_k"]]
    x, y = r * np.cos(th), r * np.sin(th)
    u = np.tile(np.asarray(case.u0, np.float64), (case.mesh.n_cells, 1))
    u[:, 1] += 0.1 * U * np.exp(-((x - 1.5) ** 2 + y ** 2))
    s = S.Solver.from_case(case, precision).init(None, u)
    every = max(2, int(round(sample_dt / case.dt)))
    n_samples = int(t_end / (every * case.dt))
    t, cd, cl = [], [], []
    t0 = time.perf_counter()
    for q in range(n_samples):
        s.step(every - 1)
        F = s.step_forces()
        t.append((q + 1) * every * case.dt)
        cd.append(F[0, 0] / (0.5 * U * U * D))
        cl.append(F[0, 1] / (0.5 * U * U * D))
    wall = time.perf_counter() - t0
    eps, _ = s.residual()
    out = shedding_analysis(t, cd, cl, D, U, t_from)
    St_fit = -3.3265 / Re + 0.1816 + 1.6e-4 * Re
    paper = {60.0: (1.4228, 0.1377), 80.0: (1.375, 0.1523), 100.0: (1.349, 0.1653)}.get(float(Re))
    out.update({"case": f"cylinder {n_theta}x{n_r} O-mesh Re {Re:g} (r_far {r_far:g}, first {first:g})",
                "precision": precision, "steps": n_samples * every, "t_end": t[-1], "t_from": t_from,
                "wall_s": wall, "cell_steps_per_s": case.mesh.n_cells * n_samples * every / wall,
                "St_fit_parallel_shedding": St_fit, "finite": bool(np.isfinite(eps) or eps == math.inf)})
    if paper:
        out.update({"paper_Cd_mean": paper[0], "paper_St": paper[1]})
    return out


def shedding(res=(60.0, 80.0, 100.0)):
    for Re in res:
        print(json.dumps(cylinder_unsteady(Re)), flush=True)


def flat_plate_run(nx_up=24, nx_plate=72, ny=64, t_end=3000.0, precision="fp32", interval=20000):
    """Laminar flat plate at Re_L = 1e5 to steady state: drag of the plate (one side)
    against the Blasius value 1.328 / sqrt(Re_L), and the wall shear along it."""
    import torch
    from . import meshes as M
    from . import sdugks as S
    torch.cuda.set_device(0)
    case = M.flat_plate(nx_up, nx_plate, ny)
    U, L, Re = case.meta["U"], case.meta["L"], case.meta["Re_L"]
    u = np.tile(np.asarray(case.u0, np.float64), (case.mesh.n_cells, 1))
    s = S.Solver.from_case(case, precision).init(None, u)
    steps, hist = 0, []
    t0 = time.perf_counter()
    n_int = int(t_end / case.dt / interval) + 1
    for _ in range(n_int):
        s.step(interval - 1)
        F = s.step_forces()
        steps += interval
        eps, _ = s.residual()
        hist.append((steps * case.dt, eps, F[4, 0] / (0.5 * U * U * L)))
    wall = time.perf_counter() - t0
    cd = hist[-1][2]
    blasius = 1.328 / math.sqrt(Re)
    return {"case": f"flat plate {case.mesh.n_cells} cells, Re_L {Re:g}, U {U}", "precision": precision,
            "steps": steps, "t": steps * case.dt, "eps_last": hist[-1][1], "Cd": cd, "Cd_blasius": blasius,
            "Cd_rel_diff": cd / blasius - 1.0, "paper_Cd": 4.237e-3, "wall_s": wall,
            "history_Cd": [h[2] for h in hist[-5:]]}


def plate():
    print(json.dumps(flat_plate_run()), flush=True)


if __name__ == "__main__":
    argv = sys.argv[1:]
    max_steps = 600000
    if "--max-steps" in argv:                              # e.g. cylinder fp32 --max-steps 3000000
        i = argv.index("--max-steps")
        max_steps = int(argv[i + 1])
        argv = argv[:i] + argv[i + 2:]
    what = argv[0] if argv else "cylinder"
    if what == "shedding" and len(argv) > 1:
        shedding(tuple(float(x) for x in argv[1:]))
    elif what == "cylinder":
        precisions = tuple(argv[1:]) or ("fp64", "fp32", "bf16dev")   # e.g. cylinder fp16dev bf16dev
        cylinder(max_steps=max_steps, precisions=precisions)
    else:
        {"shedding": shedding, "plate": plate}[what]()
