"""Full-length validation of the 256^2 lid-driven cavity (Re 1000, lid 0.1): 20,000 FP32
steps of the library against the FP64 oracle from the same initial state, with the
tolerances stated beside each measured number (relative L2 of u, centreline profiles
over U, mass drift of both).  Test infrastructure: needs a GPU; run from the repository
root as

    python tests/validate_cavity.py [steps]

Writes one JSON line to stdout.
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def cavity(steps=20000):
    import torch
    import oracle as O
    from paper_2007_07347_gb300 import meshes as M
    from paper_2007_07347_gb300 import sdugks as S
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


if __name__ == "__main__":
    cavity(int(sys.argv[1]) if len(sys.argv) > 1 else 20000)
