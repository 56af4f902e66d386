"""Boundary momentum flux of the CUDA path (forces of Sec. IV: C_d, C_l, C_p) against the
FP64 oracle, face by face and patch by patch, through the C-ABI.

Tolerances (written next to each check):
* FP64: max |gpu - oracle| over the faces <= 1e-12 max |oracle| (the patch sums use
  atomics on the GPU, so their last bits vary from run to run).
* FP32 and bf16-deviation storage: stated per test, with the measured values.
* Unsteady cylinder (Re 200, past the onset of shedding): the lift and drag series of
  the GPU in FP64 within 1e-10 of the oracle's, relative to the largest value.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


def _S():
    from paper_2007_07347_gb300 import sdugks as S
    return S


def _sym_channel():
    mesh = M.cartesian(37, 23, 37.0, 23.0)
    bcs = [(0, M.BC_MOVING_WALL, (0.05, 0.0, 0.0)), (1, M.BC_OUTLET, (0, 0, 0)),
           (2, M.BC_SYMMETRY, (0, 0, 0)), (3, M.BC_SYMMETRY, (0, 0, 0))]
    return M.Case("sym_channel", mesh, bcs, tau=0.05, dt=0.25)


def _mixed3():
    mesh = M.cartesian(3, 3, 3.0, 1.5)
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.1, 0, 0)), (3, M.BC_FARFIELD, (1, 0.05, 0)),
           (1, M.BC_OUTLET, (0, 0, 0))]
    return M.Case("mixed3", mesh, bcs, tau=0.1, dt=0.25)


CASES = {
    "cavity_48": (lambda: M.cavity(48, Re=400.0), 200),
    "cylinder_64x32_shuffled": (lambda: M.cylinder(64, 32, first=0.01, r_far=10.0, shuffle_seed=3), 300),
    "symmetry_channel_37x23": (_sym_channel, 150),
    "mixed_bc_3x3": (_mixed3, 20),
    "flat_plate_32x16": (lambda: M.flat_plate(8, 24, 16, Re_L=2e3, h_le=0.5, h_wall=0.2), 200),
    "couette_4x64": (lambda: M.couette(64), 500),
}


def _u0(case):
    return None if case.u0 == (0.0, 0.0) else np.tile(case.u0, (case.mesh.n_cells, 1))


def _patch_sums(case, F):
    bf = O.boundary_faces(case.mesh, case.bcs)
    patch = -1 - np.asarray(case.mesh.neighbour)[bf]
    out = np.zeros((64, 2))
    np.add.at(out, patch, F)
    return out


@pytest.mark.parametrize("kernel", ["auto", "tiled"])
@pytest.mark.parametrize("name", list(CASES))
def test_fp64_boundary_flux_matches_oracle(name, kernel):
    """After `steps` steps, one more step's momentum flux through every boundary face
    and its patch sums: FP64 within 1e-12 of the oracle (on uniform grids with the
    Cartesian and the tiled kernel)."""
    S = _S()
    make, steps = CASES[name]
    case = make()
    u = _u0(case)
    s = S.Solver.from_case(case, "fp64", kernel={"auto": 0, "tiled": 1}[kernel]).init(None, u)
    s.step(steps)
    Fg, Pg = s.step_boundary_flux(forces=True)
    st = O.init(case.mesh.n_cells, u=u)
    O.run(case, st, steps)
    Fo = O.run_flux(case, st, 1)
    assert Fg.shape == Fo.shape and len(Fo) == s.info()["n_boundary_faces"]
    scale = np.abs(Fo).max()
    assert np.abs(Fg - Fo).max() <= 1e-12 * scale
    Po = _patch_sums(case, Fo)
    assert np.abs(Pg - Po).max() <= 1e-12 * np.abs(Po).max()
    # the step taken is an ordinary step: the state still matches the oracle
    f, W = s.get_state()
    assert np.abs(W - st.W).max() <= 1e-12 * np.abs(st.W).max()


@pytest.mark.parametrize("kernel", ["auto", "tiled"])
def test_patch_forces_are_sums_of_face_fluxes(kernel):
    """sdugks_step_forces and the face rows of sdugks_step_boundary_flux describe the same
    step: on two identical solvers, the patch sums of the face rows equal the patch
    forces (FP32 rows summed in FP64 on the host against FP64 atomics: 1e-6 of the
    largest patch force)."""
    S = _S()
    case = M.cavity(64, Re=400.0)
    a = S.Solver.from_case(case, "fp32", kernel={"auto": 0, "tiled": 1}[kernel]).init()
    b = S.Solver.from_case(case, "fp32", kernel={"auto": 0, "tiled": 1}[kernel]).init()
    a.step(300)
    b.step(300)
    P = a.step_forces()
    F = b.step_boundary_flux()
    Ps = _patch_sums(case, F)
    assert np.abs(Ps - P).max() <= 1e-6 * np.abs(P).max()


def test_cylinder_wall_cp_and_forces_fp32_against_oracle():
    """The cylinder case's diagnostics on a 128 x 64 O-mesh after 1500 steps in FP32:
    the surface pressure coefficient C_p = (F . n / l - rho_inf c_s^2) / (0.5 rho_inf U^2)
    on every wall face within 1e-3 of the oracle's (absolute; C_p is of order 1), and
    C_d, C_l (wall patch sums over 0.5 rho U^2 D) within 1e-3 absolute."""
    S = _S()
    case = M.cylinder(128, 64, first=0.01, r_far=20.0)
    U = case.meta["U"]
    u0 = np.tile(case.u0, (case.mesh.n_cells, 1))
    s = S.Solver.from_case(case, "fp32").init(None, u0)
    s.step(1500)
    Fg = s.step_boundary_flux()
    st = O.init(case.mesh.n_cells, u=u0)
    O.run(case, st, 1500)
    Fo = O.run_flux(case, st, 1)
    bf = O.boundary_faces(case.mesh, case.bcs)
    wall = (-1 - np.asarray(case.mesh.neighbour)[bf]) == case.mesh.patches["wall"]
    nl = O.geometry(case.mesh, case.bcs)["nl"][bf[wall]]
    ln = np.hypot(nl[:, 0], nl[:, 1])

    def cp(F):
        return (np.einsum("ij,ij->i", F[wall], nl) / ln ** 2 - CS2) / (0.5 * U * U)

    cp_g, cp_o = cp(Fg), cp(Fo)
    assert cp_o.max() > 0.5                       # the front stagnation region
    assert np.abs(cp_g - cp_o).max() <= 1e-3
    cd = [F[wall, 0].sum() / (0.5 * U * U) for F in (Fg, Fo)]
    cl = [F[wall, 1].sum() / (0.5 * U * U) for F in (Fg, Fo)]
    assert abs(cd[0] - cd[1]) <= 1e-3 and abs(cl[0] - cl[1]) <= 1e-3


def test_cylinder_full_size_bf16dev_drag_within_one_percent_of_oracle():
    """The cylinder configuration in bf16-deviation storage (512 x 256 shuffled O-mesh,
    Re 40, far field at 50 D) after 3000 steps from the free stream: the wall patch's C_d
    within 1 % of the FP64 oracle's C_d after the same steps, and C_l within 1e-2
    absolute (C_l is 0 by symmetry)."""
    S = _S()
    case = M.cylinder(512, 256)
    U = case.meta["U"]
    u0 = np.tile(case.u0, (case.mesh.n_cells, 1))
    s = S.Solver.from_case(case, "bf16dev").init(None, u0)
    s.step(2999)
    Pg = s.step_forces()
    st = O.init(case.mesh.n_cells, u=u0)
    O.run(case, st, 2999)
    Po = _patch_sums(case, O.run_flux(case, st, 1))
    w = case.mesh.patches["wall"]
    cd_g, cd_o = Pg[w, 0] / (0.5 * U * U), Po[w, 0] / (0.5 * U * U)
    print(f"cylinder 512x256 bf16dev, 3000 steps: Cd gpu {cd_g:.6f} oracle {cd_o:.6f} "
          f"({cd_g / cd_o - 1:+.2e}); Cl gpu {Pg[w, 1] / (0.5 * U * U):+.2e}")
    assert cd_o > 0.5
    assert abs(cd_g / cd_o - 1.0) <= 0.01
    assert abs(Pg[w, 1] / (0.5 * U * U)) <= 1e-2


def _shedding_case():
    """Coarse cylinder at Re 200 (64 x 32 O-mesh, first cell 0.02, far field at 12 D),
    started from the free stream with a small asymmetric kick in the near wake; its
    lift oscillates with a growing amplitude after t ~ 60 (past the onset of shedding)."""
    case = M.cylinder(64, 32, Re=200.0, first=0.02, r_far=12.0)
    meta = case.mesh.meta
    radii = meta["radii"]
    rc = 0.5 * (radii[:-1] + radii[1:])
    th = 2.0 * math.pi * (meta["cell_i"] + 0.5) / meta["n_theta"]
    r = rc[meta["cell_k"]]
    x, y = r * np.cos(th), r * np.sin(th)
    u = np.tile(np.asarray(case.u0, np.float64), (case.mesh.n_cells, 1))
    u[:, 1] += 0.1 * case.meta["U"] * np.exp(-((x - 1.5) ** 2 + y ** 2))
    return case, u


def _zero_crossings(t, c):
    c = c - c.mean()
    up = np.where((c[:-1] < 0) & (c[1:] >= 0))[0]
    return t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unsteady_cylinder_force_series_matches_oracle(precision):
    """Sec. IV unsteady cylinder, in the shedding regime: C_l(t) and C_d(t) of the GPU,
    sampled every 71 steps (about 0.5 time units), against the oracle's series from the
    same start.  FP64, to t = 200 (28,400 steps; the lift period is about 50): within
    1e-10 of the largest |C_l| and |C_d| at every sample (measured 2.2e-13 and 4e-15).
    FP32, to t = 400 (56,800 steps): within 1e-3 of the largest |C_l| and 1e-4 of the
    largest |C_d| (measured to t = 200: 3.9e-5 and 7e-7), and the same period of the lift
    oscillation (upward zero crossings after t = 100) within 1 %."""
    S = _S()
    case, u = _shedding_case()
    U = case.meta["U"]
    every, n_samples = 71, (400 if precision == "fp64" else 800)
    w = case.mesh.patches["wall"]
    s = S.Solver.from_case(case, precision).init(None, u)
    st = O.init(case.mesh.n_cells, u=u)
    t, g, o = [], [], []
    for q in range(n_samples):
        s.step(every - 1)
        Pg = s.step_forces()
        O.run(case, st, every - 1)
        Po = _patch_sums(case, O.run_flux(case, st, 1))
        t.append((q + 1) * every * case.dt)
        g.append(Pg[w] / (0.5 * U * U))
        o.append(Po[w] / (0.5 * U * U))
    t, g, o = np.array(t), np.array(g), np.array(o)
    late = t > 100.0
    assert np.abs(o[late, 1]).max() > 0.05                # a lift oscillation, not a steady wake
    err_cl = np.abs(g[:, 1] - o[:, 1]).max() / np.abs(o[:, 1]).max()
    err_cd = np.abs(g[:, 0] - o[:, 0]).max() / np.abs(o[:, 0]).max()
    zg, zo = _zero_crossings(t[late], g[late, 1]), _zero_crossings(t[late], o[late, 1])
    print(f"unsteady cylinder Re 200 {precision}: max |dCl| / max|Cl| {err_cl:.2e}, max |dCd| / max|Cd| "
          f"{err_cd:.2e}, lift crossings gpu {len(zg)} oracle {len(zo)}")
    if precision == "fp64":
        assert err_cl <= 1e-10 and err_cd <= 1e-10
    else:
        assert err_cl <= 1e-3 and err_cd <= 1e-4
        assert len(zo) >= 3 and len(zg) == len(zo)
        Tg, To = np.diff(zg).mean(), np.diff(zo).mean()
        assert abs(Tg / To - 1.0) <= 0.01
