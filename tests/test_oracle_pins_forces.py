"""Pins of the oracle's boundary momentum flux (the forces of Sec. IV: C_d, C_l from
the momentum the fluid gives to the wall; C_p from the normal part) against closed
forms and an invariant, on the CPU.

* a fluid at rest: every boundary face carries the pressure rho c_s^2 n l only;
* a uniform stream through far-field faces of any orientation:
  rho c_s^2 n l + rho u (u . n l) (the second moment of the equilibrium);
* plane Couette flow at steady state: the shear stress mu U / H on every wall face,
  of opposite signs on the two walls, with mu = rho tau c_s^2;
* any state: the momentum the fluid loses in a step is the sum of the boundary
  fluxes of that step times dt (interior faces cancel).

The face normals of the closed forms are computed here from the mesh points, not
taken from the oracle.
"""
import dataclasses

import numpy as np

import oracle as O
from paper_2007_07347_gb300 import meshes as M

CS2 = 1.0 / 3.0


def _normals_out(mesh, faces):
    """n l of each face from its end points, turned away from the owner cell (the mean
    of the owner's vertices lies inside a convex cell)."""
    pts = np.asarray(mesh.points)
    fp = np.asarray(mesh.face_pts)
    own = np.asarray(mesh.owner)
    # vertex mean of every cell from the faces that bound it
    acc = np.zeros((mesh.n_cells, 2))
    cnt = np.zeros(mesh.n_cells)
    nb = np.asarray(mesh.neighbour)
    for side, cells in ((0, own), (1, nb)):
        sel = cells >= 0
        for end in (0, 1):
            np.add.at(acc, cells[sel], pts[fp[sel, end]])
            np.add.at(cnt, cells[sel], 1.0)
    centre = acc / cnt[:, None]
    p0, p1 = pts[fp[faces, 0]], pts[fp[faces, 1]]
    nl = np.stack([p1[:, 1] - p0[:, 1], -(p1[:, 0] - p0[:, 0])], 1)
    mid = 0.5 * (p0 + p1)
    flip = np.einsum("ij,ij->i", mid - centre[own[faces]], nl) < 0
    nl[flip] *= -1.0
    return nl


def _cylinder(farfield_everywhere=False, rho=1.0, u=(0.0, 0.0)):
    case = M.cylinder(24, 12, first=0.05, r_far=6.0, shuffle_seed=2)
    if farfield_everywhere:
        bcs = [(p, M.BC_FARFIELD, (rho, u[0], u[1])) for p, _, _ in case.bcs]
    else:
        bcs = [(p, k, (rho, u[0], u[1]) if k == M.BC_FARFIELD else par) for p, k, par in case.bcs]
    return dataclasses.replace(case, bcs=bcs)


def test_fluid_at_rest_pushes_with_its_pressure_only():
    """rho = 1.3 at rest around the cylinder (wall and far field at rest): every boundary
    face gets F = rho c_s^2 n l, with n out of the fluid."""
    case = _cylinder(rho=1.3)
    st = O.init(case.mesh.n_cells, rho=np.full(case.mesh.n_cells, 1.3))
    F = O.run_flux(case, st, 1)
    bf = O.boundary_faces(case.mesh, case.bcs)
    expect = 1.3 * CS2 * _normals_out(case.mesh, bf)
    assert len(bf) == 2 * 24
    assert np.abs(F - expect).max() <= 1e-14


def test_uniform_stream_through_far_field_faces():
    """A uniform stream rho = 1.02, u = (0.08, -0.03) with every boundary face a far-field
    face of that state stays uniform, and each face carries the equilibrium's second
    moment: F = rho c_s^2 n l + rho u (u . n l), for faces of every orientation."""
    rho, u = 1.02, np.array([0.08, -0.03])
    case = _cylinder(farfield_everywhere=True, rho=rho, u=u)
    n = case.mesh.n_cells
    st = O.init(n, rho=np.full(n, rho), u=np.tile(u, (n, 1)))
    W0 = st.W.copy()
    F = O.run_flux(case, st, 2)
    assert np.abs(st.W - W0).max() <= 1e-14
    nl = _normals_out(case.mesh, O.boundary_faces(case.mesh, case.bcs))
    expect = rho * CS2 * nl + rho * np.outer(nl @ u, u)
    assert np.abs(F - expect).max() <= 1e-14
    assert np.abs(expect - rho * CS2 * nl).max() > 1e-4       # the convective part is really there


def test_couette_wall_shear_is_mu_u_over_h():
    """Plane Couette flow (4 x 16, U = 0.1, Re = 10) at steady state: on every face of the
    resting bottom wall F_x = mu U / H l and on every face of the moving top wall
    F_x = -mu U / H l (the fluid gives x-momentum to the bottom wall and takes it from
    the lid), mu = rho tau c_s^2; F_y = -+ rho c_s^2 l (pressure)."""
    case = M.couette(16)
    st = O.init(case.mesh.n_cells)
    for _ in range(400):
        Ws = st.W.copy()
        O.run(case, st, 500)
        eps, _ = O.residual(st.W, Ws)
        if eps < 1e-12:
            break
    assert eps < 1e-12
    F = O.run_flux(case, st, 1)
    bf = O.boundary_faces(case.mesh, case.bcs)
    patch = -1 - np.asarray(case.mesh.neighbour)[bf]
    U, H, l = case.meta["U"], 1.0, 1.0 / 16
    tau_w = case.tau * CS2 * U / H
    bottom, top = patch == 0, patch == 2
    assert bottom.sum() == 4 and top.sum() == 4 and len(bf) == 8
    np.testing.assert_allclose(F[bottom, 0], tau_w * l, rtol=1e-10)
    np.testing.assert_allclose(F[top, 0], -tau_w * l, rtol=1e-10)
    np.testing.assert_allclose(F[bottom, 1], -CS2 * l, rtol=1e-10)
    np.testing.assert_allclose(F[top, 1], CS2 * l, rtol=1e-10)


def test_boundary_flux_balances_the_momentum_change():
    """Jittered closed box with a moving lid after 60 steps from rest: the momentum the
    fluid loses in the next step, -(P^{n+1} - P^n) with P = sum V rho u, equals dt times
    the sum of that step's boundary fluxes (the interior faces cancel pairwise)."""
    mesh = M.cartesian(14, 11, 1.4, 1.1, jitter=0.2, seed=9)
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (1, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.1, 0.0, 0.0)),
           (3, M.BC_WALL, (0, 0, 0))]
    case = M.Case("box", mesh, bcs, tau=0.02, dt=0.02)
    st = O.init(mesh.n_cells)
    O.run(case, st, 60)
    vol = O.geometry(mesh, bcs)["vol"]
    P0 = vol @ st.W[:, 1:]
    F = O.run_flux(case, st, 1)
    P1 = vol @ st.W[:, 1:]
    lhs = -(P1 - P0)
    rhs = case.dt * F.sum(0)
    assert np.abs(F[:, 0]).max() > 1e-4
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13 * np.abs(F).sum() * case.dt)
