"""CPU pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test names what it pins.  None of them compares the oracle with a retyped copy
of its own formulas: the checks are moment identities, closed-form special cases,
invariants (fixed points, conservation, mirror symmetry), the Couette closed form of
Sec. IV and its second-order convergence, and an independent exact-rational hand
stepper on tiny meshes.
"""
import dataclasses
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from oracle import handstep as H
from paper_2007_07347_gb300 import meshes as M

XI = O.XI


# ------------------------------------------------------------------ P1 equilibrium

@pytest.mark.parametrize("seed", range(5))
def test_feq_moments(seed):
    """Eqs. Feq/Macro: the discrete equilibrium carries the conserved moments
    sum feq = rho, sum xi feq = rho u and the Euler stress sum xi xi feq = rho u u + rho c_s^2 I."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0)
    u = rng.uniform(-0.2, 0.2, 2)
    fe = O.feq(rho, *u)
    assert abs(fe.sum() - rho) <= 1e-15 * rho
    np.testing.assert_allclose(XI.T @ fe, rho * u, rtol=0, atol=1e-15)
    P = np.einsum("a,ai,aj->ij", fe, XI, XI)
    np.testing.assert_allclose(P, rho * np.outer(u, u) + rho / 3.0 * np.eye(2), rtol=0, atol=1e-15)


def test_feq_rest_weights():
    """At rest the equilibrium is rho times the lattice weights (4/9, 1/9, 1/36)."""
    fe = O.feq(2.0, 0.0, 0.0)
    np.testing.assert_array_equal(fe, 2.0 * np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4))


# ------------------------------------------------------------------ geometry, LLSR

def _walls(m):
    return [(p, M.BC_WALL, (0.0, 0.0, 0.0)) for p in m.patches.values()]


def test_geometry_jittered_quads():
    """Areas sum to the box, each cell is closed (sum n l = 0), normals point out of
    the owner with |n l| = edge length, and centroids match a two-triangle split."""
    nx, ny, lx, ly = 5, 4, 2.5, 1.0
    m = M.cartesian(nx, ny, lx, ly, jitter=0.2, seed=11)
    g = O.geometry(m, _walls(m))
    assert abs(g["vol"].sum() - lx * ly) < 1e-14
    P = m.points
    for c in range(m.n_cells):
        i, j = c % nx, c // nx
        q = [i + (nx + 1) * j, i + 1 + (nx + 1) * j, i + 1 + (nx + 1) * (j + 1), i + (nx + 1) * (j + 1)]
        tri = [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
        A, C = 0.0, np.zeros(2)
        for t in tri:
            a, b, d = P[list(t)]
            at = 0.5 * abs((b[0] - a[0]) * (d[1] - a[1]) - (d[0] - a[0]) * (b[1] - a[1]))
            A += at
            C += at * (a + b + d) / 3
        assert abs(g["vol"][c] - A) < 1e-14
        np.testing.assert_allclose(g["xc"][c], C / A, atol=1e-14)
    close = np.zeros((m.n_cells, 2))
    for f in range(m.n_faces):
        p0, p1 = P[m.face_pts[f]]
        assert abs(np.hypot(*g["nl"][f]) - np.hypot(*(p1 - p0))) < 1e-14
        assert np.dot(g["xf"][f] - g["xc"][m.owner[f]], g["nl"][f]) > 0
        close[m.owner[f]] += g["nl"][f]
        if m.neighbour[f] >= 0:
            close[m.neighbour[f]] -= g["nl"][f]
    assert np.abs(close).max() < 1e-14


def test_llsr_exact_for_linear_fields():
    """The least-squares gradient reproduces the gradient of any linear field on any
    mesh, boundary cells included."""
    m = M.cartesian(7, 6, 1.4, 0.9, jitter=0.22, seed=3)
    bcs = _walls(m)
    xc = O.geometry(m, bcs)["xc"]
    phi = 2.5 + 0.7 * xc[:, 0] - 1.3 * xc[:, 1]
    g = O.gradient(m, bcs, phi)
    np.testing.assert_allclose(g, np.tile([0.7, -1.3], (m.n_cells, 1)), atol=1e-12)


def test_llsr_cartesian_special_cases():
    """On a uniform grid the LLSR gradient is the central difference inside, and the
    one-sided difference across a wall (boundary faces add no term)."""
    nx, ny, dx, dy = 6, 5, 1.0, 0.5
    m = M.cartesian(nx, ny, nx * dx, ny * dy)
    rng = np.random.default_rng(7)
    phi = rng.normal(size=m.n_cells)
    g = O.gradient(m, _walls(m), phi)
    P = phi.reshape(ny, nx)
    G = g.reshape(ny, nx, 2)
    np.testing.assert_allclose(G[1:-1, 1:-1, 0], (P[1:-1, 2:] - P[1:-1, :-2]) / (2 * dx), atol=1e-14)
    np.testing.assert_allclose(G[1:-1, 1:-1, 1], (P[2:, 1:-1] - P[:-2, 1:-1]) / (2 * dy), atol=1e-14)
    np.testing.assert_allclose(G[0, 1:-1, 1], (P[1, 1:-1] - P[0, 1:-1]) / dy, atol=1e-14)
    np.testing.assert_allclose(G[0, 1:-1, 0], (P[0, 2:] - P[0, :-2]) / (2 * dx), atol=1e-14)
    np.testing.assert_allclose(G[-1, 0, 0], (P[-1, 1] - P[-1, 0]) / dx, atol=1e-14)


def test_llsr_periodic_wraps():
    """Periodic boundaries (Sec. III): the ghost of a periodic face is the partner
    patch's inner cell at its shifted position, so the gradient is the central
    difference across the seam."""
    c = M.periodic_box(5, 4, lx=2.5, ly=2.0)
    rng = np.random.default_rng(1)
    phi = rng.normal(size=c.mesh.n_cells)
    g = O.gradient(c.mesh, c.bcs, phi)
    P = phi.reshape(4, 5)
    G = g.reshape(4, 5, 2)
    np.testing.assert_allclose(G[..., 0], (np.roll(P, -1, 1) - np.roll(P, 1, 1)) / (2 * 0.5), atol=1e-13)
    np.testing.assert_allclose(G[..., 1], (np.roll(P, -1, 0) - np.roll(P, 1, 0)) / (2 * 0.5), atol=1e-13)


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("seed", [0, 1])
def test_uniform_state_is_fixed_point(seed):
    """A uniform equilibrium on a fully periodic mesh stays put: the LLSR gradient is
    zero, every interface gets feq(rho0, u0) and a closed cell has sum n l = 0."""
    rng = np.random.default_rng(seed)
    case = M.periodic_box(6, 5, jitter=0.2, seed=seed, tau=0.07, dt=0.3)
    u0 = rng.uniform(-0.1, 0.1, 2)
    st = O.init(case.mesh.n_cells, rho0=1.3, u0=u0)
    f0 = st.f.copy()
    O.run(case, st, 40)
    assert np.abs(st.f - f0).max() <= 1e-14 * np.abs(f0).max()
    np.testing.assert_allclose(st.u, np.tile(u0, (case.mesh.n_cells, 1)), rtol=0, atol=1e-15)


def test_rest_with_walls_is_fixed_point():
    """Closed cavity with all walls at rest: rest at uniform density is exact."""
    base = M.cavity(5)
    bcs = [(p, M.BC_MOVING_WALL if k == M.BC_MOVING_WALL else k, (0.0, 0.0, 0.0)) for p, k, _ in base.bcs]
    case = dataclasses.replace(base, bcs=bcs, tau=0.1, dt=0.3)
    st = O.init(case.mesh.n_cells)
    f0 = st.f.copy()
    O.run(case, st, 30)
    assert np.abs(st.f - f0).max() <= 1e-15
    assert np.abs(st.W[:, 1:]).max() <= 1e-16


def test_conservation_periodic():
    """Mass and momentum are conserved (Eq. MacroUpdate with telescoping face
    fluxes), and sum_j V_j sum_a f_j stays equal to the mass carried by W."""
    case = M.periodic_box(12, 10, jitter=0.2, seed=5, tau=0.05, dt=0.2)
    rho, u = M.smooth_field(case, seed=2)
    vol = O.geometry(case.mesh, case.bcs)["vol"]
    st = O.init(case.mesh.n_cells, rho=rho, u=u)
    m0 = vol @ st.W
    O.run(case, st, 1500)
    m1 = vol @ st.W
    assert abs(m1[0] - m0[0]) <= 1e-13 * abs(m0[0])
    assert np.abs(m1[1:] - m0[1:]).max() <= 1e-13 * abs(m0[0])
    assert abs(vol @ st.f.sum(1) - m1[0]) <= 1e-13 * abs(m0[0])
    assert np.abs(st.u).max() > 1e-4          # the field actually evolved


# ------------------------------------------------------------------ P5 brute force
# Exact rationals grow quickly through the nonlinear equilibrium (u = rho u / rho):
# three steps on 2x2 and two on 3x3; the second step already carries a nonzero
# non-equilibrium part into every term, boundary rules included.

def _hand_vs_oracle(nx, ny, dx, dy, sides, bcs, tau, dt, steps, seed):
    rng = np.random.default_rng(seed)
    n = nx * ny
    rho = [Fr(int(k), 256) + 1 for k in rng.integers(-20, 21, n)]
    u = [(Fr(int(a), 1024), Fr(int(b), 1024)) for a, b in rng.integers(-60, 61, (n, 2))]
    f, W = H.run(H.Grid(nx, ny, dx, dy, sides), Fr(tau), Fr(dt), rho, u, steps)
    mesh = M.cartesian(nx, ny, nx * dx, ny * dy)
    case = M.Case("hand", mesh, bcs, tau=float(tau), dt=float(dt))
    st = O.init(n, rho=np.array([float(x) for x in rho]), u=np.array([[float(a), float(b)] for a, b in u]))
    O.run(case, st, steps)
    for got, exact in ((st.f, f), (st.W, W)):
        ex = np.array([[float(x) for x in row] for row in exact])
        assert np.abs(got - ex).max() <= 1e-14 * max(np.abs(ex).max(), 1e-300)


def test_handstep_2x2_periodic():
    sides = dict(bottom=("periodic",), top=("periodic",), left=("periodic",), right=("periodic",))
    bcs = [(3, M.BC_PERIODIC, (1, 2.0, 0)), (1, M.BC_PERIODIC, (3, -2.0, 0)),
           (0, M.BC_PERIODIC, (2, 0, 1.0)), (2, M.BC_PERIODIC, (0, 0, -1.0))]
    _hand_vs_oracle(2, 2, 1.0, 0.5, sides, bcs, Fr(1, 10), Fr(1, 4), 3, seed=0)


def test_handstep_3x3_periodic():
    sides = dict(bottom=("periodic",), top=("periodic",), left=("periodic",), right=("periodic",))
    bcs = [(3, M.BC_PERIODIC, (1, 3.0, 0)), (1, M.BC_PERIODIC, (3, -3.0, 0)),
           (0, M.BC_PERIODIC, (2, 0, 1.5)), (2, M.BC_PERIODIC, (0, 0, -1.5))]
    _hand_vs_oracle(3, 3, 1.0, 0.5, sides, bcs, Fr(1, 8), Fr(3, 10), 2, seed=1)


def test_handstep_3x3_moving_wall():
    """Periodic in x, wall at rest below, moving wall above (the Couette set-up)."""
    sides = dict(bottom=("wall", 0, 0), top=("wall", Fr(1, 10), 0), left=("periodic",), right=("periodic",))
    bcs = [(3, M.BC_PERIODIC, (1, 3.0, 0)), (1, M.BC_PERIODIC, (3, -3.0, 0)),
           (0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.1, 0, 0))]
    _hand_vs_oracle(3, 3, 1.0, 0.5, sides, bcs, Fr(1, 10), Fr(1, 4), 2, seed=2)


def test_handstep_3x3_all_boundary_kinds():
    """Wall, moving wall, far field and outlet on the four sides of a 3x3 mesh."""
    sides = dict(bottom=("wall", 0, 0), top=("wall", Fr(1, 10), 0),
                 left=("farfield", 1, Fr(1, 20), 0), right=("outlet",))
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.1, 0, 0)),
           (3, M.BC_FARFIELD, (1, 0.05, 0)), (1, M.BC_OUTLET, (0, 0, 0))]
    _hand_vs_oracle(3, 3, 1.0, 0.5, sides, bcs, Fr(1, 10), Fr(1, 4), 2, seed=3)


# ------------------------------------------------------------------ P6 Couette

def _run_to_residual(case, st, tol, interval=1000, cap=200000):
    n = 0
    while n < cap:
        Ws = st.W.copy()
        O.run(case, st, interval)
        n += interval
        eps, _ = O.residual(st.W, Ws)
        if eps < tol:
            return n, eps
    return n, eps


def test_couette_linear_profile():
    """Sec. IV Couette flow: from rest the steady state is the analytic profile
    u = U y / H, v = 0 (on uniform quads the scheme keeps it to round-off)."""
    case = M.couette(16)
    st = O.init(case.mesh.n_cells)
    n, eps = _run_to_residual(case, st, 1e-10)
    assert eps < 1e-10
    y = case.mesh.meta["cell_xy_nominal"][:, 1]
    U = case.meta["U"]
    err = np.sqrt(np.sum((st.u[:, 0] - U * y) ** 2) / np.sum((U * y) ** 2))
    assert err < 1e-8
    assert np.abs(st.u[:, 1]).max() < 1e-12 * U


def test_couette_second_order_on_distorted_meshes():
    """Sec. IV: the L2 error of u decays at second order on unstructured
    (jittered) 4 x {8, 16, 32, 64} meshes.  The fitted slope on these seeded meshes is
    2.21 (local orders 2.06, 2.23, 2.34); the band is that value +- 0.15, so a first-order
    term or an extra term that changes the rate fails it."""
    errs, hs = [], []
    for ny in (8, 16, 32, 64):
        base = M.couette(ny)
        dy = 1.0 / ny
        mesh = M.cartesian(4, ny, 4 * dy, 1.0, jitter=0.15, seed=3)
        case = dataclasses.replace(base, mesh=mesh)
        y = O.geometry(mesh, case.bcs)["xc"][:, 1]
        U = case.meta["U"]
        st = O.init(mesh.n_cells, u=np.stack([U * y, 0 * y], 1))
        _, eps = _run_to_residual(case, st, 1e-10)
        assert eps < 1e-10
        errs.append(np.sqrt(np.sum((st.u[:, 0] - U * y) ** 2) / np.sum((U * y) ** 2)))
        hs.append(dy)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 2.06 <= slope <= 2.36, (slope, errs)


# ------------------------------------------------------------------ P7 mirror symmetry

def test_cylinder_mirror_symmetry():
    """Flow past a cylinder is symmetric about the wake axis at every step:
    rho and u_x even, u_y odd under y -> -y (a sign or index slip in any y term breaks it)."""
    nt, nr = 32, 16
    case = M.cylinder(nt, nr, Re=40.0, first=0.02, r_far=10.0, shuffle_seed=None)
    st = O.init(case.mesh.n_cells, u0=(0.1, 0.0))
    O.run(case, st, 200)
    i = case.mesh.meta["cell_i"]
    k = case.mesh.meta["cell_k"]
    mirror = (nt - 1 - i) + nt * k
    assert np.abs(st.u[:, 1]).max() > 1e-4
    np.testing.assert_allclose(st.W[:, 0], st.W[mirror, 0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(st.u[:, 0], st.u[mirror, 0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(st.u[:, 1], -st.u[mirror, 1], rtol=0, atol=1e-13)


# ------------------------------------------------------------------ residual

def test_residual_closed_form():
    """Residual of Sec. IV (cavity): sqrt(sum dU^2 + dV^2) / sqrt(sum U0^2 + V0^2)."""
    n = 10
    Ws = np.tile([2.0, 2.0 * 3.0, 2.0 * 4.0], (n, 1))       # U0 = 3, V0 = 4
    W = np.tile([2.0, 2.0 * 3.0, 2.0 * 4.5], (n, 1))        # V = 4.5
    eps, mass = O.residual(W, Ws, vol=np.full(n, 0.5))
    assert abs(eps - 0.1) < 1e-15
    assert mass == 10.0
    eps0, _ = O.residual(W, np.tile([1.0, 0.0, 0.0], (n, 1)))
    assert math.isinf(eps0)


# ------------------------------------------------------------------ symmetric boundary
# Sec. III: a symmetric boundary puts a ghost cell at the mirror image of the inner
# cell, with the same density and the mirrored velocity.  Pinned against the scheme
# without that rule: the same flow on the mirror-doubled mesh, where the symmetry
# line is an ordinary row of interior faces.

def _channel_half(jitter, seed):
    return M.cartesian(8, 4, 8.0, 4.0, jitter=jitter, seed=seed)


@pytest.mark.parametrize("jitter,seed", [(0.0, None), (0.2, 3)])
def test_symmetry_line_equals_the_mirrored_domain(jitter, seed):
    """Periodic channel with a moving bottom wall and a symmetry line on top against
    the mirror-doubled channel (walls at both ends) from a mirror-symmetric start:
    the lower half of the doubled flow is the half-domain flow."""
    half = _channel_half(jitter, seed)
    full = M.mirror_y(half, half.patches["top"])
    n = half.n_cells
    per = [(3, M.BC_PERIODIC, (1, 8.0, 0.0)), (1, M.BC_PERIODIC, (3, -8.0, 0.0))]
    wall = [(0, M.BC_MOVING_WALL, (0.05, 0.0, 0.0))]
    c_half = M.Case("half", half, per + wall + [(2, M.BC_SYMMETRY, (0.0, 0.0, 0.0))], tau=0.05, dt=0.2)
    c_full = M.Case("full", full, per + wall, tau=0.05, dt=0.2)
    xy = half.meta["cell_xy_nominal"]
    X, Y = 2 * np.pi * xy[:, 0] / 8.0, np.pi * xy[:, 1] / 4.0
    rho = 1.0 + 0.02 * np.cos(X) * np.cos(Y)
    u = np.stack([0.03 * np.sin(X) + 0.01 * Y, 0.02 * np.sin(X) * np.sin(0.5 * Y)], 1)
    s_half = O.init(n, rho=rho, u=u)
    u_m = u.copy()
    u_m[:, 1] *= -1.0
    s_full = O.init(2 * n, rho=np.concatenate([rho, rho]), u=np.concatenate([u, u_m]))
    O.run(c_half, s_half, 40)
    O.run(c_full, s_full, 40)
    assert np.abs(s_half.W[:, 2]).max() > 1e-4                 # normal velocity near the line
    np.testing.assert_allclose(s_half.f, s_full.f[:n], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s_half.W, s_full.W[:n], rtol=0, atol=1e-13)
    # the doubled flow itself stays mirror-symmetric
    mx = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5])
    np.testing.assert_allclose(s_full.f[n:], s_full.f[:n][:, mx], rtol=0, atol=1e-13)


def _transposed(mesh):
    """The mesh with x and y exchanged (the same ids; a line of constant y becomes a
    line of constant x)."""
    meta = dict(mesh.meta)
    if "cell_xy_nominal" in meta:
        meta["cell_xy_nominal"] = meta["cell_xy_nominal"][:, ::-1].copy()
    return M.Mesh(mesh.points[:, ::-1].copy(), mesh.face_pts, mesh.owner, mesh.neighbour, mesh.n_cells,
                  mesh.patches, meta)


@pytest.mark.parametrize("jitter,seed", [(0.0, None), (0.2, 3)])
def test_symmetry_line_of_constant_x_equals_the_mirrored_domain(jitter, seed):
    """The previous check with x and y exchanged: the symmetry line is a line of
    constant x (the mirror of the other axis, its own ghost position and gradient
    reflection), periodic in y, the moving wall at x = 0."""
    half = _channel_half(jitter, seed)
    full = M.mirror_y(half, half.patches["top"])
    half, full = _transposed(half), _transposed(full)
    n = half.n_cells
    per = [(3, M.BC_PERIODIC, (1, 0.0, 8.0)), (1, M.BC_PERIODIC, (3, 0.0, -8.0))]
    wall = [(0, M.BC_MOVING_WALL, (0.0, 0.05, 0.0))]
    c_half = M.Case("half_t", half, per + wall + [(2, M.BC_SYMMETRY, (0.0, 0.0, 0.0))], tau=0.05, dt=0.2)
    c_full = M.Case("full_t", full, per + wall, tau=0.05, dt=0.2)
    xy = half.meta["cell_xy_nominal"]                         # (y, x) of the untransposed channel
    X, Y = 2 * np.pi * xy[:, 1] / 8.0, np.pi * xy[:, 0] / 4.0
    rho = 1.0 + 0.02 * np.cos(X) * np.cos(Y)
    u = np.stack([0.02 * np.sin(X) * np.sin(0.5 * Y), 0.03 * np.sin(X) + 0.01 * Y], 1)
    s_half = O.init(n, rho=rho, u=u)
    u_m = u.copy()
    u_m[:, 0] *= -1.0
    s_full = O.init(2 * n, rho=np.concatenate([rho, rho]), u=np.concatenate([u, u_m]))
    O.run(c_half, s_half, 40)
    O.run(c_full, s_full, 40)
    assert np.abs(s_half.W[:, 1]).max() > 1e-4                 # normal velocity near the line
    np.testing.assert_allclose(s_half.f, s_full.f[:n], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s_half.W, s_full.W[:n], rtol=0, atol=1e-13)
    my = np.array([0, 3, 2, 1, 4, 6, 5, 8, 7])                # mirror in x
    np.testing.assert_allclose(s_full.f[n:], s_full.f[:n][:, my], rtol=0, atol=1e-13)


def test_symmetry_uniform_stream_is_fixed_point():
    """A uniform stream along two symmetry lines (periodic in x) is a fixed point."""
    m = M.cartesian(6, 5, 6.0, 5.0, jitter=0.2, seed=8)
    bcs = [(3, M.BC_PERIODIC, (1, 6.0, 0.0)), (1, M.BC_PERIODIC, (3, -6.0, 0.0)),
           (0, M.BC_SYMMETRY, (0.0, 0.0, 0.0)), (2, M.BC_SYMMETRY, (0.0, 0.0, 0.0))]
    case = M.Case("sym_stream", m, bcs, tau=0.07, dt=0.3)
    st = O.init(m.n_cells, rho0=1.1, u0=(0.08, 0.0))
    f0 = st.f.copy()
    O.run(case, st, 40)
    assert np.abs(st.f - f0).max() <= 1e-14 * np.abs(f0).max()


def test_symmetry_channel_conserves_mass_and_streamwise_momentum():
    """Symmetry lines pass no mass and no tangential momentum (the interface
    distribution is even in the normal velocity component), so a channel periodic in
    x between two symmetry lines conserves mass and x-momentum."""
    m = M.cartesian(10, 8, 10.0, 8.0, jitter=0.2, seed=9)
    bcs = [(3, M.BC_PERIODIC, (1, 10.0, 0.0)), (1, M.BC_PERIODIC, (3, -10.0, 0.0)),
           (0, M.BC_SYMMETRY, (0.0, 0.0, 0.0)), (2, M.BC_SYMMETRY, (0.0, 0.0, 0.0))]
    case = M.Case("sym_channel", m, bcs, tau=0.05, dt=0.2)
    xy = m.meta["cell_xy_nominal"]
    X, Y = 2 * np.pi * xy[:, 0] / 10.0, 2 * np.pi * xy[:, 1] / 8.0
    rho = 1.0 + 0.03 * np.cos(X + 0.3) * np.sin(Y)
    u = np.stack([0.04 * np.sin(Y) + 0.02 * np.cos(X), 0.03 * np.sin(X) * np.cos(Y)], 1)
    vol = O.geometry(m, bcs)["vol"]
    st = O.init(m.n_cells, rho=rho, u=u)
    m0 = vol @ st.W
    O.run(case, st, 400)
    m1 = vol @ st.W
    assert abs(m1[0] - m0[0]) <= 1e-13 * abs(m0[0])
    assert abs(m1[1] - m0[1]) <= 1e-13 * abs(m0[0])
    assert abs(m1[2] - m0[2]) > 1e-6 * abs(m0[0])             # normal momentum is not conserved (pressure)


def test_symmetry_rejects_a_slanted_line():
    """Mirrored D2Q9 velocities stay on the lattice only for lines of constant x or y."""
    case = M.cylinder(16, 8, first=0.05, r_far=3.0, shuffle_seed=None)
    bcs = [(0, M.BC_SYMMETRY, (0.0, 0.0, 0.0)), (1, M.BC_FARFIELD, (1.0, 0.1, 0.0))]
    with pytest.raises(RuntimeError):
        O.run(dataclasses.replace(case, bcs=bcs), O.init(case.mesh.n_cells), 1)


# ------------------------------------------------------------------ triangles and hybrid cells

def _periodic_bcs(lx, ly):
    return [(3, M.BC_PERIODIC, (1, lx, 0.0)), (1, M.BC_PERIODIC, (3, -lx, 0.0)),
            (0, M.BC_PERIODIC, (2, 0.0, ly)), (2, M.BC_PERIODIC, (0, 0.0, -ly))]


def test_hybrid_geometry_and_linear_llsr():
    """Quad/triangle mesh: areas tile the box, every cell closes, and the LLSR
    gradient is exact for linear fields wherever the neighbours span the plane (a
    corner triangle with one neighbour gets the zero gradient of a degenerate stencil)."""
    m = M.hybrid(7, 6, 1.4, 0.9, tri_from=0.4, jitter=0.2, seed=3)
    bcs = _walls(m)
    g = O.geometry(m, bcs)
    assert abs(g["vol"].sum() - 1.4 * 0.9) < 1e-14
    cs = np.zeros((m.n_cells, 2))
    np.add.at(cs, m.owner, g["nl"])
    inner = m.neighbour >= 0
    np.add.at(cs, m.neighbour[inner], -g["nl"][inner])
    assert np.abs(cs).max() < 1e-14
    phi = 2.5 + 0.7 * g["xc"][:, 0] - 1.3 * g["xc"][:, 1]
    grad = O.gradient(m, bcs, phi)
    ok = np.abs(g["ainv"]).sum(1) > 0
    assert ok.sum() >= m.n_cells - 2 and m.meta["n_triangles"] > 0
    np.testing.assert_allclose(grad[ok], np.tile([0.7, -1.3], (ok.sum(), 1)), atol=1e-12)
    assert np.all(grad[~ok] == 0.0)


def test_hybrid_uniform_state_is_fixed_point():
    m = M.hybrid(6, 5, 6.0, 5.0, tri_from=0.3, jitter=0.2, seed=2)
    case = M.Case("hyb_fixed", m, _periodic_bcs(6.0, 5.0), tau=0.07, dt=0.3)
    st = O.init(m.n_cells, rho0=1.2, u0=(0.05, -0.03))
    f0 = st.f.copy()
    O.run(case, st, 40)
    assert np.abs(st.f - f0).max() <= 1e-14 * np.abs(f0).max()


def test_hybrid_conservation_periodic():
    m = M.hybrid(12, 10, 12.0, 10.0, tri_from=0.5, jitter=0.2, seed=6)
    bcs = _periodic_bcs(12.0, 10.0)
    case = M.Case("hyb_cons", m, bcs, tau=0.05, dt=0.15)
    xy = m.meta["cell_xy_nominal"]
    X, Y = 2 * np.pi * xy[:, 0] / 12.0, 2 * np.pi * xy[:, 1] / 10.0
    rho = 1.0 + 0.03 * np.sin(X) * np.cos(Y)
    u = np.stack([0.04 * np.cos(Y), 0.03 * np.sin(X + Y)], 1)
    vol = O.geometry(m, bcs)["vol"]
    st = O.init(m.n_cells, rho=rho, u=u)
    m0 = vol @ st.W
    O.run(case, st, 500)
    m1 = vol @ st.W
    assert np.abs(m1 - m0).max() <= 1e-13 * abs(m0[0])
    assert np.abs(st.u).max() > 1e-4


def test_couette_second_order_on_triangles():
    """Sec. IV Couette flow on hybrid meshes 4 x {8, 16, 32, 64}: triangles everywhere
    but a layer of quads along the two walls; the L2 error of u decays at second
    order, approached from below on these coarse meshes (measured local orders 1.61
    and 1.71 between 16, 32 and 64 rows, fitted slope 1.66; a first-order scheme would
    give 1).  The band is the fitted slope +- 0.12.  dt follows the CFL rule of the
    triangles (half the quads' step)."""
    errs, hs = [], []
    for ny in (8, 16, 32, 64):
        base = M.couette(ny)
        dy = 1.0 / ny
        mesh = M.hybrid(4, ny, 4 * dy, 1.0, tri_from=0.0, jitter=0.1, seed=5, quad_rows=1)
        case = dataclasses.replace(base, mesh=mesh, dt=0.5 * base.dt)
        y = O.geometry(mesh, case.bcs)["xc"][:, 1]
        U = case.meta["U"]
        st = O.init(mesh.n_cells, u=np.stack([U * y, 0 * y], 1))
        _, eps = _run_to_residual(case, st, 1e-10)
        assert eps < 1e-10
        errs.append(np.sqrt(np.sum((st.u[:, 0] - U * y) ** 2) / np.sum((U * y) ** 2)))
        hs.append(dy)
    slope = np.polyfit(np.log(hs[1:]), np.log(errs[1:]), 1)[0]
    assert 1.54 <= slope <= 1.78, (slope, errs)
    assert errs[-1] < 1e-5
