"""CPU pins of the rarefied (discrete velocity grid) oracle.

The rarefied variant runs the same scheme on a Q-node velocity grid with the
Maxwellian of Eq. Feq and diffuse walls (Sec. III).  Pinned against: closed-form
truncated Gaussian integrals of the grid (error bound of the midpoint rule), the
uniform equilibrium as a fixed point, exact conservation of mass, momentum and
energy on periodic meshes, the zero mass flux of a diffuse wall, the collisionless
Couette flow between diffuse plates, whose steady state is known in closed form on any
velocity grid, and one collisionless step of a quadratic field, which fixes the
characteristic reconstruction (the sign of its xi dt term, the upwind side, the
gradient) and the sign of the flux balance, the BGK relaxation of a uniform state
(the rate dt/tau of Eq. fn+1), and the decay of a shear wave at the Navier-Stokes rate
nu k^2 with nu = tau R T (the interface distribution of Eq. f_t_n+1), and the mirror
symmetry of a symmetric state on a grid with velocities tangential to the faces (the
tie rule of reading A5), the equilibrium of the conserved moments (its temperature
and its moments), and by brute force: three steps on 3 x 3 grids (periodic, between
diffuse walls, in a closed box; with and without tangential velocities) against an
independent 40-digit restatement of the step
(``oracle/handstep_dvm.py``).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_07347_gb300 import meshes as M


def _erf_mass(a, b, mu, s):
    """int_a^b N(x; mu, s^2) dx."""
    return 0.5 * (math.erf((b - mu) / (s * math.sqrt(2))) - math.erf((a - mu) / (s * math.sqrt(2))))


@pytest.mark.parametrize("nv,vmax,ux,uy,RT", [(100, 2.0, 0.1, 0.0, 0.5), (40, 3.0, -0.2, 0.15, 0.4)])
def test_grid_and_maxwellian_against_truncated_gaussian(nv, vmax, ux, uy, RT):
    """Eq. Feq on the midpoint grid: the discrete mass and mean velocity equal the
    Gaussian integrals over the truncated square within the midpoint-rule bound
    (h^2/24) * (2 vmax) * max|g''| per dimension."""
    xi, w = O.dvm_grid(nv, vmax)
    h = 2 * vmax / nv
    assert np.allclose(w, h * h)
    assert abs(xi[:, 0].min() + vmax - h / 2) < 1e-15 and abs(xi[:, 0].max() - vmax + h / 2) < 1e-15
    g = O.dvm_maxwell(1.3, ux, uy, RT, xi, w)
    s = math.sqrt(RT)
    Ix, Iy = _erf_mass(-vmax, vmax, ux, s), _erf_mass(-vmax, vmax, uy, s)
    bound = (h * h / 24) * (2 * vmax) / (s ** 3 * math.sqrt(2 * math.pi))     # max|g''| = 1/(s^3 sqrt(2 pi))
    rho = g.sum()
    assert abs(rho / 1.3 - Ix * Iy) <= 2.5 * bound
    # first moment along x: int x N dx = mu I + s^2 (N(a) - N(b))
    na = math.exp(-(-vmax - ux) ** 2 / (2 * RT)) / (s * math.sqrt(2 * math.pi))
    nb = math.exp(-(vmax - ux) ** 2 / (2 * RT)) / (s * math.sqrt(2 * math.pi))
    mx = ux * Ix + RT * (na - nb)
    assert abs((xi[:, 0] * g).sum() / 1.3 - mx * Iy) <= 2.5 * bound * (vmax + 2)


def test_maxwellian_of_the_conserved_moments():
    """The equilibrium a step builds from the conserved moments W = (rho, rho u,
    rho (|u|^2/2 + R T)) (Eqs. Macro, Feq: the temperature is the energy per unit mass
    less the kinetic part) is the Maxwellian of (rho, u, R T) sampled directly, and on a
    grid wide enough for the truncation to be small its moments return W.  The
    midpoint rule on a Gaussian has an error far below the truncation's; the tolerance
    is the truncated tails' share of moments up to second order, 4 t rho (1 + vmax^2)
    with t the larger one-sided tail mass of the two axes."""
    nv, vmax = 100, 4.0
    xi, w = O.dvm_grid(nv, vmax)
    rho, ux, uy, RT = 1.2, 0.3, -0.2, 0.4
    st = O.dvm_init(1, xi, w, rho0=rho, u0=(ux, uy), RT0=RT)
    g = O.dvm_maxwell(rho, ux, uy, RT, xi, w)
    assert np.abs(st.f[0] - g).max() <= 1e-13 * g.max()
    E = 0.5 * (xi ** 2).sum(1)
    mom = np.array([st.f[0].sum(), (xi[:, 0] * st.f[0]).sum(), (xi[:, 1] * st.f[0]).sum(), (E * st.f[0]).sum()])
    assert np.allclose(st.W[0], [rho, rho * ux, rho * uy, rho * (0.5 * (ux * ux + uy * uy) + RT)], rtol=1e-15)
    t = max(0.5 * math.erfc((vmax - abs(u)) / math.sqrt(2 * RT)) for u in (ux, uy))
    assert np.abs(mom - st.W[0]).max() <= 4 * t * rho * (1 + vmax ** 2)


def _periodic(lx, ly):
    return [(3, M.BC_PERIODIC, (1, lx, 0.0)), (1, M.BC_PERIODIC, (3, -lx, 0.0)),
            (0, M.BC_PERIODIC, (2, 0.0, ly)), (2, M.BC_PERIODIC, (0, 0.0, -ly))]


def test_uniform_equilibrium_is_fixed_point():
    xi, w = O.dvm_grid(12, 2.0)
    m = M.cartesian(4, 3, 1.0, 0.75, jitter=0.2, seed=2)
    st = O.dvm_init(m.n_cells, xi, w, rho0=1.1, u0=(0.1, -0.05), RT0=0.45)
    f0 = st.f.copy(); W0 = st.W.copy()
    O.dvm_run(m, _periodic(1.0, 0.75), st, xi, w, 0.5, tau=0.05, dt=0.02, n_steps=30)
    assert np.abs(st.f - f0).max() <= 1e-14 * np.abs(f0).max()
    assert np.abs(st.W - W0).max() <= 1e-14


def test_conservation_periodic():
    """Mass, momentum and energy move only through face fluxes (Eq. MacroUpdate)."""
    xi, w = O.dvm_grid(10, 2.5)
    m = M.cartesian(6, 5, 1.2, 1.0, jitter=0.2, seed=3)
    xy = m.meta["cell_xy_nominal"]
    X, Y = 2 * np.pi * xy[:, 0] / 1.2, 2 * np.pi * xy[:, 1]
    st = O.dvm_init(m.n_cells, xi, w, rho=1 + 0.05 * np.sin(X), u=np.stack([0.1 * np.cos(Y), 0.05 * np.sin(X)], 1),
                    RT=0.5 + 0.03 * np.cos(X + Y))
    vol = O.geometry(m, _periodic(1.2, 1.0))["vol"]
    W0 = vol @ st.W
    O.dvm_run(m, _periodic(1.2, 1.0), st, xi, w, 0.5, tau=0.02, dt=0.01, n_steps=60)
    W1 = vol @ st.W
    assert np.abs(W1 - W0).max() <= 1e-13 * abs(W0[0])
    assert np.abs(st.W[:, 1]).std() > 1e-4


def test_diffuse_walls_pass_no_mass():
    """A closed box with diffuse walls (one moving) keeps its mass to round-off."""
    xi, w = O.dvm_grid(16, 2.0)
    m = M.cartesian(6, 6, 1.0, 1.0, jitter=0.15, seed=4)
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (1, M.BC_WALL, (0, 0, 0)), (3, M.BC_WALL, (0, 0, 0)),
           (2, M.BC_MOVING_WALL, (0.1, 0, 0))]
    st = O.dvm_init(m.n_cells, xi, w)
    vol = O.geometry(m, bcs)["vol"]
    m0 = vol @ st.W[:, 0]
    O.dvm_run(m, bcs, st, xi, w, 0.5, tau=0.1, dt=0.01, n_steps=300)
    assert abs(vol @ st.W[:, 0] - m0) <= 1e-13 * m0
    assert np.abs(st.u).max() > 1e-3


def test_collisionless_couette_closed_form():
    """Free-molecular Couette flow between diffuse plates (bottom at rest, top moving
    at U, periodic in x): every velocity keeps the Maxwellian of the wall it left, so
    the steady state is uniform across the channel, f = A g_bottom for xi_y > 0 and
    f = B g_top for xi_y < 0, with A and B fixed by zero net mass flux at each wall and
    the total mass."""
    nv, vmax, RT, U = 8, 2.0, 0.5, 0.2
    xi, w = O.dvm_grid(nv, vmax)
    m = M.cartesian(2, 6, 1.0 / 3, 1.0)
    bcs = [(3, M.BC_PERIODIC, (1, 1.0 / 3, 0.0)), (1, M.BC_PERIODIC, (3, -1.0 / 3, 0.0)),
           (0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (U, 0, 0))]
    st = O.dvm_init(m.n_cells, xi, w, RT0=RT)
    mass0 = st.W[:, 0].mean()
    for _ in range(60):
        O.dvm_run(m, bcs, st, xi, w, RT, tau=1e12, dt=0.02, n_steps=500)
    gb = O.dvm_maxwell(1.0, 0.0, 0.0, RT, xi, w)
    gt = O.dvm_maxwell(1.0, U, 0.0, RT, xi, w)
    up, dn = xi[:, 1] > 0, xi[:, 1] < 0
    # bottom wall re-emits what arrives from the top: A sum_up xi_y gb = B sum_dn |xi_y| gt
    ratio = (np.abs(xi[dn, 1]) * gt[dn]).sum() / (xi[up, 1] * gb[up]).sum()
    f_shape = np.where(up, ratio * gb, gt)
    f_exact = f_shape * (st.f[0].sum() / f_shape.sum())
    assert np.abs(st.f - f_exact).max() <= 1e-10 * f_exact.max()
    # W moves by the same face fluxes as f: with no collisions its momentum is the
    # momentum of f (both start at zero); its mass stays at the initial mass
    np.testing.assert_allclose(st.W[:, 1], (xi[:, 0] * f_exact).sum(), rtol=1e-9)
    np.testing.assert_allclose(st.W[:, 2], 0.0, atol=1e-12)
    assert abs(st.W[:, 0].mean() - mass0) < 1e-12


def test_one_collisionless_step_of_a_quadratic_field():
    """Characteristic reconstruction (Eqs. fbpsource, fbar) and flux balance of one step
    in the free-molecular limit (tau -> infinity: fbar+ = f, f_b = fbar, f^{n+1} = f^n -
    dt/V F).  For f_q = w_q (x^2 + y^2) on a uniform mesh of unit cells, a cell two or
    more cells from the walls sees only exact central LLSR gradients (2x, 2y), and the
    upwind face values fbar = f_u + (x_f - x_u - xi dt) . sigma_u give, per axis,
    F / V = xi_x (2 x - 2 xi_x dt): the step leaves
        w_q [x^2 + y^2 - 2 dt (xi_x x + xi_y y) + 2 dt^2 (xi_x^2 + xi_y^2)]
    (the exact transport f(x - xi dt) has dt^2 where the scheme has 2 dt^2).  A flipped
    sign of xi dt in the reconstruction turns the last term into -2 dt^2; no gradient,
    a downwind side or a flux sign error change the first-order term."""
    nv, dt, n = 8, 0.1, 8
    xi, w = O.dvm_grid(nv, 2.0)
    m = M.cartesian(n, n, float(n), float(n))
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (1, M.BC_WALL, (0, 0, 0)), (3, M.BC_WALL, (0, 0, 0)),
           (2, M.BC_MOVING_WALL, (0.1, 0, 0))]
    st = O.dvm_init(m.n_cells, xi, w, RT0=0.5)
    xy = m.meta["cell_xy_nominal"]
    x, y = xy[:, 0], xy[:, 1]
    st.f[:] = w[None, :] * (x * x + y * y)[:, None]
    O.dvm_run(m, bcs, st, xi, w, 0.5, tau=1e12, dt=dt, n_steps=1)
    i, j = m.meta["cell_i"], m.meta["cell_j"]
    inner = (i >= 2) & (i <= n - 3) & (j >= 2) & (j <= n - 3)
    ex = w[None, :] * ((x * x + y * y)[:, None]
                       - 2 * dt * (xi[None, :, 0] * x[:, None] + xi[None, :, 1] * y[:, None])
                       + 2 * dt * dt * (xi[None, :, 0] ** 2 + xi[None, :, 1] ** 2))
    assert inner.sum() == (n - 4) ** 2
    err = np.abs(st.f[inner] - ex[inner]).max() / np.abs(ex[inner]).max()
    assert err <= 1e-12, err


def test_uniform_state_relaxes_at_the_bgk_rate():
    """Eq. fn+1 with no flux: a spatially uniform state on a periodic mesh has cancelling
    face fluxes, so W keeps W0 and f relaxes geometrically to its Maxwellian,
    f^n = feq(W0) + (f^0 - feq(W0)) / (1 + dt/tau)^n, whatever f^0 is."""
    xi, w = O.dvm_grid(10, 2.5)
    m = M.cartesian(4, 3, 1.0, 0.75, jitter=0.2, seed=5)
    st = O.dvm_init(m.n_cells, xi, w, rho0=1.0, u0=(0.0, 0.0), RT0=0.5)
    W0 = st.W.copy()
    geq = O.dvm_maxwell(1.0, 0.0, 0.0, 0.5, xi, w)
    g1 = O.dvm_maxwell(1.2, 0.15, -0.1, 0.65, xi, w)
    st.f[:] = g1[None, :]
    tau, dt, n = 0.05, 0.02, 7
    O.dvm_run(m, _periodic(1.0, 0.75), st, xi, w, 0.5, tau=tau, dt=dt, n_steps=n)
    ex = geq + (g1 - geq) / (1 + dt / tau) ** n
    assert np.abs(st.f - ex[None, :]).max() <= 1e-13 * np.abs(ex).max()
    assert np.abs(st.W - W0).max() <= 1e-13


def _shear_wave_decay(nx, nv, tau):
    """Decay rate of u_y = U sin(k x) on a periodic nx x 2 box of unit cells (k = 2 pi /
    nx, U = 0.01, R T = 1/2), fitted between t = 10 and t = 70."""
    m = M.cartesian(nx, 2, float(nx), 2.0)
    xi, w = O.dvm_grid(nv, 3.0)
    x = m.meta["cell_xy_nominal"][:, 0]
    k, RT = 2 * math.pi / nx, 0.5
    st = O.dvm_init(m.n_cells, xi, w, u=np.stack([0 * x, 0.01 * np.sin(k * x)], 1), RT0=RT)
    dt = 0.5 / (math.sqrt(2) * 3.0)
    bcs = _periodic(float(nx), 2.0)
    n1, n2 = int(round(10 / dt)), int(round(60 / dt))
    O.dvm_run(m, bcs, st, xi, w, RT, tau, dt, n1)
    a1 = 2 * np.mean(st.u[:, 1] * np.sin(k * x))
    O.dvm_run(m, bcs, st, xi, w, RT, tau, dt, n2)
    a2 = 2 * np.mean(st.u[:, 1] * np.sin(k * x))
    return -math.log(a2 / a1) / (n2 * dt), tau * RT * k * k


def test_shear_wave_decays_at_the_navier_stokes_rate():
    """The interface distribution f_b = c (fbar + b feq_b) (Eq. f_t_n+1) and the update
    together reproduce the BGK viscosity mu = tau p (nu = tau R T): a small shear wave
    decays at nu k^2, to within the scheme's second-order discretisation error and the
    O(Kn^2) Burnett correction.  At 32 cells per wavelength (Kn k lambda ~ 0.07) the
    rate is within 1 % of nu k^2, and the error falls by about 4 (3 to 6) from 16 to
    32 cells.  A dropped b feq_b or c factor moves the rate by far more."""
    r32, e32 = _shear_wave_decay(32, 24, 0.5)
    r16, e16 = _shear_wave_decay(16, 24, 0.5)
    d32, d16 = r32 / e32 - 1, r16 / e16 - 1
    assert abs(d32) <= 0.01, d32
    assert 3 <= d16 / d32 <= 6, (d16, d32)


def test_mirror_symmetric_state_stays_symmetric_with_tangential_nodes():
    """Reading A5 for tangential velocities (xi . n = 0: the mean of both sides' values).
    With odd nv the grid has a column xi_x = 0, tangential to every face of constant x;
    such velocities carry no flux but enter the interface moments.  On a closed box of
    walls at rest, a state symmetric under x -> L - x (rho and u_y even, u_x odd) stays
    symmetric, to round-off, only if the tie rule treats the two sides alike."""
    nx, ny, L = 6, 4, 6.0
    xi, w = O.dvm_grid(9, 2.0)
    m = M.cartesian(nx, ny, L, 4.0)
    bcs = [(p, M.BC_WALL, (0, 0, 0)) for p in range(4)]
    xy = m.meta["cell_xy_nominal"]
    X, Y = 2 * np.pi * (xy[:, 0] - L / 2) / L, np.pi * xy[:, 1] / 4.0
    st = O.dvm_init(m.n_cells, xi, w, rho=1 + 0.05 * np.cos(X),
                    u=np.stack([0.05 * np.sin(X) * np.sin(Y), 0.02 * np.cos(X) * np.sin(Y)], 1),
                    RT=0.5 + 0.02 * np.cos(X))
    O.dvm_run(m, bcs, st, xi, w, 0.5, tau=0.1, dt=0.05, n_steps=20)
    i, j = m.meta["cell_i"], m.meta["cell_j"]
    mir = (nx - 1 - i) + nx * j
    assert np.abs(st.rho - st.rho[mir]).max() <= 1e-12
    assert np.abs(st.u[:, 0] + st.u[mir, 0]).max() <= 1e-12
    assert np.abs(st.u[:, 1] - st.u[mir, 1]).max() <= 1e-12
    assert np.abs(st.RT - st.RT[mir]).max() <= 1e-12
    assert np.abs(st.u[:, 0]).max() > 1e-3


_SIDES = {
    "periodic": ({"bottom": ("periodic",), "top": ("periodic",), "left": ("periodic",), "right": ("periodic",)},
                 lambda lx, ly: _periodic(lx, ly)),
    "channel": ({"bottom": ("wall", 0.0, 0.0), "top": ("wall", 0.1, 0.0), "left": ("periodic",),
                 "right": ("periodic",)},
                lambda lx, ly: [(3, M.BC_PERIODIC, (1, lx, 0.0)), (1, M.BC_PERIODIC, (3, -lx, 0.0)),
                                (0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.1, 0, 0))]),
    "box": ({"bottom": ("wall", 0.0, 0.0), "top": ("wall", 0.1, 0.0), "left": ("wall", 0.0, 0.0),
             "right": ("wall", 0.0, 0.0)},
            lambda lx, ly: [(0, M.BC_WALL, (0, 0, 0)), (1, M.BC_WALL, (0, 0, 0)), (3, M.BC_WALL, (0, 0, 0)),
                            (2, M.BC_MOVING_WALL, (0.1, 0, 0))]),
}


@pytest.mark.parametrize("kind,nv", [("periodic", 4), ("channel", 4), ("box", 4), ("periodic", 5), ("box", 5)])
def test_hand_stepped_against_a_40_digit_restatement(kind, nv):
    """Three steps on a 3 x 3 grid of 1/3 x 1/4 cells with a 4 x 4 velocity grid (5 x 5:
    nodes at zero velocity, tangential to every face: the tie rule), from a
    non-uniform state (density, velocity and temperature vary from cell to cell),
    against ``oracle/handstep_dvm.py``: the same step written cell by cell with explicit
    neighbours and faces in 40-digit arithmetic.  Periodic sides, a channel between a
    resting and a moving diffuse wall, and a closed box (corner cells with two LLSR
    neighbours).  The FP64 oracle agrees to FP64 rounding: about 4e-16 of the largest
    value measured, 1e-14 asserted, while the state changes by about 5 % over the three
    steps."""
    mp = pytest.importorskip("mpmath")
    from oracle import handstep_dvm as H
    nx, ny, lx, ly, vmax = 3, 3, 1.0, 0.75, 2.0
    tau, dt, RTw, steps = 0.05, 0.02, 0.5, 3
    sides, bcs = _SIDES[kind]
    xi, w = O.dvm_grid(nv, vmax)
    m = M.cartesian(nx, ny, lx, ly)
    rng = np.random.default_rng(11)
    st = O.dvm_init(m.n_cells, xi, w, rho=1 + 0.1 * rng.uniform(-1, 1, m.n_cells),
                    u=0.1 * rng.uniform(-1, 1, (m.n_cells, 2)), RT=0.5 + 0.05 * rng.uniform(-1, 1, m.n_cells))
    g = H.Grid(nx, ny, lx / nx, ly / ny, sides, nv, vmax)
    fh, Wh = H.run(g, st.f, st.W, tau, dt, RTw, steps)
    O.dvm_run(m, bcs(lx, ly), st, xi, w, RTw, tau=tau, dt=dt, n_steps=steps)
    fh = np.array([[float(v) for v in row] for row in fh])
    Wh = np.array([[float(v) for v in row] for row in Wh])
    assert np.abs(st.f - fh).max() <= 1e-14 * np.abs(fh).max()
    assert np.abs(st.W - Wh).max() <= 1e-14 * np.abs(Wh).max()
    assert np.abs(Wh[:, 1:3]).max() > 1e-3                  # the state is not at rest
