"""GPU parity of the rarefied solver (sdugks_dvm, discrete velocity grid, diffuse
walls) with the FP64 oracle, through the C-ABI.

Tolerances: FP64 max |gpu - oracle| / max |oracle| <= 1e-12 for f and W (the block
reductions over the velocity grid sum in another order than the oracle's sequential
sums); FP32 (f, scratch and per-thread partial sums in FP32, moments combined and W
kept in FP64): relative L2 of u <= 1e-4 and max |rho - rho_oracle| <= 1e-5 after the
stated steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu


def _S():
    from paper_2007_07347_gb300 import sdugks as S
    return S


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cavity_jittered(n=6):
    m = M.cartesian(n, n, 1.0, 1.0, jitter=0.15, seed=4)
    bcs = [(0, M.BC_WALL, (0, 0, 0)), (1, M.BC_WALL, (0, 0, 0)), (3, M.BC_WALL, (0, 0, 0)),
           (2, M.BC_MOVING_WALL, (0.1, 0, 0))]
    return m, bcs


def _channel():
    m = M.hybrid(8, 6, 1.0, 0.75, tri_from=0.5, jitter=0.1, seed=2, quad_rows=1)
    bcs = [(3, M.BC_PERIODIC, (1, 1.0, 0.0)), (1, M.BC_PERIODIC, (3, -1.0, 0.0)),
           (0, M.BC_WALL, (0, 0, 0)), (2, M.BC_MOVING_WALL, (0.15, 0.0, 0))]
    return m, bcs


def _run(m, bcs, nv, vmax, RTw, tau, dt, steps, precision, rho=None, u=None, RT=None):
    S = _S()
    d = S.Dvm(S.Mesh(m, bcs), nv, vmax, RTw, tau, dt, precision).init(rho, u, RT)
    d.step(steps)
    xi, w = O.dvm_grid(nv, vmax)
    st = O.dvm_init(m.n_cells, xi, w, rho=rho, u=u, RT=RT, RT0=RTw)
    O.dvm_run(m, bcs, st, xi, w, RTw, tau, dt, steps)
    return d, st


@pytest.mark.parametrize("tau", [0.05, 2.0])
def test_fp64_cavity_matches_oracle(tau):
    m, bcs = _cavity_jittered()
    d, st = _run(m, bcs, 12, 2.0, 0.5, tau, 0.01, 60, "fp64")
    f, W = d.get_state()
    assert relmax(f, st.f) <= 1e-12
    assert relmax(W, st.W) <= 1e-12
    assert np.abs(st.u).max() > 1e-3


@pytest.mark.parametrize("nv", [9, 11])
def test_fp64_odd_velocity_grid_matches_oracle(nv):
    """Odd nv: the kernels take one velocity per thread at a time (nv a multiple of 4
    takes 16-byte vectors of 4 velocities; the nv = 10 channel below is even but also
    takes one at a time)."""
    m, bcs = _cavity_jittered(5)
    d, st = _run(m, bcs, nv, 2.0, 0.5, 0.1, 0.01, 40, "fp64")
    f, W = d.get_state()
    assert relmax(f, st.f) <= 1e-12
    assert relmax(W, st.W) <= 1e-12


@pytest.mark.parametrize("nv", [144, 145])
def test_fp64_rows_beyond_the_shared_buffer_match_oracle(nv):
    """Q x 8 bytes above the kernels' 160 KB shared-memory buffer: the face and cell
    kernels keep the interface values and flux sums in global memory instead (nv = 144
    with vectors of 4 velocities, 145 with one)."""
    m, bcs = _cavity_jittered(4)
    d, st = _run(m, bcs, nv, 2.0, 0.5, 0.1, 0.01, 12, "fp64")
    f, W = d.get_state()
    assert relmax(f, st.f) <= 1e-12
    assert relmax(W, st.W) <= 1e-12
    assert np.abs(st.u).max() > 1e-3


def test_fp32_rows_beyond_the_shared_buffer_match_oracle():
    """FP32 rows above the 160 KB buffer (nv = 204, Q x 4 bytes = 166 KB)."""
    m, bcs = _cavity_jittered(4)
    d, st = _run(m, bcs, 204, 2.0, 0.5, 0.1, 0.01, 30, "fp32")
    rho, u, RT = d.macros()
    assert np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2)) <= 1e-4
    assert np.abs(rho - st.rho).max() <= 1e-5
    assert np.abs(RT - st.RT).max() <= 1e-5


def test_fp64_periodic_hybrid_channel_matches_oracle():
    m, bcs = _channel()
    rng = np.random.default_rng(3)
    rho = 1 + 0.02 * rng.uniform(-1, 1, m.n_cells)
    u = 0.03 * rng.uniform(-1, 1, (m.n_cells, 2))
    RT = 0.5 + 0.01 * rng.uniform(-1, 1, m.n_cells)
    d, st = _run(m, bcs, 10, 2.5, 0.5, 0.1, 0.008, 50, "fp64", rho, u, RT)
    f, W = d.get_state()
    assert relmax(f, st.f) <= 1e-12
    assert relmax(W, st.W) <= 1e-12


def test_fp32_micro_cavity_matches_oracle():
    case = M.micro_cavity(16, Kn=0.5, nv=24)
    m, bcs = case.mesh, case.bcs
    d, st = _run(m, bcs, 24, 2.0, 0.5, case.tau, case.dt, 300, "fp32")
    rho, u, RT = d.macros()
    assert np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2)) <= 1e-4
    assert np.abs(rho - st.rho).max() <= 1e-5
    assert np.abs(RT - st.RT).max() <= 1e-5


def test_fp32_one_velocity_per_thread_matches_oracle():
    """FP32 with nv = 10 (not a multiple of 4): the kernels take one velocity per
    thread at a time."""
    case = M.micro_cavity(12, Kn=0.5, nv=10)
    m, bcs = case.mesh, case.bcs
    d, st = _run(m, bcs, 10, 2.0, 0.5, case.tau, case.dt, 200, "fp32")
    rho, u, RT = d.macros()
    assert np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2)) <= 1e-4
    assert np.abs(rho - st.rho).max() <= 1e-5
    assert np.abs(RT - st.RT).max() <= 1e-5


def test_diffuse_walls_conserve_mass_fp32():
    case = M.micro_cavity(20, Kn=1.0, nv=32)
    S = _S()
    d = S.Dvm.from_case(case, "fp32").init()
    rho0, _, _ = d.macros()
    d.step(2000)
    rho, u, RT = d.macros()
    assert np.all(np.isfinite(rho)) and np.abs(u).max() > 1e-3
    assert abs(rho.sum() / rho0.sum() - 1.0) <= 1e-6


def test_full_size_micro_cavity_fp64_against_oracle():
    """The paper's grid: 40 x 40 cells, 100 x 100 velocities on [-2, 2]^2, Kn = 1."""
    case = M.micro_cavity(40, Kn=1.0)
    d, st = _run(case.mesh, case.bcs, 100, 2.0, 0.5, case.tau, case.dt, 10, "fp64")
    f, W = d.get_state()
    assert relmax(f, st.f) <= 1e-12
    assert relmax(W, st.W) <= 1e-12


def test_dvm_errors_are_status_codes():
    S = _S()
    m, bcs = _cavity_jittered(4)
    mesh = S.Mesh(m, bcs)
    with pytest.raises(S.SdugksError) as e:
        S.Dvm(mesh, 1, 2.0, 0.5, 0.1, 0.01)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(S.SdugksError) as e:
        S.Dvm(mesh, 8, 2.0, 0.5, 0.1, 0.01, "bf16dev")
    assert e.value.name == "INVALID_ARG"
    d = S.Dvm(mesh, 8, 2.0, 0.5, 0.1, 0.01)
    with pytest.raises(S.SdugksError) as e:
        d.step(1)
    assert e.value.name == "STATE"
