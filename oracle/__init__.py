"""FP64 CPU oracle of the S-DUGKS step -- TEST INFRASTRUCTURE.

Only tests/, the package smoke check and the benchmark's CPU-baseline leg import
this.  It builds ``sdugks_oracle.c`` with gcc (FP64, ``-ffp-contract=off``, OpenMP
over independent cell and face loops) and wraps it with ctypes.  It shares no code
with the CUDA library.

Every routine is pinned by the CPU tests in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdugks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsdugks_oracle.so")
_lock = threading.Lock()
_lib = None

NQ = 9
KIND_PERIODIC = 1          # boundary kind codes as the oracle's C source numbers them
XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)


def compile_library(src: str, out: str) -> str:
    """gcc with the oracle's flags (FP64, no contraction, OpenMP); returns ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_library(_SRC, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # SDUGKS_ORACLE_LIB: another build of this source (the planted-mistake sweep
            # of tests/oracle_mutation_sweep.py); otherwise the in-tree build
            lib = C.CDLL(os.environ.get("SDUGKS_ORACLE_LIB") or build())
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            mesh_args = [i64, P, i64, P, P, P, i64, i32, P, P]
            lib.oracle_feq.argtypes = [dbl, dbl, dbl, P]
            lib.oracle_geometry.argtypes = mesh_args + [P, P, P, P, P, P]
            lib.oracle_gradient.argtypes = mesh_args + [P, P]
            lib.oracle_run.argtypes = mesh_args + [dbl, dbl, i64, P, P]
            lib.oracle_run_flux.argtypes = mesh_args + [dbl, dbl, i64, P, P, P]
            lib.oracle_init.argtypes = [i64, P, P, P, P]
            lib.oracle_residual.argtypes = [i64, P, P, P, P, P]
            lib.oracle_set_threads.argtypes = [i32]
            lib.oracle_dvm_grid.argtypes = [i32, dbl, P, P]
            lib.oracle_dvm_maxwell.argtypes = [dbl, dbl, dbl, dbl, i32, P, P, P]
            lib.oracle_dvm_init.argtypes = [i64, i32, P, P, P, P, P, P, P]
            lib.oracle_dvm_run.argtypes = mesh_args + [i32, P, P, dbl, dbl, dbl, i64, P, P]
            for fn in ("oracle_feq", "oracle_geometry", "oracle_gradient", "oracle_run", "oracle_run_flux",
                       "oracle_init", "oracle_residual", "oracle_set_threads", "oracle_dvm_grid",
                       "oracle_dvm_maxwell", "oracle_dvm_init", "oracle_dvm_run"):
                getattr(lib, fn).restype = C.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


class _MeshArgs:
    """Keeps contiguous copies of the mesh/BC arrays alive for a call."""

    def __init__(self, mesh, bcs):
        self.xy = np.ascontiguousarray(mesh.points, np.float64)
        self.fp = np.ascontiguousarray(mesh.face_pts, np.int64)
        self.own = np.ascontiguousarray(mesh.owner, np.int64)
        self.nbr = np.ascontiguousarray(mesh.neighbour, np.int64)
        npatch = max([p for p, _, _ in bcs] + [int(-1 - mesh.neighbour.min()) if mesh.neighbour.min() < 0 else -1]) + 1
        self.kind = np.zeros(max(npatch, 1), np.int32)
        self.par = np.zeros((max(npatch, 1), 3), np.float64)
        for p, k, par in bcs:
            self.kind[p] = k
            self.par[p] = par
        self.npatch = len(self.kind)
        self.nc = int(mesh.n_cells)
        self.nf = int(self.fp.shape[0])
        self.np = int(self.xy.shape[0])

    def args(self):
        return [self.np, _p(self.xy), self.nf, _p(self.fp), _p(self.own), _p(self.nbr), self.nc,
                self.npatch, _p(self.kind), _p(self.par)]


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.empty(NQ)
    _check(_load().oracle_feq(rho, ux, uy, _p(out)), "feq")
    return out


def geometry(mesh, bcs):
    m = _MeshArgs(mesh, bcs)
    vol = np.empty(m.nc); xc = np.empty((m.nc, 2)); ainv = np.empty((m.nc, 3))
    nl = np.empty((m.nf, 2)); xf = np.empty((m.nf, 2)); ghost = np.empty(m.nf, np.int64)
    _check(_load().oracle_geometry(*m.args(), _p(vol), _p(xc), _p(ainv), _p(nl), _p(xf), _p(ghost)),
           "geometry")
    return dict(vol=vol, xc=xc, ainv=ainv, nl=nl, xf=xf, ghost=ghost)


def gradient(mesh, bcs, phi):
    m = _MeshArgs(mesh, bcs)
    phi = np.ascontiguousarray(phi, np.float64)
    g = np.empty((m.nc, 2))
    _check(_load().oracle_gradient(*m.args(), _p(phi), _p(g)), "gradient")
    return g


class State:
    """Oracle state at t_n: f [N,9], W [N,3] = (rho, rho u)."""

    def __init__(self, f, W):
        self.f, self.W = f, W

    def copy(self):
        return State(self.f.copy(), self.W.copy())

    @property
    def rho(self):
        return self.W[:, 0]

    @property
    def u(self):
        return self.W[:, 1:] / self.W[:, :1]


def init(n_cells: int, rho=None, u=None, rho0: float = 1.0, u0=(0.0, 0.0)) -> State:
    rho = np.full(n_cells, rho0) if rho is None else np.ascontiguousarray(rho, np.float64)
    u = np.tile(np.asarray(u0, float), (n_cells, 1)) if u is None else np.ascontiguousarray(u, np.float64)
    f = np.empty((n_cells, NQ)); W = np.empty((n_cells, 3))
    _check(_load().oracle_init(n_cells, _p(rho), _p(u), _p(f), _p(W)), "init")
    return State(f, W)


def run(case, state: State, n_steps: int, *, tau=None, dt=None) -> State:
    """Advance ``state`` in place by n_steps steps of the case's mesh/BCs."""
    m = _MeshArgs(case.mesh, case.bcs)
    for a in (state.f, state.W):
        assert a.flags.c_contiguous and a.dtype == np.float64
    _check(_load().oracle_run(*m.args(), float(case.tau if tau is None else tau),
                              float(case.dt if dt is None else dt), int(n_steps),
                              _p(state.f), _p(state.W)), "run")
    return state


def boundary_faces(mesh, bcs) -> np.ndarray:
    """Ids of the faces that get a row in run_flux: neighbour < 0 and a patch that is
    not periodic, in ascending face id."""
    kind = {p: k for p, k, _ in bcs}
    nb = np.asarray(mesh.neighbour)
    return np.array([f for f in range(len(nb)) if nb[f] < 0 and kind.get(int(-1 - nb[f])) != KIND_PERIODIC],
                    np.int64)


def run_flux(case, state: State, n_steps: int, *, tau=None, dt=None) -> np.ndarray:
    """Advance ``state`` in place by n_steps >= 1 steps and return the momentum that
    left the fluid through each non-periodic boundary face in the last step,
    [len(boundary_faces), 2] (sum_a xi_a (xi_a . n l) f_b,a, n l out of the fluid)."""
    m = _MeshArgs(case.mesh, case.bcs)
    for a in (state.f, state.W):
        assert a.flags.c_contiguous and a.dtype == np.float64
    nb = len(boundary_faces(case.mesh, case.bcs))
    # room for a row per face, the rows past the boundary faces' marked: a row count
    # other than the boundary faces' shows up as an error instead of a buffer overrun
    out = np.full((m.nf, 2), np.nan)
    _check(_load().oracle_run_flux(*m.args(), float(case.tau if tau is None else tau),
                                   float(case.dt if dt is None else dt), int(n_steps),
                                   _p(state.f), _p(state.W), _p(out)), "run_flux")
    if not np.isnan(out[nb:]).all():
        raise RuntimeError("oracle run_flux wrote more rows than there are non-periodic boundary faces")
    return out[:nb].copy()


def residual(W, Ws, vol=None):
    W = np.ascontiguousarray(W, np.float64); Ws = np.ascontiguousarray(Ws, np.float64)
    eps = np.empty(1); mass = np.empty(1)
    v = None if vol is None else np.ascontiguousarray(vol, np.float64)
    _check(_load().oracle_residual(W.shape[0], _p(W), _p(Ws), None if v is None else _p(v),
                                   _p(eps), _p(mass)), "residual")
    return float(eps[0]), float(mass[0])


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return int(_load().oracle_set_threads(int(n)))


# ---------------------------------------------------------------- rarefied (discrete velocity grid)

def dvm_grid(nv: int, vmax: float):
    """Velocity nodes xi [Q, 2] (x fastest) and weights w [Q] of the nv x nv midpoint grid on
    [-vmax, vmax]^2."""
    xi = np.empty((nv * nv, 2)); w = np.empty(nv * nv)
    _check(_load().oracle_dvm_grid(nv, vmax, _p(xi), _p(w)), "dvm_grid")
    return xi, w


def dvm_maxwell(rho, ux, uy, RT, xi, w) -> np.ndarray:
    xi = np.ascontiguousarray(xi, np.float64); w = np.ascontiguousarray(w, np.float64)
    out = np.empty(len(w))
    _check(_load().oracle_dvm_maxwell(rho, ux, uy, RT, len(w), _p(xi), _p(w), _p(out)), "dvm_maxwell")
    return out


class DvmState:
    """Rarefied oracle state: f [N, Q] (weighted), W [N, 4] = (rho, rho u, rho E)."""

    def __init__(self, f, W):
        self.f, self.W = f, W

    @property
    def rho(self):
        return self.W[:, 0]

    @property
    def u(self):
        return self.W[:, 1:3] / self.W[:, :1]

    @property
    def RT(self):
        u = self.u
        return self.W[:, 3] / self.W[:, 0] - 0.5 * (u ** 2).sum(1)


def dvm_init(n_cells, xi, w, rho=None, u=None, RT=None, rho0=1.0, u0=(0.0, 0.0), RT0=0.5) -> DvmState:
    xi = np.ascontiguousarray(xi, np.float64); w = np.ascontiguousarray(w, np.float64)
    rho = np.full(n_cells, rho0) if rho is None else np.ascontiguousarray(rho, np.float64)
    u = np.tile(np.asarray(u0, float), (n_cells, 1)) if u is None else np.ascontiguousarray(u, np.float64)
    RT = np.full(n_cells, RT0) if RT is None else np.ascontiguousarray(RT, np.float64)
    Q = len(w)
    f = np.empty((n_cells, Q)); W = np.empty((n_cells, 4))
    _check(_load().oracle_dvm_init(n_cells, Q, _p(xi), _p(w), _p(rho), _p(u), _p(RT), _p(f), _p(W)), "dvm_init")
    return DvmState(f, W)


def dvm_run(mesh, bcs, state: DvmState, xi, w, RT_wall: float, tau: float, dt: float, n_steps: int) -> DvmState:
    """Advance the rarefied state in place (diffuse walls at R T_wall, periodic faces)."""
    m = _MeshArgs(mesh, bcs)
    xi = np.ascontiguousarray(xi, np.float64); w = np.ascontiguousarray(w, np.float64)
    for a in (state.f, state.W):
        assert a.flags.c_contiguous and a.dtype == np.float64
    _check(_load().oracle_dvm_run(*m.args(), len(w), _p(xi), _p(w), RT_wall, tau, dt, n_steps,
                                  _p(state.f), _p(state.W)), "dvm_run")
    return state
