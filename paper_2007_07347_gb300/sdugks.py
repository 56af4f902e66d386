"""ctypes binding of libsdugks (include/sdugks.h): argument marshalling only.

Every step of the S-DUGKS update runs in the library's CUDA kernels; this module
converts numpy arrays and torch tensors to pointers and raises ``SdugksError`` on a
non-zero status.  There is no fallback: if the library cannot be built or loaded,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

from . import build as _build
from . import meshes as _meshes

_lock = threading.Lock()
_lib = None

FP64, FP32, FP32_BF16DEV, FP32_FP16DEV = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_TILED, KERNEL_CARTESIAN = 0, 1, 2
STAGING_LOADS, STAGING_TMA = 0, 1
STAGINGS = {"loads": STAGING_LOADS, "tma": STAGING_TMA}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16dev": FP32_BF16DEV, "fp16dev": FP32_FP16DEV}
ERRORS = {-1: "INVALID_ARG", -2: "INVALID_MESH", -3: "BAD_BC", -4: "OOM", -5: "DIVERGED", -6: "TIMEOUT",
          -7: "CUDA", -8: "STATE", -9: "FULL"}


class SdugksError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("dt", C.c_double), ("precision", C.c_int32), ("kernel", C.c_int32),
                ("tile_cells", C.c_int32), ("graph_steps", C.c_int32), ("staging", C.c_int32),
                ("tma_wait_us", C.c_int32)]


class TuneInfo(C.Structure):
    _fields_ = [("ns_per_step", C.c_double), ("candidates", C.c_int32), ("from_cache", C.c_int32),
                ("kernel", C.c_int32), ("pad_", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("n_tiles", C.c_int64), ("halo_cells", C.c_int64),
                ("steps_done", C.c_int64), ("device_bytes", C.c_int64), ("state_bytes_per_cell_step", C.c_double),
                ("mesh_bytes_per_cell_step", C.c_double), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("tile_cells", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("staging", C.c_int32),
                ("one_code_path", C.c_int32), ("n_boundary_faces", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def header_functions() -> list[str]:
    """Names of the functions declared in include/sdugks.h."""
    with open(os.path.join(_build.INCLUDE, "sdugks.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdugks_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Build (if stale) and load libsdugks; raises if that is not possible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            P, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            sig = {
                "sdugks_mesh_create": [i64, P, i64, P, P, P, i64, P],
                "sdugks_set_bc": [P, i32, i32, P],
                "sdugks_mesh_cfl_dt": [P, dbl, P],
                "sdugks_mesh_sizes": [P, P, P, P],
                "sdugks_solver_create": [P, P, P, P],
                "sdugks_init": [P, P, P],
                "sdugks_step": [P, i64],
                "sdugks_get_macros": [P, P, P],
                "sdugks_get_macros_device": [P, P, P],
                "sdugks_residual": [P, P, P],
                "sdugks_get_state": [P, P, P],
                "sdugks_set_state": [P, P, P],
                "sdugks_get_state_raw": [P, P, P],
                "sdugks_set_state_raw": [P, P, i64],
                "sdugks_solver_info": [P, P],
                "sdugks_step_forces": [P, P],
                "sdugks_step_boundary_flux": [P, P, P],
                "sdugks_autotune": [P, P, i64, P, P, P],
                "sdugks_residual_noalloc": [i64, P, P, P, P, P],
                "sdugks_batch_create": [i64, i32, i32, P, P],
                "sdugks_batch_footprint": [P, P, P],
                "sdugks_batch_add": [P, P, dbl, dbl, P, P, P],
                "sdugks_batch_remove": [P, i64],
                "sdugks_batch_step": [P, i64],
                "sdugks_batch_residual": [P, P, P, P, P, P],
                "sdugks_batch_get_macros": [P, i64, P, P],
                "sdugks_batch_autotune": [P, i64],
                "sdugks_batch_info": [P, P],
                "sdugks_dvm_create": [P, P, P, P],
                "sdugks_dvm_init": [P, P, P, P],
                "sdugks_dvm_step": [P, i64],
                "sdugks_dvm_get_macros": [P, P, P, P],
                "sdugks_dvm_get_state": [P, P, P],
                "sdugks_dvm_sizes": [P, P, P, P, P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.sdugks_mesh_destroy.argtypes = [P]
            L.sdugks_mesh_destroy.restype = None
            L.sdugks_solver_destroy.argtypes = [P]
            L.sdugks_solver_destroy.restype = None
            L.sdugks_batch_destroy.argtypes = [P]
            L.sdugks_batch_destroy.restype = None
            L.sdugks_dvm_destroy.argtypes = [P]
            L.sdugks_dvm_destroy.restype = None
            L.sdugks_autotune_clear.argtypes = []
            L.sdugks_autotune_clear.restype = None
            L.sdugks_last_error.restype = C.c_char_p
            L.sdugks_version.restype = C.c_char_p
            _lib = L
    return _lib


def _ck(rc: int, what: str):
    if rc != 0:
        raise SdugksError(rc, what, lib().sdugks_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Mesh:
    """sdugks_mesh: geometry from a face-based owner/neighbour mesh plus boundary table."""

    def __init__(self, mesh: _meshes.Mesh, bcs=()):
        L = lib()
        self._h = C.c_void_p()
        xy = _f64(mesh.points)
        fp = np.ascontiguousarray(mesh.face_pts, np.int64)
        own = np.ascontiguousarray(mesh.owner, np.int64)
        nbr = np.ascontiguousarray(mesh.neighbour, np.int64)
        _ck(L.sdugks_mesh_create(xy.shape[0], _ptr(xy), fp.shape[0], _ptr(fp), _ptr(own), _ptr(nbr),
                                 int(mesh.n_cells), C.byref(self._h)), "sdugks_mesh_create")
        self.n_cells = int(mesh.n_cells)
        for patch, kind, par in bcs:
            self.set_bc(patch, kind, par)

    def set_bc(self, patch: int, kind: int, params=(0.0, 0.0, 0.0)):
        p = _f64(list(params) + [0.0] * (3 - len(params)))
        _ck(lib().sdugks_set_bc(self._h, int(patch), int(kind), _ptr(p)), "sdugks_set_bc")

    def cfl_dt(self, cfl: float) -> float:
        out = C.c_double()
        _ck(lib().sdugks_mesh_cfl_dt(self._h, float(cfl), C.byref(out)), "sdugks_mesh_cfl_dt")
        return out.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sdugks_mesh_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """sdugks_solver on the current CUDA device; ``stream`` is a torch.cuda.Stream,
    a raw cudaStream_t integer, or None for the default stream.  ``staging`` ("loads" or
    "tma") picks how the Cartesian kernel stages its interior blocks."""

    def __init__(self, mesh: Mesh, tau: float, dt: float, precision="fp32", *, kernel=KERNEL_AUTO,
                 tile_cells=0, graph_steps=0, staging="loads", tma_wait_us=0, stream=None):
        L = lib()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        stg = STAGINGS[staging] if isinstance(staging, str) else int(staging)
        self.params = Params(float(tau), float(dt), prec, int(kernel), int(tile_cells), int(graph_steps), stg,
                             int(tma_wait_us))
        sh = getattr(stream, "cuda_stream", stream)
        self._h = C.c_void_p()
        _ck(L.sdugks_solver_create(mesh._h, C.byref(self.params), C.c_void_p(sh or 0), C.byref(self._h)),
            "sdugks_solver_create")
        self.n = mesh.n_cells

    @classmethod
    def from_case(cls, case: _meshes.Case, precision="fp32", **kw):
        m = Mesh(case.mesh, case.bcs)
        s = cls(m, case.tau, case.dt, precision, **kw)
        s._mesh = m
        return s

    @classmethod
    def tuned(cls, case: _meshes.Case, precision="fp32", *, kernel=KERNEL_AUTO, steps=256, stream=None):
        """A solver of the case with the launch configuration sdugks_autotune picks (the
        tuning result is cached per mesh, precision and kernel request); the chosen
        configuration and its measured time are in ``.tune``."""
        m = Mesh(case.mesh, case.bcs)
        t = autotune(m, case.tau, case.dt, precision, kernel=kernel, steps=steps, stream=stream)
        s = cls(m, case.tau, case.dt, precision, kernel=kernel, tile_cells=t["tile_cells"],
                graph_steps=t["graph_steps"], staging=t["staging"], stream=stream)
        s._mesh = m
        s.tune = t
        return s

    def init(self, rho=None, u=None):
        r = None if rho is None else _f64(rho, (self.n,))
        v = None if u is None else _f64(u, (self.n, 2))
        _ck(lib().sdugks_init(self._h, _ptr(r), _ptr(v)), "sdugks_init")
        return self

    def step(self, n: int = 1):
        _ck(lib().sdugks_step(self._h, int(n)), "sdugks_step")
        return self

    def step_forces(self) -> np.ndarray:
        """One step; returns [64, 2]: the force of the fluid on each boundary patch."""
        out = np.zeros((64, 2))
        _ck(lib().sdugks_step_forces(self._h, _ptr(out)), "sdugks_step_forces")
        return out

    def step_boundary_flux(self, forces: bool = False):
        """One step; returns [n_boundary_faces, 2]: the momentum leaving the fluid through
        each non-periodic boundary face (caller's face order), and with ``forces`` also
        the [64, 2] patch sums of sdugks_step_forces."""
        out = np.zeros((self.info()["n_boundary_faces"], 2))
        frc = np.zeros((64, 2)) if forces else None
        _ck(lib().sdugks_step_boundary_flux(self._h, _ptr(frc), _ptr(out)), "sdugks_step_boundary_flux")
        return (out, frc) if forces else out

    def macros(self):
        rho = np.empty(self.n)
        u = np.empty((self.n, 2))
        _ck(lib().sdugks_get_macros(self._h, _ptr(rho), _ptr(u)), "sdugks_get_macros")
        return rho, u

    def macros_device(self, rho_t=None, u_t=None):
        """Write rho [n] and u [n, 2] (FP64 torch CUDA tensors) on the solver's stream."""
        _ck(lib().sdugks_get_macros_device(self._h, C.c_void_p(rho_t.data_ptr() if rho_t is not None else 0),
                                           C.c_void_p(u_t.data_ptr() if u_t is not None else 0)),
            "sdugks_get_macros_device")

    def residual(self):
        eps, mass = C.c_double(), C.c_double()
        _ck(lib().sdugks_residual(self._h, C.byref(eps), C.byref(mass)), "sdugks_residual")
        return eps.value, mass.value

    def get_state(self):
        f = np.empty((self.n, 9)); W = np.empty((self.n, 3))
        _ck(lib().sdugks_get_state(self._h, _ptr(f), _ptr(W)), "sdugks_get_state")
        return f, W

    def get_state_into(self, f, W):
        """Like get_state into caller-provided (e.g. pinned) float64 arrays."""
        _ck(lib().sdugks_get_state(self._h, _ptr(f), _ptr(W)), "sdugks_get_state")

    def get_state_raw(self) -> np.ndarray:
        """The state in the solver's own storage (bytes): restores bit for bit."""
        n = C.c_int64(0)
        _ck(lib().sdugks_get_state_raw(self._h, None, C.byref(n)), "sdugks_get_state_raw")
        buf = np.empty(n.value, np.uint8)
        _ck(lib().sdugks_get_state_raw(self._h, _ptr(buf), C.byref(n)), "sdugks_get_state_raw")
        return buf

    def set_state_raw(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        _ck(lib().sdugks_set_state_raw(self._h, _ptr(buf), int(buf.size)), "sdugks_set_state_raw")
        return self

    def set_state(self, f, W):
        f = _f64(f, (self.n, 9)); W = _f64(W, (self.n, 3))
        _ck(lib().sdugks_set_state(self._h, _ptr(f), _ptr(W)), "sdugks_set_state")
        return self

    def info(self) -> dict:
        out = Info()
        _ck(lib().sdugks_solver_info(self._h, C.byref(out)), "sdugks_solver_info")
        return out.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sdugks_solver_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(mesh: Mesh, tau: float, dt: float, precision="fp32", *, kernel=KERNEL_AUTO, steps=256,
             stream=None) -> dict:
    """sdugks_autotune: the fastest launch configuration of a solve on this device, as
    {tile_cells, graph_steps, staging, ns_per_step, candidates, from_cache, kernel}."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    base = Params(float(tau), float(dt), prec, int(kernel), 0, 0, STAGINGS["loads"], 0)
    best = Params()
    info = TuneInfo()
    sh = getattr(stream, "cuda_stream", stream)
    _ck(lib().sdugks_autotune(mesh._h, C.byref(base), int(steps), C.c_void_p(sh or 0), C.byref(best),
                              C.byref(info)), "sdugks_autotune")
    return {"tile_cells": best.tile_cells, "graph_steps": best.graph_steps, "staging": best.staging,
            "ns_per_step": info.ns_per_step, "candidates": info.candidates, "from_cache": info.from_cache,
            "kernel": info.kernel}


def autotune_clear():
    lib().sdugks_autotune_clear()


class BatchStatus(C.Structure):
    _fields_ = [("instances", C.c_int64), ("cells", C.c_int64), ("items", C.c_int64), ("pool_bytes", C.c_int64),
                ("pool_used", C.c_int64), ("steps", C.c_int64), ("grid", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("graph_steps", C.c_int32), ("precision", C.c_int32), ("per_item", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Batch:
    """sdugks_batch: many uniform-grid solves advanced by one batched kernel per step."""

    def __init__(self, pool_bytes: int, precision="fp32", max_instances: int = 1024, stream=None):
        L = lib()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        sh = getattr(stream, "cuda_stream", stream)
        self._h = C.c_void_p()
        _ck(L.sdugks_batch_create(int(pool_bytes), prec, int(max_instances), C.c_void_p(sh or 0), C.byref(self._h)),
            "sdugks_batch_create")
        self.max_instances = int(max_instances)
        self.n_cells = {}

    def footprint(self, mesh: Mesh) -> int:
        out = C.c_int64()
        _ck(lib().sdugks_batch_footprint(self._h, mesh._h, C.byref(out)), "sdugks_batch_footprint")
        return out.value

    def add(self, mesh: Mesh, tau: float, dt: float, rho=None, u=None) -> int:
        r = None if rho is None else _f64(rho, (mesh.n_cells,))
        v = None if u is None else _f64(u, (mesh.n_cells, 2))
        out = C.c_int64()
        _ck(lib().sdugks_batch_add(self._h, mesh._h, float(tau), float(dt), _ptr(r), _ptr(v), C.byref(out)),
            "sdugks_batch_add")
        self.n_cells[out.value] = mesh.n_cells
        return out.value

    def add_case(self, case: _meshes.Case, rho=None, u=None) -> int:
        m = Mesh(case.mesh, case.bcs)
        return self.add(m, case.tau, case.dt, rho, u)

    def remove(self, ident: int):
        _ck(lib().sdugks_batch_remove(self._h, int(ident)), "sdugks_batch_remove")
        self.n_cells.pop(ident, None)

    def step(self, n: int = 1):
        _ck(lib().sdugks_batch_step(self._h, int(n)), "sdugks_batch_step")
        return self

    def residual(self) -> dict:
        """{id: (eps, mass, steps since admission)} for every active instance."""
        m = self.max_instances
        ids = np.empty(m, np.int64); eps = np.empty(m); mass = np.empty(m); steps = np.empty(m, np.int64)
        cnt = C.c_int64()
        _ck(lib().sdugks_batch_residual(self._h, _ptr(ids), _ptr(eps), _ptr(mass), _ptr(steps), C.byref(cnt)),
            "sdugks_batch_residual")
        k = cnt.value
        return {int(i): (float(e), float(ms), int(st)) for i, e, ms, st in zip(ids[:k], eps[:k], mass[:k], steps[:k])}

    def macros(self, ident: int):
        n = self.n_cells[ident]
        rho = np.empty(n); u = np.empty((n, 2))
        _ck(lib().sdugks_batch_get_macros(self._h, int(ident), _ptr(rho), _ptr(u)), "sdugks_batch_get_macros")
        return rho, u

    def autotune(self, steps: int = 20):
        _ck(lib().sdugks_batch_autotune(self._h, int(steps)), "sdugks_batch_autotune")

    def info(self) -> dict:
        out = BatchStatus()
        _ck(lib().sdugks_batch_info(self._h, C.byref(out)), "sdugks_batch_info")
        return out.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sdugks_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DvmParams(C.Structure):
    _fields_ = [("nv", C.c_int32), ("vmax", C.c_double), ("RT_wall", C.c_double), ("tau", C.c_double),
                ("dt", C.c_double), ("precision", C.c_int32), ("graph_steps", C.c_int32)]


class Dvm:
    """sdugks_dvm: the rarefied solver on an nv x nv velocity grid (diffuse walls)."""

    def __init__(self, mesh: Mesh, nv: int, vmax: float, RT_wall: float, tau: float, dt: float, precision="fp32",
                 graph_steps: int = 0, stream=None):
        L = lib()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        prm = DvmParams(int(nv), float(vmax), float(RT_wall), float(tau), float(dt), prec, int(graph_steps))
        sh = getattr(stream, "cuda_stream", stream)
        self._h = C.c_void_p()
        _ck(L.sdugks_dvm_create(mesh._h, C.byref(prm), C.c_void_p(sh or 0), C.byref(self._h)), "sdugks_dvm_create")
        self.mesh = mesh
        self.n = mesh.n_cells
        self.Q = int(nv) * int(nv)

    @classmethod
    def from_case(cls, case: _meshes.Case, precision="fp32", **kw):
        """A micro-cavity-style case (meta: nv, vmax, RT0)."""
        mt = case.meta
        return cls(Mesh(case.mesh, case.bcs), mt["nv"], mt["vmax"], mt["RT0"], case.tau, case.dt, precision, **kw)

    def init(self, rho=None, u=None, RT=None):
        r = None if rho is None else _f64(rho, (self.n,))
        v = None if u is None else _f64(u, (self.n, 2))
        t = None if RT is None else _f64(RT, (self.n,))
        _ck(lib().sdugks_dvm_init(self._h, _ptr(r), _ptr(v), _ptr(t)), "sdugks_dvm_init")
        return self

    def step(self, n: int = 1):
        _ck(lib().sdugks_dvm_step(self._h, int(n)), "sdugks_dvm_step")

    def macros(self):
        rho = np.empty(self.n); u = np.empty((self.n, 2)); RT = np.empty(self.n)
        _ck(lib().sdugks_dvm_get_macros(self._h, _ptr(rho), _ptr(u), _ptr(RT)), "sdugks_dvm_get_macros")
        return rho, u, RT

    def get_state(self):
        f = np.empty((self.n, self.Q)); W = np.empty((self.n, 4))
        _ck(lib().sdugks_dvm_get_state(self._h, _ptr(f), _ptr(W)), "sdugks_dvm_get_state")
        return f, W

    def sizes(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _ck(lib().sdugks_dvm_sizes(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "sdugks_dvm_sizes")
        return {"n_cells": a.value, "n_faces": b.value, "Q": c.value, "device_bytes": d.value}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sdugks_dvm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
