"""CPU checks of the C-ABI library: it builds, loads, exports every function that
include/sdugks.h declares, and its host-only entry points (mesh geometry, boundary
table, CFL time step, argument validation) behave as documented.  No kernel runs."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2007_07347_gb300 import meshes as M
from paper_2007_07347_gb300 import sdugks as S


def test_library_exports_every_declared_function():
    L = S.lib()
    names = S.header_functions()
    assert "sdugks_step" in names and "sdugks_mesh_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.sdugks_version().decode().startswith("sdugks")


def test_mesh_create_and_cfl_dt():
    case = M.cavity(8)
    m = S.Mesh(case.mesh, case.bcs)
    # dx_min = 1 (unit squares): dt = cfl / sqrt(2)
    assert abs(m.cfl_dt(0.5) - 0.5 / math.sqrt(2)) < 1e-15
    cyl = M.cylinder(64, 32, first=0.01, r_far=10.0)
    m2 = S.Mesh(cyl.mesh, cyl.bcs)
    dt = m2.cfl_dt(0.5)
    # area / longest face of the first ring is just under its radial thickness 0.01
    assert 0.5 * 0.0098 / math.sqrt(2) < dt <= 0.5 * 0.01 / math.sqrt(2)


def test_mesh_sizes():
    case = M.couette(16)
    m = S.Mesh(case.mesh, case.bcs)
    nc, nf, npch = C.c_int64(), C.c_int64(), C.c_int32()
    S._ck(S.lib().sdugks_mesh_sizes(m._h, C.byref(nc), C.byref(nf), C.byref(npch)), "sizes")
    assert (nc.value, nf.value, npch.value) == (64, case.mesh.n_faces, 4)


def test_invalid_mesh_rejected():
    mesh = M.cartesian(3, 3)
    bad = M.Mesh(mesh.points, mesh.face_pts.copy(), mesh.owner.copy(), mesh.neighbour.copy(), mesh.n_cells,
                 mesh.patches)
    bad.face_pts[4] = [0, 0]                      # degenerate face
    with pytest.raises(S.SdugksError) as e:
        S.Mesh(bad)
    assert e.value.name == "INVALID_MESH"
    open_cell = M.Mesh(mesh.points, mesh.face_pts[1:], mesh.owner[1:], mesh.neighbour[1:], mesh.n_cells, mesh.patches)
    with pytest.raises(S.SdugksError) as e:
        S.Mesh(open_cell)                         # cell 0 lost a face: 3 faces, not closed
    assert e.value.name == "INVALID_MESH"


def test_bad_bc_arguments():
    m = S.Mesh(M.cartesian(2, 2))
    with pytest.raises(S.SdugksError) as e:
        m.set_bc(70, M.BC_WALL)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(S.SdugksError):
        m.set_bc(0, 99)
    with pytest.raises(S.SdugksError):
        m.set_bc(0, M.BC_FARFIELD, (0.0, 0.1, 0.0))


def test_solver_create_validates_before_touching_the_device():
    case = M.cavity(4)
    m = S.Mesh(case.mesh, [])                      # no boundary conditions
    with pytest.raises(S.SdugksError) as e:
        S.Solver(m, 0.1, 0.1)
    assert e.value.name in ("BAD_BC",)
    m2 = S.Mesh(case.mesh, case.bcs)
    with pytest.raises(S.SdugksError) as e:
        S.Solver(m2, -1.0, 0.1)
    assert e.value.name == "INVALID_ARG"
    # a periodic patch whose faces do not match its partner's
    c = M.periodic_box(3, 3)
    bcs = list(c.bcs)
    bcs[0] = (3, M.BC_PERIODIC, (1, 2.0, 0.0))     # wrong shift
    m3 = S.Mesh(c.mesh, bcs)
    with pytest.raises(S.SdugksError) as e:
        S.Solver(m3, 0.1, 0.1)
    assert e.value.name == "BAD_BC"


def test_tma_staging_is_validated_on_the_host():
    """TMA staging exists only in the Cartesian kernel; unknown values are rejected."""
    with pytest.raises(S.SdugksError) as e:
        S.Solver.from_case(M.cylinder(32, 16), "fp32", staging="tma")
    assert e.value.name == "INVALID_ARG" and "Cartesian" in str(e.value)
    with pytest.raises(S.SdugksError) as e:
        S.Solver.from_case(M.cavity(48), "fp32", kernel=S.KERNEL_TILED, staging="tma")
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(S.SdugksError) as e:
        S.Solver.from_case(M.cavity(48), "fp32", staging=7)
    assert e.value.name == "INVALID_ARG"


def test_ctypes_structs_match_the_c_header(tmp_path):
    """The binding's Params and Info have the sizes and field offsets the C compiler
    gives sdugks_params and sdugks_info."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    fields = {"sdugks_params": S.Params, "sdugks_info": S.Info, "sdugks_tune_info": S.TuneInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sdugks.h"', "int main(void) {"]
    for cname, py in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for py in fields.values():
        want.append(C.sizeof(py))
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert got == want


def test_last_error_message_is_set():
    with pytest.raises(S.SdugksError) as e:
        S.Mesh(M.Mesh(np.zeros((0, 2)), np.zeros((0, 2), np.int64), np.zeros(0, np.int64),
                      np.zeros(0, np.int64), 0, {}))
    assert "empty" in str(e.value)


@pytest.mark.parametrize("tile", [0, 32])
@pytest.mark.parametrize("make", [lambda: M.couette(64), lambda: M.cavity(64),
                                  lambda: M.cylinder(128, 64, first=0.01, r_far=10.0),
                                  lambda: M.periodic_box(24, 20, jitter=0.2, seed=4),
                                  lambda: M.flat_plate(8, 24, 16, Re_L=2e3, h_le=0.5, h_wall=0.2)])
def test_tile_construction_passes_host_index_checks(make, tile):
    """solver_create builds the tiles, halo rings and slot tables and checks every
    index the kernel will use before it touches the device: without a GPU it must get
    as far as the device allocation (CUDA error), never to an INVALID_MESH."""
    import torch
    case = make()
    try:
        s = S.Solver.from_case(case, "fp32", tile_cells=tile, kernel=S.KERNEL_TILED)
    except S.SdugksError as e:
        assert e.name == "CUDA" and not torch.cuda.is_available(), str(e)
    else:
        assert s.info()["n_tiles"] >= 1


def test_slanted_symmetry_line_is_rejected_on_the_host():
    """Mirror images of D2Q9 velocities are lattice velocities only in lines of
    constant x or y: a symmetry patch on the cylinder wall is BAD_BC, found before
    any device work."""
    import dataclasses
    case = M.cylinder(32, 16, first=0.05, r_far=4.0)
    bcs = [(0, M.BC_SYMMETRY, (0.0, 0.0, 0.0)), (1, M.BC_FARFIELD, (1.0, 0.1, 0.0))]
    with pytest.raises(S.SdugksError) as e:
        S.Solver.from_case(dataclasses.replace(case, bcs=bcs), "fp32")
    assert e.value.name == "BAD_BC"


def test_rarefied_solver_checks_its_boundaries_on_the_host():
    """The rarefied solver takes periodic faces and diffuse walls only; other kinds
    are BAD_BC before any device work, and bad grid parameters INVALID_ARG."""
    import torch
    case = M.flat_plate(8, 24, 16, Re_L=2e3, h_le=0.5, h_wall=0.2)
    with pytest.raises(S.SdugksError) as e:
        S.Dvm(S.Mesh(case.mesh, case.bcs), 8, 2.0, 0.5, 0.1, 0.01)
    assert e.value.name == "BAD_BC"
    mc = M.micro_cavity(8, nv=8)
    with pytest.raises(S.SdugksError) as e:
        S.Dvm(S.Mesh(mc.mesh, mc.bcs), 1, 2.0, 0.5, 0.1, 0.01)
    assert e.value.name == "INVALID_ARG"
    try:
        S.Dvm.from_case(mc)
    except S.SdugksError as e:
        assert e.name == "CUDA" and not torch.cuda.is_available(), str(e)


def test_missing_library_fails_loudly(monkeypatch):
    """Without the compiled library there is no fallback path: loading it, and so every
    solver call, raises."""
    saved = S._lib
    try:
        S._lib = None
        monkeypatch.setattr(S._build, "build", lambda *a, **k: "/nonexistent/libsdugks.so")
        with pytest.raises(OSError):
            S.lib()
        with pytest.raises(OSError):
            S.Solver.from_case(M.cavity(8), "fp32")

        def no_toolchain(*a, **k):
            raise RuntimeError("nvcc failed")

        monkeypatch.setattr(S._build, "build", no_toolchain)
        with pytest.raises(RuntimeError):
            S.lib()
    finally:
        S._lib = saved


def test_product_code_does_not_use_the_oracle():
    """The package and its C/CUDA sources never import, link or call the oracle (only the
    tests, smoke() and bench.py's CPU arms do)."""
    import ast
    import pathlib
    root = pathlib.Path(__file__).resolve().parent.parent
    pkg = root / "paper_2007_07347_gb300"
    for py in pkg.rglob("*.py"):
        for node in ast.walk(ast.parse(py.read_text())):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), py
    for src in list((pkg / "csrc").iterdir()) + list((root / "include").iterdir()):
        if src.suffix in (".h", ".cuh", ".cu", ".cpp"):
            assert "oracle" not in src.read_text().lower(), src
