"""sdugks_residual_noalloc: the residual/mass reduction for callers that may not
allocate device memory (their device memory is owned and budgeted by another runtime,
or the call sits on a path that must not enter the allocator).  It reduces over
caller-owned device arrays with a fixed scratch array inside the library.

Checked through the C-ABI against the solver's own sdugks_residual on the same state,
two calls in a row, with the tolerances of the residual parity test (1e-10 relative
on eps, 1e-12 on the mass).  The file sorts last so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu


def _entry():
    from paper_2007_07347_gb300 import sdugks as S
    L = S.lib()
    fn = L.sdugks_residual_noalloc
    fn.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return S, L, fn


def test_residual_noalloc_matches_solver_residual_twice():
    import torch
    S, L, fn = _entry()
    torch.cuda.set_device(0)
    case = M.cavity(48, Re=400.0)
    n = case.mesh.n_cells
    s = S.Solver.from_case(case, "fp64").init()
    s.step(100)
    s.residual()                                   # solver snapshot at step 100
    _, W0 = s.get_state()
    dev = torch.device("cuda", 0)
    d_vol = torch.tensor(O.geometry(case.mesh, case.bcs)["vol"], dtype=torch.float64, device=dev)
    d_snap = torch.tensor(W0[:, 1:] / W0[:, :1], dtype=torch.float64, device=dev).contiguous()
    d_out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        s.step(150)
        eps_ref, mass_ref = s.residual()
        _, W = s.get_state()
        d_W = torch.tensor(W, dtype=torch.float64, device=dev).contiguous()
        rc = fn(n, d_W.data_ptr(), d_vol.data_ptr(), d_snap.data_ptr(), d_out.data_ptr(), stream)
        assert rc == 0, L.sdugks_last_error().decode()
        torch.cuda.synchronize()
        eps, mass, bad = d_out.tolist()
        assert np.isfinite(eps_ref) and eps_ref > 0
        assert abs(eps - eps_ref) <= 1e-10 * eps_ref
        assert abs(mass - mass_ref) <= 1e-12 * mass_ref
        assert bad == 0.0
        # the snapshot now holds this call's (U, V), ready for the next call
        np.testing.assert_allclose(d_snap.cpu().numpy(), W[:, 1:] / W[:, :1], rtol=0, atol=0)


def test_residual_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    S, L, fn = _entry()
    torch.cuda.set_device(0)
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    rc = fn(4194304 + 1, p, p, p, p, None)
    assert rc == -1                                # SDUGKS_ERR_INVALID_ARG
    assert "scratch limit" in L.sdugks_last_error().decode()
    assert fn(0, p, p, p, p, None) == -1
