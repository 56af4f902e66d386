"""Physics checks of the GPU path against the paper's numbers (loose; not parity).

The paper's meshes are not available, so these run on the synthetic meshes of the
stated geometry, coarser than the validation runs, and the bands are wide enough for
the mesh difference (the measured values are written beside each band).
"""
import math

import pytest

from paper_2007_07347_gb300 import validate as V

pytestmark = pytest.mark.gpu


def test_cylinder_sheds_vortices_at_the_strouhal_number():
    """Sec. IV unsteady cylinder, Re 100: periodic vortex shedding with St close to the
    paper's 0.1653 (and the parallel-shedding fit -3.3265/Re + 0.1816 + 1.6e-4 Re =
    0.1643), on a 256 x 128 O-mesh out to 25 D (measured: St 0.1635, mean Cd 1.345;
    the 512 x 256 mesh to 50 D gives St 0.1646 and mean Cd 1.3445 against the paper's
    0.1653 and 1.349)."""
    out = V.cylinder_unsteady(100.0, n_theta=256, n_r=128, first=0.01, r_far=25.0, t_end=700.0, t_from=350.0)
    assert out["periods"] >= 4, out
    assert out["Cl_amp"] > 0.1, out
    assert abs(out["St"] / 0.1653 - 1.0) < 0.08, out
    assert abs(out["Cd_mean"] / 1.349 - 1.0) < 0.12, out


def test_flat_plate_drag_near_blasius():
    """Sec. IV laminar flat plate, Re_L = 1e5: the plate's drag coefficient against
    the Blasius value 1.328/sqrt(Re_L) = 4.20e-3 (the paper reports 4.237e-3; the
    96 x 64 validation mesh gives 4.375e-3 at t = 3100, still decreasing)."""
    out = V.flat_plate_run(16, 48, 48, t_end=3000.0, interval=20000)
    assert math.isfinite(out["Cd"]), out
    assert abs(out["Cd_rel_diff"]) < 0.15, out
