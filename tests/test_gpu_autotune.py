"""The autotuner (sdugks_autotune, through the C-ABI): it times the candidate launch
configurations on the device, caches the winner per mesh, and the configuration it
picks does not change results (bit for bit in FP64 on the tiled kernel; to FP32
rounding across Cartesian block shapes)."""
import numpy as np
import pytest

from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu


def _S():
    from paper_2007_07347_gb300 import sdugks as S
    return S


def rel_l2(a, b):
    return np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))


def test_cartesian_fp32_tuning_is_a_candidate_cached_and_keeps_results():
    S = _S()
    S.autotune_clear()
    case = M.cavity(100, Re=400.0)
    s = S.Solver.tuned(case, "fp32", steps=128)
    t = s.tune
    assert t["kernel"] == S.KERNEL_CARTESIAN and t["from_cache"] == 0
    assert t["candidates"] == 3 * 2 * 3                    # shapes x stagings x graph lengths
    assert t["tile_cells"] in (256, 224, 128) and t["staging"] in (0, 1) and t["graph_steps"] in (32, 64, 128)
    assert t["ns_per_step"] > 0
    assert s.info()["tile_cells"] == t["tile_cells"] and s.info()["staging"] == t["staging"]
    again = S.Solver.tuned(case, "fp32", steps=128).tune
    assert again["from_cache"] == 1 and again["candidates"] == 0
    assert (again["tile_cells"], again["staging"], again["graph_steps"]) == \
        (t["tile_cells"], t["staging"], t["graph_steps"])
    ref = S.Solver.from_case(case, "fp32").init()
    s.init()
    ref.step(300)
    s.step(300)
    assert rel_l2(s.macros()[1], ref.macros()[1]) <= 1e-5


def test_tiled_fp64_tuning_is_bitwise_neutral():
    S = _S()
    case = M.cylinder(96, 48, first=0.01, r_far=10.0, shuffle_seed=1)
    u = np.tile(case.u0, (case.mesh.n_cells, 1))
    s = S.Solver.tuned(case, "fp64", steps=64)
    t = s.tune
    assert t["kernel"] == S.KERNEL_TILED and t["candidates"] == 5 * 3
    assert t["tile_cells"] in (64, 96, 108, 120, 128)
    ref = S.Solver.from_case(case, "fp64").init(None, u)
    s.init(None, u)
    ref.step(150)
    s.step(150)
    for a, b in zip(s.get_state(), ref.get_state()):
        np.testing.assert_array_equal(a, b)


def test_different_meshes_are_tuned_separately():
    S = _S()
    S.autotune_clear()
    a = S.Solver.tuned(M.cavity(44, Re=100.0), "fp32", steps=64).tune
    b = S.Solver.tuned(M.cavity(52, Re=100.0), "fp32", steps=64).tune
    assert a["from_cache"] == 0 and b["from_cache"] == 0       # a new mesh is timed
    c = S.Solver.tuned(M.cavity(44, Re=3000.0), "fp32", steps=64).tune
    assert c["from_cache"] == 1                                # tau and dt do not change the work of a step
    d = S.Solver.tuned(M.cavity(44, Re=100.0), "bf16dev", steps=64).tune
    assert d["from_cache"] == 0                                # another precision is tuned on its own
