"""Batched solves (sdugks_batch): one kernel launch per step over the (instance, block)
work list of many uniform-grid solves of different sizes and Reynolds numbers.

Within the batched kernel an instance's arithmetic does not depend on the other
instances: its results are compared bit for bit alone and in a mix, including an
instance admitted mid-run.  Against the single-solver Cartesian kernel (the same
device function inlined into another kernel, where the compiler may contract
products and sums differently) the results agree within the FP32 parity tolerance
that both meet against the FP64 oracle: relative L2 of u <= 1e-4 (1e-3 for bf16
storage), max |rho| difference <= 1e-5 (1e-4 for bf16 storage, which keeps 8
significant bits of the scaled deviation (f - feq)/w: two kernels that round a
product differently drift apart by a few 1e-5 in rho over 300 steps).  One instance is also checked against the
FP64 oracle with the FP32 tolerance of the parity tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_07347_gb300 import meshes as M

pytestmark = pytest.mark.gpu


def _S():
    from paper_2007_07347_gb300 import sdugks as S
    return S


def _single(case, steps, precision="fp32"):
    S = _S()
    s = S.Solver.from_case(case, precision).init()
    s.step(steps)
    return s.macros()


def _close_to_single(rho, u, rho1, u1, tol_u=1e-4, tol_rho=1e-5):
    assert np.sqrt(np.sum((u - u1) ** 2) / np.sum(u1 ** 2)) <= tol_u
    assert np.abs(rho - rho1).max() <= tol_rho


MIX = [lambda: M.cavity(40, Re=400.0), lambda: M.cavity(100, Re=1000.0), lambda: M.couette(64),
       lambda: M.cavity(64, Re=100.0)]


@pytest.mark.parametrize("precision", ["fp32", "bf16dev", "fp16dev"])
def test_batch_instances_equal_single_solvers(precision):
    S = _S()
    b = S.Batch(256 << 20, precision, max_instances=16)
    cases = [mk() for mk in MIX]
    ids = [b.add_case(c) for c in cases]
    b.step(300)                                   # graph of 64 steps + single launches
    for ident, case in zip(ids, cases):
        rho, u = b.macros(ident)
        rho1, u1 = _single(case, 300, precision)
        _close_to_single(rho, u, rho1, u1, *{"fp32": (1e-4, 1e-5), "bf16dev": (1e-3, 1e-4), "fp16dev": (1e-3, 1e-4)}[precision])


def test_result_same_alone_and_in_the_mix_and_late_admission():
    S = _S()
    case = M.cavity(48, Re=400.0)
    alone = S.Batch(64 << 20, "fp32", max_instances=4)
    a = alone.add_case(case)
    alone.step(201)
    mix = S.Batch(256 << 20, "fp32", max_instances=8)
    others = [mix.add_case(mk()) for mk in MIX[:2]]
    mix.step(37)                                  # odd step count: the buffer parity flips
    late = mix.add_case(case)
    mix.add_case(MIX[2]())
    mix.step(201)
    np.testing.assert_array_equal(alone.macros(a)[1], mix.macros(late)[1])
    res = mix.residual()
    assert res[late][2] == 201 and res[others[0]][2] == 238


def test_step_graph_follows_the_work_list():
    """With one CTA per work item, the step graph's grids have the item count it was
    captured with; an admission or a removal captures it again.  An instance admitted
    after the capture (its items lie past the old grid) and one whose items move in the
    list after a removal give bit for bit the results they give alone."""
    S = _S()
    case, extra = M.cavity(48, Re=400.0), MIX[1]()
    alone = S.Batch(64 << 20, "fp32", max_instances=4)
    a = alone.add_case(case)
    alone.step(3 * 130)
    alone_x = S.Batch(64 << 20, "fp32", max_instances=4)
    ax = alone_x.add_case(extra)
    alone_x.step(130)
    mix = S.Batch(256 << 20, "fp32", max_instances=8)
    first = mix.add_case(MIX[0]())
    mine = mix.add_case(case)
    mix.step(130)                                 # a graph of 64 steps for these items
    assert mix.info()["per_item"] == 1
    late = mix.add_case(extra)                    # more items than the graph's grids
    mix.step(130)
    np.testing.assert_array_equal(alone_x.macros(ax)[1], mix.macros(late)[1])
    mix.remove(first)                             # the others' items move forward
    mix.remove(late)
    mix.step(130)
    np.testing.assert_array_equal(alone.macros(a)[1], mix.macros(mine)[1])
    assert mix.info()["items"] == alone.info()["items"]


def test_batch_against_oracle():
    S = _S()
    case = M.cavity(32, Re=100.0)
    b = S.Batch(32 << 20, "fp32", max_instances=2)
    ident = b.add_case(case)
    b.step(500)
    rho, u = b.macros(ident)
    st = O.init(case.mesh.n_cells)
    O.run(case, st, 500)
    assert np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2)) <= 1e-4
    assert np.abs(rho - st.W[:, 0]).max() <= 1e-5


def test_batch_workload_sample_against_oracle_and_single_solves():
    """The batch workload itself (256 cavities, N ~ logU[32, 512], Re ~ logU[100, 5000],
    seed 1), 60 steps in one batch.  Every instance is checked against its own
    single-solver run, and a seeded sample of 8 (the smallest, the largest and 6 drawn
    with seed 7) against the FP64 oracle.  Sixty steps from rest is an early transient:
    far from the lid u is near zero, so a relative norm of u measures FP32 rounding
    against a vanishing signal.  The criterion is therefore the FP32 profile
    tolerance, max |u - u_ref| <= 1e-4 U (lid speed U = 0.1), with
    max |rho - rho_ref| <= 1e-5."""
    S = _S()
    cases = [M.cavity(n, Re=re) for n, re in M.batch_cavities(256, seed=1)]
    probe = S.Batch(1 << 20, "fp32", 4)
    need = sum(probe.footprint(S.Mesh(c.mesh, c.bcs)) for c in cases)
    b = S.Batch(need + (64 << 20), "fp32", 512)
    ids = [b.add_case(c) for c in cases]
    steps, U = 60, 0.1
    b.step(steps)
    sizes = [c.mesh.n_cells for c in cases]
    lo, hi = int(np.argmin(sizes)), int(np.argmax(sizes))
    rng = np.random.default_rng(7)
    sample = {lo, hi} | {int(i) for i in rng.choice([i for i in range(len(cases)) if i not in (lo, hi)], 6,
                                                   replace=False)}
    assert len(sample) == 8
    for i, (c, ident) in enumerate(zip(cases, ids)):
        rho, u = b.macros(ident)
        rho1, u1 = _single(c, steps)
        assert np.abs(u - u1).max() <= 1e-4 * U
        assert np.abs(rho - rho1).max() <= 1e-5
        if i in sample:
            st = O.init(c.mesh.n_cells)
            O.run(c, st, steps)
            assert np.abs(st.u).max() > 1e-3                 # the lid has set the fluid moving
            assert np.abs(u - st.u).max() <= 1e-4 * U
            assert np.abs(rho - st.W[:, 0]).max() <= 1e-5


def test_batch_residual_matches_single_solver():
    S = _S()
    case = M.cavity(64, Re=100.0)
    b = S.Batch(64 << 20, "fp32", max_instances=2)
    ident = b.add_case(case)
    s = S.Solver.from_case(case, "fp32").init()
    for k in range(2):
        b.step(128)
        s.step(128)
        eps_b, mass_b, _ = b.residual()[ident]
        eps_s, mass_s = s.residual()
        if k == 0:
            assert np.isinf(eps_b) and np.isinf(eps_s)
        else:
            assert abs(eps_b - eps_s) <= 1e-4 * eps_s
        assert abs(mass_b - mass_s) <= 1e-9 * mass_s


def test_admission_by_footprint_and_reuse():
    S = _S()
    probe = S.Batch(1 << 20, "fp32", max_instances=4)
    mesh = S.Mesh(M.cavity(64).mesh, M.cavity(64).bcs)
    fp = probe.footprint(mesh)
    assert fp > 64 * 64 * 120
    b = S.Batch(2 * fp, "fp32", max_instances=8)
    c = M.cavity(64, Re=100.0)
    i1 = b.add_case(c)
    i2 = b.add_case(c)
    with pytest.raises(S.SdugksError) as e:
        b.add_case(c)
    assert e.value.name == "FULL"
    b.step(10)
    b.remove(i1)
    i3 = b.add_case(c)                           # the freed block is reused
    b.step(10)
    info = b.info()
    assert info["instances"] == 2 and info["pool_used"] == 2 * fp
    assert set(b.residual()) == {i2, i3}
    with pytest.raises(S.SdugksError):
        b.add_case(M.cylinder(32, 16, first=0.02, r_far=10.0))   # not a uniform grid


def test_autotune_keeps_results():
    S = _S()
    b = S.Batch(256 << 20, "fp32", max_instances=8)
    ids = [b.add_case(mk()) for mk in MIX]
    b.autotune(4)
    done = b.residual()[ids[0]][2]
    b.step(64)
    rho, u = b.macros(ids[1])
    rho1, u1 = _single(MIX[1](), done + 64)
    _close_to_single(rho, u, rho1, u1)


def test_batch_symmetry_and_periodic_instances_against_oracle():
    """Batched instances carry every side rule of the Cartesian kernel: a channel with
    a symmetry line (mirror ghosts), periodic sides and a moving wall, beside a cavity."""
    S = _S()
    mesh = M.cartesian(40, 20, 40.0, 20.0)
    bcs = [(3, M.BC_PERIODIC, (1, 40.0, 0.0)), (1, M.BC_PERIODIC, (3, -40.0, 0.0)),
           (0, M.BC_MOVING_WALL, (0.05, 0.0, 0.0)), (2, M.BC_SYMMETRY, (0.0, 0.0, 0.0))]
    chan = M.Case("sym_channel", mesh, bcs, tau=0.05, dt=0.25)
    b = S.Batch(64 << 20, "fp32", max_instances=4)
    ic = b.add_case(chan)
    b.add_case(M.cavity(36, Re=300.0))
    b.step(400)
    rho, u = b.macros(ic)
    st = O.init(mesh.n_cells)
    O.run(chan, st, 400)
    assert np.sqrt(np.sum((u - st.u) ** 2) / np.sum(st.u ** 2)) <= 1e-4
    assert np.abs(rho - st.rho).max() <= 1e-5
