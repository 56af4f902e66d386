"""CPU pins of the synthetic workloads against their stated recipe (the paper's meshes and
data are not available, so seeded generators stand in for them).

Couette (Sec. IV, 4 x 64 cells, U = 0.1, Re = 10): tau = 3 nu = 0.03 and
dt = CFL dy / sqrt(2) with CFL 0.5.  Cavity (Sec. IV, 256^2 unit cells, Re 1000,
lid 0.1): tau = 0.0768, dt = 0.5 / sqrt(2).  Cylinder (Sec. IV, Re 40): a 512 x 256
O-mesh from r = 0.5 with a first cell of 0.005 to r = 50, the radii geometric with the
ratio that makes 256 cells span that range (about 1.02111: the paper's 1.03 with 256
cells would reach 322 D), cell ids shuffled so that the unstructured path is exercised,
tau = 3 U D / Re, dt = CFL 0.005 / sqrt(2).  Batch: 256 cavities, N ~ logU[32, 512],
Re ~ logU[100, 5000], seed 1.  Rarefied micro cavity (Sec. IV, Kn 1): 40 x 40 cells,
100 x 100 velocities on [-2, 2]^2, tau = Kn L sqrt(2 / (pi R T0)) from the mean free
path lambda = (mu / p) sqrt(pi R T0 / 2), dt = CFL (L / n) / (largest node speed).
"""
import math

import numpy as np

from paper_2007_07347_gb300 import meshes as M


def test_couette_recipe():
    c = M.couette()
    assert c.mesh.n_cells == 4 * 64
    assert math.isclose(c.tau, 0.03, rel_tol=1e-14)
    assert math.isclose(c.dt, 0.5 * (1 / 64) / math.sqrt(2), rel_tol=1e-14)
    assert math.isclose(c.dt / c.tau, 0.18414, rel_tol=1e-4)


def test_cavity_recipe():
    c = M.cavity(256, Re=1000.0)
    assert c.mesh.n_cells == 65536
    assert math.isclose(c.tau, 3 * 0.1 * 256 / 1000, rel_tol=1e-14)
    assert math.isclose(c.dt, 0.5 / math.sqrt(2), rel_tol=1e-14)


def test_cylinder_recipe():
    c = M.cylinder(512, 256)
    assert c.mesh.n_cells == 512 * 256
    assert math.isclose(c.tau, 3 * 0.1 * 1.0 / 40, rel_tol=1e-14)
    assert math.isclose(c.dt, 0.5 * 0.005 / math.sqrt(2), rel_tol=1e-14)
    assert c.u0 == (0.1, 0.0)
    om = M.o_mesh(512, 256)
    r = np.hypot(om.points[:, 0], om.points[:, 1]).reshape(257, 512)
    assert np.abs(r - r[:, :1]).max() <= 1e-12 * 50         # rings of constant radius
    r = r[:, 0]
    h = np.diff(r)
    q = h[1:] / h[:-1]
    assert abs(r[0] - 0.5) <= 1e-15 and abs(h[0] - 0.005) <= 1e-15 and r[-1] == 50.0
    assert np.abs(q - q[0]).max() <= 1e-9 and abs(q[0] - 1.02111) <= 1e-5
    # the paper's ratio 1.03 over 256 cells would reach far beyond 50 D
    assert 0.5 + 0.005 * (1.03 ** 256 - 1) / 0.03 > 300
    # ids shuffled: the same mesh with cells in another order
    plain = M.cylinder(64, 32, first=0.01, r_far=10.0, shuffle_seed=None)
    shuf = M.cylinder(64, 32, first=0.01, r_far=10.0)
    assert plain.mesh.n_cells == shuf.mesh.n_cells and (plain.mesh.owner != shuf.mesh.owner).mean() > 0.9


def test_batch_recipe():
    specs = M.batch_cavities(256, seed=1)
    ns = np.array([n for n, _ in specs])
    res = np.array([re for _, re in specs])
    assert len(specs) == 256 and ns.min() >= 32 and ns.max() <= 512
    assert res.min() >= 100 and res.max() <= 5000
    assert int((ns.astype(np.int64) ** 2).sum()) == 11_677_249
    # log-uniform: the medians of log N and log Re lie near the middle of their ranges
    assert abs(np.median(np.log(ns)) - 0.5 * (math.log(32) + math.log(512))) < 0.25
    assert abs(np.median(np.log(res)) - 0.5 * (math.log(100) + math.log(5000))) < 0.35


def test_micro_cavity_recipe():
    c = M.micro_cavity(40, Kn=1.0)
    assert c.mesh.n_cells == 1600
    assert math.isclose(c.tau, math.sqrt(2 / (math.pi * 0.5)), rel_tol=1e-14)
    h = 4.0 / 100
    vmax_node = (2.0 - h / 2) * math.sqrt(2)
    assert math.isclose(c.dt, 0.5 * (1.0 / 40) / vmax_node, rel_tol=1e-12)
