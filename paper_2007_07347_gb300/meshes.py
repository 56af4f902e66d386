"""Seeded synthetic inputs: face-based quad meshes, boundary tables and case parameters.

This module is the only code shared by the FP64 oracle side and the CUDA side.  It
holds none of the method's arithmetic: it writes point coordinates, face-to-point
lists, owner/neighbour arrays and plain case numbers (tau from the Reynolds number,
dt from the known smallest cell side), nothing that the S-DUGKS step computes.

Mesh convention (the face-based owner/neighbour form of an unstructured FV mesh):

* ``points``   float64 [n_points, 2]
* ``face_pts`` int64   [n_faces, 2]   the two end points of each straight face
* ``owner``    int64   [n_faces]      cell on one side
* ``neighbour`` int64  [n_faces]      cell on the other side, or ``-1 - patch`` on a
  boundary face of boundary patch ``patch``
* ``n_cells``  int

Boundary kinds and their three parameters (the same numbers the C-ABI takes):

* PERIODIC     (partner patch, shift_x, shift_y): face centre + shift lands on the partner face
* WALL         ()                                 no-slip wall at rest
* MOVING_WALL  (u_x, u_y)                         no-slip wall moving tangentially
* FARFIELD     (rho, u_x, u_y)                    free stream
* OUTLET       ()                                 density and velocity from the inner cell

D2Q9 lattice units: c = 1, c_s^2 = 1/3, so tau = 3 nu.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_UNSET, BC_PERIODIC, BC_WALL, BC_MOVING_WALL, BC_FARFIELD, BC_OUTLET, BC_SYMMETRY = 0, 1, 2, 3, 4, 5, 6


@dataclass
class Mesh:
    points: np.ndarray
    face_pts: np.ndarray
    owner: np.ndarray
    neighbour: np.ndarray
    n_cells: int
    patches: dict
    meta: dict = field(default_factory=dict)

    @property
    def n_faces(self) -> int:
        return int(self.face_pts.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.points.shape[0])


@dataclass
class Case:
    """A mesh with its boundary table and flow parameters (lattice units)."""
    name: str
    mesh: Mesh
    bcs: list          # [(patch, kind, (p0, p1, p2))]
    tau: float
    dt: float
    rho0: float = 1.0
    u0: tuple = (0.0, 0.0)
    meta: dict = field(default_factory=dict)


def _bc_params(*p):
    q = [float(x) for x in p] + [0.0] * (3 - len(p))
    return tuple(q[:3])


def cartesian(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, *, jitter: float = 0.0,
              seed: int | None = None) -> Mesh:
    """Uniform (optionally jittered) nx x ny quad mesh on [0,lx] x [0,ly].

    Patches: 0 bottom (y=0), 1 right (x=lx), 2 top (y=ly), 3 left (x=0).
    Cell (i, j) has id i + nx*j; point (i, j) has id i + (nx+1)*j.
    ``jitter`` moves interior points by up to jitter*min(dx,dy) (seeded), which keeps
    the quads convex for jitter < 0.25.
    """
    dx, dy = lx / nx, ly / ny
    # arrays filled in place by broadcasting, row by row (row j of the points, faces
    # and cells is contiguous), with the ids of the docstring
    px = np.empty((ny + 1, nx + 1))
    px[:] = np.arange(nx + 1) * dx
    py = np.empty((ny + 1, nx + 1))
    py[:] = (np.arange(ny + 1) * dy)[:, None]
    px, py = px.ravel(), py.ravel()
    if jitter:
        rng = np.random.default_rng(seed)
        inner = np.zeros((ny + 1, nx + 1), bool)
        inner[1:ny, 1:nx] = True
        inner = inner.ravel()
        h = jitter * min(dx, dy)
        px[inner] += rng.uniform(-h, h, inner.sum())
        py[inner] += rng.uniform(-h, h, inner.sum())
    points = np.empty((px.size, 2))
    points[:, 0], points[:, 1] = px, py

    nfx, nfy = (nx + 1) * ny, nx * (ny + 1)
    fp = np.empty((nfx + nfy, 2), np.int64)
    own = np.empty(nfx + nfy, np.int64)
    nbr = np.empty(nfx + nfy, np.int64)
    # faces of constant x (between cells (i-1, j) and (i, j)), row by row
    ii, jj = np.arange(nx + 1)[None, :], np.arange(ny)[:, None]
    p0 = ii + (nx + 1) * jj
    fp[:nfx, 0], fp[:nfx, 1] = p0.ravel(), (p0 + (nx + 1)).ravel()
    o = np.empty((ny, nx + 1), np.int64)
    o[:] = ii - 1 + nx * jj
    o[:, 0] = nx * jj[:, 0]
    own[:nfx] = o.ravel()
    k = np.empty((ny, nx + 1), np.int64)
    k[:] = ii + nx * jj
    k[:, 0], k[:, nx] = -1 - 3, -1 - 1
    nbr[:nfx] = k.ravel()
    # faces of constant y (between cells (i, j-1) and (i, j))
    ii, jj = np.arange(nx)[None, :], np.arange(ny + 1)[:, None]
    p0 = ii + (nx + 1) * jj
    fp[nfx:, 0], fp[nfx:, 1] = p0.ravel(), (p0 + 1).ravel()
    o = np.empty((ny + 1, nx), np.int64)
    o[:] = ii + nx * (jj - 1)
    o[0, :] = ii[0]
    own[nfx:] = o.ravel()
    k = np.empty((ny + 1, nx), np.int64)
    k[:] = ii + nx * jj
    k[0, :], k[ny, :] = -1 - 0, -1 - 2
    nbr[nfx:] = k.ravel()

    ci = np.empty((ny, nx), np.int64)
    ci[:] = np.arange(nx)
    cj = np.empty((ny, nx), np.int64)
    cj[:] = np.arange(ny)[:, None]
    ci, cj = ci.ravel(), cj.ravel()
    xyn = np.empty((nx * ny, 2))
    xyn[:, 0], xyn[:, 1] = (ci + 0.5) * dx, (cj + 0.5) * dy
    meta = dict(kind="cartesian", nx=nx, ny=ny, lx=lx, ly=ly, dx=dx, dy=dy,
                cell_i=ci, cell_j=cj, cell_xy_nominal=xyn)
    return Mesh(points, fp, own, nbr, nx * ny, dict(bottom=0, right=1, top=2, left=3), meta)


def mirror_y(mesh: Mesh, patch: int) -> Mesh:
    """The mesh doubled by its mirror image in the horizontal line of boundary patch
    ``patch``: cell c + n is the mirror of cell c, the patch faces become interior
    faces between c and c + n (same face ids), and the mirrored copies of every
    other face follow with the same boundary patches."""
    y0s = mesh.points[np.unique(mesh.face_pts[mesh.neighbour == -1 - patch])][:, 1]
    y0 = float(y0s[0])
    assert np.all(y0s == y0), "patch is not a horizontal line"
    n, npt = mesh.n_cells, mesh.n_points
    on = mesh.points[:, 1] == y0
    mp = np.where(on, np.arange(npt), npt + np.cumsum(~on) - 1)
    q = mesh.points[~on].copy()
    q[:, 1] = 2.0 * y0 - q[:, 1]
    points = np.concatenate([mesh.points, q])
    sym = mesh.neighbour == -1 - patch
    nbr0 = np.where(sym, mesh.owner + n, mesh.neighbour)
    keep = ~sym
    fp_m = mp[mesh.face_pts[keep]]
    own_m = mesh.owner[keep] + n
    nbr_m = np.where(mesh.neighbour[keep] >= 0, mesh.neighbour[keep] + n, mesh.neighbour[keep])
    meta = dict(kind="mirror_y", base=mesh.meta.get("kind"), y0=y0)
    return Mesh(points, np.concatenate([mesh.face_pts, fp_m]).astype(np.int64),
                np.concatenate([mesh.owner, own_m]).astype(np.int64),
                np.concatenate([nbr0, nbr_m]).astype(np.int64), 2 * n,
                {k: v for k, v in mesh.patches.items() if v != patch}, meta)


def stretched(xs: np.ndarray, ys: np.ndarray) -> Mesh:
    """Tensor-product quad mesh on the (increasing) point coordinates xs, ys: cells of
    varying size, so it is not a uniform grid.  Patches and numbering as cartesian()."""
    nx, ny = len(xs) - 1, len(ys) - 1
    m = cartesian(nx, ny, 1.0, 1.0)
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    m.points = np.stack([np.asarray(xs, np.float64)[I.ravel()], np.asarray(ys, np.float64)[J.ravel()]], 1)
    xc = 0.5 * (xs[:-1] + xs[1:])
    yc = 0.5 * (ys[:-1] + ys[1:])
    m.meta = dict(kind="stretched", nx=nx, ny=ny, cell_i=m.meta["cell_i"], cell_j=m.meta["cell_j"],
                  cell_xy_nominal=np.stack([xc[m.meta["cell_i"]], yc[m.meta["cell_j"]]], 1))
    return m


def _graded(a: float, b: float, h_a: float, n: int) -> np.ndarray:
    """n cells from a to b, first cell h_a at a, geometric growth (ratio by bisection)."""
    if abs(h_a * n - (b - a)) < 1e-12 * (b - a):
        return np.linspace(a, b, n + 1)
    q = o_mesh_ratio(n, 0.0, h_a, b - a)
    x = a + h_a * (q ** np.arange(n + 1) - 1.0) / (q - 1.0)
    x[-1] = b
    return x


def flat_plate(nx_up: int = 24, nx_plate: int = 72, ny: int = 64, *, U: float = 0.1, Re_L: float = 1e5,
               L: float = 100.0, x_up: float = 50.0, height: float = 100.0, h_le: float = 0.05,
               h_wall: float = 0.02, cfl: float = 0.5) -> Case:
    """Laminar flow over a flat plate of length L on [-x_up, L] x [0, height]: far-field
    inflow at x = -x_up and at the top, an outlet at x = L, a symmetry line on y = 0
    upstream of the leading edge and a no-slip wall (the plate) along 0 <= x <= L.
    Cells cluster at the leading edge (first width h_le on both sides of x = 0) and
    at the wall (first height h_wall).  Patches: 0 symmetry, 1 outlet, 2 top, 3 inflow,
    4 plate."""
    xs = np.concatenate([-_graded(0.0, x_up, h_le, nx_up)[::-1], _graded(0.0, L, h_le, nx_plate)[1:]])
    ys = _graded(0.0, height, h_wall, ny)
    m = stretched(xs, ys)
    # split the bottom patch at the leading edge: faces with both points at x >= 0
    bot = np.where(m.neighbour == -1 - 0)[0]
    on_plate = m.points[m.face_pts[bot]][:, :, 0].min(1) >= 0.0
    m.neighbour[bot[on_plate]] = -1 - 4
    m.patches = dict(symmetry=0, outlet=1, top=2, inflow=3, plate=4)
    nu = U * L / Re_L
    dmin = min(h_le, h_wall)
    bcs = [(0, BC_SYMMETRY, _bc_params()), (1, BC_OUTLET, _bc_params()),
           (2, BC_FARFIELD, _bc_params(1.0, U, 0.0)), (3, BC_FARFIELD, _bc_params(1.0, U, 0.0)),
           (4, BC_WALL, _bc_params())]
    return Case(f"flat_plate_{len(xs) - 1}x{ny}", m, bcs, tau=3.0 * nu, dt=cfl * dmin / math.sqrt(2.0),
                u0=(U, 0.0), meta=dict(U=U, Re_L=Re_L, L=L, xs=xs, ys=ys, cfl=cfl))


def from_polygons(points: np.ndarray, cells: list, side_of) -> Mesh:
    """Face-based mesh from cell polygons (vertex lists, either orientation): every
    edge becomes one face, owned by the first cell that lists it; an edge of one cell
    only is a boundary face of patch side_of(midpoint)."""
    edge = {}
    fpts, own, nbr = [], [], []
    for c, poly in enumerate(cells):
        k = len(poly)
        for q in range(k):
            a, b = int(poly[q]), int(poly[(q + 1) % k])
            key = (a, b) if a < b else (b, a)
            f = edge.get(key)
            if f is None:
                edge[key] = len(fpts)
                fpts.append((a, b)); own.append(c); nbr.append(-1)
            else:
                assert nbr[f] == -1, "edge shared by more than two cells"
                nbr[f] = c
    fpts = np.asarray(fpts, np.int64)
    own = np.asarray(own, np.int64)
    nbr = np.asarray(nbr, np.int64)
    mid = 0.5 * (points[fpts[:, 0]] + points[fpts[:, 1]])
    for f in np.where(nbr == -1)[0]:
        nbr[f] = -1 - int(side_of(mid[f]))
    return Mesh(np.asarray(points, np.float64), fpts, own, nbr, len(cells), {})


def hybrid(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, *, tri_from: float = 0.5, jitter: float = 0.0,
           seed: int | None = None, quad_rows: int = 0) -> Mesh:
    """Quad/triangle hybrid mesh on [0,lx] x [0,ly]: the quads of the uniform (optionally
    jittered) nx x ny grid whose column index is >= tri_from * nx are each split into
    two triangles (diagonals alternating in a checkerboard), except in the quad_rows
    rows next to the bottom and to the top (a layer of quads along walls, as hybrid
    meshes keep at solid boundaries).  Patches and point numbering as cartesian(); the
    cell order is row by row, a split quad giving its lower then its upper triangle."""
    base = cartesian(nx, ny, lx, ly, jitter=jitter, seed=seed)
    P = base.points
    pid = lambda i, j: i + (nx + 1) * j  # noqa: E731
    cells, n_tri = [], 0
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = pid(i, j), pid(i + 1, j), pid(i + 1, j + 1), pid(i, j + 1)
            if i >= tri_from * nx and quad_rows <= j < ny - quad_rows:
                if (i + j) % 2 == 0:
                    cells += [[a, b, c], [a, c, d]]
                else:
                    cells += [[a, b, d], [b, c, d]]
                n_tri += 2
            else:
                cells.append([a, b, c, d])
    eps = 1e-9 * max(lx, ly)

    def side_of(x):
        if abs(x[1]) <= eps:
            return 0
        if abs(x[0] - lx) <= eps:
            return 1
        if abs(x[1] - ly) <= eps:
            return 2
        return 3

    m = from_polygons(P, cells, side_of)
    m.patches = dict(bottom=0, right=1, top=2, left=3)
    m.meta = dict(kind="hybrid", nx=nx, ny=ny, lx=lx, ly=ly, n_triangles=n_tri,
                  cell_xy_nominal=np.array([P[c].mean(0) for c in cells]))
    return m


def o_mesh_ratio(n_r: int, r0: float, first: float, r_far: float) -> float:
    """Geometric ratio q with r0 + first*(q^n_r - 1)/(q - 1) = r_far (bisection)."""
    lo, hi = 1.0 + 1e-12, 2.0
    span = r_far - r0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = first * (q ** n_r - 1.0) / (q - 1.0)
        lo, hi = (q, hi) if s < span else (lo, q)
    return 0.5 * (lo + hi)


def o_mesh(n_theta: int, n_r: int, *, diameter: float = 1.0, first: float = 0.005,
           r_far: float = 50.0) -> Mesh:
    """Body-fitted O-mesh around a circular cylinder centred at the origin.

    n_theta cells around, n_r cells out, radii geometric from D/2 with first cell
    thickness ``first`` (in units of D) out to ``r_far`` (in units of D).
    Patches: 0 cylinder wall, 1 far field.  Cell (i, k) has id i + n_theta*k.
    """
    r0 = 0.5 * diameter
    q = o_mesh_ratio(n_r, r0, first * diameter, r_far * diameter)
    radii = np.empty(n_r + 1)
    radii[0] = r0
    h = first * diameter
    for k in range(n_r):
        radii[k + 1] = radii[k] + h
        h *= q
    radii[-1] = r_far * diameter
    th = 2.0 * np.pi * np.arange(n_theta) / n_theta
    R, T = np.meshgrid(radii, th, indexing="ij")          # [n_r+1, n_theta]
    points = np.stack([(R * np.cos(T)).ravel(), (R * np.sin(T)).ravel()], 1)

    # radial faces at angle th_i, between cells (i-1, k) and (i, k), ring by ring
    kk, ii = np.meshgrid(np.arange(n_r), np.arange(n_theta), indexing="ij")
    ii, kk = ii.ravel(), kk.ravel()
    fpr = np.stack([ii + n_theta * kk, ii + n_theta * (kk + 1)], 1)
    ownr = (ii - 1) % n_theta + n_theta * kk
    nbrr = ii + n_theta * kk
    # circumferential faces at radius r_k, between cells (i, k-1) and (i, k)
    kk, ii = np.meshgrid(np.arange(n_r + 1), np.arange(n_theta), indexing="ij")
    ii, kk = ii.ravel(), kk.ravel()
    fpc = np.stack([ii + n_theta * kk, (ii + 1) % n_theta + n_theta * kk], 1)
    ownc = np.where(kk == 0, ii, np.where(kk == n_r, ii + n_theta * (n_r - 1), ii + n_theta * (kk - 1)))
    nbrc = np.where(kk == 0, -1 - 0, np.where(kk == n_r, -1 - 1, ii + n_theta * kk))
    fp = np.concatenate([fpr, fpc]).astype(np.int64)
    own = np.concatenate([ownr, ownc]).astype(np.int64)
    nbr = np.concatenate([nbrr, nbrc]).astype(np.int64)
    ci, ck = np.meshgrid(np.arange(n_theta), np.arange(n_r), indexing="xy")
    meta = dict(kind="o_mesh", n_theta=n_theta, n_r=n_r, ratio=q, radii=radii,
                cell_i=ci.ravel(), cell_k=ck.ravel(), diameter=diameter, first=first * diameter)
    return Mesh(points, fp, own, nbr, n_theta * n_r, dict(wall=0, farfield=1), meta)


def shuffled(mesh: Mesh, seed: int) -> Mesh:
    """Same mesh with cell ids, face ids and each face's point order permuted (seeded)."""
    rng = np.random.default_rng(seed)
    cperm = rng.permutation(mesh.n_cells)          # new id of old cell c is cperm[c]
    fperm = rng.permutation(mesh.n_faces)          # new face k is old face fperm[k]
    flip = rng.integers(0, 2, mesh.n_faces).astype(bool)
    own = cperm[mesh.owner[fperm]]
    nb_old = mesh.neighbour[fperm]
    nbr = np.where(nb_old >= 0, cperm[np.maximum(nb_old, 0)], nb_old)
    fp = mesh.face_pts[fperm].copy()
    fp[flip] = fp[flip][:, ::-1]
    meta = dict(mesh.meta)
    inv = np.empty_like(cperm)
    inv[cperm] = np.arange(mesh.n_cells)
    for key, val in mesh.meta.items():
        if isinstance(val, np.ndarray) and val.shape[:1] == (mesh.n_cells,):
            meta[key] = val[inv]
    meta["cell_perm"] = cperm
    return Mesh(mesh.points.copy(), fp, own, nbr, mesh.n_cells, dict(mesh.patches), meta)


# ----------------------------------------------------------------------------- cases

def couette(ny: int = 64, nx: int = 4, *, U: float = 0.1, Re: float = 10.0, cfl: float = 0.5,
            height: float = 1.0) -> Case:
    """Plane Couette flow: nx x ny square cells, unit height, periodic in x,
    bottom wall at rest, top wall moving at U; nu = U*H/Re."""
    dy = height / ny
    m = cartesian(nx, ny, nx * dy, height)
    w = nx * dy
    bcs = [(m.patches["left"], BC_PERIODIC, _bc_params(m.patches["right"], w, 0.0)),
           (m.patches["right"], BC_PERIODIC, _bc_params(m.patches["left"], -w, 0.0)),
           (m.patches["bottom"], BC_WALL, _bc_params()),
           (m.patches["top"], BC_MOVING_WALL, _bc_params(U, 0.0))]
    nu = U * height / Re
    return Case(f"couette_{nx}x{ny}", m, bcs, tau=3.0 * nu, dt=cfl * dy / math.sqrt(2.0),
                meta=dict(U=U, Re=Re, cfl=cfl, height=height))


def cavity(n: int = 256, *, U: float = 0.1, Re: float = 1000.0, cfl: float = 0.5) -> Case:
    """Lid-driven square cavity of n x n unit cells (L = n), lid (top) moving at U."""
    m = cartesian(n, n, float(n), float(n))
    bcs = [(m.patches["bottom"], BC_WALL, _bc_params()),
           (m.patches["right"], BC_WALL, _bc_params()),
           (m.patches["left"], BC_WALL, _bc_params()),
           (m.patches["top"], BC_MOVING_WALL, _bc_params(U, 0.0))]
    nu = U * n / Re
    return Case(f"cavity_{n}", m, bcs, tau=3.0 * nu, dt=cfl * 1.0 / math.sqrt(2.0),
                meta=dict(U=U, Re=Re, cfl=cfl, L=float(n)))


def cylinder(n_theta: int = 512, n_r: int = 256, *, U: float = 0.1, Re: float = 40.0,
             cfl: float = 0.5, first: float = 0.005, r_far: float = 50.0,
             shuffle_seed: int | None = 0) -> Case:
    """Flow past a circular cylinder of diameter 1 on an O-mesh; far field at r_far."""
    m = o_mesh(n_theta, n_r, first=first, r_far=r_far)
    if shuffle_seed is not None:
        m = shuffled(m, shuffle_seed)
    bcs = [(m.patches["wall"], BC_WALL, _bc_params()),
           (m.patches["farfield"], BC_FARFIELD, _bc_params(1.0, U, 0.0))]
    nu = U * 1.0 / Re
    # the smallest cell side is the first radial spacing (the circumferential side
    # of the first ring, pi*D/n_theta, is longer for n_theta <= 628)
    dmin = min(first, math.pi / n_theta)
    return Case(f"cylinder_{n_theta}x{n_r}", m, bcs, tau=3.0 * nu, dt=cfl * dmin / math.sqrt(2.0),
                u0=(U, 0.0), meta=dict(U=U, Re=Re, cfl=cfl))


def micro_cavity(n: int = 40, Kn: float = 1.0, *, U: float = 0.1, L: float = 1.0, nv: int = 100,
                 vmax: float = 2.0, RT0: float = 0.5, cfl: float = 0.5) -> Case:
    """Rarefied lid-driven micro cavity (Sec. IV): n x n cells on an L x L square,
    diffuse walls at R T0, lid moving at U, on an nv x nv velocity grid over
    [-vmax, vmax]^2.  The relaxation time follows from the Knudsen number with the
    mean free path lambda = (mu / p) sqrt(pi R T0 / 2): tau = Kn L sqrt(2 / (pi R T0));
    dt = cfl * (L / n) / (largest node speed)."""
    m = cartesian(n, n, L, L)
    bcs = [(m.patches["bottom"], BC_WALL, _bc_params()), (m.patches["right"], BC_WALL, _bc_params()),
           (m.patches["left"], BC_WALL, _bc_params()), (m.patches["top"], BC_MOVING_WALL, _bc_params(U, 0.0))]
    tau = Kn * L * math.sqrt(2.0 / (math.pi * RT0))
    h = 2.0 * vmax / nv
    vfast = math.sqrt(2.0) * (vmax - 0.5 * h)
    return Case(f"micro_cavity_{n}_Kn{Kn:g}", m, bcs, tau=tau, dt=cfl * (L / n) / vfast,
                meta=dict(U=U, Kn=Kn, nv=nv, vmax=vmax, RT0=RT0, L=L, cfl=cfl))


def periodic_box(nx: int, ny: int, *, lx: float | None = None, ly: float | None = None,
                 jitter: float = 0.0, seed: int | None = None, tau: float = 0.05,
                 dt: float = 0.1) -> Case:
    """Fully periodic nx x ny box (no walls): for fixed-point and conservation checks."""
    lx = float(nx) if lx is None else lx
    ly = float(ny) if ly is None else ly
    m = cartesian(nx, ny, lx, ly, jitter=jitter, seed=seed)
    bcs = [(3, BC_PERIODIC, _bc_params(1, lx, 0.0)), (1, BC_PERIODIC, _bc_params(3, -lx, 0.0)),
           (0, BC_PERIODIC, _bc_params(2, 0.0, ly)), (2, BC_PERIODIC, _bc_params(0, 0.0, -ly))]
    return Case(f"periodic_{nx}x{ny}", m, bcs, tau=tau, dt=dt)


def smooth_field(case: Case, seed: int, amp_rho: float = 0.05, amp_u: float = 0.05):
    """Seeded smooth initial (rho [N], u [N,2]) on a Cartesian-generated case, built from
    low Fourier modes of the nominal cell centres (periodic in the box)."""
    rng = np.random.default_rng(seed)
    xy = case.mesh.meta["cell_xy_nominal"]
    lx, ly = case.mesh.meta["lx"], case.mesh.meta["ly"]
    X = 2 * np.pi * xy[:, 0] / lx
    Y = 2 * np.pi * xy[:, 1] / ly

    def field_():
        out = np.zeros(len(X))
        for kx in range(0, 3):
            for ky in range(0, 3):
                a, b = rng.normal(size=2)
                out += a * np.cos(kx * X + ky * Y) + b * np.sin(kx * X + ky * Y)
        return out / 9.0

    rho = 1.0 + amp_rho * field_()
    u = np.stack([amp_u * field_(), amp_u * field_()], 1)
    return rho, u


def batch_cavities(count: int = 256, *, seed: int = 1, n_lo: int = 32, n_hi: int = 512,
                   re_lo: float = 100.0, re_hi: float = 5000.0, U: float = 0.1, cfl: float = 0.5):
    """Sizes and Reynolds numbers of a batch of lid-driven cavities, drawn log-uniformly (seeded)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))
    ns = np.clip(np.rint(ns).astype(int), n_lo, n_hi)
    res = np.exp(rng.uniform(math.log(re_lo), math.log(re_hi), count))
    return [(int(n), float(re)) for n, re in zip(ns, res)]
