"""High-precision hand stepper of the rarefied step on tiny grids -- TEST INFRASTRUCTURE.

A second, independent restatement of the S-DUGKS step on a discrete velocity grid
(Sec. II with the Maxwellian of Eq. Feq, diffuse walls of Sec. III) in 40-digit
arithmetic (mpmath), written cell-by-(i, j) on an nx x ny grid of dx x dy rectangles
with explicit neighbours and faces, instead of the face-based mesh machinery of
``sdugks_oracle.c``.  The Maxwellian needs exp, so the result is not exact as in the
D2Q9 hand stepper; at 40 digits its own rounding is far below FP64's, so the FP64
oracle must agree with it to FP64 rounding.

Readings shared with the oracle (readings of the paper, not code): the velocity grid
is the nv x nv midpoint grid on [-vmax, vmax]^2 with equal weights h^2, velocity
q = j + nv i with j along x; the distributions are weighted (moments are plain sums);
psi = (1, xi, |xi|^2/2) and R T = E / rho - |u|^2 / 2 with E the energy per unit mass;
the macroscopic flux of Eq. MacroUpdate is the moment of the same step's mesoscopic
flux; the LLSR neighbours are the face neighbours (periodic images at shifted
positions, none across a wall); upwind by the sign of xi . n, the mean of both sides'
reconstructions for a velocity tangential to the face (at a wall, the inner side's); a
diffuse wall sends back rho_w times its Maxwellian (rho 1, wall velocity, R T_w) into
the fluid and takes the leaving velocities from the inner reconstruction with rho_w
times the wall Maxwellian as their equilibrium, rho_w such that no mass crosses the
wall.
"""
from __future__ import annotations

import mpmath as mp

mp.mp.dps = 40


class Grid:
    """nx x ny rectangles of dx x dy on [0, nx dx] x [0, ny dy]; ``sides`` maps
    'bottom', 'right', 'top', 'left' to ('periodic',) or ('wall', u_x, u_y); cell (i, j)
    has id i + nx j.  nv x nv velocity nodes on [-vmax, vmax]^2."""

    def __init__(self, nx, ny, dx, dy, sides, nv, vmax):
        self.nx, self.ny = nx, ny
        self.dx, self.dy = mp.mpf(dx), mp.mpf(dy)
        self.sides = sides
        assert (sides["left"][0] == "periodic") == (sides["right"][0] == "periodic")
        assert (sides["bottom"][0] == "periodic") == (sides["top"][0] == "periodic")
        h = 2 * mp.mpf(vmax) / nv
        axis = [-mp.mpf(vmax) + (k + mp.mpf(1) / 2) * h for k in range(nv)]
        self.nodes = [(axis[j], axis[i]) for i in range(nv) for j in range(nv)]
        self.wq = h * h

    def cid(self, i, j):
        return i + self.nx * j

    def centre(self, i, j):
        return ((i + mp.mpf(1) / 2) * self.dx, (j + mp.mpf(1) / 2) * self.dy)

    def llsr_neighbours(self, i, j):
        """[(cell id, offset to its (image) centre)]: east, west, north, south."""
        out = []
        for di, dj, side in ((1, 0, "right"), (-1, 0, "left"), (0, 1, "top"), (0, -1, "bottom")):
            ii, jj = i + di, j + dj
            inside = 0 <= ii < self.nx and 0 <= jj < self.ny
            if not inside and self.sides[side][0] != "periodic":
                continue
            out.append((self.cid(ii % self.nx, jj % self.ny), (di * self.dx, dj * self.dy)))
        return out

    def faces(self):
        """[(owner, neighbour or None, unit normal owner -> neighbour (outward at a wall),
        length, face centre, offset from the owner's centre to the neighbour's (image)
        centre, wall velocity)]: every cell's east and north face, and the west and south
        faces of the first column and row where those sides are walls."""
        out = []
        for j in range(self.ny):
            for i in range(self.nx):
                c = self.cid(i, j)
                x, y = self.centre(i, j)
                # east face
                xb = (x + self.dx / 2, y)
                if i + 1 < self.nx or self.sides["right"][0] == "periodic":
                    out.append((c, self.cid((i + 1) % self.nx, j), (1, 0), self.dy, xb, (self.dx, 0), None))
                else:
                    out.append((c, None, (1, 0), self.dy, xb, None, self.sides["right"][1:]))
                # north face
                xb = (x, y + self.dy / 2)
                if j + 1 < self.ny or self.sides["top"][0] == "periodic":
                    out.append((c, self.cid(i, (j + 1) % self.ny), (0, 1), self.dx, xb, (0, self.dy), None))
                else:
                    out.append((c, None, (0, 1), self.dx, xb, None, self.sides["top"][1:]))
                if i == 0 and self.sides["left"][0] != "periodic":
                    out.append((c, None, (-1, 0), self.dy, (x - self.dx / 2, y), None, self.sides["left"][1:]))
                if j == 0 and self.sides["bottom"][0] != "periodic":
                    out.append((c, None, (0, -1), self.dx, (x, y - self.dy / 2), None, self.sides["bottom"][1:]))
        return out


def maxwell(g: Grid, rho, ux, uy, RT):
    """Eq. Feq (D = 2) at every node, times the node weight."""
    pre = rho / (2 * mp.pi * RT)
    return [g.wq * pre * mp.exp(-((x - ux) ** 2 + (y - uy) ** 2) / (2 * RT)) for x, y in g.nodes]


def moments(g: Grid, vals):
    """(sum, sum xi_x, sum xi_y, sum |xi|^2 / 2) of a weighted distribution."""
    m = [mp.mpf(0)] * 4
    for (x, y), v in zip(g.nodes, vals):
        m[0] += v
        m[1] += x * v
        m[2] += y * v
        m[3] += (x * x + y * y) / 2 * v
    return m


def maxwell_W(g: Grid, W):
    rho = W[0]
    ux, uy = W[1] / rho, W[2] / rho
    return maxwell(g, rho, ux, uy, W[3] / rho - (ux * ux + uy * uy) / 2)


def step(g: Grid, f, W, tau, dt, RTw):
    """One step in place: f[c] lists of Q values, W[c] = [rho, rho u_x, rho u_y, rho E]."""
    tau, dt, RTw = mp.mpf(tau), mp.mpf(dt), mp.mpf(RTw)
    a = (2 * tau - dt) / (2 * tau)
    b = dt / (2 * tau)
    cf = 2 * tau / (2 * tau + dt)
    r = dt / tau
    n_cells, Q = g.nx * g.ny, len(g.nodes)
    vol = g.dx * g.dy
    # Eq. fbarplus
    fbp = []
    for c in range(n_cells):
        eq = maxwell_W(g, W[c])
        fbp.append([a * f[c][q] + b * eq[q] for q in range(Q)])
    # LLSR gradient per cell and velocity: sigma = A^-1 sum_k d_k (fbp_k - fbp_c)
    sig = []
    for j in range(g.ny):
        for i in range(g.nx):
            c = g.cid(i, j)
            nb = g.llsr_neighbours(i, j)
            axx = sum(d[0] * d[0] for _, d in nb)
            axy = sum(d[0] * d[1] for _, d in nb)
            ayy = sum(d[1] * d[1] for _, d in nb)
            det = axx * ayy - axy * axy
            row = []
            for q in range(Q):
                bx = sum(d[0] * (fbp[k][q] - fbp[c][q]) for k, d in nb)
                by = sum(d[1] * (fbp[k][q] - fbp[c][q]) for k, d in nb)
                row.append(((ayy * bx - axy * by) / det, (axx * by - axy * bx) / det))
            sig.append(row)
    centres = [None] * n_cells
    for j in range(g.ny):
        for i in range(g.nx):
            centres[g.cid(i, j)] = g.centre(i, j)
    # interface distributions and the flux sum of every cell (Eqs. fbpsource, fbar,
    # Macro, Feq, f_t_n+1, MesoFlux)
    F = [[mp.mpf(0)] * Q for _ in range(n_cells)]
    for o, k, n, length, xb, off, wall in g.faces():
        xo = centres[o]
        s = [x * n[0] + y * n[1] for x, y in g.nodes]

        def recon(cell, pos, q):
            x, y = g.nodes[q]
            return (fbp[cell][q] + (xb[0] - x * dt - pos[0]) * sig[cell][q][0]
                    + (xb[1] - y * dt - pos[1]) * sig[cell][q][1])

        if k is not None:
            xk = (xo[0] + off[0], xo[1] + off[1])      # the neighbour's (image) centre
            fbar = [recon(o, xo, q) if s[q] > 0 else
                    (recon(k, xk, q) if s[q] < 0 else (recon(o, xo, q) + recon(k, xk, q)) / 2) for q in range(Q)]
            gb = maxwell_W(g, moments(g, fbar))
            fb = [cf * (fbar[q] + b * gb[q]) for q in range(Q)]
        else:
            gw = maxwell(g, mp.mpf(1), mp.mpf(wall[0]), mp.mpf(wall[1]), RTw)
            fbar = [recon(o, xo, q) if s[q] >= 0 else None for q in range(Q)]
            s_out = sum(s[q] * fbar[q] for q in range(Q) if s[q] >= 0)
            g_out = sum(s[q] * gw[q] for q in range(Q) if s[q] >= 0)
            g_in = sum(s[q] * gw[q] for q in range(Q) if s[q] < 0)
            rho_w = -cf * s_out / (cf * b * g_out + g_in)
            fb = [rho_w * gw[q] if s[q] < 0 else cf * (fbar[q] + b * rho_w * gw[q]) for q in range(Q)]
        for q in range(Q):
            flux = s[q] * length * fb[q]
            F[o][q] += flux
            if k is not None:
                F[k][q] -= flux
    # Eqs. MacroFlux, MacroUpdate, fn+1
    for c in range(n_cells):
        M = moments(g, F[c])
        W[c] = [W[c][d] - dt / vol * M[d] for d in range(4)]
        eq = maxwell_W(g, W[c])
        f[c] = [(f[c][q] - dt / vol * F[c][q] + r * eq[q]) / (1 + r) for q in range(Q)]


def run(g: Grid, f, W, tau, dt, RTw, n_steps):
    """n_steps steps from FP64 (or exact) starting values; returns (f, W) as mpf lists."""
    f = [[mp.mpf(v) for v in row] for row in f]
    W = [[mp.mpf(v) for v in row] for row in W]
    for _ in range(n_steps):
        step(g, f, W, tau, dt, RTw)
    return f, W
