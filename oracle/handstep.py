"""Exact-rational hand stepper for tiny structured meshes -- TEST INFRASTRUCTURE.

A second, independent restatement of the S-DUGKS step (Sec. II, boundary rules of
Sec. III) in exact rational arithmetic (``fractions.Fraction``) on an nx x ny grid of
dx x dy rectangles, written cell-by-(i, j) with explicit neighbours instead of the
face-based mesh machinery of ``sdugks_oracle.c``.  It pins the C oracle by brute
force on 2x2 and 3x3 meshes over a few steps: with rational tau, dt, dx, dy and the
polynomial D2Q9 equilibrium every quantity of the step is rational, so this result
is exact and the FP64 oracle must agree with it to rounding.

Readings shared with the oracle (they are readings of the paper, not code): D2Q9 with
c_s^2 = 1/3, the macroscopic flux of Eq. MacroUpdate = moments of the same step's
mesoscopic flux (the moment of Eq. Integration), upwind by the sign of xi.n with the
two-sided mean for tangential
velocities, wall/far-field/outlet by non-equilibrium extrapolation for incoming
velocities and interior reconstruction with the boundary Maxwellian otherwise.
"""
from __future__ import annotations

from fractions import Fraction as Fr

XI = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W9 = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4


def feq(rho, ux, uy):
    """Second-order Hermite equilibrium, 3 = 1/c_s^2."""
    out = []
    uu = ux * ux + uy * uy
    for (ex, ey), w in zip(XI, W9):
        eu = ex * ux + ey * uy
        out.append(w * rho * (1 + 3 * eu + Fr(9, 2) * eu * eu - Fr(3, 2) * uu))
    return out


def feq_W(W):
    return feq(W[0], W[1] / W[0], W[2] / W[0])


class Grid:
    """nx x ny rectangles of size dx x dy; ``sides`` maps 'bottom','right','top','left'
    to ('periodic',) | ('wall', ux, uy) | ('farfield', rho, ux, uy) | ('outlet',)."""

    def __init__(self, nx, ny, dx, dy, sides):
        self.nx, self.ny, self.dx, self.dy = nx, ny, Fr(dx), Fr(dy)
        self.sides = sides
        assert (sides["left"][0] == "periodic") == (sides["right"][0] == "periodic")
        assert (sides["bottom"][0] == "periodic") == (sides["top"][0] == "periodic")

    def cid(self, i, j):
        return i + self.nx * j

    def centre(self, i, j):
        return ((i + Fr(1, 2)) * self.dx, (j + Fr(1, 2)) * self.dy)

    def neighbours(self, i, j):
        """[(cell id, offset vector to its (image) centre)] over the four sides."""
        out = []
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            ii, jj = i + di, j + dj
            if 0 <= ii < self.nx and 0 <= jj < self.ny:
                out.append((self.cid(ii, jj), (di * self.dx, dj * self.dy)))
                continue
            side = {(1, 0): "right", (-1, 0): "left", (0, 1): "top", (0, -1): "bottom"}[(di, dj)]
            if self.sides[side][0] == "periodic":
                out.append((self.cid(ii % self.nx, jj % self.ny), (di * self.dx, dj * self.dy)))
        return out


def step(g: Grid, tau, dt, f, W):
    """One step; f[c][9], W[c][3] lists of Fractions.  Returns the new (f, W)."""
    tau, dt = Fr(tau), Fr(dt)
    n = g.nx * g.ny
    vol = g.dx * g.dy
    ap, bp, cf, r = (2 * tau - dt) / (2 * tau), dt / (2 * tau), 2 * tau / (2 * tau + dt), dt / tau
    feqn = [feq_W(W[c]) for c in range(n)]
    fbp = [[ap * f[c][a] + bp * feqn[c][a] for a in range(9)] for c in range(n)]
    # least-squares gradient: solve (sum d d^T) sigma = sum d (phi_k - phi_j)
    sig = []
    for j in range(g.ny):
        for i in range(g.nx):
            c = g.cid(i, j)
            nb = g.neighbours(i, j)
            axx = sum(d[0] * d[0] for _, d in nb)
            axy = sum(d[0] * d[1] for _, d in nb)
            ayy = sum(d[1] * d[1] for _, d in nb)
            det = axx * ayy - axy * axy
            s = []
            for a in range(9):
                bx = sum(d[0] * (fbp[k][a] - fbp[c][a]) for k, d in nb)
                by = sum(d[1] * (fbp[k][a] - fbp[c][a]) for k, d in nb)
                if det == 0:
                    s.append((Fr(0), Fr(0)))
                else:
                    s.append(((ayy * bx - axy * by) / det, (axx * by - axy * bx) / det))
            sig.append(s)

    def extrap(c, xc, xb, a):
        ex, ey = XI[a]
        px, py = xb[0] - ex * dt, xb[1] - ey * dt
        return fbp[c][a] + (px - xc[0]) * sig[c][a][0] + (py - xc[1]) * sig[c][a][1]

    F = [[Fr(0)] * 9 for _ in range(n)]

    def add_flux(c, nl_out, fb):
        for a in range(9):
            F[c][a] += (XI[a][0] * nl_out[0] + XI[a][1] * nl_out[1]) * fb[a]

    def interior_face(cl, xl, cr, xr, xb, nl):
        """Face with outward normal*length nl from cell cl (centre xl) toward cr (xr)."""
        fbar = []
        for a in range(9):
            s = XI[a][0] * nl[0] + XI[a][1] * nl[1]
            el, er = extrap(cl, xl, xb, a), extrap(cr, xr, xb, a)
            fbar.append(el if s > 0 else er if s < 0 else (el + er) / 2)
        rho = sum(fbar)
        mx = sum(XI[a][0] * fbar[a] for a in range(9))
        my = sum(XI[a][1] * fbar[a] for a in range(9))
        fe = feq(rho, mx / rho, my / rho)
        return [(fbar[a] + bp * fe[a]) * cf for a in range(9)]

    def boundary_face(c, xc, xb, nl, side):
        kind = g.sides[side]
        if kind[0] == "wall":
            rho, ux, uy = W[c][0], Fr(kind[1]), Fr(kind[2])
        elif kind[0] == "farfield":
            rho, ux, uy = Fr(kind[1]), Fr(kind[2]), Fr(kind[3])
        elif kind[0] == "outlet":
            rho, ux, uy = W[c][0], W[c][1] / W[c][0], W[c][2] / W[c][0]
        else:
            raise ValueError(kind)
        fe = feq(rho, ux, uy)
        out = []
        for a in range(9):
            s = XI[a][0] * nl[0] + XI[a][1] * nl[1]
            if s < 0:
                out.append(fe[a] + f[c][a] - feqn[c][a])
            else:
                out.append((extrap(c, xc, xb, a) + bp * fe[a]) * cf)
        return out

    dx, dy = g.dx, g.dy
    # faces of constant x: between (i-1, j) and (i, j), normal +x, length dy
    for j in range(g.ny):
        for i in range(g.nx + 1):
            xb = (i * dx, (j + Fr(1, 2)) * dy)
            nl = (dy, Fr(0))
            if 0 < i < g.nx:
                L, R = g.cid(i - 1, j), g.cid(i, j)
                fb = interior_face(L, g.centre(i - 1, j), R, g.centre(i, j), xb, nl)
                add_flux(L, nl, fb); add_flux(R, (-nl[0], -nl[1]), fb)
            elif i == 0 and g.sides["left"][0] == "periodic":
                continue                               # counted once, at i == nx
            elif i == g.nx and g.sides["right"][0] == "periodic":
                L, R = g.cid(g.nx - 1, j), g.cid(0, j)
                xr = (g.nx * dx + dx / 2, (j + Fr(1, 2)) * dy)   # image of cell (0, j)
                fb = interior_face(L, g.centre(g.nx - 1, j), R, xr, xb, nl)
                add_flux(L, nl, fb); add_flux(R, (-nl[0], -nl[1]), fb)
            elif i == 0:
                c = g.cid(0, j)
                add_flux(c, (-dy, Fr(0)), boundary_face(c, g.centre(0, j), xb, (-dy, Fr(0)), "left"))
            else:
                c = g.cid(g.nx - 1, j)
                add_flux(c, nl, boundary_face(c, g.centre(g.nx - 1, j), xb, nl, "right"))
    # faces of constant y: between (i, j-1) and (i, j), normal +y, length dx
    for j in range(g.ny + 1):
        for i in range(g.nx):
            xb = ((i + Fr(1, 2)) * dx, j * dy)
            nl = (Fr(0), dx)
            if 0 < j < g.ny:
                B, T = g.cid(i, j - 1), g.cid(i, j)
                fb = interior_face(B, g.centre(i, j - 1), T, g.centre(i, j), xb, nl)
                add_flux(B, nl, fb); add_flux(T, (-nl[0], -nl[1]), fb)
            elif j == 0 and g.sides["bottom"][0] == "periodic":
                continue
            elif j == g.ny and g.sides["top"][0] == "periodic":
                B, T = g.cid(i, g.ny - 1), g.cid(i, 0)
                xt = ((i + Fr(1, 2)) * dx, g.ny * dy + dy / 2)
                fb = interior_face(B, g.centre(i, g.ny - 1), T, xt, xb, nl)
                add_flux(B, nl, fb); add_flux(T, (-nl[0], -nl[1]), fb)
            elif j == 0:
                c = g.cid(i, 0)
                add_flux(c, (Fr(0), -dx), boundary_face(c, g.centre(i, 0), xb, (Fr(0), -dx), "bottom"))
            else:
                c = g.cid(i, g.ny - 1)
                add_flux(c, nl, boundary_face(c, g.centre(i, g.ny - 1), xb, nl, "top"))

    f_new, W_new = [], []
    for c in range(n):
        mac = [sum(F[c]), sum(XI[a][0] * F[c][a] for a in range(9)), sum(XI[a][1] * F[c][a] for a in range(9))]
        w1 = [W[c][d] - dt / vol * mac[d] for d in range(3)]
        fe1 = feq_W(w1)
        f_new.append([(f[c][a] - dt / vol * F[c][a] + r * fe1[a]) / (1 + r) for a in range(9)])
        W_new.append(w1)
    return f_new, W_new


def run(g: Grid, tau, dt, rho, u, n_steps):
    """Start from f = feq(rho, u) and take n_steps steps; returns (f, W)."""
    n = g.nx * g.ny
    W = [[Fr(rho[c]), Fr(rho[c]) * Fr(u[c][0]), Fr(rho[c]) * Fr(u[c][1])] for c in range(n)]
    f = [feq(Fr(rho[c]), Fr(u[c][0]), Fr(u[c][1])) for c in range(n)]
    for _ in range(n_steps):
        f, W = step(g, tau, dt, f, W)
    return f, W
