"""Planted-mistake sweep of the oracle's CPU pins (test infrastructure).

Each entry plants one plausible mistake (a dropped term, a wrong sign, a wrong factor,
the wrong side) in a copy of oracle/sdugks_oracle.c, compiles the copy in a temporary
folder with the oracle's flags, and runs the pins against it (SDUGKS_ORACLE_LIB).  A
mistake that no pin catches is a gap in the pins.  The in-tree oracle is never edited.
Run from the repository root:

    python tests/oracle_mutation_sweep.py        # exit status 1 if a mistake goes uncaught
"""
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

D2Q9, DVM = "tests/test_oracle_pins.py", "tests/test_oracle_pins_dvm.py"
FORCES = "tests/test_oracle_pins_forces.py"

# (what, pins, text in the oracle, replacement, which occurrence: 0 first, -1 last)
MUTATIONS = [
    ("D2Q9: sign of xi dt in the reconstruction", D2Q9,
     "double px = xb[0] - XI[a][0] * dt, py = xb[1] - XI[a][1] * dt;",
     "double px = xb[0] + XI[a][0] * dt, py = xb[1] + XI[a][1] * dt;", 0),
    ("D2Q9: b feq_b dropped from f_b", D2Q9,
     "fbf[a] = (fbar[a] + b_plus * feqb[a]) * c_face;", "fbf[a] = fbar[a] * c_face;", 0),
    ("D2Q9: c dropped from f_b", D2Q9,
     "fbf[a] = (fbar[a] + b_plus * feqb[a]) * c_face;", "fbf[a] = (fbar[a] + b_plus * feqb[a]);", 0),
    ("D2Q9: relaxation rate dt/(2 tau)", D2Q9,
     "const double r = dt / tau;", "const double r = dt / (2.0 * tau);", 0),
    ("D2Q9: Hermite coefficient of (xi.u)^2", D2Q9,
     "(eu * eu) / (2.0 * CS2 * CS2)", "(eu * eu) / (2.5 * CS2 * CS2)", 0),
    ("D2Q9: sign of the W update", D2Q9,
     "W[3 * j + d] - dt / m->vol[j] * Mj[d]", "W[3 * j + d] + dt / m->vol[j] * Mj[d]", 0),
    ("LLSR: sign of the inverse's off-diagonal", D2Q9,
     "m->ainv[3 * c + 1] = -axy / det;", "m->ainv[3 * c + 1] = axy / det;", 0),
    ("D2Q9: downwind side", D2Q9,
     "if (s > TIE) fbar[a] = from_o;\n                else if (s < -TIE) fbar[a] = from_k;",
     "if (s > TIE) fbar[a] = from_k;\n                else if (s < -TIE) fbar[a] = from_o;", 0),
    ("D2Q9: coefficient a of fbar+", D2Q9,
     "(2.0 * tau - dt) / (2.0 * tau);  /* Eq. fbarplus */",
     "(2.0 * tau - 0.5 * dt) / (2.0 * tau);  /* Eq. fbarplus */", 0),
    ("D2Q9: wall's non-equilibrium part dropped", D2Q9,
     "fbf[a] = feqb[a] + (f[NQ * o + a] - w->feqn[NQ * o + a]);", "fbf[a] = feqb[a];", 0),
    ("D2Q9: far-field velocity components swapped", D2Q9,
     "*rho = par[0]; *ux = par[1]; *uy = par[2]; break;", "*rho = par[0]; *ux = par[2]; *uy = par[1]; break;", 0),
    ("D2Q9: sign of the outlet's tangential velocity", D2Q9,
     "*rho = Wo[0]; *ux = Wo[1] / Wo[0]; *uy = Wo[2] / Wo[0]; break;",
     "*rho = Wo[0]; *ux = Wo[1] / Wo[0]; *uy = -Wo[2] / Wo[0]; break;", 0),
    ("D2Q9: sign of the moving wall's velocity", D2Q9,
     "*rho = Wo[0]; *ux = par[0]; *uy = par[1]; break;", "*rho = Wo[0]; *ux = -par[0]; *uy = par[1]; break;", 0),
    ("symmetry: mirror ghost's gradient not reflected", D2Q9,
     "else if (mir == 2) { ak = MIRROR_Y[a]; gsy = -1.0; }", "else if (mir == 2) { ak = MIRROR_Y[a]; gsy = 1.0; }", 0),
    ("geometry: centroid divisor", D2Q9,
     "cen[0] = ox + cx / (3.0 * a2);", "cen[0] = ox + cx / (6.0 * a2);", 0),
    ("residual: denominator without V0", D2Q9,
     "den += U0 * U0 + V0 * V0;", "den += U0 * U0;", 0),
    ("D2Q9: tangential velocities take the owner's side", D2Q9,
     "else fbar[a] = 0.5 * (from_o + from_k);", "else fbar[a] = from_o;", 0),
    ("D2Q9: interface momentum from the wrong component", D2Q9,
     "Wb[1] += XI[a][0] * fbar[a];", "Wb[1] += XI[a][1] * fbar[a];", 0),
    ("D2Q9: wall's leaving values without b feq_b", D2Q9,
     "fbf[a] = (fbar + b_plus * feqb[a]) * c_face;", "fbf[a] = fbar * c_face;", 0),
    ("D2Q9: sign of the wall's non-equilibrium part", D2Q9,
     "fbf[a] = feqb[a] + (f[NQ * o + a] - w->feqn[NQ * o + a]);", "fbf[a] = feqb[a] - (f[NQ * o + a] - w->feqn[NQ * o + a]);", 0),
    ("D2Q9: coefficient of u^2 in feq", D2Q9,
     "- uu / (2.0 * CS2));", "- uu / (3.0 * CS2));", 0),
    ("D2Q9: a diagonal weight", D2Q9,
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 35.0};", 0),
    ("LLSR: sign of the offset d = x_k - x_j", D2Q9,
     "bx += (px - m->xc[2 * c]) * dphi;", "bx += (m->xc[2 * c] - px) * dphi;", 0),
    ("D2Q9: neighbour side adds the face flux", D2Q9,
     "double sg = (m->own[fc] == j) ? 1.0 : -1.0;", "double sg = 1.0;", 0),
    ("geometry: periodic image without its shift", D2Q9,
     "m->gpos[2 * f] = m->xc[2 * other] - sx;", "m->gpos[2 * f] = m->xc[2 * other];", 0),
    ("geometry: symmetry ghost at half its distance (lines of constant y)", D2Q9,
     "m->gpos[2 * f + 1] = xo[1] + 2.0 * dn * Ny;", "m->gpos[2 * f + 1] = xo[1] + dn * Ny;", 0),
    ("geometry: symmetry ghost at half its distance (lines of constant x)", D2Q9,
     "m->gpos[2 * f] = xo[0] + 2.0 * dn * Nx;", "m->gpos[2 * f] = xo[0] + dn * Nx;", 0),
    ("symmetry: ghost's x-gradient not reflected", D2Q9,
     "if (mir == 1) { ak = MIRROR_X[a]; gsx = -1.0; }", "if (mir == 1) { ak = MIRROR_X[a]; gsx = 1.0; }", 0),
    ("forces: x-momentum flux from the y component of xi", FORCES,
     "px += XI[a][0] * s * fb[NQ * fc + a];", "px += XI[a][1] * s * fb[NQ * fc + a];", 0),
    ("forces: flux without the normal velocity s", FORCES,
     "py += XI[a][1] * s * fb[NQ * fc + a];", "py += XI[a][1] * fb[NQ * fc + a];", 0),
    ("forces: rows for periodic faces too", FORCES,
     "if (m->nbr[fc] >= 0 || m->bck[-1 - m->nbr[fc]] == KIND_PERIODIC) continue;",
     "if (m->nbr[fc] >= 0) continue;", 0),
    ("forces: the previous step's interface values", FORCES,
     "    if (!rc && bflux) boundary_flux(&m, w.fb, bflux);\n",
     "    if (!rc && bflux) { one_step(&m, tau, dt, f, W, &w); boundary_flux(&m, w.fb, bflux); }\n", 0),
    ("D2Q9: cell update without the 1/(1 + r)", D2Q9,
     "f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]) / (1.0 + r);",
     "f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]);", 0),
    ("D2Q9: sign of the flux in the f update", D2Q9,
     "f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]) / (1.0 + r);",
     "f[NQ * j + a] = (f[NQ * j + a] + dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]) / (1.0 + r);", 0),
    ("D2Q9: f update with the old equilibrium", D2Q9,
     "f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * feq1[a]) / (1.0 + r);",
     "f[NQ * j + a] = (f[NQ * j + a] - dt / m->vol[j] * w->F[NQ * j + a] + r * w->feqn[NQ * j + a]) / (1.0 + r);", 0),
    ("D2Q9: c = 2 tau / (2 tau - dt)", D2Q9,
     "const double c_face = 2.0 * tau / (2.0 * tau + dt);    /* Eq. f_t_n+1 */",
     "const double c_face = 2.0 * tau / (2.0 * tau - dt);    /* Eq. f_t_n+1 */", 0),
    ("D2Q9: b feq_b doubled in f_b", D2Q9,
     "fbf[a] = (fbar[a] + b_plus * feqb[a]) * c_face;", "fbf[a] = (fbar[a] + 2.0 * b_plus * feqb[a]) * c_face;", 0),
    ("D2Q9: tangential velocities take the neighbour's side", D2Q9,
     "else fbar[a] = 0.5 * (from_o + from_k);", "else fbar[a] = from_k;", 0),
    ("D2Q9: interface density without the rest velocity", D2Q9,
     "                Wb[0] += fbar[a];\n", "                Wb[0] += a ? fbar[a] : 0.0;\n", 0),
    ("equilibrium: velocity not divided by rho", D2Q9,
     "feq_of(W[0], W[1] / W[0], W[2] / W[0], out);", "feq_of(W[0], W[1], W[2], out);", 0),
    ("walls: incoming values from fbar+ instead of f", D2Q9,
     "fbf[a] = feqb[a] + (f[NQ * o + a] - w->feqn[NQ * o + a]);",
     "fbf[a] = feqb[a] + (w->fbp[NQ * o + a] - w->feqn[NQ * o + a]);", 0),
    ("walls: leaving values without the gradient term", D2Q9,
     "double fbar = w->fbp[NQ * o + a] + (px - xo[0]) * w->sig[2 * (NQ * o + a)] +\n"
     "                                  (py - xo[1]) * w->sig[2 * (NQ * o + a) + 1];",
     "double fbar = w->fbp[NQ * o + a];", 0),
    ("walls: moving wall's density fixed at 1", D2Q9,
     "*rho = Wo[0]; *ux = par[0]; *uy = par[1]; break;", "*rho = 1.0; *ux = par[0]; *uy = par[1]; break;", 0),
    ("outlet: velocity not divided by rho", D2Q9,
     "*rho = Wo[0]; *ux = Wo[1] / Wo[0]; *uy = Wo[2] / Wo[0]; break;",
     "*rho = Wo[0]; *ux = Wo[1]; *uy = Wo[2]; break;", 0),
    ("symmetry: ghost velocity not mirrored (lines of constant x)", D2Q9,
     "if (mir == 1) { ak = MIRROR_X[a]; gsx = -1.0; }", "if (mir == 1) { gsx = -1.0; }", 0),
    ("LLSR: diagonal entries of the inverse swapped", D2Q9,
     "m->ainv[3 * c] = ayy / det;", "m->ainv[3 * c] = axx / det;", 0),
    ("forces: y-momentum from the x component of xi", FORCES,
     "py += XI[a][1] * s * fb[NQ * fc + a];", "py += XI[a][0] * s * fb[NQ * fc + a];", 0),
    ("forces: sign of the face normal", FORCES,
     "double s = XI[a][0] * m->nl[2 * fc] + XI[a][1] * m->nl[2 * fc + 1];\n            px +=",
     "double s = -(XI[a][0] * m->nl[2 * fc] + XI[a][1] * m->nl[2 * fc + 1]);\n            px +=", 0),
    ("forces: the flux halved", FORCES,
     "px += XI[a][0] * s * fb[NQ * fc + a];\n            py += XI[a][1] * s * fb[NQ * fc + a];",
     "px += XI[a][0] * s * fb[NQ * fc + a] * 0.5;\n            py += XI[a][1] * s * fb[NQ * fc + a] * 0.5;", 0),
    ("rarefied: sign of the W update", DVM,
     "W[4 * j + d] -= dt / m->vol[j] * Mj[d];", "W[4 * j + d] += dt / m->vol[j] * Mj[d];", -1),
    ("rarefied: wall density without its b G_out term", DVM,
     "double rho_w = -c_face * S_out / (c_face * b_plus * G_out + G_in);",
     "double rho_w = -c_face * S_out / (G_in);", -1),
    ("rarefied: wall's leaving values without b rho_w g", DVM,
     "fbf[q] = s < -TIE ? rho_w * g[q] : (fbar[q] + b_plus * rho_w * g[q]) * c_face;",
     "fbf[q] = s < -TIE ? rho_w * g[q] : fbar[q] * c_face;", -1),
    ("rarefied: Maxwellian prefactor", DVM,
     "const double pre = rho / (2.0 * M_PI * RT);", "const double pre = rho / (M_PI * RT);", -1),
    ("rarefied: Maxwellian exponent", DVM,
     "exp(-(cx * cx + cy * cy) / (2.0 * RT));", "exp(-(cx * cx + cy * cy) / (RT));", -1),
    ("rarefied: a and b of fbar+ swapped", DVM,
     "k->fbp[(size_t)Q * j + q] = a_plus * f[(size_t)Q * j + q] + b_plus * fe[q];",
     "k->fbp[(size_t)Q * j + q] = b_plus * f[(size_t)Q * j + q] + a_plus * fe[q];", -1),
    ("rarefied: tangential velocities take the owner's side", DVM,
     "fbar[q] = s > TIE ? from_o : (s < -TIE ? from_k : 0.5 * (from_o + from_k));",
     "fbar[q] = s > TIE ? from_o : (s < -TIE ? from_k : from_o);", -1),
    ("rarefied: downwind side", DVM,
     "fbar[q] = s > TIE ? from_o : (s < -TIE ? from_k : 0.5 * (from_o + from_k));",
     "fbar[q] = s > TIE ? from_k : (s < -TIE ? from_o : 0.5 * (from_o + from_k));", -1),
    ("rarefied: sign of xi dt in the reconstruction", DVM,
     "double px = xb[0] - xi[2 * q] * dt, py = xb[1] - xi[2 * q + 1] * dt;\n                    const double *so = &k->sig[2 * ((size_t)Q * o + q)], *sk",
     "double px = xb[0] + xi[2 * q] * dt, py = xb[1] + xi[2 * q + 1] * dt;\n                    const double *so = &k->sig[2 * ((size_t)Q * o + q)], *sk", -1),
    ("rarefied: b feq_b dropped from f_b", DVM,
     "fbf[q] = (fbar[q] + b_plus * g[q]) * c_face;   /* step 7 */", "fbf[q] = fbar[q] * c_face;   /* step 7 */", -1),
    ("rarefied: relaxation rate dt/(2 tau)", DVM,
     "    const double r = dt / tau;\n", "    const double r = dt / (2.0 * tau);\n", -1),
    ("rarefied: temperature from the total energy", DVM,
     "double RT = W[3] / rho - 0.5 * (ux * ux + uy * uy);", "double RT = W[3] / rho;", -1),
    ("rarefied: energy moment without its 1/2", DVM,
     "W[3] += 0.5 * (x * x + y * y) * g[q];", "W[3] += (x * x + y * y) * g[q];", -1),
    ("rarefied: moving wall's velocity reversed", DVM,
     "if (m->bck[p] == KIND_MOVING_WALL) { uwx = m->bcp[3 * p]; uwy = m->bcp[3 * p + 1]; }",
     "if (m->bck[p] == KIND_MOVING_WALL) { uwx = -m->bcp[3 * p]; uwy = -m->bcp[3 * p + 1]; }", -1),
    ("rarefied: wall Maxwellian at twice the wall temperature", DVM,
     "dvm_maxwell(1.0, uwx, uwy, RTw, Q, xi, w, g);", "dvm_maxwell(1.0, uwx, uwy, 2.0 * RTw, Q, xi, w, g);", -1),
    ("rarefied: wall density without c", DVM,
     "double rho_w = -c_face * S_out / (c_face * b_plus * G_out + G_in);",
     "double rho_w = -S_out / (c_face * b_plus * G_out + G_in);", -1),
    ("rarefied: first-order reconstruction (no gradient term)", DVM,
     "double from_o = k->fbp[(size_t)Q * o + q] + (px - xo[0]) * so[0] + (py - xo[1]) * so[1];",
     "double from_o = k->fbp[(size_t)Q * o + q];", -1),
    ("rarefied: cell update without the 1/(1 + r)", DVM,
     "f[(size_t)Q * j + q] = (f[(size_t)Q * j + q] - dt / m->vol[j] * Fj[q] + r * fe[q]) / (1.0 + r);",
     "f[(size_t)Q * j + q] = (f[(size_t)Q * j + q] - dt / m->vol[j] * Fj[q] + r * fe[q]);", -1),
]


def main() -> int:
    with open(os.path.join(ROOT, "oracle", "sdugks_oracle.c")) as fh:
        src = fh.read()
    missed = 0
    with tempfile.TemporaryDirectory() as tmp:
        for k, (what, pins, old, new, which) in enumerate(MUTATIONS):
            if old not in src:
                print(f"{what}: text not found in the oracle")
                missed += 1
                continue
            i = src.index(old) if which == 0 else src.rindex(old)
            c_path, so_path = os.path.join(tmp, f"m{k}.c"), os.path.join(tmp, f"m{k}.so")
            with open(c_path, "w") as fh:
                fh.write(src[:i] + new + src[i + len(old):])
            oracle.compile_library(c_path, so_path)
            r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider"],
                               cwd=ROOT, capture_output=True, text=True,
                               env=dict(os.environ, SDUGKS_ORACLE_LIB=so_path))
            caught = [ln.split("::")[1].split(" ")[0] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
            if not caught and r.returncode not in (0, 1):       # the pins' process died: the mistake showed
                caught = [f"a crash of the pins (exit status {r.returncode})"]
            print(f"{what}: " + (f"caught by {caught[0]}" if caught else "NOT CAUGHT"), flush=True)
            missed += not caught
    print(f"{len(MUTATIONS) - missed} of {len(MUTATIONS)} planted mistakes caught")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
